// Grid transfers, Krylov vector passes, small dense solves and set-up kernels.
//
// Reductions are deterministic: each block reduces its elements in a fixed
// tree (per-thread partial sums in the working precision, block and grid
// combination in double), writes per-block partials, and the last block to
// arrive (atomic arrival counter, no waiting) combines them in block order
// and runs a small epilogue on the result.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "hz_gram_solve.cuh"
#include "hz_kernels.h"

namespace hz {

constexpr int VB = 256;          // threads per block of vector kernels
constexpr int KMAX = 16;         // largest Krylov basis handled by one pass

static int vec_blocks(long long n) {
  long long b = (n + VB * 4 - 1) / (VB * 4);
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 8));
}
// reduction kernels use fewer, fuller blocks: fewer partial sums to combine
static int red_blocks(long long n) {
  long long b = (n + VB * 4 - 1) / (VB * 4);
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 4));
}

// ----------------------------------------------------------------------------
// transfers
// ----------------------------------------------------------------------------
// Both transfer kernels map threads to (x, y) of one plane of one right-hand
// side (blockIdx.z = rhs * planes + z): no integer division per node, 32-bit
// offsets within a field (fewer than 2^31 nodes).
constexpr int TRX = 64, TRY = 4;

// full weighting (Eq. restriction): c = R f, weights (1/4, 1/2, 1/4) per axis
template <class R>
__global__ void __launch_bounds__(TRX * TRY) k_restrict(const cx<R>* __restrict__ f, cx<R>* __restrict__ c, int nxf,
                                                         int nyf, int nzf) {
  const int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1, nzc = (nzf - 1) / 2 + 1;
  const int X = blockIdx.x * TRX + threadIdx.x, Y = blockIdx.y * TRY + threadIdx.y;
  if (X >= nxc || Y >= nyc) return;
  const int r = blockIdx.z / nzc, Z = blockIdx.z - r * nzc;
  const cx<R>* F = f + (long long)r * nxf * nyf * nzf;
  cx<R> acc = mkc<R>(0, 0);
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = 2 * Z + dz;
    if (z < 0 || z >= nzf) continue;
    const R wz = dz == 0 ? (R)0.5 : (R)0.25;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = 2 * Y + dy;
      if (y < 0 || y >= nyf) continue;
      const R wzy = wz * (dy == 0 ? (R)0.5 : (R)0.25);
      const cx<R>* row = F + (z * nyf + y) * nxf;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = 2 * X + dx;
        if (x < 0 || x >= nxf) continue;
        acc += (wzy * (dx == 0 ? (R)0.5 : (R)0.25)) * row[x];
      }
    }
  }
  c[(long long)r * nxc * nyc * nzc + (Z * nyc + Y) * nxc + X] = acc;
}

// trilinear interpolation (Eq. prolongation) added to base: f = base + P c
template <class R>
__global__ void __launch_bounds__(TRX * TRY) k_prolong_add(const cx<R>* __restrict__ c, const cx<R>* __restrict__ base,
                                                            cx<R>* __restrict__ f, int nxf, int nyf, int nzf) {
  const int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1, nzc = (nzf - 1) / 2 + 1;
  const int x = blockIdx.x * TRX + threadIdx.x, y = blockIdx.y * TRY + threadIdx.y;
  if (x >= nxf || y >= nyf) return;
  const int r = blockIdx.z / nzf, z = blockIdx.z - r * nzf;
  const cx<R>* C = c + (long long)r * nxc * nyc * nzc;
  // an odd fine index sits halfway between coarse nodes X0 and X0 + 1 (both
  // inside the grid); an even one on X0 (the second term then has weight 0)
  const int X0 = x >> 1, Y0 = y >> 1, Z0 = z >> 1;
  const int ox = x & 1, oy = y & 1, oz = z & 1;
  const R hx = ox ? (R)0.5 : (R)1, hy = oy ? (R)0.5 : (R)1, hz = oz ? (R)0.5 : (R)1;
  const R gx = ox ? (R)0.5 : (R)0, gy = oy ? (R)0.5 : (R)0, gz = oz ? (R)0.5 : (R)0;
  auto row = [&](int Z, int Y) {
    const cx<R>* p = C + (Z * nyc + Y) * nxc + X0;
    return hx * p[0] + gx * p[ox];
  };
  const cx<R> a0 = hy * row(Z0, Y0) + gy * row(Z0, Y0 + oy);
  const cx<R> a1 = hy * row(Z0 + oz, Y0) + gy * row(Z0 + oz, Y0 + oy);
  const cx<R> acc = hz * a0 + gz * a1;
  const long long t = (long long)r * nxf * nyf * nzf + (z * nyf + y) * nxf + x;
  f[t] = base ? base[t] + acc : acc;
}

template <class R>
void launch_restrict(const cx<R>* fine, cx<R>* coarse, int nxf, int nyf, int nzf, int nrhs, cudaStream_t s) {
  const int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1, nzc = (nzf - 1) / 2 + 1;
  const long long Nf = (long long)nxf * nyf * nzf, Nc = (long long)nxc * nyc * nzc;
  const int chunk = std::max(1, 65535 / nzc);  // grid.z limit
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int nr = std::min(chunk, nrhs - r0);
    const dim3 grid((nxc + TRX - 1) / TRX, (nyc + TRY - 1) / TRY, nzc * nr);
    count_launch();
    k_restrict<R><<<grid, dim3(TRX, TRY), 0, s>>>(fine + r0 * Nf, coarse + r0 * Nc, nxf, nyf, nzf);
  }
}
template <class R>
void launch_prolong_add(const cx<R>* coarse, const cx<R>* base, cx<R>* fine, int nxf, int nyf, int nzf, int nrhs,
                        cudaStream_t s) {
  const int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1, nzc = (nzf - 1) / 2 + 1;
  const long long Nf = (long long)nxf * nyf * nzf, Nc = (long long)nxc * nyc * nzc;
  const int chunk = std::max(1, 65535 / nzf);  // grid.z limit
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int nr = std::min(chunk, nrhs - r0);
    const dim3 grid((nxf + TRX - 1) / TRX, (nyf + TRY - 1) / TRY, nzf * nr);
    count_launch();
    k_prolong_add<R><<<grid, dim3(TRX, TRY), 0, s>>>(coarse + r0 * Nc, base ? base + r0 * Nf : nullptr,
                                                      fine + r0 * Nf, nxf, nyf, nzf);
  }
}

// ----------------------------------------------------------------------------
// multi-value grid reduction
//   stage 1 (every block): per-thread sums in R, warp sums in R, the 8 warp
//     results combined in double, written as partial[(v * nrhs + rhs) * nblk + blk];
//   stage 2 (last block to arrive): every thread sums a fixed stride of the
//     blocks for all values, then a block tree in double.  Fixed order: the
//     result does not depend on block scheduling.
// ----------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Double-single sums for the complex64 path: an unevaluated pair hi + lo of
// floats added with the error-free two-sum, so the cross-warp and cross-block
// stages keep about 48 mantissa bits in FP32 arithmetic (the FP64 rate of this
// GPU is a small fraction of its FP32 rate).  The pair occupies the 8 bytes of
// a partial-sum slot.
struct dsf {
  float hi, lo;
};
__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  dsf r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
__device__ __forceinline__ dsf ds_warp_sum(dsf a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dsf b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a = ds_add(a, b);
  }
  return a;
}

template <class R, int NV>
__device__ __forceinline__ void block_partials(const R* acc, double* sm /* [VB/32][NV] */, double* partial, int nrhs,
                                               int rhs, unsigned nblk, unsigned blk, int tid) {
  const int lane = tid & 31, w = tid >> 5;
  float* sf = reinterpret_cast<float*>(sm);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    R x = warp_sum_r<R>(acc[v]);
    if (lane == 0) {
      if constexpr (sizeof(R) == sizeof(float)) sf[w * NV + v] = x;
      else sm[w * NV + v] = (double)x;
    }
  }
  __syncthreads();
  for (int v = tid; v < NV; v += VB) {
    if constexpr (sizeof(R) == sizeof(float)) {
      dsf t{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < VB / 32; ++k) t = ds_add(t, dsf{sf[k * NV + v], 0.f});
      reinterpret_cast<dsf*>(partial)[((size_t)v * nrhs + rhs) * nblk + blk] = t;
    } else {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < VB / 32; ++k) t += sm[k * NV + v];
      partial[((size_t)v * nrhs + rhs) * nblk + blk] = t;
    }
  }
}

// Stage 2; result for value v in out[v] (shared memory), valid after return.
// One warp per value (warp w takes values w, w + 8, ...): its lanes sum a fixed
// stride of the block partials, then a warp tree; no block-wide barrier between
// values and few live accumulators.
constexpr int kCombineChunk = 8;
template <class R, int NV>
__device__ __forceinline__ void combine_partials(const double* partial, int nrhs, int rhs, unsigned nblk,
                                                 double* sm /* unused */, double* out, int tid) {
  (void)sm;
  const int lane = tid & 31, w = tid >> 5;
  __syncthreads();
#pragma unroll 1
  for (int v = w; v < NV; v += VB / 32) {
    if constexpr (sizeof(R) == sizeof(float)) {
      const float2* pp = reinterpret_cast<const float2*>(partial) + ((size_t)v * nrhs + rhs) * nblk;
      dsf a{0.f, 0.f}, b{0.f, 0.f};
      unsigned k = lane;
      for (; k + 32 < nblk; k += 64) {  // two independent chains
        const float2 q0 = __ldcg(pp + k), q1 = __ldcg(pp + k + 32);
        a = ds_add(a, dsf{q0.x, q0.y});
        b = ds_add(b, dsf{q1.x, q1.y});
      }
      if (k < nblk) {
        const float2 q0 = __ldcg(pp + k);
        a = ds_add(a, dsf{q0.x, q0.y});
      }
      const dsf t = ds_warp_sum(ds_add(a, b));
      if (lane == 0) out[v] = (double)t.hi + (double)t.lo;
    } else {
      const double* pp = partial + ((size_t)v * nrhs + rhs) * nblk;
      double a = 0.0, b = 0.0;
      unsigned k = lane;
      for (; k + 32 < nblk; k += 64) {
        a += __ldcg(pp + k);
        b += __ldcg(pp + k + 32);
      }
      if (k < nblk) a += __ldcg(pp + k);
      const double t = warp_sum(a + b);
      if (lane == 0) out[v] = t;
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// classical Gram-Schmidt passes
// ----------------------------------------------------------------------------
struct CgsArgs {
  int n, nrhs, kn, ld;
  long long vstride;
  const double* coef;   // [rhs][ld] complex
  bool update, dots, norm;
  double* dots_out;     // [rhs][ld] complex
  double* nrm_out;      // [rhs]
  int epi;
  double* H;            // per rhs: column-major (ldh x m) complex, ldh = ld
  int col;
  int hcols;            // m (columns per rhs)
  double* scale_out;    // [rhs]
  double* beta_out;     // [rhs]
  Reduce red;
  int* skip;            // see KrylovCall::skip
  double* coef_final;
};

template <class R, int KN>
__global__ void __launch_bounds__(VB) k_cgs(const cx<R>* __restrict__ V, cx<R>* __restrict__ w, CgsArgs a) {
  constexpr int NV = 2 * KN + 1;
  __shared__ double sm[(VB / 32) * (NV > kCombineChunk ? NV : kCombineChunk)];
  __shared__ double sres[NV];
  __shared__ R scoef[2 * KMAX + 2];
  const int tid = threadIdx.x;
  const int rhs = blockIdx.y;
  const long long N = a.n;
  // second Arnoldi pass of a right-hand side whose first pass needed no
  // reorthogonalisation: nothing to do (uniform per block; no block of this
  // rhs arrives at the reduction, whose counter therefore stays at zero)
  if (a.epi == EPI_ARNOLDI_SECOND && a.skip && a.skip[rhs]) return;
  if (a.update && tid < KN) {
    scoef[2 * tid] = (R)a.coef[(size_t)rhs * a.ld * 2 + 2 * tid];
    scoef[2 * tid + 1] = (R)a.coef[(size_t)rhs * a.ld * 2 + 2 * tid + 1];
  }
  __syncthreads();
  R acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0;
  cx<R>* W = w + rhs * N;
  const cx<R>* Vr = V + rhs * N;
  // two elements per iteration, all their loads issued before the arithmetic
  auto body = [&](const cx<R>* v, cx<R> wi, long long i) {
    if (a.update) {
#pragma unroll
      for (int k = 0; k < KN; ++k) wi -= mkc<R>(scoef[2 * k], scoef[2 * k + 1]) * v[k];
      W[i] = wi;
    }
    if (a.dots) {
#pragma unroll
      for (int k = 0; k < KN; ++k) {
        const cx<R> p = cjmul(v[k], wi);
        acc[2 * k] += p.x;
        acc[2 * k + 1] += p.y;
      }
    }
    if (a.norm) acc[2 * KN] += abs2(wi);
  };
  const long long stride = (long long)gridDim.x * VB;
  long long i = blockIdx.x * (long long)VB + tid;
  for (; i + stride < N; i += 2 * stride) {
    cx<R> v0[KN > 0 ? KN : 1], v1[KN > 0 ? KN : 1];
#pragma unroll
    for (int k = 0; k < KN; ++k) {
      v0[k] = Vr[k * a.vstride + i];
      v1[k] = Vr[k * a.vstride + i + stride];
    }
    const cx<R> w0 = W[i], w1 = W[i + stride];
    body(v0, w0, i);
    body(v1, w1, i + stride);
  }
  if (i < N) {
    cx<R> v0[KN > 0 ? KN : 1];
#pragma unroll
    for (int k = 0; k < KN; ++k) v0[k] = Vr[k * a.vstride + i];
    body(v0, W[i], i);
  }
  const unsigned nblk = gridDim.x;
  block_partials<R, NV>(acc, sm, a.red.partial, a.nrhs, rhs, nblk, blockIdx.x, tid);
  if (!last_block_arrive(a.red.count + rhs, nblk, tid)) return;
  combine_partials<R, NV>(a.red.partial, a.nrhs, rhs, nblk, sm, sres, tid);
  if (tid == 0) {
    a.red.count[rhs] = 0;
    double* Hc = a.H ? a.H + ((size_t)rhs * a.hcols + (a.col >= 0 ? a.col : 0)) * a.ld * 2 : nullptr;
    double* dout = a.dots_out ? a.dots_out + (size_t)rhs * a.ld * 2 : nullptr;
    switch (a.epi) {
      case EPI_STORE:
        if (dout)
          for (int k = 0; k < KN; ++k) {
            dout[2 * k] = sres[2 * k];
            dout[2 * k + 1] = sres[2 * k + 1];
          }
        if (a.nrm_out) a.nrm_out[rhs] = sres[2 * KN];
        break;
      case EPI_ARNOLDI_FIRST: {
        double h1sq = 0.0;
        for (int k = 0; k < KN; ++k) {
          Hc[2 * k] = sres[2 * k];
          Hc[2 * k + 1] = sres[2 * k + 1];
          dout[2 * k] = sres[2 * k];
          dout[2 * k + 1] = sres[2 * k + 1];
          h1sq += sres[2 * k] * sres[2 * k] + sres[2 * k + 1] * sres[2 * k + 1];
        }
        if (a.skip) {
          // ||w - V h1||^2 = ||w||^2 - ||h1||^2 (orthonormal V); without severe
          // cancellation (more than half of ||w||^2 left) one pass suffices
          const double w2 = sres[2 * KN], nu2 = w2 - h1sq;
          const bool one_pass = nu2 > 0.5 * w2 && nu2 > 1e-300;
          a.skip[rhs] = one_pass ? 1 : 0;
          if (one_pass) {
            const double nu = sqrt(nu2);
            Hc[2 * KN] = nu;
            Hc[2 * KN + 1] = 0.0;
            a.scale_out[rhs] = 1.0 / nu;
            double* cf = a.coef_final + (size_t)rhs * a.ld * 2;
            for (int k = 0; k < 2 * KN; ++k) cf[k] = sres[k];
          }
        }
        break;
      }
      case EPI_ARNOLDI_SECOND: {
        // second Gram-Schmidt pass: add the correction to the column; the norm
        // of w - V h2 is ||w||^2 - ||h2||^2 for orthonormal V (h2 is tiny)
        double h2sq = 0.0;
        for (int k = 0; k < KN; ++k) {
          Hc[2 * k] += sres[2 * k];
          Hc[2 * k + 1] += sres[2 * k + 1];
          dout[2 * k] = sres[2 * k];
          dout[2 * k + 1] = sres[2 * k + 1];
          h2sq += sres[2 * k] * sres[2 * k] + sres[2 * k + 1] * sres[2 * k + 1];
        }
        if (a.norm) {
          double nrm = sqrt(fmax(sres[2 * KN] - h2sq, 0.0));
          Hc[2 * KN] = nrm;
          Hc[2 * KN + 1] = 0.0;
          // an exactly zero (or denormal) norm ends the Krylov space: the next
          // basis vector is set to zero and the small solve ignores it
          if (a.scale_out) a.scale_out[rhs] = (nrm > 1e-300) ? 1.0 / nrm : 0.0;
        }
        break;
      }
      case EPI_NORMALISE: {
        double nrm = sqrt(sres[2 * KN]);
        if (a.col >= 0) {
          Hc[2 * KN] = nrm;
          Hc[2 * KN + 1] = 0.0;
        }
        if (a.beta_out) a.beta_out[rhs] = nrm;
        if (a.scale_out) a.scale_out[rhs] = (nrm > 1e-300) ? 1.0 / nrm : 0.0;
        break;
      }
    }
  }
}

// w <- (w - sum_k coef[r][k] V_k) * scale[r]  (third Gram-Schmidt pass fused with
// the normalisation; no reduction)
template <class R, int KN>
__global__ void __launch_bounds__(VB) k_update_scale(const cx<R>* __restrict__ V, cx<R>* __restrict__ w,
                                                     const double* __restrict__ coef, const double* __restrict__ scale,
                                                     int n, long long vstride, int ld) {
  __shared__ R scoef[2 * KMAX + 2];
  const int rhs = blockIdx.y;
  if (threadIdx.x < 2 * KN) scoef[threadIdx.x] = (R)coef[(size_t)rhs * ld * 2 + threadIdx.x];
  __syncthreads();
  const R sc = (R)scale[rhs];
  cx<R>* W = w + (long long)rhs * n;
  const cx<R>* Vr = V + (long long)rhs * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cx<R> wi = W[i];
#pragma unroll
    for (int k = 0; k < KN; ++k) wi -= mkc<R>(scoef[2 * k], scoef[2 * k + 1]) * Vr[k * vstride + i];
    W[i] = sc * wi;
  }
}

template <class R, int KN>
static void cgs_kn(const KrylovCall& k, const cx<R>* V, cx<R>* w, const CgsArgs& a, cudaStream_t s) {
  dim3 grid(red_blocks(k.n), k.nrhs);
  count_launch();
  k_cgs<R, KN><<<grid, VB, 0, s>>>(V, w, a);
}

template <class R>
void launch_cgs(const KrylovCall& k, const cx<R>* V, cx<R>* w, const double* coef, bool update, bool dots,
                bool norm, double* dots_out, double* nrm_out, int epi, double* H, int col, double* scale_out,
                double* beta_out, const Reduce& red, cudaStream_t s) {
  CgsArgs a;
  a.n = k.n;
  a.nrhs = k.nrhs;
  a.kn = k.kn;
  a.ld = k.ld;
  a.vstride = k.vstride;
  a.coef = coef;
  a.update = update;
  a.dots = dots;
  a.norm = norm;
  a.dots_out = dots_out;
  a.nrm_out = nrm_out;
  a.epi = epi;
  a.H = H;
  a.col = col;
  a.hcols = k.ld - 1;
  a.scale_out = scale_out;
  a.beta_out = beta_out;
  a.red = red;
  a.skip = k.skip;
  a.coef_final = k.coef_final;
  switch (k.kn) {
#define HZ_KN(K) \
  case K: cgs_kn<R, K>(k, V, w, a, s); break;
    HZ_KN(0) HZ_KN(1) HZ_KN(2) HZ_KN(3) HZ_KN(4) HZ_KN(5) HZ_KN(6) HZ_KN(7) HZ_KN(8) HZ_KN(9) HZ_KN(10) HZ_KN(11)
    HZ_KN(12) HZ_KN(13) HZ_KN(14) HZ_KN(15) HZ_KN(16)
#undef HZ_KN
    default: break;
  }
}

template <class R>
void launch_update_scale(const KrylovCall& k, const cx<R>* V, cx<R>* w, const double* coef, const double* scale,
                         cudaStream_t s) {
  dim3 grid(vec_blocks(k.n), k.nrhs);
  switch (k.kn) {
#define HZ_KN(K)                                                                               \
  case K:                                                                                      \
    count_launch();                                                                            \
    k_update_scale<R, K><<<grid, VB, 0, s>>>(V, w, coef, scale, k.n, k.vstride, k.ld); \
    break;
    HZ_KN(1) HZ_KN(2) HZ_KN(3) HZ_KN(4) HZ_KN(5) HZ_KN(6) HZ_KN(7) HZ_KN(8) HZ_KN(9) HZ_KN(10) HZ_KN(11)
    HZ_KN(12) HZ_KN(13) HZ_KN(14) HZ_KN(15) HZ_KN(16)
#undef HZ_KN
    default: break;
  }
}

template <class R>
void launch_norm2(const cx<R>* v, int n, int nrhs, const Reduce& red, cudaStream_t s) {
  KrylovCall k;
  k.n = n;
  k.nrhs = nrhs;
  k.kn = 0;
  k.ld = 1;
  launch_cgs<R>(k, v, const_cast<cx<R>*>(v), nullptr, false, false, true, nullptr, red.out, EPI_STORE, nullptr, -1,
                nullptr, nullptr, red, s);
}

// ----------------------------------------------------------------------------
// scale / combine / axpy / copy
// ----------------------------------------------------------------------------
template <class R>
__global__ void k_scale(const cx<R>* __restrict__ w, cx<R>* __restrict__ out, const double* __restrict__ scale, int n,
                        int nrhs) {
  const int rhs = blockIdx.y;
  const R sc = (R)scale[rhs];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[(long long)rhs * n + i] = sc * w[(long long)rhs * n + i];
}
template <class R>
void launch_scale(const cx<R>* w, cx<R>* out, const double* scale, int n, int nrhs, cudaStream_t s) {
  count_launch();
  k_scale<R><<<dim3(vec_blocks(n), nrhs), VB, 0, s>>>(w, out, scale, n, nrhs);
}

// x = x0 + sum_k y_k Z_k (x0 may be null); the basis size is a template
// argument so that the loads of all terms are in flight together.
template <class R, int KN>
__global__ void k_combine(const cx<R>* __restrict__ Z, long long zstride, const double* __restrict__ y, int ld,
                          const cx<R>* __restrict__ x0, cx<R>* __restrict__ x, int n) {
  __shared__ R sy[2 * KMAX];
  const int rhs = blockIdx.y;
  if (threadIdx.x < 2 * KN) sy[threadIdx.x] = (R)y[(size_t)rhs * ld * 2 + threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)rhs * n + i;
    cx<R> acc = x0 ? x0[o] : mkc<R>(0, 0);
#pragma unroll
    for (int k = 0; k < KN; ++k) acc += mkc<R>(sy[2 * k], sy[2 * k + 1]) * Z[k * zstride + o];
    x[o] = acc;
  }
}
template <class R>
void launch_combine(const cx<R>* Z, long long zstride, int kn, const double* y, int ld, const cx<R>* x0, cx<R>* x,
                    int n, int nrhs, cudaStream_t s) {
  const dim3 grid(vec_blocks(n), nrhs);
  switch (kn) {
#define HZ_KN(K)                                                             \
  case K:                                                                    \
    count_launch();                                                          \
    k_combine<R, K><<<grid, VB, 0, s>>>(Z, zstride, y, ld, x0, x, n); \
    break;
    HZ_KN(1) HZ_KN(2) HZ_KN(3) HZ_KN(4) HZ_KN(5) HZ_KN(6) HZ_KN(7) HZ_KN(8) HZ_KN(9) HZ_KN(10) HZ_KN(11)
    HZ_KN(12) HZ_KN(13) HZ_KN(14) HZ_KN(15) HZ_KN(16)
#undef HZ_KN
    default: break;
  }
}

template <class R>
__global__ void k_axpy(const cx<R>* __restrict__ x, cx<R>* __restrict__ y, R ar, R ai, long long n) {
  const cx<R> a = mkc<R>(ar, ai);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
template <class R>
void launch_axpy(const cx<R>* x, cx<R>* y, double ar, double ai, long long n, cudaStream_t s) {
  count_launch();
  k_axpy<R><<<vec_blocks(n), VB, 0, s>>>(x, y, (R)ar, (R)ai, n);
}
template <class R>
__global__ void k_copy(const cx<R>* __restrict__ x, cx<R>* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}
template <class R>
void launch_copy(const cx<R>* x, cx<R>* y, long long n, cudaStream_t s) {
  count_launch();
  k_copy<R><<<vec_blocks(n), VB, 0, s>>>(x, y, n);
}
template <class R>
__global__ void k_zero(cx<R>* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = mkc<R>(0, 0);
}
template <class R>
void launch_zero(cx<R>* y, long long n, cudaStream_t s) {
  count_launch();
  k_zero<R><<<vec_blocks(n), VB, 0, s>>>(y, n);
}

__global__ void k_c128_to_c64(const cx<double>* __restrict__ in, cx<float>* __restrict__ out,
                              const double* __restrict__ scale, int n) {
  const int rhs = blockIdx.y;
  const double sc = scale ? scale[rhs] : 1.0;  // null: plain narrowing
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cx<double> v = in[(long long)rhs * n + i];
    out[(long long)rhs * n + i] = mkc<float>((float)(v.x * sc), (float)(v.y * sc));
  }
}
void launch_c128_to_c64_scaled(const cx<double>* in, cx<float>* out, const double* scale, int n, int nrhs,
                               cudaStream_t s) {
  count_launch();
  k_c128_to_c64<<<dim3(vec_blocks(n), nrhs), VB, 0, s>>>(in, out, scale, n);
}
__global__ void k_add_c64_to_c128(const cx<float>* __restrict__ d, cx<double>* __restrict__ x,
                                  const double* __restrict__ scale, int n, bool accumulate) {
  const int rhs = blockIdx.y;
  const double sc = scale ? scale[rhs] : 1.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cx<float> v = d[(long long)rhs * n + i];
    cx<double>& t = x[(long long)rhs * n + i];
    if (accumulate) {
      t.x += sc * (double)v.x;
      t.y += sc * (double)v.y;
    } else {
      t = mkc<double>(sc * (double)v.x, sc * (double)v.y);
    }
  }
}
void launch_add_c64_to_c128_scaled(const cx<float>* d, cx<double>* x, const double* scale, int n, int nrhs,
                                   cudaStream_t s) {
  count_launch();
  k_add_c64_to_c128<<<dim3(vec_blocks(n), nrhs), VB, 0, s>>>(d, x, scale, n, true);
}
void launch_c64_to_c128(const cx<float>* d, cx<double>* x, int n, int nrhs, cudaStream_t s) {
  count_launch();
  k_add_c64_to_c128<<<dim3(vec_blocks(n), nrhs), VB, 0, s>>>(d, x, nullptr, n, false);
}

// ----------------------------------------------------------------------------
// small least squares by complex Givens rotations (one thread per rhs)
// ----------------------------------------------------------------------------
// Warp-parallel Givens least squares min || beta e_1 - H y || for one (M+1) x M
// upper Hessenberg H per right-hand side (one warp each): lane k holds column
// k in registers; rotation j is formed by lane j and broadcast; the back
// substitution sums R[i][k] y_k across lanes.  T = float for the complex64
// hierarchy, double for complex128.
template <class T, int M>
__global__ void __launch_bounds__(32) k_lsq_warp(const double* __restrict__ H, const double* __restrict__ beta,
                                                 double* __restrict__ y, int ld) {
  const int r = blockIdx.x;
  const int lane = threadIdx.x;
  const double* Hr = H + (size_t)r * M * (M + 1) * 2;
  T cr[M + 1], ci[M + 1];  // column `lane`
#pragma unroll
  for (int i = 0; i <= M; ++i) {
    cr[i] = lane < M ? (T)Hr[(lane * (M + 1) + i) * 2] : (T)0;
    ci[i] = lane < M ? (T)Hr[(lane * (M + 1) + i) * 2 + 1] : (T)0;
  }
  T gr[M + 1], gi[M + 1];
#pragma unroll
  for (int i = 0; i <= M; ++i) gr[i] = gi[i] = (T)0;
  gr[0] = (T)beta[r];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    // lane j forms the rotation that zeroes its subdiagonal entry
    T c = 1, sr = 0, si = 0;
    if (lane == j) {
      const T ar = cr[j], ai = ci[j], br = cr[j + 1], bi = ci[j + 1];
      const T na = sqrt(ar * ar + ai * ai), nb = sqrt(br * br + bi * bi);
      const T rr = sqrt(na * na + nb * nb);
      if (rr == (T)0) {
        c = 1; sr = 0; si = 0;
      } else if (na == (T)0) {
        c = 0; sr = 1; si = 0;
      } else {
        c = na / rr;
        // s = (a / |a|) conj(b) / r
        const T ur = ar / na, ui = ai / na;
        sr = (ur * br + ui * bi) / rr;
        si = (ui * br - ur * bi) / rr;
      }
    }
    c = __shfl_sync(0xffffffffu, c, j);
    sr = __shfl_sync(0xffffffffu, sr, j);
    si = __shfl_sync(0xffffffffu, si, j);
    if (lane >= j && lane < M) {
      const T t1r = cr[j], t1i = ci[j], t2r = cr[j + 1], t2i = ci[j + 1];
      // [c s; -conj(s) c] [t1; t2]
      cr[j] = c * t1r + (sr * t2r - si * t2i);
      ci[j] = c * t1i + (sr * t2i + si * t2r);
      cr[j + 1] = c * t2r - (sr * t1r + si * t1i);
      ci[j + 1] = c * t2i - (sr * t1i - si * t1r);
    }
    const T g1r = gr[j], g1i = gi[j], g2r = gr[j + 1], g2i = gi[j + 1];
    gr[j] = c * g1r + (sr * g2r - si * g2i);
    gi[j] = c * g1i + (sr * g2i + si * g2r);
    gr[j + 1] = c * g2r - (sr * g1r + si * g1i);
    gi[j + 1] = c * g2i - (sr * g1i - si * g1r);
  }
  // back substitution: y_i = (g_i - sum_{k>i} R[i][k] y_k) / R[i][i]
  T yr = 0, yi = 0;  // y_lane
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
    T pr = 0, pi = 0;
    if (lane > i && lane < M) {
      pr = cr[i] * yr - ci[i] * yi;
      pi = cr[i] * yi + ci[i] * yr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pr += __shfl_xor_sync(0xffffffffu, pr, o);
      pi += __shfl_xor_sync(0xffffffffu, pi, o);
    }
    if (lane == i) {
      const T tr = gr[i] - pr, ti = gi[i] - pi;
      const T dr = cr[i], di = ci[i];
      const T d2 = dr * dr + di * di;
      if (d2 > (T)0) {
        yr = (tr * dr + ti * di) / d2;
        yi = (ti * dr - tr * di) / d2;
      } else {
        yr = yi = 0;
      }
    }
  }
  if (lane < M) {
    y[((size_t)r * ld + lane) * 2] = (double)yr;
    y[((size_t)r * ld + lane) * 2 + 1] = (double)yi;
  }
}

template <class T>
static void lsq_t(const double* H, const double* beta, double* y, int m, int ld, int nrhs, cudaStream_t s) {
  switch (m) {
#define HZ_M(MM)                                                   \
  case MM:                                                         \
    count_launch();                                                \
    k_lsq_warp<T, MM><<<nrhs, 32, 0, s>>>(H, beta, y, ld); \
    break;
    HZ_M(1) HZ_M(2) HZ_M(3) HZ_M(4) HZ_M(5) HZ_M(6) HZ_M(7) HZ_M(8) HZ_M(9) HZ_M(10) HZ_M(11) HZ_M(12) HZ_M(13)
    HZ_M(14) HZ_M(15) HZ_M(16)
#undef HZ_M
    default: break;
  }
}

void launch_lsq(const double* H, const double* beta, double* y, int m, int ld, int nrhs, cudaStream_t s,
                bool single) {
  if (single) lsq_t<float>(H, beta, y, m, ld, nrhs, s);
  else lsq_t<double>(H, beta, y, m, ld, nrhs, s);
}

// ----------------------------------------------------------------------------
// CA-GMRES bottom solve: Gram matrix of [p_0 .. p_s], CholQR, least squares
// ----------------------------------------------------------------------------
// The small Cholesky solve runs in one thread of the last block only: the
// register cap (4 blocks per SM for the usual s = 4) sizes the streaming loop,
// and whatever the solve does not fit in registers goes to local memory.
template <class R, int KN>
__global__ void __launch_bounds__(VB) k_gram(const cx<R>* __restrict__ P, long long pstride, int n,
                                                             double* y, int ld, Reduce red) {
  constexpr int NG = KN * (KN + 1) / 2;
  constexpr int NV = 2 * NG;
  constexpr int S = KN - 1;
  __shared__ double sm[(VB / 32) * (NV > kCombineChunk ? NV : kCombineChunk)];
  __shared__ double sres[NV];
  const int tid = threadIdx.x, rhs = blockIdx.y, nrhs = gridDim.y;
  R acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0;
  const cx<R>* Pr = P + (long long)rhs * n;
  for (long long i = blockIdx.x * (long long)VB + tid; i < n; i += (long long)gridDim.x * VB) {
    cx<R> p[KN];
#pragma unroll
    for (int k = 0; k < KN; ++k) p[k] = Pr[k * pstride + i];
    int q = 0;
#pragma unroll
    for (int a = 0; a < KN; ++a)
#pragma unroll
      for (int b = a; b < KN; ++b) {
        cx<R> t = cjmul(p[a], p[b]);
        acc[2 * q] += t.x;
        acc[2 * q + 1] += t.y;
        ++q;
      }
  }
  const unsigned nblk = gridDim.x;
  block_partials<R, NV>(acc, sm, red.partial, nrhs, rhs, nblk, blockIdx.x, tid);
  if (!last_block_arrive(red.count + rhs, nblk, tid)) return;
  combine_partials<R, NV>(red.partial, nrhs, rhs, nblk, sm, sres, tid);
  if (tid != 0) return;
  red.count[rhs] = 0;
  gram_lsq_solve<KN>(sres, y + (size_t)rhs * ld * 2);
}

template <class R>
void launch_gram_lsq(const cx<R>* P, long long pstride, int kn, int n, int nrhs, double* y, int ld,
                     const Reduce& red, cudaStream_t s) {
  dim3 grid(red_blocks(n), nrhs);
  switch (kn) {
    case 2: count_launch();
      k_gram<R, 2><<<grid, VB, 0, s>>>(P, pstride, n, y, ld, red); break;
    case 3: count_launch();
      k_gram<R, 3><<<grid, VB, 0, s>>>(P, pstride, n, y, ld, red); break;
    case 4: count_launch();
      k_gram<R, 4><<<grid, VB, 0, s>>>(P, pstride, n, y, ld, red); break;
    case 5: count_launch();
      k_gram<R, 5><<<grid, VB, 0, s>>>(P, pstride, n, y, ld, red); break;
    case 6: count_launch();
      k_gram<R, 6><<<grid, VB, 0, s>>>(P, pstride, n, y, ld, red); break;
    case 7: count_launch();
      k_gram<R, 7><<<grid, VB, 0, s>>>(P, pstride, n, y, ld, red); break;
    default: break;
  }
}

// ----------------------------------------------------------------------------
// set-up, sources, receivers
// ----------------------------------------------------------------------------
template <class R>
__global__ void k_setup_kappa(const double* __restrict__ c, int nxf, int nyf, int nzf, int n_pml, int stride,
                              double omega, double ell, R* __restrict__ kappa) {
  const int nx = (nxf - 1) / stride + 1, ny = (nyf - 1) / stride + 1, nz = (nzf - 1) / stride + 1;
  const long long N = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int X = (int)(i % nx), Y = (int)((i / nx) % ny), Z = (int)(i / ((long long)nx * ny));
    int fx = min(max(X * stride, n_pml), nxf - 1 - n_pml);
    int fy = min(max(Y * stride, n_pml), nyf - 1 - n_pml);
    int fz = min(max(Z * stride, n_pml), nzf - 1 - n_pml);
    double cv = c[((long long)fz * nyf + fy) * nxf + fx];
    kappa[i] = (R)(omega * ell / cv);
  }
}
template <class R>
void launch_setup_kappa(const double* c, int nxf, int nyf, int nzf, int n_pml, int stride, double omega,
                        double ell, R* kappa, cudaStream_t s) {
  long long n = (long long)((nxf - 1) / stride + 1) * ((nyf - 1) / stride + 1) * ((nzf - 1) / stride + 1);
  count_launch();
  k_setup_kappa<R><<<vec_blocks(n), VB, 0, s>>>(c, nxf, nyf, nzf, n_pml, stride, omega, ell, kappa);
}

template <class R>
__global__ void k_point_sources(const int* idx3, const double* amp, int nsrc, int nx, int ny, int nz, double scale,
                                cx<R>* f) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsrc) return;
  long long N = (long long)nx * ny * nz;
  int ix = idx3[3 * s], iy = idx3[3 * s + 1], iz = idx3[3 * s + 2];
  long long i = ((long long)iz * ny + iy) * nx + ix;
  f[(long long)s * N + i] = mkc<R>((R)(amp[2 * s] * scale), (R)(amp[2 * s + 1] * scale));
}
template <class R>
void launch_point_sources(const int* idx3, const double* amp, int nsrc, int nx, int ny, int nz, double scale,
                          cx<R>* f, cudaStream_t s) {
  count_launch();
  k_point_sources<R><<<(nsrc + 63) / 64, 64, 0, s>>>(idx3, amp, nsrc, nx, ny, nz, scale, f);
}

// b = Q_h f for one point source per right-hand side, f = amp h^-3 e_{i_s}
// (Eq. point-source): row j of Q_h (shell weights of its own eta*, Eq.
// q-operator) meets the source at offset i_s - j, so b is nonzero only on the
// in-grid nodes of the 3x3x3 block around i_s.  b must be zero on entry.
__global__ void k_source_rows(LevelView<double> L, TableView<double> T, const int* __restrict__ idx3,
                              const double* __restrict__ amp, int nsrc, double scale, cx<double>* __restrict__ b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27 * nsrc) return;
  const int s = t / 27, d = t - 27 * s;
  const int dz = d / 9 - 1, dy = (d / 3) % 3 - 1, dx = d % 3 - 1;
  const int x = idx3[3 * s] + dx, y = idx3[3 * s + 1] + dy, z = idx3[3 * s + 2] + dz;
  if (x < 0 || x >= L.nx || y < 0 || y >= L.ny || z < 0 || z >= L.nz) return;
  const long long j = ((long long)z * L.ny + y) * L.nx + x;
  double bt[3];
  table_eval<double, 5, 3>(T.coef, T.nseg, T.ds, T.inv_ds, eta_star(L.kappa[j]), bt);
  const int m = abs(dx) + abs(dy) + abs(dz);
  const double w = m == 0 ? bt[0] : m == 1 ? bt[1] / 6.0 : m == 2 ? bt[2] / 12.0 : (1.0 - bt[0] - bt[1] - bt[2]) / 8.0;
  b[(long long)s * L.N + j] = mkc<double>(w * amp[2 * s] * scale, w * amp[2 * s + 1] * scale);
}
void launch_source_rows(const LevelView<double>& lv, const TableView<double>& tab, const int* idx3,
                        const double* amp, int nsrc, double scale, cx<double>* b, cudaStream_t s) {
  count_launch();
  k_source_rows<<<(27 * nsrc + 127) / 128, 128, 0, s>>>(lv, tab, idx3, amp, nsrc, scale, b);
}

template <class R>
__global__ void k_gather(const cx<R>* u, const int* rec, int nrec, int n, int nrhs, cx<double>* out) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nrec * nrhs) return;
  int r = (int)(t / nrec), q = (int)(t % nrec);
  out[t] = cvt<double>(u[(long long)r * n + rec[q]]);
}
template <class R>
void launch_gather(const cx<R>* u, const int* rec, int nrec, int n, int nrhs, cx<double>* out, cudaStream_t s) {
  long long t = (long long)nrec * nrhs;
  count_launch();
  k_gather<R><<<(int)((t + 255) / 256), 256, 0, s>>>(u, rec, nrec, n, nrhs, out);
}
// receivers are distinct nodes, so the scatter has no write conflicts
template <class R>
__global__ void k_scatter(const cx<double>* vals, const int* rec, int nrec, int n, int nrhs, cx<R>* out) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nrec * nrhs) return;
  int r = (int)(t / nrec), q = (int)(t % nrec);
  out[(long long)r * n + rec[q]] = cvt<R>(vals[t]);
}
template <class R>
void launch_scatter(const cx<double>* vals, const int* rec, int nrec, int n, int nrhs, cx<R>* out, cudaStream_t s) {
  long long t = (long long)nrec * nrhs;
  count_launch();
  k_scatter<R><<<(int)((t + 255) / 256), 256, 0, s>>>(vals, rec, nrec, n, nrhs, out);
}

// ----------------------------------------------------------------------------
// explicit instantiations
// ----------------------------------------------------------------------------
#define HZ_INST(R)                                                                                                   \
  template void launch_restrict<R>(const cx<R>*, cx<R>*, int, int, int, int, cudaStream_t);                        \
  template void launch_prolong_add<R>(const cx<R>*, const cx<R>*, cx<R>*, int, int, int, int, cudaStream_t);       \
  template void launch_cgs<R>(const KrylovCall&, const cx<R>*, cx<R>*, const double*, bool, bool, bool, double*,   \
                              double*, int, double*, int, double*, double*, const Reduce&, cudaStream_t);          \
  template void launch_norm2<R>(const cx<R>*, int, int, const Reduce&, cudaStream_t);                              \
  template void launch_update_scale<R>(const KrylovCall&, const cx<R>*, cx<R>*, const double*, const double*,       \
                                       cudaStream_t);                              \
  template void launch_scale<R>(const cx<R>*, cx<R>*, const double*, int, int, cudaStream_t);                      \
  template void launch_combine<R>(const cx<R>*, long long, int, const double*, int, const cx<R>*, cx<R>*, int, int, \
                                  cudaStream_t);                                                                   \
  template void launch_gram_lsq<R>(const cx<R>*, long long, int, int, int, double*, int, const Reduce&,             \
                                   cudaStream_t);                                                                  \
  template void launch_axpy<R>(const cx<R>*, cx<R>*, double, double, long long, cudaStream_t);                     \
  template void launch_copy<R>(const cx<R>*, cx<R>*, long long, cudaStream_t);                                     \
  template void launch_zero<R>(cx<R>*, long long, cudaStream_t);                                                   \
  template void launch_setup_kappa<R>(const double*, int, int, int, int, int, double, double, R*, cudaStream_t);    \
  template void launch_point_sources<R>(const int*, const double*, int, int, int, int, double, cx<R>*,              \
                                        cudaStream_t);                                                             \
  template void launch_gather<R>(const cx<R>*, const int*, int, int, int, cx<double>*, cudaStream_t);               \
  template void launch_scatter<R>(const cx<double>*, const int*, int, int, int, cx<R>*, cudaStream_t);
HZ_INST(float)
HZ_INST(double)
#undef HZ_INST

}  // namespace hz

// ----------------------------------------------------------------------------
// adjoint-state gradient, PML fold, shell coefficients (double precision)
// ----------------------------------------------------------------------------
namespace hz {

__global__ void k_gradient(LevelView<double> L, TableView<double> T, double omega_h, const cx<double>* __restrict__ v,
                           const cx<double>* __restrict__ lam, const cx<double>* __restrict__ f,
                           const cx<double>* __restrict__ rr, int nrhs, double* __restrict__ g) {
  const long long N = L.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx), y = (int)((i / L.nx) % L.ny), z = (int)(i / ((long long)L.nx * L.ny));
    const double kap = L.kappa[i];
    const double eta_raw = kap * kInv2Pi;
    const double eta = eta_raw < kEtaMax ? eta_raw : kEtaMax;
    // d eta / d m with kappa^2 = (omega h)^2 m; zero where the clamp is active
    const double deta = eta_raw < kEtaMax ? (omega_h * omega_h) / (4.0 * 3.14159265358979323846 * kap) : 0.0;
    double av[5], dav[5], bv[3], dbv[3];
    table_eval_d<double, 0, 5>(T.coef, T.nseg, T.ds, T.inv_ds, eta, av, dav);
    table_eval_d<double, 5, 3>(T.coef, T.nseg, T.ds, T.inv_ds, eta, bv, dbv);
    for (int j = 0; j < 5; ++j) dav[j] *= deta;
    for (int j = 0; j < 3; ++j) dbv[j] *= deta;
    const double dt[3] = {dav[3], dav[4] * 0.25, -(dav[3] + dav[4]) * 0.25};
    const double w[4] = {av[0], av[1] / 6.0, av[2] / 12.0, (1.0 - av[0] - av[1] - av[2]) * 0.125};
    const double dw[4] = {dav[0], dav[1] / 6.0, dav[2] / 12.0, -(dav[0] + dav[1] + dav[2]) * 0.125};
    const double dq[4] = {dbv[0], dbv[1] / 6.0, dbv[2] / 12.0, -(dbv[0] + dbv[1] + dbv[2]) * 0.125};
    const double dk2 = omega_h * omega_h;  // d kappa^2 / d m
    const cx<double> ab[3] = {L.abar[0][x], L.abar[1][y], L.abar[2][z]};
    const cx<double> ac[3] = {L.achk[0][x], L.achk[1][y], L.achk[2][z]};
    double acc = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      cx<double> dAv = mkc(0.0, 0.0), dQv = mkc(0.0, 0.0), dQf = mkc(0.0, 0.0);
      for (int dz = -1; dz <= 1; ++dz) {
        const int qz = z + dz;
        if (qz < 0 || qz >= L.nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          const int qy = y + dy;
          if (qy < 0 || qy >= L.ny) continue;
          for (int dx = -1; dx <= 1; ++dx) {
            const int qx = x + dx;
            if (qx < 0 || qx >= L.nx) continue;
            const long long j = (long long)r * N + ((long long)qz * L.ny + qy) * L.nx + qx;
            const int d[3] = {dx, dy, dz};
            cx<double> st = mkc(0.0, 0.0);
            for (int a = 0; a < 3; ++a) {
              const int cls = (d[(a + 1) % 3] != 0) + (d[(a + 2) % 3] != 0);
              const cx<double> dd = d[a] == 0 ? -2.0 * ab[a] : (d[a] > 0 ? ab[a] + ac[a] : ab[a] - ac[a]);
              st += dt[cls] * dd;
            }
            const int sh = (dx != 0) + (dy != 0) + (dz != 0);
            const cx<double> dA = (-L.inv_ell2) * st - mkc(L.inv_ell2 * (dk2 * w[sh] + kap * kap * dw[sh]), 0.0);
            const cx<double> vj = v[j];
            dAv += dA * vj;
            dQv += dq[sh] * vj;
            dQf += dq[sh] * f[j];
          }
        }
      }
      const long long o = (long long)r * N + i;
      const cx<double> t1 = cjmul(lam[o], dQf - dAv);
      const cx<double> t2 = cjmul(rr[o], dQv);
      acc += t1.x + t2.x;
    }
    g[i] += acc;
  }
}

void launch_gradient(const LevelView<double>& lv, const TableView<double>& tab, double omega_h,
                     const cx<double>* v, const cx<double>* lam, const cx<double>* f, const cx<double>* rres,
                     int nrhs, double* g_ext, cudaStream_t s) {
  count_launch();
  k_gradient<<<vec_blocks(lv.N), VB, 0, s>>>(lv, tab, omega_h, v, lam, f, rres, nrhs, g_ext);
}

__global__ void k_fold_pml(const double* __restrict__ ge, double* __restrict__ g, int nx, int ny, int nz, int p) {
  const long long N = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    const int lo = p, hx = nx - 1 - p, hy = ny - 1 - p, hz = nz - 1 - p;
    if (x < lo || x > hx || y < lo || y > hy || z < lo || z > hz) {
      g[i] = 0.0;
      continue;
    }
    const int x0 = x == lo ? 0 : x, x1 = x == hx ? nx - 1 : x;
    const int y0 = y == lo ? 0 : y, y1 = y == hy ? ny - 1 : y;
    const int z0 = z == lo ? 0 : z, z1 = z == hz ? nz - 1 : z;
    double acc = 0.0;
    for (int c = z0; c <= z1; ++c)
      for (int b = y0; b <= y1; ++b)
        for (int a = x0; a <= x1; ++a) acc += ge[((long long)c * ny + b) * nx + a];
    g[i] = acc;
  }
}
void launch_fold_pml(const double* g_ext, double* g, int nx, int ny, int nz, int n_pml, cudaStream_t s) {
  count_launch();
  k_fold_pml<<<vec_blocks((long long)nx * ny * nz), VB, 0, s>>>(g_ext, g, nx, ny, nz, n_pml);
}

__global__ void k_shell_coeffs(LevelView<double> L, TableView<double> T, double* out) {
  const long long N = L.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double kap = L.kappa[i];
    double a[5];
    table_eval<double, 0, 5>(T.coef, T.nseg, T.ds, T.inv_ds, eta_star(kap), a);
    const double k2 = kap * kap;
    out[i] = 6.0 * a[3] - k2 * a[0];
    out[N + i] = -a[3] + a[4] - k2 * a[1] / 6.0;
    out[2 * N + i] = -a[4] / 2.0 + (1.0 - a[3] - a[4]) / 2.0 - k2 * a[2] / 12.0;
    out[3 * N + i] = -0.75 * (1.0 - a[3] - a[4]) - k2 * (1.0 - a[0] - a[1] - a[2]) / 8.0;
  }
}
void launch_shell_coeffs(const LevelView<double>& lv, const TableView<double>& tab, double* out, cudaStream_t s) {
  count_launch();
  k_shell_coeffs<<<vec_blocks(lv.N), VB, 0, s>>>(lv, tab, out);
}

}  // namespace hz

namespace hz {

template <class R>
__global__ void k_setup_dinv(LevelView<R> L, TableView<R> T, cx<R> shift, cx<R>* __restrict__ out) {
  const long long N = L.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx), y = (int)((i / L.nx) % L.ny), z = (int)(i / ((long long)L.nx * L.ny));
    const R kap = L.kappa[i];
    R av[5];
    table_eval<R, 0, 5>(T.coef, T.nseg, T.ds, T.inv_ds, eta_star(kap), av);
    const cx<R> sab = L.abar[0][x] + L.abar[1][y] + L.abar[2][z];
    const cx<R> D = L.inv_ell2 * ((R)2 * av[3] * sab) - (L.inv_ell2 * kap * kap * av[0]) * shift;
    out[i] = cinv(D);
  }
}

template <class R>
void launch_setup_dinv(const LevelView<R>& lv, const TableView<R>& tab, cx<R> shift, cx<R>* out, cudaStream_t s) {
  count_launch();
  k_setup_dinv<R><<<vec_blocks(lv.N), VB, 0, s>>>(lv, tab, shift, out);
}
template void launch_setup_dinv<float>(const LevelView<float>&, const TableView<float>&, cx<float>, cx<float>*,
                                       cudaStream_t);
template void launch_setup_dinv<double>(const LevelView<double>&, const TableView<double>&, cx<double>, cx<double>*,
                                        cudaStream_t);

}  // namespace hz
