// Shared device-side definitions of the GB300 three-grid IOFD Helmholtz library.
//
// Grid fields are stored x-fastest, [rhs][z][y][x], complex interleaved
// (re, im).  Nodes outside 0..n carry u = 0 (paper Eq. helmholtz-pml).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hz {

// ----------------------------------------------------------------------------
// complex arithmetic on an aligned pair (8 B for float, 16 B for double)
// ----------------------------------------------------------------------------
template <class R>
struct __align__(2 * sizeof(R)) cx {
  R x, y;
};

template <class R> __host__ __device__ __forceinline__ cx<R> mkc(R a, R b) { cx<R> r; r.x = a; r.y = b; return r; }
template <class R> __host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mkc<R>(a.x + b.x, a.y + b.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mkc<R>(a.x - b.x, a.y - b.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a) { return mkc<R>(-a.x, -a.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mkc<R>(s * a.x, s * a.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mkc<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R> __host__ __device__ __forceinline__ cx<R>& operator+=(cx<R>& a, cx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <class R> __host__ __device__ __forceinline__ cx<R>& operator-=(cx<R>& a, cx<R> b) { a.x -= b.x; a.y -= b.y; return a; }
template <class R> __host__ __device__ __forceinline__ cx<R> conjc(cx<R> a) { return mkc<R>(a.x, -a.y); }
// conj(a) * b
template <class R> __host__ __device__ __forceinline__ cx<R> cjmul(cx<R> a, cx<R> b) {
  return mkc<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// 1/d: a correctly rounded reciprocal instead of an IEEE division in single precision
__host__ __device__ __forceinline__ float recip(float d) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(d);
#else
  return 1.0f / d;
#endif
}
__host__ __device__ __forceinline__ double recip(double d) { return 1.0 / d; }
template <class R> __host__ __device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) {
  const R r = recip(b.x * b.x + b.y * b.y);
  return mkc<R>((a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r);
}
template <class R> __host__ __device__ __forceinline__ cx<R> cinv(cx<R> b) {
  const R r = recip(b.x * b.x + b.y * b.y);
  return mkc<R>(b.x * r, -b.y * r);
}
template <class R> __host__ __device__ __forceinline__ R abs2(cx<R> a) { return a.x * a.x + a.y * a.y; }
template <class R, class S> __host__ __device__ __forceinline__ cx<R> cvt(cx<S> a) { return mkc<R>((R)a.x, (R)a.y); }

// ----------------------------------------------------------------------------
// IOFD coefficient functions: cubic Hermite data (paper Sec. 2.2) converted
// once on the host to a power basis per segment, p(u) = c0 + u (c1 + u (c2 + u c3)),
// u = s - s_k.  Functions: 0..4 = alpha_1..alpha_5, 5..7 = beta_1..beta_3.
// ----------------------------------------------------------------------------
constexpr int kMaxSeg = 32;
constexpr int kNumFn = 8;
constexpr double kEtaMax = 0.4;       // Eq. iofd-clamped-coordinate
constexpr double kInv2Pi = 0.15915494309189533576888376337251;

template <class R>
struct TableView {
  const R* coef;   // [seg][fn][4]
  int nseg;
  R ds, inv_ds;
};

// The four power-basis coefficients of one function on one segment (the table
// is 16-byte aligned: one 128-bit load for float, two for double).
__device__ __forceinline__ void load_coef4(const float* p, float& c0, float& c1, float& c2, float& c3) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  c0 = v.x; c1 = v.y; c2 = v.z; c3 = v.w;
}
__device__ __forceinline__ void load_coef4(const double* p, double& c0, double& c1, double& c2, double& c3) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  c0 = a.x; c1 = a.y; c2 = b.x; c3 = b.y;
}

// Evaluate functions [F0, F0+NF) at eta (eta already clamped to [0, 0.4]).
template <class R, int F0, int NF>
__device__ __forceinline__ void table_eval(const R* __restrict__ tab, int nseg, R ds, R inv_ds, R eta, R* out) {
  int seg = (int)(eta * inv_ds);
  seg = seg < 0 ? 0 : (seg > nseg - 1 ? nseg - 1 : seg);
  R u = eta - (R)seg * ds;
  const R* c = tab + (seg * kNumFn + F0) * 4;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    R c0, c1, c2, c3;
    load_coef4(c + 4 * f, c0, c1, c2, c3);
    out[f] = c0 + u * (c1 + u * (c2 + u * c3));
  }
}

// Same, also returning d/deta (for the gradient).
template <class R, int F0, int NF>
__device__ __forceinline__ void table_eval_d(const R* __restrict__ tab, int nseg, R ds, R inv_ds, R eta, R* out, R* dout) {
  int seg = (int)(eta * inv_ds);
  seg = seg < 0 ? 0 : (seg > nseg - 1 ? nseg - 1 : seg);
  R u = eta - (R)seg * ds;
  const R* c = tab + (seg * kNumFn + F0) * 4;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    out[f] = c[4 * f] + u * (c[4 * f + 1] + u * (c[4 * f + 2] + u * c[4 * f + 3]));
    dout[f] = c[4 * f + 1] + u * ((R)2 * c[4 * f + 2] + (R)3 * u * c[4 * f + 3]);
  }
}

template <class R>
__device__ __forceinline__ R eta_star(R kappa) {
  R e = kappa * (R)kInv2Pi;
  return e < (R)kEtaMax ? e : (R)kEtaMax;
}

// ----------------------------------------------------------------------------
// One level of the hierarchy as the kernels see it.
// PML per axis a (0 = x, 1 = y, 2 = z): abar = (d+ + d-)/2, achk = (d+ - d-)/2
// with d+- = xi_i^{-1} xi_{i+-1/2}^{-1} (Eq. pml-second-difference), so that
// the directional term is abar (T(+1)+T(-1)-2T(0)) + achk (T(+1)-T(-1)).
// plain_lo/hi: index range of an axis where abar = 1 and achk = 0 exactly.
// ----------------------------------------------------------------------------
template <class R>
struct LevelView {
  int level;                      // 0 = h, 1 = 2h, 2 = 4h
  int nx, ny, nz;                 // nodes per axis (intervals + 1)
  long long N;                    // nodes
  const R* kappa;                 // k(x_i) * ell per node
  const cx<R>* abar[3];
  const cx<R>* achk[3];
  // PML correction factors of the forward kernel, per axis and node:
  // eps[a][0] = -(abar - 1 + achk) / ell^2, eps[a][1] = -(abar - 1 - achk) / ell^2
  // (zero where the axis is not stretched)
  const cx<R>* eps[3][2];
  // precombined coefficient polynomials of this level (layout in hz_fwd.cuh)
  const R* ctab;
  int plain_lo[3], plain_hi[3];
  R inv_ell2;                     // 1 / ell^2
  int zblock;                     // planes per CTA of the forward stencil (0: heuristic)
  int zblock_f;                   // the same for the PML-frame launch (0: as zblock)
};

// ----------------------------------------------------------------------------
// Deterministic block reduction helpers (values accumulated in double).
// ----------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum `val` over the block (tid = linear thread id, nthreads = block size, a
// multiple of 32); result valid in thread 0.  `scratch` >= 32 doubles.
__device__ __forceinline__ double block_sum(double val, double* scratch, int tid, int nthreads) {
  val = warp_sum(val);
  int lane = tid & 31, w = tid >> 5;
  int nw = nthreads >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = val;
  __syncthreads();
  double r = 0.0;
  if (tid < 32) {
    r = (tid < nw) ? scratch[tid] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Arrival of one block at a grid-wide reduction of group `counter`.  Thread 0
// must have written this block's partials before the call.  Returns true in
// every thread of the last block to arrive; that block then reads all
// partials (use __ldcg) and must reset *counter to 0.  No thread waits for
// another block, so the pattern cannot hang.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter, unsigned nblk, int tid) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(counter, 1u) == nblk - 1u);
  __syncthreads();
  return s_last;
}

}  // namespace hz
