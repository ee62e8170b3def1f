// Block Krylov kernels of block flexible GMRES over several right-hand sides
// (the block Krylov method for multiple right-hand sides of Sec. 7): the
// Gram block G = X^H Y of two sets of basis columns and the block update
// Y = beta Y + X C with a small dense coefficient matrix C.
//
// Both are tall-skinny products over the grid (p, q <= a few dozen columns of
// N nodes).  The Gram kernel gives each block a PT x QT tile of G and a
// contiguous chunk of nodes, accumulates conj(x) y per thread in the working
// precision, reduces the block in double and writes one partial per chunk; a
// second kernel sums the chunks in chunk order (deterministic).  Chunks are
// the slow grid index, so the blocks of all tiles of one chunk run together
// and the columns' chunk is read from L2 after its first use.
#include <algorithm>

#include "hz_kernels.h"

namespace hz {

namespace {

constexpr int BT = 256;       // threads per block
constexpr int GPT = 4, GQT = 4;  // Gram tile

template <class R>
__device__ __forceinline__ const cx<R>* col_ptr(const BlockCols& c, int t) {
  return reinterpret_cast<const cx<R>*>(c.base) + (long long)(t / c.s) * c.bstride + (long long)(t % c.s) * c.n;
}

template <class R>
__global__ void __launch_bounds__(BT) k_block_gram(BlockCols X, BlockCols Y, long long chunk, double* partial) {
  const int ntq = (Y.count + GQT - 1) / GQT;
  const int tp = blockIdx.x / ntq, tq = blockIdx.x % ntq;
  const int p0 = tp * GPT, q0 = tq * GQT;
  const long long i0 = blockIdx.y * chunk, i1 = min(i0 + chunk, X.n);
  const cx<R>* xp[GPT];
  const cx<R>* yp[GQT];
#pragma unroll
  for (int a = 0; a < GPT; ++a) xp[a] = p0 + a < X.count ? col_ptr<R>(X, p0 + a) : nullptr;
#pragma unroll
  for (int b = 0; b < GQT; ++b) yp[b] = q0 + b < Y.count ? col_ptr<R>(Y, q0 + b) : nullptr;
  cx<R> acc[GPT][GQT];
#pragma unroll
  for (int a = 0; a < GPT; ++a)
#pragma unroll
    for (int b = 0; b < GQT; ++b) acc[a][b] = mkc<R>(0, 0);
  for (long long i = i0 + threadIdx.x; i < i1; i += BT) {
    cx<R> xv[GPT], yv[GQT];
#pragma unroll
    for (int a = 0; a < GPT; ++a) xv[a] = xp[a] ? xp[a][i] : mkc<R>(0, 0);
#pragma unroll
    for (int b = 0; b < GQT; ++b) yv[b] = yp[b] ? yp[b][i] : mkc<R>(0, 0);
#pragma unroll
    for (int a = 0; a < GPT; ++a)
#pragma unroll
      for (int b = 0; b < GQT; ++b) acc[a][b] += cjmul(xv[a], yv[b]);
  }
  // block reduction in double: value v of warp w in red[w][v]
  __shared__ double red[BT / 32][2 * GPT * GQT];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < GPT; ++a)
#pragma unroll
    for (int b = 0; b < GQT; ++b) {
      const double re = warp_sum((double)acc[a][b].x), im = warp_sum((double)acc[a][b].y);
      if (lane == 0) {
        red[w][2 * (a * GQT + b)] = re;
        red[w][2 * (a * GQT + b) + 1] = im;
      }
    }
  __syncthreads();
  if (threadIdx.x < 2 * GPT * GQT) {
    const int v = threadIdx.x;
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < BT / 32; ++k) t += red[k][v];
    const int e = v >> 1, a = e / GQT, b = e % GQT;
    if (p0 + a < X.count && q0 + b < Y.count)
      partial[(((size_t)blockIdx.y * X.count + p0 + a) * Y.count + q0 + b) * 2 + (v & 1)] = t;
  }
}

// out[e] = sum over chunks c of partial[c][e], in chunk order
__global__ void __launch_bounds__(BT) k_block_gram_sum(const double* __restrict__ partial, int nchunk, int nval,
                                                        double* __restrict__ out) {
  const int e = blockIdx.x * BT + threadIdx.x;
  if (e >= nval) return;
  double t = 0.0;
  for (int c = 0; c < nchunk; ++c) t += partial[(size_t)c * nval + e];
  out[e] = t;
}

// Y_c = beta Y_c + sum_i X_i C[i][c] for c < q.  Each thread finishes one node
// of every output column from that node's inputs alone, so Y may be X itself
// (an in-place change of basis); the pointers are therefore not restrict.
template <class R, int QM>
__global__ void __launch_bounds__(BT) k_block_update(BlockCols X, cx<R>* Y, int q, const double* C, double beta,
                                                     long long n) {
  extern __shared__ __align__(16) unsigned char bsm[];
  cx<R>* sC = reinterpret_cast<cx<R>*>(bsm);  // [p][QM]
  const int p = X.count;
  for (int t = threadIdx.x; t < p * QM; t += BT) {
    const int i = t / QM, c = t % QM;
    sC[t] = c < q ? mkc<R>((R)C[2 * (i * q + c)], (R)C[2 * (i * q + c) + 1]) : mkc<R>(0, 0);
  }
  __syncthreads();
  for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    cx<R> acc[QM];
#pragma unroll
    for (int c = 0; c < QM; ++c) acc[c] = (beta != 0.0 && c < q) ? (R)beta * Y[(long long)c * n + i] : mkc<R>(0, 0);
    for (int t = 0; t < p; ++t) {
      const cx<R> xv = col_ptr<R>(X, t)[i];
      const cx<R>* cr = sC + t * QM;
#pragma unroll
      for (int c = 0; c < QM; ++c) acc[c] += xv * cr[c];
    }
#pragma unroll
    for (int c = 0; c < QM; ++c)
      if (c < q) Y[(long long)c * n + i] = acc[c];
  }
}

int gram_chunks(long long n) {
  // chunks of at least 16 K nodes, at most 1024 of them
  const long long c = (n + 16383) / 16384;
  return (int)std::max<long long>(1, std::min<long long>(c, 1024));
}

}  // namespace

size_t block_gram_partial_doubles(long long n, int p, int q) { return (size_t)gram_chunks(n) * p * q * 2; }

template <class R>
void launch_block_gram(const BlockCols& X, const BlockCols& Y, double* partial, double* out, cudaStream_t s) {
  const int nchunk = gram_chunks(X.n);
  const long long chunk = (X.n + nchunk - 1) / nchunk;
  const int tiles = ((X.count + GPT - 1) / GPT) * ((Y.count + GQT - 1) / GQT);
  count_launch();
  k_block_gram<R><<<dim3(tiles, nchunk), BT, 0, s>>>(X, Y, chunk, partial);
  const int nval = 2 * X.count * Y.count;
  count_launch();
  k_block_gram_sum<<<(nval + BT - 1) / BT, BT, 0, s>>>(partial, nchunk, nval, out);
}

template <class R>
void launch_block_update(const BlockCols& X, cx<R>* Y, int q, const double* C, double beta, cudaStream_t s) {
  const long long n = X.n;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((n + BT - 1) / BT, 152LL * 8));
  auto go = [&](auto qm) {
    constexpr int QM = decltype(qm)::value;
    const size_t sm = (size_t)X.count * QM * sizeof(cx<R>);
    count_launch();
    k_block_update<R, QM><<<blocks, BT, sm, s>>>(X, Y, q, C, beta, n);
  };
  if (q <= 4) go(std::integral_constant<int, 4>{});
  else if (q <= 8) go(std::integral_constant<int, 8>{});
  else go(std::integral_constant<int, 16>{});
}

// one-time attribute: the update's coefficient block can exceed 48 KB (complex128, p = 96, q = 16)
void block_init_attrs() {
  cudaFuncSetAttribute(k_block_update<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kBlockMaxP * 16 * (int)sizeof(cx<double>));
  cudaFuncSetAttribute(k_block_update<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kBlockMaxP * 16 * (int)sizeof(cx<float>));
}

template void launch_block_gram<float>(const BlockCols&, const BlockCols&, double*, double*, cudaStream_t);
template void launch_block_gram<double>(const BlockCols&, const BlockCols&, double*, double*, cudaStream_t);
template void launch_block_update<float>(const BlockCols&, cx<float>*, int, const double*, double, cudaStream_t);
template void launch_block_update<double>(const BlockCols&, cx<double>*, int, const double*, double, cudaStream_t);

}  // namespace hz
