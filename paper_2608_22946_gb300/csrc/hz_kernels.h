// Host-side launch interface of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <atomic>

#include "hz_common.cuh"

namespace hz {

// Kernels launched by this library in the process (instrumentation for the
// benchmark's launch count; graph replays add their kernel-node count).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// M_AWIN: an APPLY of the fine level from a z-window (StencilCall::zr0 .. xstride)
enum StencilMode { M_APPLY = 0, M_RESID = 1, M_J2 = 2, M_JSWEEP = 3, M_J1 = 4, M_AWIN = 5 };
enum StencilOp { OP_AB = 0, OP_Q = 1 };

// Reduction target of a kernel that finishes with a deterministic
// grid-wide sum: per-block partials, an arrival counter per group and the
// output slot per group (all device memory owned by the handle).
struct Reduce {
  double* partial = nullptr;
  unsigned* count = nullptr;
  double* out = nullptr;       // sum per group
  double* root = nullptr;      // optional sqrt(sum)
  double* inv_root = nullptr;  // optional 1/sqrt(sum) (0 when the sum is 0)
};

template <class R>
struct StencilCall {
  LevelView<R> lv;
  TableView<R> tab;
  cx<R> mass_shift;      // 1 + i sigma (B) or 1 (A)
  R omega_j = 0;         // Jacobi weight
  const cx<R>* x = nullptr;     // APPLY/RESID: x; J2/J1: g; JSWEEP: current iterate y
  const cx<R>* g = nullptr;     // RESID/JSWEEP: right-hand side
  const cx<R>* base = nullptr;  // J2: out = base + J2(g) when non-null
  const cx<R>* dinv = nullptr;  // J2 (forward): 1/diag of this operator on this level, per node
  cx<R>* y = nullptr;
  int nrhs = 1;
  Reduce red;            // RESID: ||y||^2 per rhs when red.out != nullptr
  // optional second stream: the PML-frame launch of a split application runs
  // on it beside the rectangle launch (fork / join through the two events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // z-window of a fine-level APPLY (one brick of a z-slab decomposition): rows
  // [zr0, zr1) are computed (zr1 = 0: all nz rows); input plane q is read at
  // x + rhs * xstride + (q - xz0) * plane, output row z written at
  // y + rhs * ystride + (z - zr0) * plane (strides 0: N)
  int zr0 = 0, zr1 = 0, xz0 = 0;
  long long xstride = 0, ystride = 0;
};

template <class R>
void launch_stencil(const StencilCall<R>& c, int mode, int op, bool adjoint, cudaStream_t s);
// Forward stencil of one (precision, mode) for operator kind opk (hz_fwd.cuh),
// and the one-time kernel attributes of those kernels.
template <class R, int MODE>
void launch_fwd(const StencilCall<R>& c, int opk, cudaStream_t s);
template <class R, int MODE>
void fwd_init_attrs();
// Smallest z-block (planes per CTA) of a stencil launch.
constexpr int kMinZblock = 2;
// (level 0 runs the accumulation-form kernels of hz_fwd.cuh, levels 1 and 2 the
// gather-form kernels of hz_fwd_gather.cu; each has its own launch layout)
long long stencil_blocks_per_rhs(int level, int nx, int ny, int nz, const int* plain_lo, const int* plain_hi,
                                 int nrhs, int zblock = 0, int zblock_f = 0);
// Blocks per right-hand side of an adjoint stencil launch (zblock > 0 forces it).
long long adj_blocks_per_rhs(int nx, int ny, int nz, int nrhs, int zblock = 0);
// Host replay of a forward stencil application's launch layout on a grid of
// nx x ny x nz nodes: per-node write counts of right-hand side 0 (or null) and
// the number of layout violations (defined beside the tiling).
long long replay_adj_layout(int nx, int ny, int nz, int nrhs, int zblock, unsigned char* counts, long long* blocks);
long long replay_fwd_layout(int level, int nx, int ny, int nz, const int* plain_lo, const int* plain_hi, int op,
                            int nrhs, int zblock, int zblock_f, unsigned char* counts, long long* blocks);
// Columns of a block Krylov basis: column t at base + (t / s) * bstride + (t % s) * n
// elements (blocks of s consecutive columns of n nodes, blocks bstride apart).
struct BlockCols {
  const void* base;
  long long bstride;
  long long n;
  int s;
  int count;
};
constexpr int kBlockMaxS = 16;   // right-hand sides sharing one block FGMRES basis
constexpr int kBlockMaxP = 256;  // basis columns entering one block update (m_out * s)
// doubles of the Gram kernel's per-chunk partial sums for p x q blocks of n nodes
size_t block_gram_partial_doubles(long long n, int p, int q);
// out (p x q complex double, row-major) = X^H Y; partial: block_gram_partial_doubles
template <class R>
void launch_block_gram(const BlockCols& X, const BlockCols& Y, double* partial, double* out, cudaStream_t s);
// Y_c = beta Y_c + sum_t X_t C[t][c] for the q <= 16 columns of Y (stride X.n);
// C complex double p x q row-major on the device; Y may be X itself
template <class R>
void launch_block_update(const BlockCols& X, cx<R>* Y, int q, const double* C, double beta, cudaStream_t s);
void block_init_attrs();
namespace gather {
// forward stencil of the coarse levels (hz_fwd_gather.cu)
template <class R>
void launch_fwd_gather(const StencilCall<R>& c, int mode, int op, cudaStream_t s);
long long gather_blocks_per_rhs(int nx, int ny, int nz, const int* plain_lo, const int* plain_hi, int nrhs,
                                int zblock, int zblock_f);
long long replay_gather_layout(int nx, int ny, int nz, const int* plo, const int* phi, int op, int nrhs, int zblock,
                               int zblock_f, unsigned char* counts, long long* blocks);
// The bottom solve C_4h (s-step CA-GMRES with kBottomSteps steps, two-sweep
// Jacobi maps of B_4h) as one persistent cooperative kernel.
constexpr int kBottomSteps = 4;
template <class R>
struct BottomArgs {
  StencilCall<R> c;         // level 2, B shift, omega_4h, 1/diag of B_4h; x and y are set per sweep
  cx<R>* P = nullptr;       // basis p_0 .. p_s (p_0 given), right-hand sides of one vector contiguous
  cx<R>* Zc = nullptr;      // J(p_0) .. J(p_{s-1})
  long long vs = 0;         // elements per basis vector (N_4h * nrhs)
  cx<R>* e = nullptr;       // result sum_k y_k J(p_k)
  double* y = nullptr;      // [nrhs][ld] complex coefficients (out)
  int ld = kBottomSteps + 1;
  double* partial = nullptr;  // bottom_partial_doubles(nrhs) Gram partial sums
  unsigned* bar = nullptr;    // two counters, zeroed by the launcher
  int* err = nullptr;         // set nonzero when a grid-barrier wait gave up
  unsigned spins = 1u << 23;  // polls (100 ns apart) before a barrier wait gives up
  unsigned extra = 0;         // > 0 only to test that path: arrivals the barrier waits for in vain
  int zblock = 0, ntx = 0, nty = 0, nzb = 0;  // set by the launcher
};
// Enqueue on s; false when it could not be launched (nothing enqueued then
// except, possibly, the barrier reset).
template <class R>
bool launch_bottom4h(BottomArgs<R> b, cudaStream_t s);
template <class R>
size_t bottom_partial_doubles(int nrhs);
bool coop_capture_supported();
}  // namespace gather

// Grid transfers (Eq. full-weighting, Eq. linear-prolongation).
template <class R>
void launch_restrict(const cx<R>* fine, cx<R>* coarse, int nxf, int nyf, int nzf, int nrhs, cudaStream_t s);
template <class R>
void launch_prolong_add(const cx<R>* coarse, const cx<R>* base, cx<R>* fine, int nxf, int nyf, int nzf, int nrhs,
                        cudaStream_t s);

// Krylov vector passes.  Vectors of one basis are `vstride` elements apart;
// each holds nrhs contiguous fields of n elements.  Scalars are complex
// double pairs per rhs, rows of length `ld`.
struct KrylovCall {
  int n = 0;            // elements per field
  int nrhs = 1;
  long long vstride = 0;  // elements between basis vectors
  int kn = 0;            // number of basis vectors involved
  int ld = 0;            // leading dimension of per-rhs scalar rows (complex entries)
  // selective reorthogonalisation (Arnoldi passes only): per-rhs flag set by
  // the first pass when its projection leaves more than 1/sqrt(2) of ||w||
  // (Daniel, Gragg, Kaufman and Stewart's criterion), in which case the
  // second pass returns at once and the first pass hands its coefficients,
  // norm and scale to the final update
  int* skip = nullptr;
  double* coef_final = nullptr;  // [rhs][ld] complex, read by the final update
};

// w -= sum_k coef[r][k] V_k  (optional), then dots[r][k] = <V_k, w> (optional),
// nrm2[r] = ||w||^2 (optional).  Results written by the last block, which
// then runs `epi` (see hz_vec.cu).
enum CgsEpi { EPI_STORE = 0, EPI_ARNOLDI_FIRST = 1, EPI_ARNOLDI_SECOND = 2, EPI_NORMALISE = 3 };
template <class R>
void launch_cgs(const KrylovCall& k, const cx<R>* V, cx<R>* w, const double* coef, bool update, bool dots,
                bool norm, double* dots_out, double* nrm_out, int epi, double* H, int col, double* scale_out,
                double* beta_out, const Reduce& red, cudaStream_t s);

// out = w * scale[r]  (scale real double per rhs)
template <class R>
void launch_scale(const cx<R>* w, cx<R>* out, const double* scale, int n, int nrhs, cudaStream_t s);

// x = (x0 ? x0 : 0) + sum_k y[r][k] Z_k  (y complex double, rows of length ld)
template <class R>
void launch_combine(const cx<R>* Z, long long zstride, int kn, const double* y, int ld, const cx<R>* x0, cx<R>* x,
                    int n, int nrhs, cudaStream_t s);

// Small least-squares min || beta e1 - H y || per rhs (H: (m+1) x m, column-major
// complex double, leading dim m+1, per rhs stride (m+1)*m); y rows of length ld.
void launch_lsq(const double* H, const double* beta, double* y, int m, int ld, int nrhs, cudaStream_t s,
                bool single);
// w <- (w - sum_k coef[r][k] V_k) * scale[r]: last Gram-Schmidt pass fused with the normalisation
template <class R>
void launch_update_scale(const KrylovCall& k, const cx<R>* V, cx<R>* w, const double* coef, const double* scale,
                         cudaStream_t s);

// Gram matrix of kn vectors, Cholesky, and the CA-GMRES least-squares solve
// min || p_0 - sum_{k>=1} y_{k-1} p_k ||; writes y (kn-1 entries per rhs).
template <class R>
void launch_gram_lsq(const cx<R>* P, long long pstride, int kn, int n, int nrhs, double* y, int ld,
                     const Reduce& red, cudaStream_t s);

// y = a*x + b*y style helpers
template <class R>
void launch_axpy(const cx<R>* x, cx<R>* y, double ar, double ai, long long n, cudaStream_t s);
template <class R>
void launch_copy(const cx<R>* x, cx<R>* y, long long n, cudaStream_t s);
template <class R>
void launch_zero(cx<R>* y, long long n, cudaStream_t s);

// Mixed precision glue.
void launch_c128_to_c64_scaled(const cx<double>* in, cx<float>* out, const double* scale, int n, int nrhs,
                               cudaStream_t s);
void launch_c64_to_c128(const cx<float>* d, cx<double>* x, int n, int nrhs, cudaStream_t s);
void launch_add_c64_to_c128_scaled(const cx<float>* d, cx<double>* x, const double* scale, int n, int nrhs,
                                   cudaStream_t s);
template <class R>
void launch_norm2(const cx<R>* v, int n, int nrhs, const Reduce& red, cudaStream_t s);

// Set-up: kappa_L[j] = omega * ell / c_ext[2^L j], where c_ext is c inside the
// physical box and, at a PML node, c at the closest physical node (Sec. 2.1,
// Sec. 3.1).
template <class R>
void launch_setup_kappa(const double* c, int nxf, int nyf, int nzf, int n_pml, int stride, double omega,
                        double ell, R* kappa, cudaStream_t s);

// Point sources f = h^-3 amp delta (Eq. point-source) written into zeroed fields.
template <class R>
void launch_point_sources(const int* idx3, const double* amp, int nsrc, int nx, int ny, int nz, double scale,
                          cx<R>* f, cudaStream_t s);

// Adjoint-state gradient (row-local derivatives of A and Q w.r.t. m = 1/c^2):
// g_ext[i] += sum_r Re[ conj(lam_i) (dQ_i f - dA_i v) + conj(rres_i) dQ_i v ].
void launch_gradient(const LevelView<double>& lv, const TableView<double>& tab, double omega_h,
                     const cx<double>* v, const cx<double>* lam, const cx<double>* f, const cx<double>* rres,
                     int nrhs, double* g_ext, cudaStream_t s);
// g[t] = sum of g_ext over the nodes whose velocity copies physical node t
// (identity inside, rays into the PML at its faces, edges and corners); 0 in the PML.
void launch_fold_pml(const double* g_ext, double* g, int nx, int ny, int nz, int n_pml, cudaStream_t s);
// Interior shell coefficients C_0..C_3 of A at every node (Eq. iofd-shell-coefficients), [m][node].
void launch_shell_coeffs(const LevelView<double>& lv, const TableView<double>& tab, double* out, cudaStream_t s);
void launch_source_rows(const LevelView<double>& lv, const TableView<double>& tab, const int* idx3,
                        const double* amp, int nsrc, double scale, cx<double>* b, cudaStream_t s);
// 1 / H_ii for H = A_L (sigma = 0) or B_L at every node of a level (the Jacobi diagonal,
// Eq. jacobi-map): ell^-2 [2 a4 (abar_x + abar_y + abar_z) - (1 + i sigma) kappa^2 a1].
template <class R>
void launch_setup_dinv(const LevelView<R>& lv, const TableView<R>& tab, cx<R> shift, cx<R>* out, cudaStream_t s);
// Set kernel attributes once per process/device (dynamic shared memory opt-in).
void init_kernel_attributes();

// Receivers
template <class R>
void launch_gather(const cx<R>* u, const int* rec, int nrec, int n, int nrhs, cx<double>* out, cudaStream_t s);
template <class R>
void launch_scatter(const cx<double>* vals, const int* rec, int nrec, int n, int nrhs, cx<R>* out, cudaStream_t s);

}  // namespace hz
