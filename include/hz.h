/*
 * hz.h -- C ABI of the GB300 three-grid IOFD Helmholtz library (libhz.so).
 *
 * The library solves the PML-truncated Helmholtz problem
 *     -sum_j xi_j^-1 d_j (xi_j^-1 d_j u) - k(x)^2 u = f,  u = 0 on the box boundary
 * (Sec. 2.1, Eq. helmholtz-pml) with the compact 27-point IOFD discretisation
 * P_h v = Q_h f, u = Q_h v (Sec. 2.2, Eq. iofd-complete-system), by FGMRES
 * right-preconditioned with the three-grid cycle of Algorithm 1 (Sec. 3).
 *
 * Conventions shared by every entry point
 *   - Grid: nx, ny, nz intervals per axis INCLUDING n_pml PML layers on each
 *     side; every one of the (nx+1)(ny+1)(nz+1) nodes is an unknown
 *     (Sec. 5 counts meshes this way).  nx, ny, nz and n_pml must be divisible by 4
 *     (two coarsenings, each halving the PML layers, Sec. 3.1).
 *   - Field layout: x fastest, then y, then z; for nrhs right-hand sides the
 *     fields are stacked, [rhs][z][y][x].  Complex values are interleaved
 *     (re, im): complex64 = 2 x float, complex128 = 2 x double.
 *   - Level L in {0, 1, 2} is the grid of spacing 2^L h (h, 2h, 4h), with
 *     (nx/2^L + 1)(ny/2^L + 1)(nz/2^L + 1) nodes.
 *   - Pointers named *_dev are DEVICE pointers on the handle's device;
 *     pointers named *_host are host pointers.  The caller owns every buffer
 *     it passes; the library never frees or retains them past the call.
 *     Input and output buffers must not alias unless stated.
 *   - `stream` arguments are cudaStream_t values (0 = legacy default stream)
 *     passed as void*; work is enqueued on it and the call returns without
 *     synchronising unless stated.  Part of a stencil application may run on
 *     a second stream of the handle, forked from `stream` and joined back to
 *     it with events, so stream order as seen by the caller is unchanged.
 *   - Every entry point returns an hz_status; on failure hz_last_error()
 *     gives a message.  No C++ exception crosses the ABI.  Calls on one
 *     handle must not run concurrently from several host threads.
 */
#ifndef HZ_H_
#define HZ_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HZ_OK = 0,
  HZ_EINVAL = 1,      /* bad argument (null pointer, size, divisibility, range) */
  HZ_ENOMEM = 2,      /* device allocation failed */
  HZ_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  HZ_ENOCONV = 4,     /* max_pc reached before the tolerance (results are filled) */
  HZ_ETIMEOUT = 5,    /* a bounded device wait gave up: a grid barrier of the persistent
                         bottom-solve kernel (opt-in: environment HZ_PERSISTENT=1 when the
                         handle is created; all its blocks are co-resident by a cooperative
                         launch) did not release within about a second.  The
                         kernel finishes without waiting, its results are invalid, and the
                         next helmholtz_solve or helmholtz_adjoint_grad on the handle
                         returns this status (threegrid_precond, being asynchronous, does
                         not read it).  The context stays usable. */
  HZ_ENONFINITE = 6   /* a NaN/Inf appeared in a residual norm */
} hz_status;

/* precision of a call */
enum { HZ_C64 = 0, HZ_C128 = 1 };

/* operators for iofd_apply */
enum {
  HZ_OP_A = 0,      /* A_ell = L_ell - M_ell            (Eq. physical-iofd-levels)   */
  HZ_OP_B = 1,      /* B_ell = L_ell - (1+i sigma) M_ell (Eq. shifted-iofd-levels)   */
  HZ_OP_Q = 2,      /* Q_h amplitude correction, level 0 only (Eq. q-operator)       */
  HZ_OP_A_ADJ = 3,  /* A_ell^H                                                        */
  HZ_OP_B_ADJ = 4,  /* B_ell^H                                                        */
  HZ_OP_Q_ADJ = 5   /* Q_h^H, level 0 only                                            */
};

typedef struct {
  int nx, ny, nz;      /* intervals per axis, PML included */
  int n_pml;           /* PML layers per side on the fine grid */
  double h;            /* fine spacing */
  double omega;        /* angular frequency (time dependence exp(-i omega t)) */
  double gamma_max;    /* PML stretch amplitude (Eq. pml-profile); Table 4: 1.119058 */
} hz_grid;

typedef struct {
  int ix, iy, iz;      /* source node */
  double amp_re, amp_im;  /* f_h = amp h^-3 delta_{i,i_s} (Eq. point-source) */
} hz_source;

/* Solver configuration; hz_default_params() fills Table 4 of the paper
 * (tol 1e-4 there; the mixed-versus-FP64 study uses 1e-6). */
typedef struct {
  double tol;          /* stop when ||A v - b|| / ||b|| <= tol (Eq. relative-residual) */
  int max_pc;          /* cap on preconditioner calls (outer FGMRES steps) */
  int m_out;           /* outer FGMRES restart length */
  int m_h, nJ_h;       /* fine smoother: GMRES(m_h) right-preconditioned by nJ_h Jacobi sweeps */
  int c_2h, m_2h;      /* 2h solve: c_2h FGMRES(m_2h) cycles on A_2h */
  int nJ_2h;           /* Jacobi sweeps of the shifted 2h cycle */
  int m_4h, nJ_4h;     /* 4h bottom: m_4h CA-GMRES steps, nJ_4h Jacobi sweeps */
  double w_h, w_2h, w_4h;  /* Jacobi weights */
  double sigma;        /* complex shift of B_2h, B_4h */
  int precision;       /* HZ_C64: complex64 hierarchy and inner solves, FP64 outer
                          Krylov scalars and FP64 iterative refinement;
                          HZ_C128: everything in complex128 */
  double inner_tol;    /* HZ_C64 only: floor of the relative tolerance of each
                          complex64 correction solve inside the refinement loop */
  int max_refine;      /* HZ_C64 only: cap on refinement passes */
  int autotune;        /* nonzero: hz_create times the forward stencil on every level for a
                          set of z-block sizes (planes per thread block) and keeps the
                          fastest; zero: a fixed heuristic */
  int refine;          /* HZ_C64 only.  1: FP64 iterative refinement around complex64
                          corrections, each FP64 true residual deciding convergence
                          (default).  0: the paper's protocol (Sec. 5.2, Table 4): one
                          complex64 FGMRES(m_out) solve stopped by its own complex64 true
                          residual at tol, no refinement pass; rel_res is that residual */
  int block;           /* 0: an independent FGMRES(m_out) per right-hand side in flight
                          (batched operator and preconditioner applications; default).
                          1: block flexible GMRES (the block Krylov method for multiple
                          right-hand sides of Sec. 7): the right-hand sides in flight, in
                          groups of at most 16, share one basis; each block step applies
                          the preconditioner to the group's basis block and counts as one
                          preconditioner call; each right-hand side takes the minimal
                          residual over the whole block space.  A numerically
                          rank-deficient initial block (a zero or repeated right-hand
                          side) falls back to the independent method for that solve. */
} hz_params;

typedef struct {
  int pc_calls;        /* preconditioner calls = outer FGMRES steps, all passes */
  int refine_passes;   /* refinement-loop passes (HZ_C64), each ending in the FP64
                          true residual; that of the zero initial guess is b itself */
  double rel_res;      /* final ||A v - b|| / ||b||, max over right-hand sides */
  double t_setup;      /* seconds, per-level coefficients and tables */
  double t_solve;      /* seconds */
  size_t device_bytes; /* device memory held by the handle */
  int zblock[3];       /* z-block of the forward stencil per level (autotuned or heuristic):
                          the whole grid, or the PML-free rectangle of a split launch */
  int zblock_frame[3]; /* z-block of the PML-frame launch per level (split launches) */
} hz_stats;

typedef struct hz_handle hz_handle;

/* Table 4 defaults (Sec. 6.1): m_out 5, m_h 2 / nJ_h 2 / w_h 0.8, c_2h 2,
 * m_2h 10, nJ_2h 2 / w_2h 0.8, m_4h 4 / nJ_4h 2 / w_4h 0.2, sigma 0.9,
 * tol 1e-4, precision HZ_C64, inner_tol 1e-5, max_pc 1000, max_refine 8, autotune 1, refine 1,
 * block 0. */
void hz_default_params(hz_params* p);

/* Create a solver for one frequency and velocity model.
 *   c_dev       DEVICE, double, (nx+1)(ny+1)(nz+1) wave speeds on every fine
 *               node; values inside the PML are ignored and replaced by the
 *               nearest physical value (Sec. 2.1).  Read during the call only.
 *   table_host  HOST, double, table_rows x 17 IOFD Hermite data, one row per
 *               uniform node s_k on [0, 0.4]: s, alpha_1..5, d alpha_1..5/ds,
 *               beta_1..3, d beta_1..3/ds (Sec. 2.2: alpha_j, beta_j are cubic
 *               Hermite interpolants of tabulated values).  2 <= rows <= 33.
 *   max_nrhs    largest nrhs any later call will use (sizes the workspaces).
 *   stream      stream for set-up work; the call synchronises it.
 * Returns HZ_EINVAL for bad sizes, HZ_ENOMEM if the workspaces do not fit. */
hz_status hz_create(const hz_grid* grid, const double* c_dev, const hz_params* params, const double* table_host,
                    int table_rows, int max_nrhs, void* stream, hz_handle** out);
hz_status hz_destroy(hz_handle* h);
const char* hz_last_error(const hz_handle* h);
/* Number of kernels this library has launched in this process (each CUDA
 * graph replay counts the kernels it contains).  Instrumentation only. */
unsigned long long hz_kernel_launches(void);
/* Device bytes hz_create would allocate for these sizes. */
hz_status hz_workspace_bytes(const hz_grid* grid, const hz_params* params, int max_nrhs, size_t* bytes);
/* Replace the solver parameters (e.g. tolerance); cached CUDA graphs are dropped. */
hz_status hz_set_params(hz_handle* h, const hz_params* params);

/* Host-only check of a stencil application's launch layout; no GPU work and
 * no counterpart in the paper.  Replays, for level `level` of `grid` (the same
 * checks as hz_create), how one application of op (forward: HZ_OP_A,
 * HZ_OP_B, or HZ_OP_Q on level 0; adjoint: HZ_OP_A_ADJ, HZ_OP_B_ADJ) with
 * nrhs right-hand sides and the given z-blocks (0: the built-in heuristic;
 * zblock_f: the PML-frame launch of a forward application, 0 = zblock)
 * assigns grid nodes to CUDA blocks and threads.
 *   counts_host  HOST, N_L bytes, or NULL: times each node of right-hand side 0
 *                is written (saturating at 255; 1 everywhere is an exact cover).
 *   blocks       HOST, or NULL: blocks per right-hand side (the fused
 *                reductions keep one partial sum per block).
 *   violations   HOST: tiles whose threads would write outside the grid, use a
 *                row form that omits PML terms present at a written node, or
 *                repeat / overrun a block id.  0 for a valid layout.
 * Returns HZ_EINVAL for bad arguments (message in hz_last_error(NULL)). */
hz_status hz_layout_check(const hz_grid* grid, int level, int op, int nrhs, int zblock, int zblock_f,
                          unsigned char* counts_host, long long* blocks, long long* violations);

/* Per-level coefficients, for inspection (Eq. iofd-clamped-coordinate,
 * Eq. iofd-shell-coefficients).
 *   kappa_dev  DEVICE double, N_L values: kappa_{L,i} = k(x_i) 2^L h.
 *   shell_dev  DEVICE double, 4 N_L values or NULL: the interior shell
 *              coefficients C_0..C_3 of A_L at each node (times ell^2, as in
 *              the paper), laid out [m][node].  Synchronises the handle stream. */
hz_status iofd_coeffs(hz_handle* h, int level, double* kappa_dev, double* shell_dev);

/* y = Op x on level `level` for nrhs stacked fields (Sec. 2.2 and Sec. 3.1).
 *   x_dev, y_dev  DEVICE, complex64 (precision HZ_C64) or complex128, N_L*nrhs.
 * HZ_OP_Q / HZ_OP_Q_ADJ require level 0.  1 <= nrhs <= max_nrhs. */
hz_status iofd_apply(hz_handle* h, int level, int op, int precision, const void* x_dev, void* y_dev, int nrhs,
                     void* stream);

/* One brick of a z-slab decomposition of the fine level (the brick-and-halo
 * form of the paper's multi-GPU runs, Sec. 6.1): rows z0 .. z1-1 of y = Op x
 * on level 0, from the brick's planes and a one-plane halo on each side.
 *   op          HZ_OP_A or HZ_OP_B.
 *   x_win_dev   DEVICE, (z1 - z0 + 2) planes of nx*ny values per right-hand side:
 *               input planes z0-1 .. z1 (a halo plane outside 0 .. nz-1 is never
 *               read; the zero boundary applies there).
 *   y_win_dev   DEVICE, (z1 - z0) planes per right-hand side: output rows z0 .. z1-1.
 *   0 <= z0 < z1 <= nz.  Each row takes the same arithmetic as in iofd_apply. */
hz_status iofd_apply_window(hz_handle* h, int op, int precision, const void* x_win_dev, void* y_win_dev, int nrhs,
                            int z0, int z1, void* stream);

/* y = J_nsweeps(H, g; omega): the weighted Jacobi map from zero of
 * Eq. jacobi-map, the smoother inside S_h (level 0, H = A_h) and inside the
 * shifted cycle V_2h^sigma and the bottom solve C_4h (levels 1 and 2, H =
 * B_ell), with the operator's own diagonal D: y_1 = omega D^-1 g and, for two
 * sweeps, y = y_1 + omega D^-1 (g - H y_1).
 *   op             HZ_OP_A on level 0, HZ_OP_B on levels 1 and 2.
 *   nsweeps        1 or 2 (Table 4 uses 2 on every level).
 *   g_dev, y_dev   DEVICE, N_L * nrhs in `precision`; distinct. */
hz_status iofd_jacobi(hz_handle* h, int level, int op, int precision, int nsweeps, double omega, const void* g_dev,
                      void* y_dev, int nrhs, void* stream);

/* r = g - Op x and norm2[k] = ||r_k||^2 for each right-hand side k, without
 * allocating device memory during the call.  The paper has no counterpart:
 * this serves callers that cannot allocate at call time (stream capture with
 * allocation forbidden, fixed-budget real-time loops, embedding hosts).  The
 * norm's grid-wide reduction keeps its per-block partial sums and arrival
 * counters in a file-scope device array of the library (512 KiB of partial
 * sums + 64 counters, held on every device that loads the library until the
 * process exits) instead of the handle's workspace.
 *   op             HZ_OP_A, HZ_OP_B, HZ_OP_A_ADJ or HZ_OP_B_ADJ.
 *   g_dev, x_dev   DEVICE inputs, r_dev DEVICE output (N_L * nrhs, `precision`);
 *                  r must not alias g or x.
 *   norm2_dev      DEVICE double, nrhs values out.
 * Limits: nrhs <= 64 and (blocks per rhs of the launch that runs -- forward
 * or adjoint, which tile differently; hz_layout_check reports both) * nrhs
 * <= 65536; larger problems return HZ_EINVAL with a message.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and should come before
 * any stream capture.  Every call shares the one array: calls that overlap on
 * the GPU (concurrent streams, several handles) race and must be serialised. */
hz_status iofd_residual_static(hz_handle* h, int level, int op, int precision, const void* g_dev, const void* x_dev,
                               void* r_dev, double* norm2_dev, int nrhs, void* stream);

/* z = M_h^{-1} r: one application of the three-grid preconditioner of
 * Algorithm 1 (pre-smooth S_h(r;0), restrict r - A_h z_pre, K_2h, prolong and
 * correct, post-smooth S_h(r; z~)), with the shifted 2h-4h cycle of
 * Eq. shifted-auxiliary-cycle inside K_2h (Eq. unshifted-middle-solve).
 * Every inner method does its fixed work; the map depends on r nonlinearly.
 *   r_dev, z_dev  DEVICE fine-grid fields (N_0 * nrhs) in `precision`.
 *   adjoint       nonzero: the same structure built from A^H, B^H (used by
 *                 the adjoint solve of the gradient).
 * The call is enqueued as one CUDA graph launch on `stream`. */
hz_status threegrid_precond(hz_handle* h, const void* r_dev, void* z_dev, int nrhs, int adjoint, int precision,
                            void* stream);

/* Solve A_h v = Q_h f for nsrc point sources (zero initial guess) with
 * FGMRES(m_out) right-preconditioned by Algorithm 1 until
 * ||A v - b|| / ||b|| <= tol for every source (Sec. 3.3, Eq. relative-residual).
 *   src_host   HOST, nsrc sources; solved in groups of at most max_nrhs.
 *   v_dev      DEVICE complex128, N_0 * nsrc: the IOFD auxiliary field v.
 *   u_dev      DEVICE complex128, N_0 * nsrc, or NULL: the pressure u = Q_h v
 *              (evaluated in the hierarchy's precision: complex64 arithmetic
 *              for HZ_C64, complex128 for HZ_C128).
 *   stats      HOST or NULL.
 * Synchronises.  Returns HZ_ENOCONV (with v, u filled) if max_pc is reached. */
hz_status helmholtz_solve(hz_handle* h, const hz_source* src_host, int nsrc, void* v_dev, void* u_dev,
                          hz_stats* stats);

/* Receiver misfit J = 1/2 sum_s || R Q_h v_s - d_s ||^2 and its gradient
 * with respect to the squared slowness m = 1/c^2 on every fine node, by the
 * adjoint-state method (forward solves, A^H lambda = Q^H R^T (R u - d),
 * row-local derivatives of A_h and Q_h).  The PML copies the nearest physical
 * velocity, so PML entries of the gradient are 0 and their contributions are
 * added to that physical node.  (Not in the paper; its Sec. 1 motivates many
 * sources for imaging and inversion.)
 *   rec_host   HOST int, nrec x 3 node indices (ix, iy, iz), distinct.
 *   dobs_host  HOST double, nsrc x nrec complex values (re, im interleaved).
 *   misfit     HOST double out.
 *   grad_dev   DEVICE double, N_0 values out.
 * Synchronises. */
hz_status helmholtz_adjoint_grad(hz_handle* h, const hz_source* src_host, int nsrc, const int* rec_host, int nrec,
                                 const double* dobs_host, double* misfit, double* grad_dev, hz_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H_ */
