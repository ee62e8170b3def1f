// Host orchestration and C ABI of the three-grid IOFD Helmholtz library.
//
// The preconditioner (Algorithm 1) does fixed work, so one application is a
// fixed sequence of kernels whose data-dependent scalars (Arnoldi
// coefficients, Givens least-squares solutions, CA-GMRES Gram/Cholesky
// solutions) stay in device memory; it is captured once per (precision,
// nrhs, adjoint, input, output) into a CUDA graph and replayed.  Only the
// outer FGMRES talks to the host: one small copy of the new Hessenberg
// column per Arnoldi step, for the FP64 Givens update and the stopping test
// of Eq. relative-residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hz.h"
#include "hz_fwd.cuh"
#include "hz_kernels.h"

using namespace hz;

std::atomic<unsigned long long> hz::g_launches{0};

namespace {

struct Fail {
  hz_status st;
  std::string msg;
};

#define HZ_CK(x)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) throw Fail{HZ_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define HZ_LAUNCHED() HZ_CK(cudaGetLastError())
#define HZ_REQUIRE(c, msg)                      \
  do {                                          \
    if (!(c)) throw Fail{HZ_EINVAL, (msg)};     \
  } while (0)

constexpr int LDMAX = 17;  // largest (restart length + 1) of any Krylov method

// ----------------------------------------------------------------------------
// device allocation bookkeeping (also used to count bytes without allocating)
// ----------------------------------------------------------------------------
struct Alloc {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  bool count_only = false;
  template <class T>
  T* get(size_t n) {
    if (n == 0) return nullptr;
    size_t b = ((n * sizeof(T)) + 255) & ~(size_t)255;
    bytes += b;
    if (count_only) return nullptr;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail{HZ_ENOMEM, "device allocation of " + std::to_string(b) + " bytes failed (" +
                                std::to_string(bytes >> 20) + " MiB requested in total)"};
    }
    ptrs.push_back(p);
    return (T*)p;
  }
  void free_all() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

struct Level {
  int nx = 0, ny = 0, nz = 0, n_pml = 0;  // nodes per axis
  long long N = 0;
  double ell = 0;
  double* kap_d = nullptr;
  float* kap_f = nullptr;
  cx<double>* abar_d[3] = {};
  cx<double>* achk_d[3] = {};
  cx<float>* abar_f[3] = {};
  cx<float>* achk_f[3] = {};
  // PML correction factors eps+- of the forward kernel per axis, and the
  // precombined coefficient polynomials of this level
  cx<double>* eps_d[3][2] = {};
  cx<float>* eps_f[3][2] = {};
  double* ctab_d = nullptr;
  float* ctab_f = nullptr;
  int plain_lo[3] = {}, plain_hi[3] = {};
  // 1/diag of the operator each Jacobi map of Algorithm 1 uses on this level
  // ([0]: A_L, [1]: B_L); complex64 set at creation, complex128 on first use
  cx<float>* dinv_f[2] = {};
  cx<double>* dinv_d[2] = {};
  int zblock = 0;    // forward-stencil planes per thread block (autotuned; 0: heuristic)
  int zblock_f = 0;  // the same for the PML-frame launch (0: as zblock)
};

template <class R>
struct Work {
  bool ready = false;
  int nrhs = 0;
  cx<R>*Vo = nullptr, *Zo = nullptr, *Vs = nullptr, *Zs = nullptr, *zpre = nullptr, *rres = nullptr;
  cx<R>*jt[3][2] = {};
  cx<R>*r2 = nullptr, *e2 = nullptr, *Vk = nullptr, *Zk = nullptr, *vy = nullptr, *vres = nullptr, *vyt = nullptr;
  cx<R>*P = nullptr, *Zc = nullptr, *e4 = nullptr;
  double *Ho = nullptr, *Hs = nullptr, *Hk = nullptr, *coef1 = nullptr, *coef2 = nullptr;
  double *beta_o = nullptr, *beta_s = nullptr, *beta_k = nullptr, *scale_o = nullptr, *scale_s = nullptr,
         *scale_k = nullptr;
  double *yo = nullptr, *ys = nullptr, *yk = nullptr, *yc = nullptr, *nrm = nullptr;
  // block FGMRES: Gram partial sums per node chunk, one Gram block, one coefficient block
  double *bpart = nullptr, *bgram = nullptr, *bcoef = nullptr;
};

template <class R> struct Sel;

}  // namespace

struct hz_handle {
  hz_grid g{};
  hz_params p{};
  int max_nrhs = 1;
  cudaStream_t st = 0;     // stream the current call enqueues on
  cudaStream_t own = 0;    // non-blocking stream owned by the handle (solves)
  cudaStream_t side = 0;   // second stream for the PML-frame launches
  int* cgs_skip = nullptr; // per rhs: second Gram-Schmidt pass not needed
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
  Alloc al;
  Level lev[3];
  double* tab_d = nullptr;
  float* tab_f = nullptr;
  int nseg = 0;
  double ds = 0;
  Work<float> wf;
  Work<double> wd;
  // complex128 vectors of the solve (rhs, solution, residual) and sources
  cx<double>*b128 = nullptr, *r128 = nullptr, *f128 = nullptr, *x128 = nullptr;
  cx<float>*b64 = nullptr, *x64 = nullptr;
  // gradient buffers
  cx<double>*vg = nullptr, *ug = nullptr, *lg = nullptr, *rf = nullptr;
  double* g_ext = nullptr;
  cx<double>* recv = nullptr;
  int* rec_dev = nullptr;
  int rec_cap = 0;
  int* src_idx = nullptr;
  double* src_amp = nullptr;
  // reductions
  double* red_partial = nullptr;
  unsigned* red_count = nullptr;
  double *s_nrm = nullptr, *s_root = nullptr, *s_inv = nullptr;
  std::map<std::tuple<int, int, int, const void*, void*>, std::pair<cudaGraphExec_t, unsigned long long>> graphs;
  double t_setup = 0;
  bool use_graphs = true;
  // the bottom solve C_4h as one persistent cooperative kernel (forward, m_4h = 4,
  // two Jacobi sweeps; opt-in through HZ_PERSISTENT=1 at creation); its
  // grid-barrier counters, error flag and Gram partials
  bool coop_bottom = false;
  unsigned* bot_bar = nullptr;
  int* bot_err = nullptr;
  double* bot_partial_f = nullptr;
  double* bot_partial_d = nullptr;
  unsigned bot_spins = 1u << 23, bot_extra = 0;
};

namespace {

template <> struct Sel<float> {
  static Work<float>& w(hz_handle* H) { return H->wf; }
  static const float* kap(const Level& L) { return L.kap_f; }
  static const cx<float>* ab(const Level& L, int a) { return L.abar_f[a]; }
  static const cx<float>* ac(const Level& L, int a) { return L.achk_f[a]; }
  static const float* tab(hz_handle* H) { return H->tab_f; }
  static const cx<float>* dinv(const Level& L, bool shifted) { return L.dinv_f[shifted ? 1 : 0]; }
  static const cx<float>* eps(const Level& L, int a, int s) { return L.eps_f[a][s]; }
  static const float* ctab(const Level& L) { return L.ctab_f; }
  static constexpr int prec = HZ_C64;
};
template <> struct Sel<double> {
  static Work<double>& w(hz_handle* H) { return H->wd; }
  static const double* kap(const Level& L) { return L.kap_d; }
  static const cx<double>* ab(const Level& L, int a) { return L.abar_d[a]; }
  static const cx<double>* ac(const Level& L, int a) { return L.achk_d[a]; }
  static const double* tab(hz_handle* H) { return H->tab_d; }
  static const cx<double>* dinv(const Level& L, bool shifted) { return L.dinv_d[shifted ? 1 : 0]; }
  static const cx<double>* eps(const Level& L, int a, int s) { return L.eps_d[a][s]; }
  static const double* ctab(const Level& L) { return L.ctab_d; }
  static constexpr int prec = HZ_C128;
};

// ----------------------------------------------------------------------------
// set-up on the host: PML factors (Eq. pml-profile, Eq. pml-second-difference)
// ----------------------------------------------------------------------------
void pml_axis(int n, int p, double gmax, std::vector<std::complex<double>>& abar,
              std::vector<std::complex<double>>& achk, int& lo, int& hi) {
  auto gam = [&](int i) {
    if (p == 0) return 0.0;
    double d = std::max(std::max((double)(p - i), (double)(i - (n - p))), 0.0);
    d = std::min(d, (double)p);  // ghost node outside the box: gamma_max
    return gmax * (1.0 - std::cos(M_PI * d / (2.0 * p)));
  };
  const std::complex<double> I(0, 1);
  abar.resize(n + 1);
  achk.resize(n + 1);
  lo = n + 1;
  hi = -1;
  for (int i = 0; i <= n; ++i) {
    double gi = gam(i), gp = gam(i + 1), gm = gam(i - 1);
    std::complex<double> xin = 1.0 / (1.0 + I * gi);
    std::complex<double> xhp = 1.0 / (1.0 + I * (0.5 * (gi + gp)));  // average gamma, then invert
    std::complex<double> xhm = 1.0 / (1.0 + I * (0.5 * (gm + gi)));
    std::complex<double> dp = xin * xhp, dm = xin * xhm;
    abar[i] = 0.5 * (dp + dm);
    achk[i] = 0.5 * (dp - dm);
    if (abar[i] == std::complex<double>(1.0, 0.0) && achk[i] == std::complex<double>(0.0, 0.0)) {
      lo = std::min(lo, i);
      hi = std::max(hi, i);
    }
  }
  if (hi < lo) {
    lo = 1;
    hi = 0;
  }
}

// cubic Hermite rows -> power basis per segment (Sec. 2.2)
void build_table(const double* rows, int K, std::vector<double>& coef, double& ds) {
  ds = rows[17] - rows[0];
  for (int k = 0; k + 1 < K; ++k)
    HZ_REQUIRE(std::fabs((rows[(k + 1) * 17] - rows[k * 17]) - ds) < 1e-9 * std::max(1.0, ds),
               "IOFD table nodes must be uniformly spaced");
  HZ_REQUIRE(std::fabs(rows[0]) < 1e-12, "IOFD table must start at s = 0");
  HZ_REQUIRE(std::fabs(rows[(K - 1) * 17] - kEtaMax) < 1e-9, "IOFD table must end at s = 0.4");
  coef.assign((size_t)kMaxSeg * kNumFn * 4, 0.0);
  for (int k = 0; k + 1 < K; ++k) {
    for (int f = 0; f < kNumFn; ++f) {
      int vc = f < 5 ? 1 + f : 11 + (f - 5);
      int dc = f < 5 ? 6 + f : 14 + (f - 5);
      double v0 = rows[k * 17 + vc], v1 = rows[(k + 1) * 17 + vc];
      double d0 = rows[k * 17 + dc], d1 = rows[(k + 1) * 17 + dc];
      double sl = (v1 - v0) / ds;
      double* c = &coef[((size_t)k * kNumFn + f) * 4];
      c[0] = v0;
      c[1] = d0;
      c[2] = (3.0 * sl - 2.0 * d0 - d1) / ds;
      c[3] = (d0 + d1 - 2.0 * sl) / (ds * ds);
    }
  }
}

// ----------------------------------------------------------------------------
// precombined coefficient polynomials of the forward kernel (hz_fwd.cuh)
// ----------------------------------------------------------------------------
using Poly = std::array<double, 6>;  // power basis, degree <= 5

Poly poly_shift(const double* c, int deg, double d) {  // p(u + d) of p(u) = sum c_i u^i
  Poly out{};
  for (int i = deg; i >= 0; --i) {  // Horner in polynomials: out = out * (u + d) + c_i
    Poly t{};
    for (int j = 0; j < 5; ++j) {
      t[j + 1] += out[j];
      t[j] += d * out[j];
    }
    t[0] += c[i];
    out = t;
  }
  return out;
}
Poly poly_lin(double a0, const Poly& p, double s) {  // a0 + s p
  Poly o{};
  for (int j = 0; j < 6; ++j) o[j] = s * p[j];
  o[0] += a0;
  return o;
}
Poly poly_add(const Poly& a, const Poly& b, double sb) {  // a + sb b
  Poly o{};
  for (int j = 0; j < 6; ++j) o[j] = a[j] + sb * b[j];
  return o;
}
Poly poly_mul_quad(const Poly& p, double q0, double q1, double q2) {  // p (q0 + q1 u + q2 u^2), deg p <= 3
  Poly o{};
  for (int j = 0; j < 4; ++j) {
    o[j] += q0 * p[j];
    o[j + 1] += q1 * p[j];
    o[j + 2] += q2 * p[j];
  }
  return o;
}

// Coefficient polynomials of one level, laid out [kind][segment][power][function]
// as hz_fwd.cuh describes.  On segment k the kernel evaluates at u = eta - s_o
// with s_o = (R)k * (R)ds rounded as it rounds it (single: float, double:
// double), so each Hermite cubic (power basis about the table node s_k) is
// re-expanded about s_o and kappa^2 = (2 pi)^2 (s_o + u)^2.  Segment nseg
// (eta >= 0.4) holds the clamped, constant alpha's and beta's.
//   C_m = (L_m - kappa^2 M_m) / ell^2,  K_m = kappa^2 M_m / ell^2,
//   L = (6 a4, a5 - a4, (1 - a4 - 2 a5) / 2, -3 (1 - a4 - a5) / 4),
//   M = (a1, a2 / 6, a3 / 12, (1 - a1 - a2 - a3) / 8),
//   Q = (b1, b2 / 6, b3 / 12, (1 - b1 - b2 - b3) / 8)
// (Eq. iofd-shell-coefficients, Eq. q-operator).
void build_coef_tables(const std::vector<double>& coef, const double* rows, int K, double ds, double ell,
                       bool single, std::vector<double>& out) {
  const int nseg = K - 1, ns = K;
  out.assign((size_t)kCtPerSeg * ns, 0.0);
  const double four_pi2 = 4.0 * M_PI * M_PI, inv_l2 = 1.0 / (ell * ell);
  for (int k = 0; k <= nseg; ++k) {
    const double s_o = single ? (double)((float)k * (float)ds) : (double)k * ds;
    Poly P[kNumFn];
    for (int f = 0; f < kNumFn; ++f) {
      if (k < nseg) {
        P[f] = poly_shift(&coef[((size_t)k * kNumFn + f) * 4], 3, s_o - rows[k * 17]);
      } else {
        P[f] = Poly{};
        P[f][0] = rows[(K - 1) * 17 + (f < 5 ? 1 + f : 11 + (f - 5))];
      }
    }
    const Poly &a1 = P[0], &a2 = P[1], &a3 = P[2], &a4 = P[3], &a5 = P[4], &b1 = P[5], &b2 = P[6], &b3 = P[7];
    Poly Lm[4], Mm[4], Qm[4];
    Lm[0] = poly_lin(0.0, a4, 6.0);
    Lm[1] = poly_add(a5, a4, -1.0);
    Lm[2] = poly_add(poly_lin(0.5, a4, -0.5), a5, -1.0);
    Lm[3] = poly_add(poly_lin(-0.75, a4, 0.75), a5, 0.75);
    Mm[0] = a1;
    Mm[1] = poly_lin(0.0, a2, 1.0 / 6.0);
    Mm[2] = poly_lin(0.0, a3, 1.0 / 12.0);
    Mm[3] = poly_add(poly_add(poly_lin(0.125, a1, -0.125), a2, -0.125), a3, -0.125);
    Qm[0] = b1;
    Qm[1] = poly_lin(0.0, b2, 1.0 / 6.0);
    Qm[2] = poly_lin(0.0, b3, 1.0 / 12.0);
    Qm[3] = poly_add(poly_add(poly_lin(0.125, b1, -0.125), b2, -0.125), b3, -0.125);
    // kappa^2 = (2 pi)^2 (s_o + u)^2
    const double q0 = four_pi2 * s_o * s_o, q1 = 2.0 * four_pi2 * s_o, q2 = four_pi2;
    for (int m = 0; m < 4; ++m) {
      const Poly Km = poly_lin(0.0, poly_mul_quad(Mm[m], q0, q1, q2), inv_l2);
      const Poly Cm = poly_add(poly_lin(0.0, Lm[m], inv_l2), Km, -1.0);
      for (int j = 0; j < 6; ++j) {
        out[(size_t)k * kCtCA + 4 * j + m] = Cm[j];
        out[ct_off_K(ns) + (size_t)k * kCtK + 4 * j + m] = Km[j];
      }
      for (int j = 0; j < 4; ++j) out[ct_off_Q(ns) + (size_t)k * kCtQ + 4 * j + m] = Qm[m][j];
    }
    for (int j = 0; j < 4; ++j) {
      out[ct_off_T(ns) + (size_t)k * kCtT + 2 * j] = a4[j];
      out[ct_off_T(ns) + (size_t)k * kCtT + 2 * j + 1] = a5[j];
    }
  }
}

template <class R>
LevelView<R> view(hz_handle* H, int L) {
  const Level& lv = H->lev[L];
  LevelView<R> v;
  v.level = L;
  v.nx = lv.nx;
  v.ny = lv.ny;
  v.nz = lv.nz;
  v.N = lv.N;
  v.kappa = Sel<R>::kap(lv);
  for (int a = 0; a < 3; ++a) {
    v.abar[a] = Sel<R>::ab(lv, a);
    v.achk[a] = Sel<R>::ac(lv, a);
    v.eps[a][0] = Sel<R>::eps(lv, a, 0);
    v.eps[a][1] = Sel<R>::eps(lv, a, 1);
    v.plain_lo[a] = lv.plain_lo[a];
    v.plain_hi[a] = lv.plain_hi[a];
  }
  v.ctab = Sel<R>::ctab(lv);
  v.inv_ell2 = (R)(1.0 / (lv.ell * lv.ell));
  v.zblock = lv.zblock;
  v.zblock_f = lv.zblock_f;
  return v;
}
template <class R>
TableView<R> tview(hz_handle* H) {
  TableView<R> t;
  t.coef = Sel<R>::tab(H);
  t.nseg = H->nseg;
  t.ds = (R)H->ds;
  t.inv_ds = (R)(1.0 / H->ds);
  return t;
}

// Jacobi diagonals used by Algorithm 1: A_h on level 0, B_2h and B_4h (Eq. jacobi-map).
template <class R>
void compute_dinv(hz_handle* H, cx<R>* (&d0)[2], cx<R>* (&d1)[2], cx<R>* (&d2)[2]) {
  const cx<R> one = mkc<R>((R)1, (R)0), sh = mkc<R>((R)1, (R)H->p.sigma);
  launch_setup_dinv<R>(view<R>(H, 0), tview<R>(H), one, d0[0], H->st);
  launch_setup_dinv<R>(view<R>(H, 1), tview<R>(H), sh, d1[1], H->st);
  launch_setup_dinv<R>(view<R>(H, 2), tview<R>(H), sh, d2[1], H->st);
}

void prepare_dinv_double(hz_handle* H) {
  if (H->lev[0].dinv_d[0]) return;
  H->lev[0].dinv_d[0] = H->al.get<cx<double>>(H->lev[0].N);
  H->lev[1].dinv_d[1] = H->al.get<cx<double>>(H->lev[1].N);
  H->lev[2].dinv_d[1] = H->al.get<cx<double>>(H->lev[2].N);
  compute_dinv<double>(H, H->lev[0].dinv_d, H->lev[1].dinv_d, H->lev[2].dinv_d);
  HZ_CK(cudaGetLastError());
}

Reduce reducer(hz_handle* H, double* out, double* root = nullptr, double* inv = nullptr) {
  Reduce r;
  r.partial = H->red_partial;
  r.count = H->red_count;
  r.out = out;
  r.root = root;
  r.inv_root = inv;
  return r;
}

// ----------------------------------------------------------------------------
// operator building blocks
// ----------------------------------------------------------------------------
template <class R>
StencilCall<R> call(hz_handle* H, int L, bool shifted, int nrhs) {
  StencilCall<R> c;
  c.lv = view<R>(H, L);
  c.tab = tview<R>(H);
  c.mass_shift = mkc<R>((R)1, shifted ? (R)H->p.sigma : (R)0);
  c.nrhs = nrhs;
  c.side = H->side;
  c.fork = H->ev_fork;
  c.join = H->ev_join;
  return c;
}

template <class R>
void apply(hz_handle* H, int L, bool shifted, bool adj, const cx<R>* x, cx<R>* y, int nrhs) {
  StencilCall<R> c = call<R>(H, L, shifted, nrhs);
  c.x = x;
  c.y = y;
  launch_stencil<R>(c, M_APPLY, OP_AB, adj, H->st);
  HZ_LAUNCHED();
}

template <class R>
void resid(hz_handle* H, int L, bool shifted, bool adj, const cx<R>* g, const cx<R>* x, cx<R>* y, int nrhs,
           Reduce red = Reduce()) {
  StencilCall<R> c = call<R>(H, L, shifted, nrhs);
  c.x = x;
  c.g = g;
  c.y = y;
  c.red = red;
  launch_stencil<R>(c, M_RESID, OP_AB, adj, H->st);
  HZ_LAUNCHED();
}

template <class R>
void q_apply(hz_handle* H, bool adj, const cx<R>* x, cx<R>* y, int nrhs) {
  StencilCall<R> c = call<R>(H, 0, false, nrhs);
  c.x = x;
  c.y = y;
  launch_stencil<R>(c, M_APPLY, OP_Q, adj, H->st);
  HZ_LAUNCHED();
}

// y = J_nJ(H_L, g; w) (Eq. jacobi-map), optionally out = base + J(...)
template <class R>
void jacobi(hz_handle* H, int L, bool shifted, bool adj, const cx<R>* g, cx<R>* y, int nJ, double w, int nrhs,
            const cx<R>* base = nullptr) {
  Work<R>& W = Sel<R>::w(H);
  StencilCall<R> c = call<R>(H, L, shifted, nrhs);
  c.omega_j = (R)w;
  const long long n = H->lev[L].N * nrhs;
  if (nJ == 1) {
    c.x = g;
    c.y = y;
    c.base = base;
    launch_stencil<R>(c, M_J1, OP_AB, adj, H->st);
    HZ_LAUNCHED();
    return;
  }
  c.dinv = Sel<R>::dinv(H->lev[L], shifted);
  HZ_REQUIRE(adj || c.dinv, "internal: Jacobi diagonal of this level/operator was not prepared");
  if (nJ == 2) {
    c.x = g;
    c.y = y;
    c.base = base;
    launch_stencil<R>(c, M_J2, OP_AB, adj, H->st);
    HZ_LAUNCHED();
    return;
  }
  // nJ > 2: two fused sweeps, then single sweeps ping-ponging between temporaries
  cx<R>* a = W.jt[L][0];
  cx<R>* b = W.jt[L][1];
  c.x = g;
  c.y = a;
  c.base = nullptr;
  launch_stencil<R>(c, M_J2, OP_AB, adj, H->st);
  HZ_LAUNCHED();
  for (int s = 2; s < nJ; ++s) {
    StencilCall<R> d = c;
    d.x = a;
    d.g = g;
    d.y = b;
    launch_stencil<R>(d, M_JSWEEP, OP_AB, adj, H->st);
    HZ_LAUNCHED();
    std::swap(a, b);
  }
  if (base) {
    launch_copy<R>(base, y, n, H->st);
    launch_axpy<R>(a, y, 1.0, 0.0, n, H->st);
  } else {
    launch_copy<R>(a, y, n, H->st);
  }
  HZ_LAUNCHED();
}

// Arnoldi step j on device: w = V[j+1] holds A z_j; orthogonalise against
// V[0..j] by classical Gram-Schmidt with one reorthogonalisation, write the
// Hessenberg column j and normalise V[j+1].
template <class R>
void arnoldi_orth(hz_handle* H, int L, int nrhs, cx<R>* V, int j, double* Hm, int m, double* scale) {
  Work<R>& W = Sel<R>::w(H);
  KrylovCall k;
  k.n = (int)H->lev[L].N;
  k.nrhs = nrhs;
  k.vstride = H->lev[L].N * nrhs;
  k.kn = j + 1;
  k.ld = m + 1;
  cx<R>* w = V + (j + 1) * k.vstride;
  Reduce red = reducer(H, nullptr);
  k.skip = H->cgs_skip;
  k.coef_final = W.coef2;
  // pass 1: h1 = V^H w and ||w||^2 (decides whether pass 2 is needed)
  launch_cgs<R>(k, V, w, nullptr, false, true, true, W.coef1, nullptr, EPI_ARNOLDI_FIRST, Hm, j, scale, nullptr,
                red, H->st);
  // pass 2: w -= V h1, then h2 = V^H w and ||w||^2 -> column += h2, subdiagonal, 1/norm
  launch_cgs<R>(k, V, w, W.coef1, true, true, true, W.coef2, nullptr, EPI_ARNOLDI_SECOND, Hm, j, scale, nullptr,
                red, H->st);
  // pass 3: v_{j+1} = (w - V h2) / norm
  launch_update_scale<R>(k, V, w, W.coef2, scale, H->st);
  HZ_LAUNCHED();
}

// One right-preconditioned (flexible) GMRES cycle of m steps on A_L (unshifted)
// for A x = g from x0 (nullptr = 0); x may equal x0.  Minv(v, z) applies the
// right preconditioner.  All scalars stay on the device.
template <class R, class MF>
void gmres_cycle(hz_handle* H, int L, bool adj, const cx<R>* g, const cx<R>* x0, cx<R>* x, int m, MF Minv, cx<R>* V,
                 cx<R>* Z, double* Hm, double* beta, double* scale, double* y, int nrhs) {
  Work<R>& W = Sel<R>::w(H);
  const int n = (int)H->lev[L].N;
  const long long vs = H->lev[L].N * nrhs;
  if (x0) {
    resid<R>(H, L, false, adj, g, x0, V, nrhs, reducer(H, W.nrm, beta, scale));
  } else {
    KrylovCall k;
    k.n = n;
    k.nrhs = nrhs;
    k.kn = 0;
    k.ld = m + 1;
    launch_cgs<R>(k, g, const_cast<cx<R>*>(g), nullptr, false, false, true, nullptr, nullptr, EPI_NORMALISE, nullptr,
                  -1, scale, beta, reducer(H, nullptr), H->st);
    HZ_LAUNCHED();
  }
  launch_scale<R>(x0 ? V : g, V, scale, n, nrhs, H->st);
  HZ_LAUNCHED();
  for (int j = 0; j < m; ++j) {
    Minv(V + j * vs, Z + j * vs);
    apply<R>(H, L, false, adj, Z + j * vs, V + (j + 1) * vs, nrhs);
    arnoldi_orth<R>(H, L, nrhs, V, j, Hm, m, scale);
  }
  launch_lsq(Hm, beta, y, m, m + 1, nrhs, H->st, sizeof(R) == sizeof(float));
  launch_combine<R>(Z, vs, m, y, m + 1, x0, x, n, nrhs, H->st);
  HZ_LAUNCHED();
}

// C_4h: m_4h CA-GMRES steps on B_4h e = g from zero, right-preconditioned by
// J_{nJ,4h}(B_4h, .; w_4h).  P[0] holds g on entry.  Monomial s-step basis
// p_{k+1} = B J(p_k), one Gram pass, Cholesky QR and the small least squares.
template <class R>
void bottom_4h(hz_handle* H, bool adj, cx<R>* e, int nrhs) {
  Work<R>& W = Sel<R>::w(H);
  const hz_params& p = H->p;
  const long long vs = H->lev[2].N * nrhs;
  const int s = p.m_4h;
  // the persistent form where launch latency dominates: 4h grids below 2^20 nodes
  // (larger ones keep the tuned rectangle/frame launches)
  if (H->coop_bottom && !adj && s == gather::kBottomSteps && p.nJ_4h == 2 && H->lev[2].N < (1LL << 20)) {
    gather::BottomArgs<R> b;
    b.c = call<R>(H, 2, true, nrhs);
    b.c.omega_j = (R)p.w_4h;
    b.c.dinv = Sel<R>::dinv(H->lev[2], true);
    HZ_REQUIRE(b.c.dinv, "internal: Jacobi diagonal of B_4h was not prepared");
    b.P = W.P;
    b.Zc = W.Zc;
    b.vs = vs;
    b.e = e;
    b.y = W.yc;
    b.ld = s + 1;
    b.partial = sizeof(R) == 4 ? H->bot_partial_f : H->bot_partial_d;
    b.bar = H->bot_bar;
    b.err = H->bot_err;
    b.spins = H->bot_spins;
    b.extra = H->bot_extra;
    if (!gather::launch_bottom4h<R>(b, H->st)) {
      H->coop_bottom = false;
      cudaGetLastError();
      throw Fail{HZ_ECUDA, "cooperative launch of the persistent bottom solve failed (disabled for this handle)"};
    }
    HZ_LAUNCHED();
    return;
  }
  for (int k = 0; k < s; ++k) {
    jacobi<R>(H, 2, true, adj, W.P + k * vs, W.Zc + k * vs, p.nJ_4h, p.w_4h, nrhs);
    apply<R>(H, 2, true, adj, W.Zc + k * vs, W.P + (k + 1) * vs, nrhs);
  }
  launch_gram_lsq<R>(W.P, vs, s + 1, (int)H->lev[2].N, nrhs, W.yc, s + 1, reducer(H, nullptr), H->st);
  launch_combine<R>(W.Zc, vs, s, W.yc, s + 1, nullptr, e, (int)H->lev[2].N, nrhs, H->st);
  HZ_LAUNCHED();
}

// V_2h^sigma (Eq. shifted-auxiliary-cycle): q -> out on the 2h grid.
template <class R>
void vcycle(hz_handle* H, bool adj, const cx<R>* q, cx<R>* out, int nrhs) {
  Work<R>& W = Sel<R>::w(H);
  const hz_params& p = H->p;
  const Level& L1 = H->lev[1];
  jacobi<R>(H, 1, true, adj, q, W.vy, p.nJ_2h, p.w_2h, nrhs);                 // y = J(B, q)
  resid<R>(H, 1, true, adj, q, W.vy, W.vres, nrhs);                           // q - B y
  launch_restrict<R>(W.vres, W.P, L1.nx, L1.ny, L1.nz, nrhs, H->st);           // q_4h -> P[0]
  HZ_LAUNCHED();
  bottom_4h<R>(H, adj, W.e4, nrhs);                                            // e_4h = C_4h(q_4h)
  launch_prolong_add<R>(W.e4, W.vy, W.vyt, L1.nx, L1.ny, L1.nz, nrhs, H->st);  // y~ = y + P e
  HZ_LAUNCHED();
  resid<R>(H, 1, true, adj, q, W.vyt, W.vres, nrhs);                          // q - B y~
  jacobi<R>(H, 1, true, adj, W.vres, out, p.nJ_2h, p.w_2h, nrhs, W.vyt);      // y~ + J(B, .)
}

// Algorithm 1: z = M_h^{-1} r.
template <class R>
void precond_enqueue(hz_handle* H, const cx<R>* r, cx<R>* z, int nrhs, bool adj) {
  Work<R>& W = Sel<R>::w(H);
  const hz_params& p = H->p;
  const Level& L0 = H->lev[0];
  auto Mh = [&](const cx<R>* v, cx<R>* zz) { jacobi<R>(H, 0, false, adj, v, zz, p.nJ_h, p.w_h, nrhs); };
  auto M2 = [&](const cx<R>* v, cx<R>* zz) { vcycle<R>(H, adj, v, zz, nrhs); };
  // 1: pre-smooth S_h(r; 0)
  gmres_cycle<R>(H, 0, adj, r, nullptr, W.zpre, p.m_h, Mh, W.Vs, W.Zs, W.Hs, W.beta_s, W.scale_s, W.ys, nrhs);
  // 2: restrict the fine residual
  resid<R>(H, 0, false, adj, r, W.zpre, W.rres, nrhs);
  launch_restrict<R>(W.rres, W.r2, L0.nx, L0.ny, L0.nz, nrhs, H->st);
  HZ_LAUNCHED();
  // 3: K_2h = c_2h FGMRES(m_2h) cycles on A_2h from zero, right PC V_2h^sigma
  for (int c = 0; c < p.c_2h; ++c)
    gmres_cycle<R>(H, 1, adj, W.r2, c == 0 ? nullptr : W.e2, W.e2, p.m_2h, M2, W.Vk, W.Zk, W.Hk, W.beta_k, W.scale_k,
                   W.yk, nrhs);
  // 4: prolong and correct
  launch_prolong_add<R>(W.e2, W.zpre, W.zpre, L0.nx, L0.ny, L0.nz, nrhs, H->st);
  HZ_LAUNCHED();
  // 5: post-smooth S_h(r; z~)
  gmres_cycle<R>(H, 0, adj, r, W.zpre, z, p.m_h, Mh, W.Vs, W.Zs, W.Hs, W.beta_s, W.scale_s, W.ys, nrhs);
}

void destroy_streams(hz_handle* H) {
  if (H->ev_fork) cudaEventDestroy(H->ev_fork);
  if (H->ev_join) cudaEventDestroy(H->ev_join);
  if (H->side) cudaStreamDestroy(H->side);
  if (H->own) cudaStreamDestroy(H->own);
}

void drop_graphs(hz_handle* H) {
  for (auto& kv : H->graphs) cudaGraphExecDestroy(kv.second.first);
  H->graphs.clear();
}

template <class R>
void precond(hz_handle* H, const cx<R>* r, cx<R>* z, int nrhs, bool adj) {
  // the legacy default stream cannot be captured: enqueue directly there
  if (!H->use_graphs || H->st == 0 || H->st == cudaStreamLegacy || H->st == cudaStreamPerThread) {
    precond_enqueue<R>(H, r, z, nrhs, adj);
    return;
  }
  auto key = std::make_tuple(Sel<R>::prec, nrhs, adj ? 1 : 0, (const void*)r, (void*)z);
  auto it = H->graphs.find(key);
  if (it == H->graphs.end()) {
    if (H->graphs.size() >= 64) drop_graphs(H);  // bound the cache (new buffers each call)
    cudaGraph_t graph = nullptr;
    const unsigned long long c0 = g_launches.load();
    HZ_CK(cudaStreamBeginCapture(H->st, cudaStreamCaptureModeThreadLocal));
    try {
      precond_enqueue<R>(H, r, z, nrhs, adj);
    } catch (...) {
      cudaStreamEndCapture(H->st, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      g_launches.store(c0);
      throw;
    }
    HZ_CK(cudaStreamEndCapture(H->st, &graph));
    const unsigned long long nodes = g_launches.load() - c0;  // kernels recorded, not run
    g_launches.store(c0);
    cudaGraphExec_t exec;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    HZ_CK(e);
    it = H->graphs.emplace(key, std::make_pair(exec, nodes)).first;
  }
  HZ_CK(cudaGraphLaunch(it->second.first, H->st));
  count_launch(it->second.second);
}

// ----------------------------------------------------------------------------
// workspaces
// ----------------------------------------------------------------------------
template <class R>
void plan_work(Alloc& al, Work<R>& W, const Level* lev, const hz_params& p, int nrhs) {
  auto vec = [&](int L, int count) { return al.get<cx<R>>((size_t)lev[L].N * nrhs * count); };
  W.nrhs = nrhs;
  W.Vo = vec(0, p.m_out + 1);
  W.Zo = vec(0, p.m_out);
  W.Vs = vec(0, p.m_h + 1);
  W.Zs = vec(0, p.m_h);
  W.zpre = vec(0, 1);
  W.rres = vec(0, 1);
  W.r2 = vec(1, 1);
  W.e2 = vec(1, 1);
  W.Vk = vec(1, p.m_2h + 1);
  W.Zk = vec(1, p.m_2h);
  W.vy = vec(1, 1);
  W.vres = vec(1, 1);
  W.vyt = vec(1, 1);
  W.P = vec(2, p.m_4h + 1);
  W.Zc = vec(2, p.m_4h);
  W.e4 = vec(2, 1);
  const int nj[3] = {p.nJ_h, p.nJ_2h, p.nJ_4h};
  for (int L = 0; L < 3; ++L)
    if (nj[L] > 2) {
      W.jt[L][0] = vec(L, 1);
      W.jt[L][1] = vec(L, 1);
    }
  auto sc = [&](size_t n) { return al.get<double>(n); };
  W.Ho = sc((size_t)nrhs * (p.m_out + 1) * p.m_out * 2);
  W.Hs = sc((size_t)nrhs * (p.m_h + 1) * p.m_h * 2);
  W.Hk = sc((size_t)nrhs * (p.m_2h + 1) * p.m_2h * 2);
  W.coef1 = sc((size_t)nrhs * LDMAX * 2);
  W.coef2 = sc((size_t)nrhs * LDMAX * 2);
  W.yo = sc((size_t)nrhs * LDMAX * 2);
  W.ys = sc((size_t)nrhs * LDMAX * 2);
  W.yk = sc((size_t)nrhs * LDMAX * 2);
  W.yc = sc((size_t)nrhs * LDMAX * 2);
  W.beta_o = sc(nrhs);
  W.beta_s = sc(nrhs);
  W.beta_k = sc(nrhs);
  W.scale_o = sc(nrhs);
  W.scale_s = sc(nrhs);
  W.scale_k = sc(nrhs);
  W.nrm = sc(nrhs);
  if (nrhs >= 2) {
    const int S = std::min(nrhs, kBlockMaxS);
    W.bpart = sc(block_gram_partial_doubles(lev[0].N, p.m_out * S, S));
    W.bgram = sc((size_t)p.m_out * S * S * 2);
    W.bcoef = sc((size_t)p.m_out * S * S * 2);
  }
  W.ready = !al.count_only;
}

void check_params(const hz_params& p) {
  HZ_REQUIRE(p.m_out >= 1 && p.m_out <= LDMAX - 1, "m_out must be in [1, 16]");
  HZ_REQUIRE(p.m_h >= 1 && p.m_h <= LDMAX - 1, "m_h must be in [1, 16]");
  HZ_REQUIRE(p.m_2h >= 1 && p.m_2h <= LDMAX - 1, "m_2h must be in [1, 16]");
  HZ_REQUIRE(p.m_4h >= 1 && p.m_4h <= 6, "m_4h must be in [1, 6]");
  HZ_REQUIRE(p.c_2h >= 1, "c_2h must be >= 1");
  HZ_REQUIRE(p.nJ_h >= 1 && p.nJ_2h >= 1 && p.nJ_4h >= 1, "Jacobi sweep counts must be >= 1");
  HZ_REQUIRE(p.tol > 0 && p.max_pc >= 1, "tol must be > 0 and max_pc >= 1");
  HZ_REQUIRE(p.precision == HZ_C64 || p.precision == HZ_C128, "precision must be HZ_C64 or HZ_C128");
  HZ_REQUIRE(p.block == 0 || p.block == 1, "block must be 0 or 1");
}

void check_grid(const hz_grid& g) {
  HZ_REQUIRE(g.nx >= 4 && g.ny >= 4 && g.nz >= 4, "grid needs at least 4 intervals per axis");
  HZ_REQUIRE(g.nx % 4 == 0 && g.ny % 4 == 0 && g.nz % 4 == 0, "intervals per axis must be divisible by 4");
  HZ_REQUIRE(g.n_pml >= 0 && g.n_pml % 4 == 0, "n_pml must be a non-negative multiple of 4");
  HZ_REQUIRE(2 * g.n_pml < std::min(g.nx, std::min(g.ny, g.nz)), "PML layers leave no physical domain");
  HZ_REQUIRE(g.h > 0 && g.omega > 0 && g.gamma_max >= 0, "h and omega must be positive, gamma_max >= 0");
  HZ_REQUIRE((long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1) < (1LL << 31), "grid too large (2^31 nodes)");
}

void level_dims(const hz_grid& g, int L, Level& lv) {
  int f = 1 << L;
  lv.nx = g.nx / f + 1;
  lv.ny = g.ny / f + 1;
  lv.nz = g.nz / f + 1;
  lv.n_pml = g.n_pml / f;
  lv.N = (long long)lv.nx * lv.ny * lv.nz;
  lv.ell = g.h * f;
  // PML-free index ranges (the launch layout and its block counts depend on them)
  const int nn[3] = {g.nx / f, g.ny / f, g.nz / f};
  std::vector<std::complex<double>> ab, ac;
  for (int a = 0; a < 3; ++a) pml_axis(nn[a], lv.n_pml, g.gamma_max, ab, ac, lv.plain_lo[a], lv.plain_hi[a]);
}

// Block partial sums of one fused stencil reduction (forward or adjoint
// launch) on level lv with nrhs right-hand sides, at the z-blocks it will run.
long long resid_blocks(const Level& lv, int level, int nrhs, bool adjoint) {
  return adjoint ? adj_blocks_per_rhs(lv.nx, lv.ny, lv.nz, nrhs)
                 : stencil_blocks_per_rhs(level, lv.nx, lv.ny, lv.nz, lv.plain_lo, lv.plain_hi, nrhs, lv.zblock,
                                          lv.zblock_f);
}

// Per-block partial sums: the vector reductions use at most 1216 x 56, a fused
// stencil reduction one per block -- forward or adjoint launch -- at the
// smallest z-block (4 planes) the planners or the autotuner can pick.
size_t red_partial_size(const Level* lev, int nrhs) {
  size_t m = 1216 * 56;
  for (int L = 0; L < 3; ++L) {
    const long long f = stencil_blocks_per_rhs(L, lev[L].nx, lev[L].ny, lev[L].nz, lev[L].plain_lo, lev[L].plain_hi,
                                               1, kMinZblock, kMinZblock);
    const long long a = adj_blocks_per_rhs(lev[L].nx, lev[L].ny, lev[L].nz, 1, kMinZblock);
    m = std::max(m, (size_t)std::max(f, a));
  }
  return m * nrhs;
}

// Allocation plan shared by hz_create and hz_workspace_bytes.
void plan_all(hz_handle* H, bool count_only) {
  Alloc& al = H->al;
  al.count_only = count_only;
  for (int L = 0; L < 3; ++L) {
    Level& lv = H->lev[L];
    level_dims(H->g, L, lv);
    lv.kap_d = al.get<double>(lv.N);
    lv.kap_f = al.get<float>(lv.N);
    const int nn[3] = {lv.nx, lv.ny, lv.nz};
    for (int a = 0; a < 3; ++a) {
      lv.abar_d[a] = al.get<cx<double>>(nn[a]);
      lv.achk_d[a] = al.get<cx<double>>(nn[a]);
      lv.abar_f[a] = al.get<cx<float>>(nn[a]);
      lv.achk_f[a] = al.get<cx<float>>(nn[a]);
      for (int sgn = 0; sgn < 2; ++sgn) {
        lv.eps_d[a][sgn] = al.get<cx<double>>(nn[a]);
        lv.eps_f[a][sgn] = al.get<cx<float>>(nn[a]);
      }
    }
    lv.ctab_d = al.get<double>((size_t)kCtPerSeg * (kMaxSeg + 1));
    lv.ctab_f = al.get<float>((size_t)kCtPerSeg * (kMaxSeg + 1));
  }
  H->lev[0].dinv_f[0] = al.get<cx<float>>(H->lev[0].N);
  H->lev[1].dinv_f[1] = al.get<cx<float>>(H->lev[1].N);
  H->lev[2].dinv_f[1] = al.get<cx<float>>(H->lev[2].N);
  H->tab_d = al.get<double>((size_t)kMaxSeg * kNumFn * 4);
  H->tab_f = al.get<float>((size_t)kMaxSeg * kNumFn * 4);
  const int nr = H->max_nrhs;
  H->red_partial = al.get<double>(red_partial_size(H->lev, nr));
  H->red_count = al.get<unsigned>(nr);
  H->cgs_skip = al.get<int>(nr);
  H->s_nrm = al.get<double>(nr);
  H->s_root = al.get<double>(nr);
  H->s_inv = al.get<double>(nr);
  H->src_idx = al.get<int>((size_t)3 * nr);
  H->src_amp = al.get<double>((size_t)2 * nr);
  const size_t N0 = (size_t)H->lev[0].N * nr;
  H->b128 = al.get<cx<double>>(N0);
  H->f128 = al.get<cx<double>>(N0);
  H->r128 = al.get<cx<double>>(N0);
  if (H->p.precision == HZ_C64) {
    plan_work<float>(al, H->wf, H->lev, H->p, nr);
    H->b64 = al.get<cx<float>>(N0);
    H->x64 = al.get<cx<float>>(N0);
  } else {
    plan_work<double>(al, H->wd, H->lev, H->p, nr);
  }
}

void prepare_dinv_double(hz_handle* H);

template <class R>
void ensure_work(hz_handle* H) {
  Work<R>& W = Sel<R>::w(H);
  if (W.ready) return;
  H->al.count_only = false;
  plan_work<R>(H->al, W, H->lev, H->p, H->max_nrhs);
  if (sizeof(R) == sizeof(double)) prepare_dinv_double(H);
}

// Launch-shape autotuner: on every level, time the forward stencil (the A_h
// apply on the fine level, the Jacobi map of B on the coarse levels; nrhs =
// max_nrhs, the hierarchy's precision) for a set of z-block sizes on two
// workspace vectors and keep the fastest; where the level splits into the
// PML-free rectangle and the PML frame, the frame's z-block is then tuned with
// the rectangle's fixed.  Runs once, at creation.
// Tuned z-blocks are kept per process, keyed by device, precision, right-hand
// sides and level shapes, so handles created again for the same problem size
// skip the timing.
struct TuneKey {
  int dev, prec, nrhs, dims[9];
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, prec, nrhs) < std::tie(o.dev, o.prec, o.nrhs) ||
           (std::tie(dev, prec, nrhs) == std::tie(o.dev, o.prec, o.nrhs) &&
            std::lexicographical_compare(dims, dims + 9, o.dims, o.dims + 9));
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 6>> g_tune_cache;

template <class R>
void autotune_zblocks(hz_handle* H) {
  Work<R>& W = Sel<R>::w(H);
  const int nr = H->max_nrhs;
  TuneKey key{};
  HZ_CK(cudaGetDevice(&key.dev));
  key.prec = (int)sizeof(R);
  key.nrhs = nr;
  for (int L = 0; L < 3; ++L) {
    key.dims[3 * L] = H->lev[L].nx;
    key.dims[3 * L + 1] = H->lev[L].ny;
    key.dims[3 * L + 2] = H->lev[L].nz * 1024 + H->lev[L].n_pml;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int L = 0; L < 3; ++L) {
        H->lev[L].zblock = it->second[2 * L];
        H->lev[L].zblock_f = it->second[2 * L + 1];
      }
      return;
    }
  }
  cx<R>* src[3] = {W.Vo, W.Vk, W.P};
  cudaEvent_t e0, e1;
  HZ_CK(cudaEventCreate(&e0));
  HZ_CK(cudaEventCreate(&e1));
  const int cand[] = {kMinZblock, 3, 4, 6, 8, 10, 12, 16, 22, 28, 34, 46, 64};
  for (int L = 0; L < 3; ++L) {
    Level& lv = H->lev[L];
    const long long n = lv.N * nr;
    launch_zero<R>(src[L], n, H->st);
    HZ_LAUNCHED();
    // the launch each level runs most: the A_h apply on the fine level, the
    // two-sweep Jacobi map of the shifted operator on the coarse levels
    // (the V-cycle and the bottom solve)
    const int mode = L == 0 ? M_APPLY : M_J2;
    auto time_apply = [&]() {
      StencilCall<R> c = call<R>(H, L, L > 0, nr);
      c.x = src[L];
      c.y = src[L] + n;  // the next basis vector of the same workspace
      if (L > 0) {
        c.dinv = Sel<R>::dinv(H->lev[L], true);
        c.omega_j = (R)(L == 1 ? H->p.w_2h : H->p.w_4h);
      }
      launch_stencil<R>(c, mode, OP_AB, false, H->st);  // warm-up
      float ms = 0.f;
      // short launches (coarse levels) are timed over more repetitions
      for (int reps : {3, 24}) {
        HZ_CK(cudaEventRecord(e0, H->st));
        for (int rep = 0; rep < reps; ++rep) launch_stencil<R>(c, mode, OP_AB, false, H->st);
        HZ_CK(cudaEventRecord(e1, H->st));
        HZ_LAUNCHED();
        HZ_CK(cudaEventSynchronize(e1));
        HZ_CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= (float)reps;
        if (ms * reps >= 0.2f) break;
      }
      return ms;
    };
    const bool split =
        stencil_blocks_per_rhs(L, lv.nx, lv.ny, lv.nz, lv.plain_lo, lv.plain_hi, nr, kMinZblock, 64) !=
        stencil_blocks_per_rhs(L, lv.nx, lv.ny, lv.nz, lv.plain_lo, lv.plain_hi, nr, kMinZblock, kMinZblock);
    for (int pass = 0; pass < (split ? 2 : 1); ++pass) {
      float best_t = 1e30f;
      int best = 0;
      for (int zb : cand) {
        if (zb > lv.nz && zb != cand[0]) continue;
        if (pass == 0) lv.zblock = zb;
        lv.zblock_f = zb;
        const float ms = time_apply();
        if (ms < best_t) {
          best_t = ms;
          best = zb;
        }
      }
      if (pass == 0) lv.zblock = best;
      lv.zblock_f = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::array<int, 6> tuned;
  for (int L = 0; L < 3; ++L) {
    tuned[2 * L] = H->lev[L].zblock;
    tuned[2 * L + 1] = H->lev[L].zblock_f;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = tuned;
}

std::vector<double> host_copy(const double* d, int n, cudaStream_t st) {
  std::vector<double> h(n);
  HZ_CK(cudaMemcpyAsync(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  HZ_CK(cudaStreamSynchronize(st));
  return h;
}

// ----------------------------------------------------------------------------
// outer FGMRES(m_out) with FP64 Givens on the host (Sec. 3.3, Table 4)
// ----------------------------------------------------------------------------
// With `inner` set (the complex64 correction solve of the refinement loop) a
// cycle whose Arnoldi estimate reaches tol ends the solve without a further
// true residual, and the solve also ends when a restart cycle no longer
// reduces the true residual by 10%: the FP64 refinement loop measures and
// corrects what complex64 cannot resolve.
template <class R>
double outer_fgmres(hz_handle* H, const cx<R>* b, cx<R>* x, int nrhs, bool adj, const std::vector<double>& bn,
                    double tol, int max_pc, int& pc, bool inner = false) {
  Work<R>& W = Sel<R>::w(H);
  const int m = H->p.m_out, ld = m + 1;
  const long long N = H->lev[0].N, vs = N * nrhs;
  double relmax = 0.0, prev_rel = HUGE_VAL;
  bool est_converged = false;
  for (;;) {
    resid<R>(H, 0, false, adj, b, x, W.Vo, nrhs, reducer(H, W.nrm, W.beta_o, W.scale_o));
    std::vector<double> beta = host_copy(W.beta_o, nrhs, H->st);
    relmax = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      if (!std::isfinite(beta[r])) throw Fail{HZ_ENONFINITE, "non-finite residual norm in the outer FGMRES"};
      relmax = std::max(relmax, bn[r] > 0 ? beta[r] / bn[r] : 0.0);
    }
    if (relmax <= tol || pc >= max_pc) break;
    if (inner && relmax > 0.9 * prev_rel) break;  // complex64 stagnation: hand back to the refinement
    prev_rel = relmax;
    launch_scale<R>(W.Vo, W.Vo, W.scale_o, (int)N, nrhs, H->st);
    HZ_LAUNCHED();
    using C = std::complex<double>;
    std::vector<std::vector<C>> Rm(nrhs, std::vector<C>((size_t)ld * m)), gv(nrhs, std::vector<C>(ld));
    std::vector<std::vector<double>> cs(nrhs, std::vector<double>(m));
    std::vector<std::vector<C>> sn(nrhs, std::vector<C>(m));
    for (int r = 0; r < nrhs; ++r) gv[r][0] = beta[r];
    std::vector<double> hcol((size_t)nrhs * ld * m * 2);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      precond<R>(H, W.Vo + j * vs, W.Zo + j * vs, nrhs, adj);
      ++pc;
      apply<R>(H, 0, false, adj, W.Zo + j * vs, W.Vo + (j + 1) * vs, nrhs);
      arnoldi_orth<R>(H, 0, nrhs, W.Vo, j, W.Ho, m, W.scale_o);
      HZ_CK(cudaMemcpyAsync(hcol.data(), W.Ho, hcol.size() * sizeof(double), cudaMemcpyDeviceToHost, H->st));
      HZ_CK(cudaStreamSynchronize(H->st));
      bool all_conv = true, breakdown = false;
      for (int r = 0; r < nrhs; ++r) {
        const double* Hr = hcol.data() + ((size_t)r * m + j) * ld * 2;
        std::vector<C>& Rr = Rm[r];
        for (int i = 0; i <= j + 1; ++i) Rr[(size_t)j * ld + i] = C(Hr[2 * i], Hr[2 * i + 1]);
        for (int i = 0; i < j; ++i) {  // previous rotations
          C t1 = Rr[(size_t)j * ld + i], t2 = Rr[(size_t)j * ld + i + 1];
          Rr[(size_t)j * ld + i] = cs[r][i] * t1 + sn[r][i] * t2;
          Rr[(size_t)j * ld + i + 1] = cs[r][i] * t2 - std::conj(sn[r][i]) * t1;
        }
        C a = Rr[(size_t)j * ld + j], bb = Rr[(size_t)j * ld + j + 1];
        double na = std::abs(a), nb = std::abs(bb), rr = std::hypot(na, nb);
        if (rr == 0.0) {
          cs[r][j] = 1.0;
          sn[r][j] = 0.0;
        } else if (na == 0.0) {
          cs[r][j] = 0.0;
          sn[r][j] = 1.0;
        } else {
          cs[r][j] = na / rr;
          sn[r][j] = (a / na) * std::conj(bb) / rr;
        }
        Rr[(size_t)j * ld + j] = cs[r][j] * a + sn[r][j] * bb;
        Rr[(size_t)j * ld + j + 1] = 0.0;
        C g1 = gv[r][j], g2 = gv[r][j + 1];
        gv[r][j] = cs[r][j] * g1 + sn[r][j] * g2;
        gv[r][j + 1] = cs[r][j] * g2 - std::conj(sn[r][j]) * g1;
        double est = bn[r] > 0 ? std::abs(gv[r][j + 1]) / bn[r] : 0.0;
        if (!std::isfinite(est)) throw Fail{HZ_ENONFINITE, "non-finite Arnoldi residual estimate"};
        if (est > tol) all_conv = false;
        if (nb == 0.0) breakdown = true;
      }
      k = j + 1;
      est_converged = all_conv;
      if (all_conv || breakdown || pc >= max_pc) break;
    }
    std::vector<double> yh((size_t)nrhs * LDMAX * 2, 0.0);
    for (int r = 0; r < nrhs; ++r) {
      std::vector<C> y(k);
      for (int i = k - 1; i >= 0; --i) {
        C t = gv[r][i];
        for (int c = i + 1; c < k; ++c) t -= Rm[r][(size_t)c * ld + i] * y[c];
        C d = Rm[r][(size_t)i * ld + i];
        y[i] = std::abs(d) > 0 ? t / d : C(0.0);
      }
      for (int i = 0; i < k; ++i) {
        yh[((size_t)r * ld + i) * 2] = y[i].real();
        yh[((size_t)r * ld + i) * 2 + 1] = y[i].imag();
      }
    }
    HZ_CK(cudaMemcpyAsync(W.yo, yh.data(), (size_t)nrhs * ld * 2 * sizeof(double), cudaMemcpyHostToDevice, H->st));
    launch_combine<R>(W.Zo, vs, k, W.yo, ld, x, x, (int)N, nrhs, H->st);
    HZ_LAUNCHED();
    if (inner && (est_converged || pc >= max_pc)) break;
  }
  return relmax;
}

// ----------------------------------------------------------------------------
// block flexible GMRES(m_out) over groups of right-hand sides (Sec. 7's block
// Krylov method for multiple right-hand sides)
// ----------------------------------------------------------------------------
// One basis per group of S <= 16 right-hand sides: the block residual
// R_0 = V_0 R_hat, then per step Z_j = M(V_j) (the three-grid preconditioner
// on the S columns), W = A Z_j, block classical Gram-Schmidt against
// V_0 .. V_j in two passes, W = V_{j+1} H_{j+1,j}.  Thin QR factors come from
// Cholesky-QR applied twice (Gram block on the device, Cholesky of the S x S
// block in FP64 on the host).  The block Hessenberg matrix is banded (S
// sub-diagonals, the last block upper triangular) and is reduced by Givens
// rotations in FP64 on the host; the rotated right-hand side block gives each
// column's residual estimate.  Column t of block j of the basis is
// Vo + j * vs + (r0 + t) * N, so the group's blocks are the same workspace
// the independent solves use.
using Cd = std::complex<double>;

// G = R^H R for an S x S Hermitian block (row-major); R upper triangular.
// False when a pivot falls below rel times the largest diagonal entry.
bool chol_upper(const std::vector<Cd>& G, int S, double rel, std::vector<Cd>& Rm) {
  Rm.assign((size_t)S * S, Cd(0.0));
  double dmax = 0.0;
  for (int i = 0; i < S; ++i) dmax = std::max(dmax, G[(size_t)i * S + i].real());
  if (!(dmax > 0.0) || !std::isfinite(dmax)) return false;
  for (int i = 0; i < S; ++i) {
    Cd d = G[(size_t)i * S + i];
    for (int k = 0; k < i; ++k) d -= std::norm(Rm[(size_t)k * S + i]);
    if (!(d.real() > rel * dmax)) return false;
    const double rii = std::sqrt(d.real());
    Rm[(size_t)i * S + i] = rii;
    for (int j = i + 1; j < S; ++j) {
      Cd t = G[(size_t)i * S + j];
      for (int k = 0; k < i; ++k) t -= std::conj(Rm[(size_t)k * S + i]) * Rm[(size_t)k * S + j];
      Rm[(size_t)i * S + j] = t / rii;
    }
  }
  return true;
}

// inverse of an upper-triangular S x S matrix (row-major)
std::vector<Cd> upper_inverse(const std::vector<Cd>& Rm, int S) {
  std::vector<Cd> X((size_t)S * S, Cd(0.0));
  for (int c = 0; c < S; ++c)
    for (int i = c; i >= 0; --i) {
      Cd t = (i == c) ? Cd(1.0) : Cd(0.0);
      for (int k = i + 1; k <= c; ++k) t -= Rm[(size_t)i * S + k] * X[(size_t)k * S + c];
      X[(size_t)i * S + c] = t / Rm[(size_t)i * S + i];
    }
  return X;
}

template <class R>
struct BlockGroup {
  hz_handle* H;
  Work<R>& W;
  long long N, vs;
  int r0, S;
  BlockCols cols(const cx<R>* base, int count) const { return BlockCols{base + (long long)r0 * N, vs, N, S, count}; }
  cx<R>* blk(cx<R>* base, int j) const { return base + (long long)j * vs + (long long)r0 * N; }
  // G = X^H Y, p x q row-major, on the host
  std::vector<Cd> gram(const BlockCols& X, const BlockCols& Y) const {
    launch_block_gram<R>(X, Y, W.bpart, W.bgram, H->st);
    HZ_LAUNCHED();
    std::vector<double> g = host_copy(W.bgram, 2 * X.count * Y.count, H->st);
    std::vector<Cd> G((size_t)X.count * Y.count);
    for (size_t e = 0; e < G.size(); ++e) G[e] = Cd(g[2 * e], g[2 * e + 1]);
    return G;
  }
  // Y = beta Y + X C (C: p x q row-major)
  void update(const BlockCols& X, cx<R>* Y, const std::vector<Cd>& Cm, double beta) const {
    HZ_CK(cudaMemcpyAsync(W.bcoef, Cm.data(), Cm.size() * sizeof(Cd), cudaMemcpyHostToDevice, H->st));
    launch_block_update<R>(X, Y, S, W.bcoef, beta, H->st);
    HZ_LAUNCHED();
  }
  // thin QR of block j of the basis in place by Cholesky-QR twice; R (S x S, upper)
  bool cholqr2(int j, std::vector<Cd>& Rout) const {
    // pivots below this fraction mean a condition number beyond what two
    // Cholesky-QR passes orthogonalise in the working precision
    const double rel = sizeof(R) == 4 ? 1e-7 : 1e-14;
    const BlockCols B = cols(W.Vo + (long long)j * vs, S);
    cx<R>* Bp = blk(W.Vo, j);
    std::vector<Cd> R1, R2;
    if (!chol_upper(gram(B, B), S, rel, R1)) return false;
    update(B, Bp, upper_inverse(R1, S), 0.0);
    if (!chol_upper(gram(B, B), S, 1e-3, R2)) return false;
    update(B, Bp, upper_inverse(R2, S), 0.0);
    Rout.assign((size_t)S * S, Cd(0.0));
    for (int i = 0; i < S; ++i)
      for (int c = i; c < S; ++c) {
        Cd t = 0.0;
        for (int k = i; k <= c; ++k) t += R2[(size_t)i * S + k] * R1[(size_t)k * S + c];
        Rout[(size_t)i * S + c] = t;
      }
    return true;
  }
};

// One group of S right-hand sides starting at r0; returns the largest relative
// true residual of the group's last restart, or a negative value when the
// initial block is numerically rank-deficient (nothing has been changed then).
template <class R>
double block_fgmres_group(hz_handle* H, const cx<R>* b, cx<R>* x, int nrhs, int r0, int S, bool adj,
                          const std::vector<double>& bn, double tol, int max_pc, int& pc, bool inner) {
  Work<R>& W = Sel<R>::w(H);
  const int m = H->p.m_out;
  const long long N = H->lev[0].N, vs = N * nrhs;
  BlockGroup<R> G{H, W, N, vs, r0, S};
  const int ldE = (m + 1) * S;
  double relmax = 0.0, prev_rel = HUGE_VAL;
  bool est_converged = false, first = true;
  for (;;) {
    cx<R>* V0 = G.blk(W.Vo, 0);
    resid<R>(H, 0, false, adj, b + (long long)r0 * N, x + (long long)r0 * N, V0, S,
             reducer(H, W.nrm, W.beta_o, W.scale_o));
    std::vector<double> beta = host_copy(W.beta_o, S, H->st);
    relmax = 0.0;
    for (int c = 0; c < S; ++c) {
      if (!std::isfinite(beta[c])) throw Fail{HZ_ENONFINITE, "non-finite residual norm in the block FGMRES"};
      relmax = std::max(relmax, bn[r0 + c] > 0 ? beta[c] / bn[r0 + c] : 0.0);
    }
    if (relmax <= tol || pc >= max_pc) break;
    if (inner && relmax > 0.9 * prev_rel) break;
    prev_rel = relmax;
    std::vector<Cd> Rh;
    if (!G.cholqr2(0, Rh)) {
      if (first) return -1.0;
      break;  // a later rank-deficient residual block: the caller's true residual decides
    }
    first = false;
    // banded Hessenberg (column-major, ld ldE), rotated right-hand side block E
    std::vector<Cd> Hh((size_t)ldE * m * S, Cd(0.0)), E((size_t)ldE * S, Cd(0.0));
    for (int i = 0; i < S; ++i)
      for (int c = i; c < S; ++c) E[(size_t)c * ldE + i] = Rh[(size_t)i * S + c];
    struct Rot {
      int i;
      double c;
      Cd s;
    };
    std::vector<Rot> rots;
    auto rotate = [](const Rot& q, Cd* v) {
      const Cd t1 = v[q.i], t2 = v[q.i + 1];
      v[q.i] = q.c * t1 + q.s * t2;
      v[q.i + 1] = q.c * t2 - std::conj(q.s) * t1;
    };
    int k = 0;
    for (int j = 0; j < m; ++j) {
      precond<R>(H, G.blk(W.Vo, j), G.blk(W.Zo, j), S, adj);
      ++pc;
      cx<R>* Wb = G.blk(W.Vo, j + 1);
      apply<R>(H, 0, false, adj, G.blk(W.Zo, j), Wb, S);
      const BlockCols Vset = G.cols(W.Vo, (j + 1) * S), Wset = G.cols(W.Vo + (long long)(j + 1) * vs, S);
      std::vector<Cd> Hacc((size_t)(j + 1) * S * S, Cd(0.0));
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<Cd> Hp = G.gram(Vset, Wset);
        std::vector<Cd> neg(Hp.size());
        for (size_t e = 0; e < Hp.size(); ++e) {
          Hacc[e] += Hp[e];
          neg[e] = -Hp[e];
        }
        G.update(Vset, Wb, neg, 1.0);
      }
      std::vector<Cd> Rsub;
      const bool full = G.cholqr2(j + 1, Rsub);
      // block column j of the Hessenberg matrix, then the old and new rotations
      for (int c = 0; c < S; ++c) {
        const int q = j * S + c;
        Cd* col = &Hh[(size_t)q * ldE];
        for (int i = 0; i < (j + 1) * S; ++i) col[i] = Hacc[(size_t)i * S + c];
        if (full)
          for (int i = 0; i <= c; ++i) col[(j + 1) * S + i] = Rsub[(size_t)i * S + c];
        for (const Rot& q2 : rots) rotate(q2, col);
        for (int r = q + S; r > q; --r) {
          const Cd a = col[r - 1], bb = col[r];
          if (bb == Cd(0.0)) continue;
          const double na = std::abs(a), nb = std::abs(bb), rr = std::hypot(na, nb);
          Rot g{r - 1, 0.0, Cd(0.0)};
          if (na == 0.0) {
            g.c = 0.0;
            g.s = 1.0;
          } else {
            g.c = na / rr;
            g.s = (a / na) * std::conj(bb) / rr;
          }
          rotate(g, col);
          col[r] = 0.0;
          for (int e = 0; e < S; ++e) rotate(g, &E[(size_t)e * ldE]);
          rots.push_back(g);
        }
      }
      k = j + 1;
      bool all_conv = true;
      for (int c = 0; c < S; ++c) {
        double e2 = 0.0;
        for (int i = k * S; i < (k + 1) * S; ++i) e2 += std::norm(E[(size_t)c * ldE + i]);
        const double est = bn[r0 + c] > 0 ? std::sqrt(e2) / bn[r0 + c] : 0.0;
        if (!std::isfinite(est)) throw Fail{HZ_ENONFINITE, "non-finite block Arnoldi residual estimate"};
        if (est > tol) all_conv = false;
      }
      // a rank-deficient block W ends the cycle; its zeroed sub-diagonal block
      // is no convergence evidence, so the next restart's true residual decides
      est_converged = all_conv && full;
      if (all_conv || !full || pc >= max_pc) break;
    }
    // Y = R^-1 E[0 : kS] (k S x S), then x += [Z_0 .. Z_{k-1}] Y
    const int KS = k * S;
    std::vector<Cd> Y((size_t)KS * S, Cd(0.0));
    for (int c = 0; c < S; ++c)
      for (int i = KS - 1; i >= 0; --i) {
        Cd t = E[(size_t)c * ldE + i];
        for (int l = i + 1; l < KS; ++l) t -= Hh[(size_t)l * ldE + i] * Y[(size_t)l * S + c];
        const Cd d = Hh[(size_t)i * ldE + i];
        Y[(size_t)i * S + c] = std::abs(d) > 0 ? t / d : Cd(0.0);
      }
    G.update(G.cols(W.Zo, KS), x + (long long)r0 * N, Y, 1.0);
    if (inner && (est_converged || pc >= max_pc)) break;
  }
  return relmax;
}

// The outer Krylov solve: block FGMRES over groups of at most kBlockMaxS
// right-hand sides when selected (independent FGMRES for a group whose initial
// block is rank-deficient), else the independent batched FGMRES.
template <class R>
double outer_solve(hz_handle* H, const cx<R>* b, cx<R>* x, int nrhs, bool adj, const std::vector<double>& bn,
                   double tol, int max_pc, int& pc, bool inner = false) {
  if (!H->p.block || nrhs < 2) return outer_fgmres<R>(H, b, x, nrhs, adj, bn, tol, max_pc, pc, inner);
  const long long N = H->lev[0].N;
  double relmax = 0.0;
  for (int r0 = 0; r0 < nrhs; r0 += kBlockMaxS) {
    const int S = std::min(kBlockMaxS, nrhs - r0);
    double rel = S >= 2 ? block_fgmres_group<R>(H, b, x, nrhs, r0, S, adj, bn, tol, max_pc, pc, inner) : -1.0;
    if (rel < 0.0) {
      // the independent method on this group alone (its own columns, scales and norms)
      std::vector<double> bg(bn.begin() + r0, bn.begin() + r0 + S);
      rel = outer_fgmres<R>(H, b + (long long)r0 * N, x + (long long)r0 * N, S, adj, bg, tol, max_pc, pc, inner);
    }
    relmax = std::max(relmax, rel);
  }
  return relmax;
}

std::vector<double> norms(hz_handle* H, const cx<double>* v, int nrhs) {
  launch_norm2<double>(v, (int)H->lev[0].N, nrhs, reducer(H, H->s_nrm), H->st);
  HZ_LAUNCHED();
  std::vector<double> n2 = host_copy(H->s_nrm, nrhs, H->st);
  for (double& t : n2) t = std::sqrt(t);
  return n2;
}

// Solve (adj ? A_h^H : A_h) x = b for nrhs complex128 fields; x is overwritten.
struct SolveOut {
  int pc = 0, passes = 0;
  double rel = 0;
};
SolveOut solve_c128(hz_handle* H, const cx<double>* b, cx<double>* x, int nrhs, bool adj) {
  SolveOut o;
  const hz_params& p = H->p;
  const long long N = H->lev[0].N;
  std::vector<double> bn = norms(H, b, nrhs);
  launch_zero<double>(x, N * nrhs, H->st);
  HZ_LAUNCHED();
  if (p.precision == HZ_C128) {
    ensure_work<double>(H);
    o.rel = outer_solve<double>(H, b, x, nrhs, adj, bn, p.tol, p.max_pc, o.pc);
    return o;
  }
  ensure_work<float>(H);
  if (!p.refine) {
    // the paper's protocol: one complex64 FGMRES solve of the scaled system to
    // tol, stopped by its complex64 true residual; v = ||b|| x64
    std::vector<double> inv(nrhs), one(nrhs);
    for (int r = 0; r < nrhs; ++r) {
      inv[r] = bn[r] > 1e-300 ? 1.0 / bn[r] : 0.0;
      one[r] = bn[r] > 0 ? 1.0 : 0.0;
    }
    HZ_CK(cudaMemcpyAsync(H->s_inv, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, H->st));
    HZ_CK(cudaMemcpyAsync(H->s_root, bn.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, H->st));
    launch_c128_to_c64_scaled(b, H->b64, H->s_inv, (int)N, nrhs, H->st);
    launch_zero<float>(H->x64, N * nrhs, H->st);
    HZ_LAUNCHED();
    o.rel = outer_solve<float>(H, H->b64, H->x64, nrhs, adj, one, p.tol, p.max_pc, o.pc);
    launch_add_c64_to_c128_scaled(H->x64, x, H->s_root, (int)N, nrhs, H->st);
    HZ_LAUNCHED();
    HZ_CK(cudaStreamSynchronize(H->st));
    return o;
  }
  // FP64 iterative refinement around complex64 corrections
  bool x_zero = true;  // the initial guess: its residual is b, whose norms are known
  std::vector<double> root(nrhs), inv(nrhs);
  for (;;) {
    std::vector<double> rn;
    const cx<double>* r = H->r128;
    if (x_zero) {
      rn = bn;
      for (int i = 0; i < nrhs; ++i) {
        root[i] = bn[i];
        inv[i] = bn[i] > 1e-300 ? 1.0 / bn[i] : 0.0;
      }
      HZ_CK(cudaMemcpyAsync(H->s_root, root.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, H->st));
      HZ_CK(cudaMemcpyAsync(H->s_inv, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, H->st));
      r = b;
    } else {
      resid<double>(H, 0, false, adj, b, x, H->r128, nrhs, reducer(H, H->s_nrm, H->s_root, H->s_inv));
      rn = host_copy(H->s_root, nrhs, H->st);
    }
    ++o.passes;
    double relmax = 0.0, need = 1.0;
    for (int r = 0; r < nrhs; ++r) {
      if (!std::isfinite(rn[r])) throw Fail{HZ_ENONFINITE, "non-finite FP64 residual norm"};
      double rel = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
      relmax = std::max(relmax, rel);
      if (rn[r] > 0) need = std::min(need, 0.5 * p.tol * bn[r] / rn[r]);
    }
    o.rel = relmax;
    if (relmax <= p.tol || o.pc >= p.max_pc || o.passes > p.max_refine) break;
    launch_c128_to_c64_scaled(r, H->b64, H->s_inv, (int)N, nrhs, H->st);
    launch_zero<float>(H->x64, N * nrhs, H->st);
    HZ_LAUNCHED();
    std::vector<double> one(nrhs);
    for (int r = 0; r < nrhs; ++r) one[r] = rn[r] > 0 ? 1.0 : 0.0;
    double inner = std::max(p.inner_tol, need);
    outer_solve<float>(H, H->b64, H->x64, nrhs, adj, one, inner, p.max_pc, o.pc, true);
    launch_add_c64_to_c128_scaled(H->x64, x, H->s_root, (int)N, nrhs, H->st);
    HZ_LAUNCHED();
    x_zero = false;
  }
  HZ_CK(cudaStreamSynchronize(H->st));  // the host norm buffers feed queued copies
  return o;
}

// A grid-barrier wait of the persistent bottom solve that gave up sets a
// device flag (the kernel then finishes without waiting, its results
// invalid); the synchronous entry points read and clear it.
void check_bottom_err(hz_handle* H) {
  if (!H->bot_err) return;
  int e = 0;
  HZ_CK(cudaMemcpyAsync(&e, H->bot_err, sizeof(int), cudaMemcpyDeviceToHost, H->st));
  HZ_CK(cudaStreamSynchronize(H->st));
  if (e) {
    HZ_CK(cudaMemsetAsync(H->bot_err, 0, sizeof(int), H->st));
    HZ_CK(cudaStreamSynchronize(H->st));
    throw Fail{HZ_ETIMEOUT, "a grid-barrier wait of the persistent bottom solve gave up; the results are invalid"};
  }
}

void upload_source_list(hz_handle* H, const hz_source* src, int ns) {
  std::vector<int> idx(3 * ns);
  std::vector<double> amp(2 * ns);
  for (int s = 0; s < ns; ++s) {
    HZ_REQUIRE(src[s].ix >= 0 && src[s].ix <= H->g.nx && src[s].iy >= 0 && src[s].iy <= H->g.ny && src[s].iz >= 0 &&
                   src[s].iz <= H->g.nz,
               "source node outside the grid");
    idx[3 * s] = src[s].ix;
    idx[3 * s + 1] = src[s].iy;
    idx[3 * s + 2] = src[s].iz;
    amp[2 * s] = src[s].amp_re;
    amp[2 * s + 1] = src[s].amp_im;
  }
  HZ_CK(cudaMemcpyAsync(H->src_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, H->st));
  HZ_CK(cudaMemcpyAsync(H->src_amp, amp.data(), amp.size() * sizeof(double), cudaMemcpyHostToDevice, H->st));
}

// the source field f = amp h^-3 e_{i_s} (Eq. point-source), one per right-hand side
void upload_sources(hz_handle* H, const hz_source* src, int ns) {
  upload_source_list(H, src, ns);
  const long long N = H->lev[0].N;
  launch_zero<double>(H->f128, N * ns, H->st);
  launch_point_sources<double>(H->src_idx, H->src_amp, ns, H->lev[0].nx, H->lev[0].ny, H->lev[0].nz,
                               1.0 / (H->g.h * H->g.h * H->g.h), H->f128, H->st);
  HZ_LAUNCHED();
}

// b = Q_h f of the point sources directly on their 27-node blocks (no field f)
void source_rhs(hz_handle* H, const hz_source* src, int ns, cx<double>* b) {
  upload_source_list(H, src, ns);
  const long long N = H->lev[0].N;
  launch_zero<double>(b, N * ns, H->st);
  launch_source_rows(view<double>(H, 0), tview<double>(H), H->src_idx, H->src_amp, ns,
                     1.0 / (H->g.h * H->g.h * H->g.h), b, H->st);
  HZ_LAUNCHED();
}



}  // namespace

// ============================================================================
// C ABI
// ============================================================================
#include <functional>

static hz_status run_guarded(hz_handle* H, const std::function<void()>& f) {
  try {
    f();
    return HZ_OK;
  } catch (const Fail& e) {
    if (H) H->err = e.msg;
    return e.st;
  } catch (const std::exception& e) {
    if (H) H->err = e.what();
    return HZ_ECUDA;
  } catch (...) {
    if (H) H->err = "unknown error";
    return HZ_ECUDA;
  }
}

static thread_local std::string g_create_error;

extern "C" {

void hz_default_params(hz_params* p) {
  if (!p) return;
  p->tol = 1e-4;
  p->max_pc = 1000;
  p->m_out = 5;
  p->m_h = 2;
  p->nJ_h = 2;
  p->c_2h = 2;
  p->m_2h = 10;
  p->nJ_2h = 2;
  p->m_4h = 4;
  p->nJ_4h = 2;
  p->w_h = 0.8;
  p->w_2h = 0.8;
  p->w_4h = 0.2;
  p->sigma = 0.9;
  p->precision = HZ_C64;
  p->inner_tol = 1e-5;
  p->max_refine = 8;
  p->autotune = 1;
  p->refine = 1;
  p->block = 0;
}

const char* hz_last_error(const hz_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

unsigned long long hz_kernel_launches(void) { return g_launches.load(); }

hz_status hz_workspace_bytes(const hz_grid* grid, const hz_params* params, int max_nrhs, size_t* bytes) {
  if (!grid || !params || !bytes || max_nrhs < 1) return HZ_EINVAL;
  hz_handle tmp;
  hz_status st = run_guarded(&tmp, [&] {
    check_grid(*grid);
    check_params(*params);
    tmp.g = *grid;
    tmp.p = *params;
    tmp.max_nrhs = max_nrhs;
    plan_all(&tmp, true);
    *bytes = tmp.al.bytes;
  });
  g_create_error = tmp.err;
  return st;
}

hz_status hz_layout_check(const hz_grid* grid, int level, int op, int nrhs, int zblock, int zblock_f,
                          unsigned char* counts_host, long long* blocks, long long* violations) {
  if (!grid || !violations) return HZ_EINVAL;
  hz_handle tmp;
  hz_status st = run_guarded(&tmp, [&] {
    check_grid(*grid);
    HZ_REQUIRE(level >= 0 && level <= 2, "level must be 0, 1 or 2");
    HZ_REQUIRE(op == HZ_OP_A || op == HZ_OP_B || op == HZ_OP_Q || op == HZ_OP_A_ADJ || op == HZ_OP_B_ADJ,
               "op must be HZ_OP_A, HZ_OP_B, HZ_OP_Q, HZ_OP_A_ADJ or HZ_OP_B_ADJ");
    HZ_REQUIRE(op != HZ_OP_Q || level == 0, "Q_h is defined on the fine level only");
    HZ_REQUIRE(nrhs >= 1 && zblock >= 0 && zblock_f >= 0, "nrhs must be >= 1, z-blocks >= 0");
    Level lv;
    level_dims(*grid, level, lv);
    if (counts_host) std::memset(counts_host, 0, (size_t)lv.N);
    if (op == HZ_OP_A_ADJ || op == HZ_OP_B_ADJ)
      *violations = replay_adj_layout(lv.nx, lv.ny, lv.nz, nrhs, zblock, counts_host, blocks);
    else
      *violations = replay_fwd_layout(level, lv.nx, lv.ny, lv.nz, lv.plain_lo, lv.plain_hi,
                                      op == HZ_OP_Q ? OP_Q : OP_AB, nrhs, zblock, zblock_f, counts_host, blocks);
  });
  g_create_error = tmp.err;
  return st;
}

hz_status hz_create(const hz_grid* grid, const double* c_dev, const hz_params* params, const double* table_host,
                    int table_rows, int max_nrhs, void* stream, hz_handle** out) {
  if (!out) return HZ_EINVAL;
  *out = nullptr;
  hz_handle* H = new hz_handle();
  hz_status st = run_guarded(H, [&] {
    HZ_REQUIRE(grid && c_dev && params && table_host, "null argument");
    HZ_REQUIRE(table_rows >= 2 && table_rows <= kMaxSeg + 1, "table_rows must be in [2, 33]");
    HZ_REQUIRE(max_nrhs >= 1, "max_nrhs must be >= 1");
    check_grid(*grid);
    check_params(*params);
    H->g = *grid;
    H->p = *params;
    H->max_nrhs = max_nrhs;
    H->st = (cudaStream_t)stream;
    HZ_CK(cudaStreamCreateWithFlags(&H->own, cudaStreamNonBlocking));
    HZ_CK(cudaStreamCreateWithFlags(&H->side, cudaStreamNonBlocking));
    HZ_CK(cudaEventCreateWithFlags(&H->ev_fork, cudaEventDisableTiming));
    HZ_CK(cudaEventCreateWithFlags(&H->ev_join, cudaEventDisableTiming));
    const char* ng = std::getenv("HZ_NO_GRAPH");
    H->use_graphs = !(ng && ng[0] == '1');
    init_kernel_attributes();
    block_init_attrs();
    HZ_LAUNCHED();
    auto t0 = std::chrono::steady_clock::now();
    plan_all(H, false);
    HZ_CK(cudaMemsetAsync(H->red_count, 0, sizeof(unsigned) * max_nrhs, H->st));
    {
      // opt-in: on the 289^3 benchmark the ten grid barriers cost more than the
      // launch gaps they replace (15.0 against 14.2-14.5 ms per preconditioner call)
      const char* pp = std::getenv("HZ_PERSISTENT");
      H->coop_bottom = (pp && pp[0] == '1') && gather::coop_capture_supported();
      const char* bt = std::getenv("HZ_BARRIER_TEST");  // makes every grid-barrier wait run out (tests)
      if (bt && bt[0] == '1') {
        H->bot_extra = 1;
        H->bot_spins = 4096;
      }
      if (H->coop_bottom) {
        H->bot_bar = H->al.get<unsigned>(2);
        H->bot_err = H->al.get<int>(1);
        H->bot_partial_f = H->al.get<double>(gather::bottom_partial_doubles<float>(max_nrhs));
        H->bot_partial_d = H->al.get<double>(gather::bottom_partial_doubles<double>(max_nrhs));
        HZ_CK(cudaMemsetAsync(H->bot_err, 0, sizeof(int), H->st));
      }
    }
    std::vector<double> coef;
    double ds;
    build_table(table_host, table_rows, coef, ds);
    H->nseg = table_rows - 1;
    H->ds = ds;
    std::vector<float> coef_f(coef.begin(), coef.end());
    HZ_CK(cudaMemcpyAsync(H->tab_d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, H->st));
    HZ_CK(cudaMemcpyAsync(H->tab_f, coef_f.data(), coef_f.size() * sizeof(float), cudaMemcpyHostToDevice, H->st));
    for (int L = 0; L < 3; ++L) {
      Level& lv = H->lev[L];
      const int f = 1 << L;
      const int nn[3] = {H->g.nx / f, H->g.ny / f, H->g.nz / f};
      for (int a = 0; a < 3; ++a) {
        std::vector<std::complex<double>> ab, ac;
        pml_axis(nn[a], lv.n_pml, H->g.gamma_max, ab, ac, lv.plain_lo[a], lv.plain_hi[a]);
        std::vector<cx<float>> abf(ab.size()), acf(ac.size());
        for (size_t i = 0; i < ab.size(); ++i) {
          abf[i] = mkc<float>((float)ab[i].real(), (float)ab[i].imag());
          acf[i] = mkc<float>((float)ac[i].real(), (float)ac[i].imag());
        }
        HZ_CK(cudaMemcpy(lv.abar_d[a], ab.data(), ab.size() * 16, cudaMemcpyHostToDevice));
        HZ_CK(cudaMemcpy(lv.achk_d[a], ac.data(), ac.size() * 16, cudaMemcpyHostToDevice));
        HZ_CK(cudaMemcpy(lv.abar_f[a], abf.data(), abf.size() * 8, cudaMemcpyHostToDevice));
        HZ_CK(cudaMemcpy(lv.achk_f[a], acf.data(), acf.size() * 8, cudaMemcpyHostToDevice));
        // eps+- = -(abar - 1 +- achk) / ell^2: zero where the axis is not stretched
        for (int sgn = 0; sgn < 2; ++sgn) {
          std::vector<std::complex<double>> e(ab.size());
          std::vector<cx<float>> ef(ab.size());
          for (size_t i = 0; i < ab.size(); ++i) {
            e[i] = -((ab[i] - 1.0) + (sgn == 0 ? ac[i] : -ac[i])) / (lv.ell * lv.ell);
            ef[i] = mkc<float>((float)e[i].real(), (float)e[i].imag());
          }
          HZ_CK(cudaMemcpy(lv.eps_d[a][sgn], e.data(), e.size() * 16, cudaMemcpyHostToDevice));
          HZ_CK(cudaMemcpy(lv.eps_f[a][sgn], ef.data(), ef.size() * 8, cudaMemcpyHostToDevice));
        }
      }
      {
        std::vector<double> ct_d, ct_s;
        build_coef_tables(coef, table_host, table_rows, ds, lv.ell, false, ct_d);
        build_coef_tables(coef, table_host, table_rows, ds, lv.ell, true, ct_s);
        std::vector<float> ct_f(ct_s.begin(), ct_s.end());
        HZ_CK(cudaMemcpy(lv.ctab_d, ct_d.data(), ct_d.size() * sizeof(double), cudaMemcpyHostToDevice));
        HZ_CK(cudaMemcpy(lv.ctab_f, ct_f.data(), ct_f.size() * sizeof(float), cudaMemcpyHostToDevice));
      }
      launch_setup_kappa<double>(c_dev, H->g.nx + 1, H->g.ny + 1, H->g.nz + 1, H->g.n_pml, f, H->g.omega, lv.ell,
                                 lv.kap_d, H->st);
      launch_setup_kappa<float>(c_dev, H->g.nx + 1, H->g.ny + 1, H->g.nz + 1, H->g.n_pml, f, H->g.omega, lv.ell,
                                lv.kap_f, H->st);
      HZ_LAUNCHED();
    }
    compute_dinv<float>(H, H->lev[0].dinv_f, H->lev[1].dinv_f, H->lev[2].dinv_f);
    HZ_LAUNCHED();
    if (H->p.precision == HZ_C128) prepare_dinv_double(H);
    if (H->p.autotune) {
      if (H->p.precision == HZ_C64) autotune_zblocks<float>(H);
      else autotune_zblocks<double>(H);
    }
    HZ_CK(cudaStreamSynchronize(H->st));
    H->t_setup = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    H->st = H->own;
  });
  if (st != HZ_OK) {
    g_create_error = H->err;
    drop_graphs(H);
    H->al.free_all();
    destroy_streams(H);
    delete H;
    return st;
  }
  *out = H;
  return HZ_OK;
}

hz_status hz_destroy(hz_handle* H) {
  if (!H) return HZ_EINVAL;
  cudaStreamSynchronize(H->own);
  cudaStreamSynchronize(H->side);
  drop_graphs(H);
  H->al.free_all();
  destroy_streams(H);
  delete H;
  return HZ_OK;
}

hz_status hz_set_params(hz_handle* H, const hz_params* params) {
  if (!H || !params) return HZ_EINVAL;
  return run_guarded(H, [&] {
    check_params(*params);
    const hz_params& o = H->p;
    HZ_REQUIRE(params->m_out == o.m_out && params->m_h == o.m_h && params->m_2h == o.m_2h &&
                   params->m_4h == o.m_4h && (params->nJ_h > 2) == (o.nJ_h > 2) &&
                   (params->nJ_2h > 2) == (o.nJ_2h > 2) && (params->nJ_4h > 2) == (o.nJ_4h > 2),
               "restart lengths and Jacobi temporaries are fixed at hz_create");
    if (params->precision != o.precision) {
      if (params->precision == HZ_C64 && !H->b64) {
        H->b64 = H->al.get<cx<float>>((size_t)H->lev[0].N * H->max_nrhs);
        H->x64 = H->al.get<cx<float>>((size_t)H->lev[0].N * H->max_nrhs);
      }
    }
    drop_graphs(H);
    H->p = *params;
    // the shift sigma enters the Jacobi diagonals of B_2h, B_4h
    H->st = H->own;
    compute_dinv<float>(H, H->lev[0].dinv_f, H->lev[1].dinv_f, H->lev[2].dinv_f);
    if (H->lev[0].dinv_d[0]) compute_dinv<double>(H, H->lev[0].dinv_d, H->lev[1].dinv_d, H->lev[2].dinv_d);
    HZ_LAUNCHED();
    HZ_CK(cudaStreamSynchronize(H->st));
  });
}

hz_status iofd_coeffs(hz_handle* H, int level, double* kappa_dev, double* shell_dev) {
  if (!H) return HZ_EINVAL;
  return run_guarded(H, [&] {
    HZ_REQUIRE(level >= 0 && level <= 2, "level must be 0, 1 or 2");
    HZ_REQUIRE(kappa_dev, "kappa_dev is null");
    const Level& lv = H->lev[level];
    H->st = H->own;
    HZ_CK(cudaMemcpyAsync(kappa_dev, lv.kap_d, lv.N * sizeof(double), cudaMemcpyDeviceToDevice, H->st));
    if (shell_dev) {
      launch_shell_coeffs(view<double>(H, level), tview<double>(H), shell_dev, H->st);
      HZ_LAUNCHED();
    }
    HZ_CK(cudaStreamSynchronize(H->st));
  });
}

hz_status iofd_apply(hz_handle* H, int level, int op, int precision, const void* x, void* y, int nrhs, void* stream) {
  if (!H) return HZ_EINVAL;
  return run_guarded(H, [&] {
    HZ_REQUIRE(level >= 0 && level <= 2, "level must be 0, 1 or 2");
    HZ_REQUIRE(op >= HZ_OP_A && op <= HZ_OP_Q_ADJ, "unknown operator");
    HZ_REQUIRE(x && y && x != y, "x and y must be distinct non-null device pointers");
    HZ_REQUIRE(nrhs >= 1 && nrhs <= H->max_nrhs, "nrhs out of range");
    HZ_REQUIRE(precision == HZ_C64 || precision == HZ_C128, "precision must be HZ_C64 or HZ_C128");
    const bool isq = (op == HZ_OP_Q || op == HZ_OP_Q_ADJ);
    HZ_REQUIRE(!isq || level == 0, "Q_h is defined on the fine level only");
    const bool adj = (op == HZ_OP_A_ADJ || op == HZ_OP_B_ADJ || op == HZ_OP_Q_ADJ);
    const bool shifted = (op == HZ_OP_B || op == HZ_OP_B_ADJ);
    cudaStream_t old = H->st;
    H->st = (cudaStream_t)stream;
    try {
      if (precision == HZ_C64) {
        StencilCall<float> c = call<float>(H, level, shifted, nrhs);
        c.x = (const cx<float>*)x;
        c.y = (cx<float>*)y;
        launch_stencil<float>(c, M_APPLY, isq ? OP_Q : OP_AB, adj, H->st);
      } else {
        StencilCall<double> c = call<double>(H, level, shifted, nrhs);
        c.x = (const cx<double>*)x;
        c.y = (cx<double>*)y;
        launch_stencil<double>(c, M_APPLY, isq ? OP_Q : OP_AB, adj, H->st);
      }
      HZ_LAUNCHED();
    } catch (...) {
      H->st = old;
      throw;
    }
    H->st = old;
  });
}

hz_status iofd_apply_window(hz_handle* H, int op, int precision, const void* x, void* y, int nrhs, int z0, int z1,
                            void* stream) {
  if (!H) return HZ_EINVAL;
  return run_guarded(H, [&] {
    HZ_REQUIRE(op == HZ_OP_A || op == HZ_OP_B, "the window apply takes HZ_OP_A or HZ_OP_B");
    HZ_REQUIRE(x && y && x != y, "x and y must be distinct non-null device pointers");
    HZ_REQUIRE(nrhs >= 1 && nrhs <= H->max_nrhs, "nrhs out of range");
    HZ_REQUIRE(precision == HZ_C64 || precision == HZ_C128, "precision must be HZ_C64 or HZ_C128");
    const Level& L0 = H->lev[0];
    HZ_REQUIRE(z0 >= 0 && z0 < z1 && z1 <= L0.nz, "need 0 <= z0 < z1 <= nz (fine-level planes)");
    const long long plane = (long long)L0.nx * L0.ny;
    auto fill = [&](auto& c) {
      c.zr0 = z0;
      c.zr1 = z1;
      c.xz0 = z0 - 1;
      c.xstride = (long long)(z1 - z0 + 2) * plane;
      c.ystride = (long long)(z1 - z0) * plane;
    };
    cudaStream_t old = H->st;
    H->st = (cudaStream_t)stream;
    try {
      if (precision == HZ_C64) {
        StencilCall<float> c = call<float>(H, 0, op == HZ_OP_B, nrhs);
        c.x = (const cx<float>*)x;
        c.y = (cx<float>*)y;
        fill(c);
        launch_stencil<float>(c, M_AWIN, OP_AB, false, H->st);
      } else {
        StencilCall<double> c = call<double>(H, 0, op == HZ_OP_B, nrhs);
        c.x = (const cx<double>*)x;
        c.y = (cx<double>*)y;
        fill(c);
        launch_stencil<double>(c, M_AWIN, OP_AB, false, H->st);
      }
      HZ_LAUNCHED();
    } catch (...) {
      H->st = old;
      throw;
    }
    H->st = old;
  });
}

hz_status iofd_jacobi(hz_handle* H, int level, int op, int precision, int nsweeps, double omega, const void* g,
                      void* y, int nrhs, void* stream) {
  if (!H) return HZ_EINVAL;
  return run_guarded(H, [&] {
    HZ_REQUIRE(level >= 0 && level <= 2, "level must be 0, 1 or 2");
    HZ_REQUIRE(op == (level == 0 ? HZ_OP_A : HZ_OP_B),
               "the Jacobi maps of Algorithm 1 smooth A_h on level 0 and B on levels 1 and 2");
    HZ_REQUIRE(nsweeps == 1 || nsweeps == 2, "nsweeps must be 1 or 2");
    HZ_REQUIRE(g && y && g != y, "g and y must be distinct non-null device pointers");
    HZ_REQUIRE(nrhs >= 1 && nrhs <= H->max_nrhs, "nrhs out of range");
    HZ_REQUIRE(precision == HZ_C64 || precision == HZ_C128, "precision must be HZ_C64 or HZ_C128");
    cudaStream_t old = H->st;
    H->st = (cudaStream_t)stream;
    try {
      if (precision == HZ_C64) {
        jacobi<float>(H, level, level != 0, false, (const cx<float>*)g, (cx<float>*)y, nsweeps, omega, nrhs);
      } else {
        prepare_dinv_double(H);
        jacobi<double>(H, level, level != 0, false, (const cx<double>*)g, (cx<double>*)y, nsweeps, omega, nrhs);
      }
    } catch (...) {
      H->st = old;
      throw;
    }
    H->st = old;
  });
}

hz_status threegrid_precond(hz_handle* H, const void* r, void* z, int nrhs, int adjoint, int precision, void* stream) {
  if (!H) return HZ_EINVAL;
  return run_guarded(H, [&] {
    HZ_REQUIRE(r && z && r != z, "r and z must be distinct non-null device pointers");
    HZ_REQUIRE(nrhs >= 1 && nrhs <= H->max_nrhs, "nrhs out of range");
    HZ_REQUIRE(precision == HZ_C64 || precision == HZ_C128, "precision must be HZ_C64 or HZ_C128");
    cudaStream_t old = H->st;
    H->st = (cudaStream_t)stream;
    try {
      if (precision == HZ_C64) {
        ensure_work<float>(H);
        precond<float>(H, (const cx<float>*)r, (cx<float>*)z, nrhs, adjoint != 0);
      } else {
        ensure_work<double>(H);
        precond<double>(H, (const cx<double>*)r, (cx<double>*)z, nrhs, adjoint != 0);
      }
    } catch (...) {
      H->st = old;
      throw;
    }
    H->st = old;
  });
}

hz_status helmholtz_solve(hz_handle* H, const hz_source* src, int nsrc, void* v_dev, void* u_dev, hz_stats* stats) {
  if (!H) return HZ_EINVAL;
  bool noconv = false;
  hz_status st = run_guarded(H, [&] {
    HZ_REQUIRE(src && v_dev && nsrc >= 1, "null argument or nsrc < 1");
    H->st = H->own;
    HZ_CK(cudaDeviceSynchronize());  // inputs written on other streams are complete
    auto t0 = std::chrono::steady_clock::now();
    const long long N = H->lev[0].N;
    SolveOut tot;
    for (int s0 = 0; s0 < nsrc; s0 += H->max_nrhs) {
      const int ns = std::min(H->max_nrhs, nsrc - s0);
      source_rhs(H, src + s0, ns, H->b128);  // b = Q_h f (Eq. iofd-complete-system)
      cx<double>* v = (cx<double>*)v_dev + (size_t)s0 * N;
      SolveOut o;
      try {
        o = solve_c128(H, H->b128, v, ns, false);
      } catch (const Fail& f) {
        if (f.st == HZ_ENONFINITE) check_bottom_err(H);  // a barrier that gave up explains the NaN
        throw;
      }
      tot.pc += o.pc;
      tot.passes += o.passes;
      tot.rel = std::max(tot.rel, o.rel);
      if (u_dev) {
        cx<double>* u = (cx<double>*)u_dev + (size_t)s0 * N;
        if (H->p.precision == HZ_C64) {
          // u = Q_h v in the hierarchy's precision (complex64), widened on output
          launch_c128_to_c64_scaled(v, H->x64, nullptr, (int)N, ns, H->st);
          q_apply<float>(H, false, H->x64, H->b64, ns);
          launch_c64_to_c128(H->b64, u, (int)N, ns, H->st);
          HZ_LAUNCHED();
        } else {
          q_apply<double>(H, false, v, u, ns);  // u = Q_h v
        }
      }
    }
    HZ_CK(cudaStreamSynchronize(H->st));
    check_bottom_err(H);
    if (stats) {
      stats->pc_calls = tot.pc;
      stats->refine_passes = tot.passes;
      stats->rel_res = tot.rel;
      stats->t_setup = H->t_setup;
      stats->t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      stats->device_bytes = H->al.bytes;
      for (int L = 0; L < 3; ++L) {
        stats->zblock[L] = H->lev[L].zblock;
        stats->zblock_frame[L] = H->lev[L].zblock_f > 0 ? H->lev[L].zblock_f : H->lev[L].zblock;
      }
    }
    noconv = !(tot.rel <= H->p.tol);
  });
  if (st == HZ_OK && noconv) {
    H->err = "max_pc or max_refine reached before the tolerance";
    return HZ_ENOCONV;
  }
  return st;
}

hz_status helmholtz_adjoint_grad(hz_handle* H, const hz_source* src, int nsrc, const int* rec, int nrec,
                                 const double* dobs, double* misfit, double* grad_dev, hz_stats* stats) {
  if (!H) return HZ_EINVAL;
  bool noconv = false;
  hz_status st = run_guarded(H, [&] {
    HZ_REQUIRE(src && rec && dobs && misfit && grad_dev && nsrc >= 1 && nrec >= 1, "null argument or empty set");
    H->st = H->own;
    HZ_CK(cudaDeviceSynchronize());
    auto t0 = std::chrono::steady_clock::now();
    const Level& L0 = H->lev[0];
    const long long N = L0.N;
    const int nr = H->max_nrhs;
    if (!H->vg) {
      H->vg = H->al.get<cx<double>>((size_t)N * nr);
      H->ug = H->al.get<cx<double>>((size_t)N * nr);
      H->lg = H->al.get<cx<double>>((size_t)N * nr);
      H->rf = H->al.get<cx<double>>((size_t)N * nr);
      H->g_ext = H->al.get<double>((size_t)N);
    }
    if (H->rec_cap < nrec) {
      H->rec_dev = H->al.get<int>((size_t)nrec);
      H->recv = H->al.get<cx<double>>((size_t)nrec * nr);
      H->rec_cap = nrec;
    }
    std::vector<int> flat(nrec);
    for (int q = 0; q < nrec; ++q) {
      int ix = rec[3 * q], iy = rec[3 * q + 1], iz = rec[3 * q + 2];
      HZ_REQUIRE(ix >= 0 && ix < L0.nx && iy >= 0 && iy < L0.ny && iz >= 0 && iz < L0.nz, "receiver outside grid");
      flat[q] = (int)(((long long)iz * L0.ny + iy) * L0.nx + ix);
    }
    {
      std::vector<int> sorted(flat);
      std::sort(sorted.begin(), sorted.end());
      HZ_REQUIRE(std::adjacent_find(sorted.begin(), sorted.end()) == sorted.end(), "receivers must be distinct");
    }
    HZ_CK(cudaMemcpyAsync(H->rec_dev, flat.data(), nrec * sizeof(int), cudaMemcpyHostToDevice, H->st));
    HZ_CK(cudaMemsetAsync(H->g_ext, 0, N * sizeof(double), H->st));
    double J = 0.0;
    SolveOut tot;
    for (int s0 = 0; s0 < nsrc; s0 += nr) {
      const int ns = std::min(nr, nsrc - s0);
      upload_sources(H, src + s0, ns);
      q_apply<double>(H, false, H->f128, H->b128, ns);
      SolveOut o = solve_c128(H, H->b128, H->vg, ns, false);
      tot.pc += o.pc;
      tot.passes += o.passes;
      tot.rel = std::max(tot.rel, o.rel);
      q_apply<double>(H, false, H->vg, H->ug, ns);
      launch_gather<double>(H->ug, H->rec_dev, nrec, (int)N, ns, H->recv, H->st);
      HZ_LAUNCHED();
      std::vector<double> uv((size_t)nrec * ns * 2);
      HZ_CK(cudaMemcpyAsync(uv.data(), H->recv, uv.size() * sizeof(double), cudaMemcpyDeviceToHost, H->st));
      HZ_CK(cudaStreamSynchronize(H->st));
      for (int s = 0; s < ns; ++s)
        for (int q = 0; q < nrec; ++q) {
          size_t i = ((size_t)s * nrec + q) * 2;
          size_t j = ((size_t)(s0 + s) * nrec + q) * 2;
          uv[i] -= dobs[j];
          uv[i + 1] -= dobs[j + 1];
          J += 0.5 * (uv[i] * uv[i] + uv[i + 1] * uv[i + 1]);
        }
      HZ_CK(cudaMemcpyAsync(H->recv, uv.data(), uv.size() * sizeof(double), cudaMemcpyHostToDevice, H->st));
      launch_zero<double>(H->rf, N * ns, H->st);
      launch_scatter<double>(H->recv, H->rec_dev, nrec, (int)N, ns, H->rf, H->st);  // R^T (R u - d)
      q_apply<double>(H, true, H->rf, H->b128, ns);                                 // Q^H R^T (R u - d)
      HZ_LAUNCHED();
      SolveOut oa = solve_c128(H, H->b128, H->lg, ns, true);                         // A^H lambda = ...
      tot.pc += oa.pc;
      tot.passes += oa.passes;
      tot.rel = std::max(tot.rel, oa.rel);
      launch_gradient(view<double>(H, 0), tview<double>(H), H->g.omega * H->g.h, H->vg, H->lg, H->f128, H->rf, ns,
                      H->g_ext, H->st);
      HZ_LAUNCHED();
    }
    launch_fold_pml(H->g_ext, grad_dev, L0.nx, L0.ny, L0.nz, L0.n_pml, H->st);
    HZ_LAUNCHED();
    HZ_CK(cudaStreamSynchronize(H->st));
    check_bottom_err(H);
    *misfit = J;
    if (stats) {
      stats->pc_calls = tot.pc;
      stats->refine_passes = tot.passes;
      stats->rel_res = tot.rel;
      stats->t_setup = H->t_setup;
      stats->t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      stats->device_bytes = H->al.bytes;
      for (int L = 0; L < 3; ++L) {
        stats->zblock[L] = H->lev[L].zblock;
        stats->zblock_frame[L] = H->lev[L].zblock_f > 0 ? H->lev[L].zblock_f : H->lev[L].zblock;
      }
    }
    noconv = !(tot.rel <= H->p.tol);
  });
  if (st == HZ_OK && noconv) {
    H->err = "max_pc or max_refine reached before the tolerance";
    return HZ_ENOCONV;
  }
  return st;
}

}  // extern "C"

// ============================================================================
// Allocation-free residual: r = g - Op x and ||r||^2 per right-hand side.
//
// For callers that cannot allocate device memory at call time: code running
// while a CUDA graph is being captured with allocation forbidden, real-time
// loops whose memory budget is fixed up front, or hosts embedding the solver
// inside an allocator they do not control.  The grid-wide reduction of the
// residual norm needs scratch (one partial sum per block and per right-hand
// side, plus an arrival counter per right-hand side); here it lives in the
// file-scope device array below instead of the handle's workspace, so the
// call itself never allocates.  The handle must already exist.
// ============================================================================
namespace {

constexpr long long kResidStaticPartials = 1 << 16;  // doubles (512 KiB)
constexpr int kResidStaticMaxRhs = 64;
// [partials (kResidStaticPartials) | arrival counters (64 unsigned, in 32 double slots)]
static __device__ __align__(256) double g_resid_static[kResidStaticPartials + kResidStaticMaxRhs / 2];

constexpr int kMaxDevices = 64;
// Device address of the array per device, written by the first call on that
// device; threads racing on that first call all write the same address, so no
// lock is taken.
double* g_resid_static_addr[kMaxDevices] = {};

// Host-side stand-in -> device address, once per device (with that device current).
double* resid_static_scratch() {
  int dev = 0;
  HZ_CK(cudaGetDevice(&dev));
  HZ_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal out of range");
  if (!g_resid_static_addr[dev]) {
    void* p = nullptr;
    HZ_CK(cudaGetSymbolAddress(&p, g_resid_static));
    g_resid_static_addr[dev] = (double*)p;
  }
  return g_resid_static_addr[dev];
}

}  // namespace

extern "C" hz_status iofd_residual_static(hz_handle* H, int level, int op, int precision, const void* g,
                                          const void* x, void* r, double* norm2, int nrhs, void* stream) {
  if (!H) return HZ_EINVAL;
  return run_guarded(H, [&] {
    HZ_REQUIRE(level >= 0 && level <= 2, "level must be 0, 1 or 2");
    HZ_REQUIRE(op == HZ_OP_A || op == HZ_OP_B || op == HZ_OP_A_ADJ || op == HZ_OP_B_ADJ,
               "operator must be A, B or their adjoints");
    HZ_REQUIRE(g && x && r && norm2 && r != x && r != g, "g, x, r, norm2 must be non-null and r distinct");
    HZ_REQUIRE(precision == HZ_C64 || precision == HZ_C128, "precision must be HZ_C64 or HZ_C128");
    HZ_REQUIRE(nrhs >= 1 && nrhs <= H->max_nrhs, "nrhs out of range");
    HZ_REQUIRE(nrhs <= kResidStaticMaxRhs, "nrhs exceeds the static scratch limit of 64 right-hand sides");
    const Level& lv = H->lev[level];
    const bool adj0 = (op == HZ_OP_A_ADJ || op == HZ_OP_B_ADJ);
    // partial sums of the launch that will run (forward and adjoint tile differently)
    const long long need = resid_blocks(lv, level, nrhs, adj0) * nrhs;
    HZ_REQUIRE(need <= kResidStaticPartials,
               "grid too large for the static scratch (" + std::to_string(need) + " block partial sums > " +
                   std::to_string(kResidStaticPartials) + ")");
    double* base = resid_static_scratch();
    cudaStream_t st = (cudaStream_t)stream;
    Reduce red;
    red.partial = base;
    red.out = norm2;
    red.count = reinterpret_cast<unsigned*>(base + kResidStaticPartials);
    // the arrival counters must start at zero (the last block also resets them)
    HZ_CK(cudaMemsetAsync(red.count, 0, sizeof(unsigned) * nrhs, st));
    const bool adj = adj0;
    const bool shifted = (op == HZ_OP_B || op == HZ_OP_B_ADJ);
    if (precision == HZ_C64) {
      StencilCall<float> c = call<float>(H, level, shifted, nrhs);
      c.x = (const cx<float>*)x;
      c.g = (const cx<float>*)g;
      c.y = (cx<float>*)r;
      c.red = red;
      launch_stencil<float>(c, M_RESID, OP_AB, adj, st);
    } else {
      StencilCall<double> c = call<double>(H, level, shifted, nrhs);
      c.x = (const cx<double>*)x;
      c.g = (const cx<double>*)g;
      c.y = (cx<double>*)r;
      c.red = red;
      launch_stencil<double>(c, M_RESID, OP_AB, adj, st);
    }
    HZ_LAUNCHED();
  });
}
