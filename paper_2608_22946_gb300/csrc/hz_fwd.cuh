// Forward 27-point IOFD stencil for sm_103a, accumulation form.
//
// Operator (Sec. 2.2, Eq. iofd-shell-form and Eq. pml-second-difference):
//   (H x)_i = -ell^-2 sum_j [ abar_j S_j + achk_j D_j ] - s kappa_i^2 ell^-2 (M x)_i
// with T_j(t) the transverse-weighted sum of x over the plane at offset t along
// axis j (weights alpha_4, alpha_5/4, (1 - alpha_4 - alpha_5)/4 of row i),
// S_j = T_j(+1) + T_j(-1) - 2 T_j(0), D_j = T_j(+1) - T_j(-1), and s = 1 (A) or
// 1 + i sigma (B, Eq. shifted-iofd-levels).  Where no axis is stretched the row
// is the shell form of Eq. iofd-shell-coefficients,
//   (H x)_z = C_0 c_z + C_1 (e_z + c_{z-1} + c_{z+1}) + C_2 (k_z + e_{z-1} + e_{z+1})
//           + C_3 (k_{z-1} + k_{z+1}),
// where c, e, k are the centre, the four face neighbours and the four corners
// of the row's column in one z-plane.  A stretched axis adds
//   eps+_j (T_j(+1) - T_j(0)) + eps-_j (T_j(-1) - T_j(0)),
//   eps+-_j = -ell^-2 (abar_j - 1 +- achk_j),
// to the shell row: the same operator written as shell part plus PML correction.
//
// Kernel design.  A block owns a tile of columns (two adjacent x columns per
// thread in the wide tiles) and marches in z.  Every plane that arrives through
// the cp.async ring is reduced once to (c, e, k) per column (and, on PML
// tiles, to the in-plane differences the corrections need) and added to the
// three rows it touches: it completes the row below (as that row's "+1"
// plane), adds to its own row, and opens the row above (as its "-1" plane).
// Live state per column: two accumulators per right-hand side and the
// coefficients of three rows.  The coefficients of a row are evaluated once,
// from kappa, and serve every right-hand side the block carries (a block
// processes RB right-hand sides of the same tile).
//
// Coefficients: C_m(kappa) = (L_m(eta) - kappa^2 M_m(eta)) / ell^2 with the
// stiffness and mass shell weights L_m, M_m of the cubic Hermite alpha's and
// eta = kappa / 2 pi clamped at 0.4 (Eq. iofd-clamped-coordinate).  On each
// table segment kappa = 2 pi (s_k + u), so C_m and K_m = kappa^2 M_m / ell^2
// are quintics in u; beyond the clamp the alpha's are constant and they are
// quadratics in u = eta - 0.4.  The host writes these polynomials once per
// level (one extra segment for the clamp), so a row costs one segment lookup
// and a Horner pass per coefficient.  B uses C_m - i sigma K_m.
#pragma once

#include <algorithm>
#include <type_traits>

#include "hz_kernels.h"

namespace hz {

// operator kinds of the forward kernel
enum { OPK_A = 0, OPK_B = 1, OPK_Q = 2 };

// Per-level coefficient table, laid out [kind][segment][power j][function m]
// with NS = nseg + 1 segments (segment nseg is eta >= 0.4), power basis in u;
// power-major so that one Horner step loads the j-th coefficient of every
// function of a kind at once:
constexpr int kCtCA = 24;  // C_0..C_3 of A_ell, 4 quintics
constexpr int kCtK = 24;   // K_0..K_3 = kappa^2 M_m / ell^2, 4 quintics
constexpr int kCtT = 8;    // alpha_4, alpha_5, 2 cubics (transverse weights of the PML rows)
constexpr int kCtQ = 16;   // Q_h shell weights, 4 cubics (Eq. q-operator)
constexpr int kCtPerSeg = kCtCA + kCtK + kCtT + kCtQ;
__host__ __device__ constexpr int ct_off_K(int ns) { return kCtCA * ns; }
__host__ __device__ constexpr int ct_off_T(int ns) { return (kCtCA + kCtK) * ns; }
__host__ __device__ constexpr int ct_off_Q(int ns) { return (kCtCA + kCtK + kCtT) * ns; }
constexpr int kMaxZb = 64;  // largest z-block of a forward launch

// Tile of NPX * TXT by TYT node columns, TXT * TYT threads.  A plane of the
// tile and its one-node halo is PWS x PHS values.
template <int NPX_, int TXT_, int TYT_>
struct FShape {
  static constexpr int NPX = NPX_, TXT = TXT_, TYT = TYT_, NT = TXT_ * TYT_;
  static constexpr int TWN = NPX_ * TXT_;
  static constexpr int PWS = TWN + 2, PHS = TYT_ + 2, PLN = PWS * PHS;
  static constexpr int NSLOT = (PLN + NT - 1) / NT;
  static_assert(NPX_ == 1 || PWS % 2 == 0, "paired columns need 16-byte aligned halo rows");
};
// Tile sets.  Fine grids (set 0): two x-adjacent columns per thread, 64 x 8
// rectangle tiles and 64 x 4 strips below / above the rectangle.  Coarse grids
// (set 1, few nodes per block: parallelism matters more than per-node work):
// one column per thread, 32 x 8 and 32 x 4.  Both: 4 x 32 strips left / right.
template <int SS>
struct Shapes;
template <>
struct Shapes<0> {
  using Rect = FShape<2, 32, 8>;
  using Wide = FShape<2, 32, 4>;
  using Tall = FShape<1, 4, 32>;
};
template <>
struct Shapes<1> {
  using Rect = FShape<1, 32, 8>;
  using Wide = FShape<1, 32, 4>;
  using Tall = FShape<1, 4, 32>;
};
// Small grids (set 2): rectangle and frame tiles in ONE launch of 256-thread
// blocks (launch latency dominates there): 32 x 8, 64 x 4 and 4 x 64.
template <>
struct Shapes<2> {
  using Rect = FShape<1, 32, 8>;
  using Wide = FShape<1, 64, 4>;
  using Tall = FShape<1, 4, 64>;
};
// grids below this many nodes use the coarse tile set, below kFusedNodes the fused launch
constexpr long long kCoarseNodes = 8LL << 20;
constexpr long long kFusedNodes = 1LL << 20;

// ring depth by precision, mode and right-hand sides per block; PREF = NSTG - 2
// planes are in flight, and the stage of the previous plane stays readable
template <class R, int MODE, int RB>
struct FStages {
  static constexpr int v = (sizeof(R) == 8 || MODE == M_J2 || RB > 1) ? 3 : 6;
};

template <class R, int MODE, int OPK, class TS, int RB>
struct FLayout {
  static constexpr int NSTG = FStages<R, MODE, RB>::v;
  static constexpr size_t CXB = sizeof(cx<R>);
  static constexpr size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
  static constexpr size_t ring = (size_t)NSTG * RB * TS::PLN * CXB;
  static constexpr size_t dring = MODE == M_J2 ? (size_t)NSTG * TS::PLN * CXB : 0;
  static constexpr size_t y1 = MODE == M_J2 ? (size_t)RB * TS::PLN * CXB : 0;
  static constexpr size_t kap = (size_t)NSTG * TS::NT * TS::NPX * sizeof(R);
  static constexpr int tabn = (OPK == OPK_Q ? kCtQ : kCtCA + (OPK == OPK_B ? kCtK : 0) + kCtT) * (kMaxSeg + 1);
  static constexpr size_t tab = (size_t)tabn * sizeof(R);
  static constexpr size_t ez = OPK == OPK_Q ? 0 : (size_t)(kMaxZb + 2) * 2 * CXB;
  static constexpr size_t o_ring = 0;
  static constexpr size_t o_dring = a16(o_ring + ring);
  static constexpr size_t o_y1 = a16(o_dring + dring);
  static constexpr size_t o_kap = a16(o_y1 + y1);
  static constexpr size_t o_tab = a16(o_kap + kap);
  static constexpr size_t o_ez = a16(o_tab + tab);
  static constexpr size_t o_red = a16(o_ez + ez);
  static constexpr size_t bytes = o_red + 32 * sizeof(double);
};

// ----------------------------------------------------------------------------
// launch layout
// ----------------------------------------------------------------------------
// Which tiles a launch covers.  Rectangle / grid launches: tile (t, blockIdx.y)
// has its origin at (ox + rw t, oy + rh blockIdx.y) and writes columns up to
// (rx1, ry1).  Frame launches: the PML frame around the PML-free rectangle
// [px0, px1] x [py0, py1], as rows of ww x wh tiles below and above it (its x
// range; only y is stretched there) followed by columns of tw x th tiles left
// and right of it (all y; x and, in the corners, y stretched).  All launches
// of one operator application share one block numbering (bid_offset,
// nblk_total) so that a fused grid reduction spans them.
struct TileMap {
  int rw = 64, rh = 8, ww = 64, wh = 4, tw = 4, th = 32;  // rectangle, wide- and tall-strip tile sizes
  int ox = 0, oy = 0, ntx = 1, nrow = 1, rx1 = 0, ry1 = 0;
  int nx = 0, ny = 0, px0 = 0, px1 = -1, py0 = 0, py1 = -1;
  int nwx = 0, nw_lo = 0, nw_hi = 0;  // 64 x 4 tiles per strip row; tile rows below / above
  int nty = 0, nt_lo = 0, nt_hi = 0;  // rows of 4 x 32 tiles; tiles left / right per row
  int count = 0;                      // frame tiles per z-block
  int bid_offset = 0, nblk_total = 1;
};

struct FrameTile {
  int x0, y0, rx1, ry1;
  bool wide;
};

__host__ __device__ __forceinline__ FrameTile decode_frame(const TileMap& m, int t) {
  FrameTile f;
  const int nw = m.nwx * (m.nw_lo + m.nw_hi);
  if (t < nw) {
    const int r = t / m.nwx, c = t - r * m.nwx;
    f.x0 = m.px0 + c * m.ww;
    f.rx1 = m.px1;
    if (r < m.nw_lo) {
      f.y0 = r * m.wh;
      f.ry1 = m.py0 - 1;
    } else {
      f.y0 = m.py1 + 1 + (r - m.nw_lo) * m.wh;
      f.ry1 = m.ny - 1;
    }
    f.wide = true;
  } else {
    const int u = t - nw, per = m.nt_lo + m.nt_hi;
    const int r = u / per, c = u - r * per;
    f.y0 = r * m.th;
    f.ry1 = m.ny - 1;
    if (c < m.nt_lo) {
      f.x0 = c * m.tw;
      f.rx1 = m.px0 - 1;
    } else {
      f.x0 = m.px1 + 1 + (c - m.nt_lo) * m.tw;
      f.rx1 = m.nx - 1;
    }
    f.wide = false;
  }
  return f;
}

// Row form of a whole-grid tile: 0 shell (x and y outside the PML), 2 general.
__host__ __device__ __forceinline__ int grid_tile_form(int x0, int y0, int tw, int th, int nx, int ny,
                                                      const int* plo, const int* phi) {
  const int xe = min(x0 + tw - 1, nx - 1), ye = min(y0 + th - 1, ny - 1);
  const bool px = x0 >= plo[0] && xe <= phi[0], py = y0 >= plo[1] && ye <= phi[1];
  return (px && py) ? 0 : 2;
}

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void fcp_async(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES),
               "r"(pred ? BYTES : 0));
}
__device__ __forceinline__ void fcp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void fcp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// N values from 16-byte (float: 8-byte when N = 2) aligned shared memory
template <int N>
__device__ __forceinline__ void lds_vec(const float* p, float* d) {
  static_assert(N % 2 == 0, "");
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 v = reinterpret_cast<const float4*>(p)[i];
      d[4 * i] = v.x;
      d[4 * i + 1] = v.y;
      d[4 * i + 2] = v.z;
      d[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 v = reinterpret_cast<const float2*>(p)[i];
      d[2 * i] = v.x;
      d[2 * i + 1] = v.y;
    }
  }
}
template <int N>
__device__ __forceinline__ void lds_vec(const double* p, double* d) {
  static_assert(N % 2 == 0, "");
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const double2 v = reinterpret_cast<const double2*>(p)[i];
    d[2 * i] = v.x;
    d[2 * i + 1] = v.y;
  }
}

// NF polynomials of degree DEG stored power-major (c[j * NF + m]), evaluated
// together at u: one vector load per power
template <class R, int NF, int DEG>
__device__ __forceinline__ void horner_pm(const R* c, R u, R* v) {
  lds_vec<NF>(c + DEG * NF, v);
#pragma unroll
  for (int j = DEG - 1; j >= 0; --j) {
    R cj[NF];
    lds_vec<NF>(c + j * NF, cj);
#pragma unroll
    for (int m = 0; m < NF; ++m) v[m] = v[m] * u + cj[m];
  }
}

// complex accumulate helpers
template <class R>
__device__ __forceinline__ void cfma(cx<R>& acc, R w, cx<R> v) {
  acc.x += w * v.x;
  acc.y += w * v.y;
}
template <class R>
__device__ __forceinline__ void cfma(cx<R>& acc, cx<R> w, cx<R> v) {
  acc.x += w.x * v.x - w.y * v.y;
  acc.y += w.x * v.y + w.y * v.x;
}
template <class R>
__device__ __forceinline__ cx<R> cmulw(R w, cx<R> v) { return mkc<R>(w * v.x, w * v.y); }
template <class R>
__device__ __forceinline__ cx<R> cmulw(cx<R> w, cx<R> v) { return w * v; }

// coefficients of one row
template <class R, bool CPLX>
struct RowC {
  R c[4];
};
template <class R>
struct RowC<R, true> {
  cx<R> c[4];
};
template <class R>
struct RowT {
  R a4, q5, qb;
};

// segment and local coordinate of kappa in the coefficient table (segment
// ns - 1 is the clamp eta >= 0.4)
template <class R>
__device__ __forceinline__ int seg_of(R kap, int ns, R ds, R inv_ds, R& u) {
  const R e = kap * (R)kInv2Pi;
  int seg = (int)(e * inv_ds);
  seg = seg < 0 ? 0 : (seg > ns - 1 ? ns - 1 : seg);
  u = e - (R)seg * ds;
  return seg;
}

// PML transverse weights (alpha_4, alpha_5 / 4, (1 - alpha_4 - alpha_5) / 4) of a
// row; tT points at the alpha_4 / alpha_5 block of the shared-memory table
template <class R>
__device__ __forceinline__ RowT<R> eval_t(const R* tT, int seg, R u) {
  R a[2];
  horner_pm<R, 2, 3>(tT + seg * kCtT, u, a);
  return RowT<R>{a[0], a[1] * (R)0.25, ((R)1 - a[0] - a[1]) * (R)0.25};
}

// Shell coefficients of a row from its kappa (segment lookup + Horner).
template <class R, int OPK>
__device__ __forceinline__ void eval_c(const R* sT, int ns, int seg, R u, cx<R> shift, RowC<R, OPK == OPK_B>& C) {
  if constexpr (OPK == OPK_Q) {
    horner_pm<R, 4, 3>(sT + seg * kCtQ, u, C.c);
  } else if constexpr (OPK == OPK_B) {
    R cr[4], km[4];
    horner_pm<R, 4, 5>(sT + seg * kCtCA, u, cr);
    horner_pm<R, 4, 5>(sT + ct_off_K(ns) + seg * kCtK, u, km);
#pragma unroll
    for (int m = 0; m < 4; ++m) C.c[m] = mkc<R>(cr[m] - (shift.x - (R)1) * km[m], -shift.y * km[m]);
  } else {
    horner_pm<R, 4, 5>(sT + seg * kCtCA, u, C.c);
  }
}

// the alpha_4 / alpha_5 block of the shared-memory table: [C][K (B only)][T]
template <int OPK>
__device__ __forceinline__ int t_block(int ns) { return OPK == OPK_B ? ct_off_T(ns) : ct_off_K(ns); }

// Contribution of one plane to a row at plane offset RHO (= plane - row):
// shell weights, PML corrections in x / y (Ac, Bc) and, in a z-PML row, the z
// correction eps * T_z with the row's own transverse weights.
template <int RHO, bool CORR, bool ZP, class R, class CT>
__device__ __forceinline__ cx<R> contrib(const CT& C, const RowT<R>& T, cx<R> c, cx<R> e, cx<R> k, cx<R> Ac,
                                         cx<R> Bc, bool zp, cx<R> ez) {
  cx<R> h;
  if constexpr (RHO == 0) {
    h = cmulw(C.c[0], c);
    cfma(h, C.c[1], e);
    cfma(h, C.c[2], k);
  } else {
    h = cmulw(C.c[1], c);
    cfma(h, C.c[2], e);
    cfma(h, C.c[3], k);
  }
  if constexpr (CORR) {
    if constexpr (RHO == 0) {
      cfma(h, T.a4, Ac);
      cfma(h, T.q5, Bc);
    } else {
      cfma(h, T.q5, Ac);
      cfma(h, T.qb, Bc);
    }
  }
  if constexpr (ZP) {
    if (zp) {
      cx<R> tau = cmulw(T.a4, c);
      cfma(tau, T.q5, e);
      cfma(tau, T.qb, k);
      h += ez * tau;
    }
  }
  return h;
}

// ----------------------------------------------------------------------------
// one block: tile (x0, y0) of shape TS writing columns up to (rx1, ry1), z-block
// blockIdx.z, right-hand sides rhs0 .. rhs0 + RB - 1
// ----------------------------------------------------------------------------
// FORM: 0 shell (x and y outside the PML), 3 y stretched, 2 x and y stretched.
// ZP: some row of the block lies in the z-PML (blocks wholly between the two
// z-layers carry no z-correction code at all).
template <class R, int MODE, int OPK, int FORM, bool ZP, class TS, int RB>
__device__ __forceinline__ void fwd_tile(const StencilCall<R>& a, unsigned char* smem, int zblock, int x0, int y0,
                                         int rx1, int ry1, int rhs0, unsigned bid, unsigned nblk) {
  using LY = FLayout<R, MODE, OPK, TS, RB>;
  constexpr int NSTG = LY::NSTG, PREF = NSTG - 2;
  constexpr int NPX = TS::NPX, PWS = TS::PWS, PLN = TS::PLN, NT = TS::NT, NSLOT = TS::NSLOT;
  constexpr bool CPLX = OPK == OPK_B;
  constexpr bool XC = FORM == 2, YC = FORM == 2 || FORM == 3, CORR = XC || YC;
  static_assert(PREF >= 1, "ring too short");
  static_assert(!ZP || OPK != OPK_Q, "Q_h has no PML terms");
  using CT = RowC<R, CPLX>;

  const LevelView<R>& Lv = a.lv;
  cx<R>* sX = reinterpret_cast<cx<R>*>(smem + LY::o_ring);
  cx<R>* sD = reinterpret_cast<cx<R>*>(smem + LY::o_dring);
  cx<R>* sY1 = reinterpret_cast<cx<R>*>(smem + LY::o_y1);
  R* sK = reinterpret_cast<R*>(smem + LY::o_kap);
  R* sT = reinterpret_cast<R*>(smem + LY::o_tab);
  cx<R>* sEz = reinterpret_cast<cx<R>*>(smem + LY::o_ez);
  double* sRed = reinterpret_cast<double*>(smem + LY::o_red);

  const int tid = threadIdx.x;
  const int tx = tid % TS::TXT, ty = tid / TS::TXT;
  const int nx = Lv.nx, ny = Lv.ny, nz = Lv.nz;
  // row window (z-slab brick): M_AWIN only; every other mode covers all rows
  constexpr bool WIN = MODE == M_AWIN;
  const int zr0 = WIN ? a.zr0 : 0, xz0 = WIN ? a.xz0 : 0;
  const int zr1 = (WIN && a.zr1 > 0) ? a.zr1 : nz;
  const int zb0 = zr0 + blockIdx.z * zblock, zb1 = min(zb0 + zblock, zr1);
  const long long xs = (WIN && a.xstride > 0) ? a.xstride : Lv.N, ys = (WIN && a.ystride > 0) ? a.ystride : Lv.N;
  const int nplanes = zb1 - zb0 + 2;
  const int plane_sz = nx * ny;
  const long long N = Lv.N;
  const int ns = a.tab.nseg + 1;
  const R ds = a.tab.ds, inv_ds = a.tab.inv_ds;
  const int zlo = Lv.plain_lo[2], zhi = Lv.plain_hi[2];

  // coefficient tables (this level) and the z-PML factors of rows zb0-1 .. zb1
  {
    const R* g = Lv.ctab;
    if constexpr (OPK == OPK_Q) {
      for (int i = tid; i < kCtQ * ns; i += NT) sT[i] = g[ct_off_Q(ns) + i];
    } else {
      const int nca = (kCtCA + (CPLX ? kCtK : 0)) * ns;
      for (int i = tid; i < nca; i += NT) sT[i] = g[i];
      if constexpr (CORR || ZP)
        for (int i = tid; i < kCtT * ns; i += NT) sT[nca + i] = g[ct_off_T(ns) + i];
      if constexpr (ZP)
        for (int t = tid; t < nplanes; t += NT) {
          const int r = zb0 - 1 + t;
          const bool ok = r >= 0 && r < nz;
          sEz[2 * t] = ok ? Lv.eps[2][0][r] : mkc<R>(0, 0);
          sEz[2 * t + 1] = ok ? Lv.eps[2][1][r] : mkc<R>(0, 0);
        }
    }
  }

  // this thread's columns
  const int gx0 = x0 + NPX * tx, gy = y0 + ty;
  bool act[NPX];
#pragma unroll
  for (int i = 0; i < NPX; ++i) act[i] = (gx0 + i <= rx1) && (gy <= ry1);
  const int col0 = gy * nx + gx0;  // used only where act
  cx<R> exp_[NPX], exm_[NPX], eyp = mkc<R>(0, 0), eym = mkc<R>(0, 0);
#pragma unroll
  for (int i = 0; i < NPX; ++i) {
    exp_[i] = mkc<R>(0, 0);
    exm_[i] = mkc<R>(0, 0);
    if constexpr (XC) {
      const int xi = min(gx0 + i, nx - 1);
      exp_[i] = Lv.eps[0][0][xi];
      exm_[i] = Lv.eps[0][1][xi];
    }
  }
  if constexpr (YC) {
    const int yi = min(gy, ny - 1);
    eyp = Lv.eps[1][0][yi];
    eym = Lv.eps[1][1][yi];
  }

  // this thread's load slots of every halo plane
  int go[NSLOT];
  bool gin[NSLOT];
#pragma unroll
  for (int j = 0; j < NSLOT; ++j) {
    const int li = tid + j * NT;
    const int ly = li / PWS, lx = li - ly * PWS;
    const int qx = x0 - 1 + lx, qy = y0 - 1 + ly;
    gin[j] = li < PLN && qx >= 0 && qx < nx && qy >= 0 && qy < ny;
    go[j] = gin[j] ? qy * nx + qx : 0;
  }
  auto slot_ok = [&](int j) { return j < NSLOT - 1 || tid + j * NT < PLN; };

  // group kk (ring stage st): halo plane zb0-1+kk of every right-hand side (and
  // of 1/diag for the Jacobi map), kappa of the tile's own columns one plane higher
  auto issue = [&](int kk, int st) {
    const int q = zb0 - 1 + kk;
    const bool zin = (unsigned)q < (unsigned)nz;
    const int zo = zin ? q * plane_sz : 0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const cx<R>* Xr = a.x + (size_t)(rhs0 + r) * (size_t)xs + (zin ? zo - (long long)xz0 * plane_sz : 0);
      cx<R>* dst = sX + ((size_t)st * RB + r) * PLN + tid;
#pragma unroll
      for (int j = 0; j < NSLOT; ++j)
        if (slot_ok(j)) fcp_async<sizeof(cx<R>)>(dst + j * NT, Xr + go[j], zin && gin[j]);
    }
    if constexpr (MODE == M_J2) {
      const cx<R>* Dp = a.dinv + zo;
      cx<R>* dst = sD + (size_t)st * PLN + tid;
#pragma unroll
      for (int j = 0; j < NSLOT; ++j)
        if (slot_ok(j)) fcp_async<sizeof(cx<R>)>(dst + j * NT, Dp + go[j], zin && gin[j]);
    }
    const int q1 = q + 1;
    const bool z1 = (unsigned)q1 < (unsigned)nz;
#pragma unroll
    for (int i = 0; i < NPX; ++i) {
      const bool pk = z1 && act[i];
      fcp_async<sizeof(R)>(sK + ((size_t)st * NT + tid) * NPX + i, Lv.kappa + (pk ? q1 * plane_sz + col0 + i : 0),
                           pk);
    }
    fcp_commit();
  };

#pragma unroll
  for (int k = 0; k < PREF; ++k) {
    if (k < nplanes) issue(k, k);
    else fcp_commit();
  }

  // accumulators of rows p (role 0 this step) and p-1 / p+1 (completed, then
  // reopened); coefficients of rows p-1, p, p+1 (slot = row mod 3).  PML tiles
  // also hold the rows' transverse weights; shell tiles in a z-PML block hold
  // the rows' kappa and evaluate the weights where a z-correction needs them.
  constexpr bool HOLD_T = CORR;
  constexpr bool HOLD_K = !CORR && ZP;
  cx<R> accP[RB][NPX], accM[RB][NPX];
  CT C[3][NPX];
  RowT<R> Th[HOLD_T ? 3 : 1][NPX];
  R kq[HOLD_K ? 3 : 1][NPX];
  R nrm2[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    nrm2[r] = 0;
#pragma unroll
    for (int i = 0; i < NPX; ++i) accP[r][i] = accM[r][i] = mkc<R>(0, 0);
  }
#pragma unroll
  for (int sl = 0; sl < (HOLD_T ? 3 : 1); ++sl)
#pragma unroll
    for (int i = 0; i < NPX; ++i) Th[sl][i] = RowT<R>{0, 0, 0};
  const R* tT = sT + t_block<OPK>(ns);
  const R om = a.omega_j;
  const int lc0 = (ty + 1) * PWS + NPX * tx + 1;  // halo index of this thread's first column
  int st = 0, stp = NSTG - 1, sti = PREF;       // ring stages of planes k, k-1 and k+PREF

  auto step = [&](auto Uc, int k) {
    constexpr int U = decltype(Uc)::value;                          // k mod 3
    constexpr int CP = U, CN = (U + 1) % 3, CM = (U + 2) % 3;      // coefficient slots of rows p, p+1, p-1
    fcp_wait<PREF - 1>();
    __syncthreads();
    if (k + PREF < nplanes) issue(k + PREF, sti);
    else fcp_commit();
    const int p = zb0 - 1 + k;             // plane that arrived
    const bool o1 = k + 3 <= nplanes;      // row p+1 lies in this z-block
    const bool o0 = k >= 1 && k + 2 <= nplanes;
    const bool o3 = k >= 2;                // row p-1 completes
    const cx<R>* Xs = sX + (size_t)st * RB * PLN;
    const cx<R>* Xsp = sX + (size_t)stp * RB * PLN;

    // own-column values of row p-1 read early (their latency overlaps the step)
    cx<R> gq[RB][NPX];
    constexpr bool WANT_G = MODE == M_RESID || MODE == M_JSWEEP || MODE == M_J2;
    if constexpr (WANT_G) {
      const cx<R>* src = (MODE == M_J2) ? a.base : a.g;
      if (o3 && src) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int i = 0; i < NPX; ++i)
            gq[r][i] = act[i] ? src[(size_t)(rhs0 + r) * (size_t)N + (p - 1) * plane_sz + col0 + i] : mkc<R>(0, 0);
      }
    }

    // coefficients of row p+1 (kappa arrived with this plane's group)
    if (o1) {
      R kv[NPX];
      const R* kp = sK + ((size_t)st * NT + tid) * NPX;
#pragma unroll
      for (int i = 0; i < NPX; ++i) kv[i] = kp[i];
#pragma unroll
      for (int i = 0; i < NPX; ++i) {
        R u;
        const int seg = seg_of(kv[i], ns, ds, inv_ds, u);
        eval_c<R, OPK>(sT, ns, seg, u, a.mass_shift, C[CN][i]);
        if constexpr (HOLD_T) Th[CN][i] = eval_t(tT, seg, u);
        if constexpr (HOLD_K) kq[CN][i] = kv[i];
      }
    }

    // z-PML rows among p-1, p, p+1 (uniform) and their correction factors
    bool zq3 = false, zq0 = false, zq1 = false;
    cx<R> ez3 = mkc<R>(0, 0), ez0 = mkc<R>(0, 0), ez1 = mkc<R>(0, 0);
    RowT<R> T3[NPX], T0[NPX], T1[NPX];
#pragma unroll
    for (int i = 0; i < NPX; ++i) {
      if constexpr (HOLD_T) {
        T3[i] = Th[CM][i];
        T0[i] = Th[CP][i];
        T1[i] = Th[CN][i];
      } else {
        T3[i] = T0[i] = T1[i] = RowT<R>{0, 0, 0};
      }
    }
    if constexpr (ZP) {
      zq1 = o1 && (p + 1 < zlo || p + 1 > zhi);
      zq0 = o0 && (p < zlo || p > zhi);
      zq3 = o3 && (p - 1 < zlo || p - 1 > zhi);
      // sEz[2 t + {0, 1}] = eps+, eps- of row zb0 - 1 + t; row p is t = k
      if (zq3) ez3 = sEz[2 * (k - 1)];
      if (zq0) ez0 = -(sEz[2 * k] + sEz[2 * k + 1]);
      if (zq1) ez1 = sEz[2 * (k + 1) + 1];
      if constexpr (HOLD_K) {
#pragma unroll
        for (int i = 0; i < NPX; ++i) {
          R u;
          if (zq3) T3[i] = eval_t(tT, seg_of(kq[CM][i], ns, ds, inv_ds, u), u);
          if (zq0) T0[i] = eval_t(tT, seg_of(kq[CP][i], ns, ds, inv_ds, u), u);
          if (zq1) T1[i] = eval_t(tT, seg_of(kq[CN][i], ns, ds, inv_ds, u), u);
        }
      }
    }

    // Jacobi map: first sweep y1 = omega D^-1 g on the whole halo plane
    if constexpr (MODE == M_J2) {
      const cx<R>* Ds = sD + (size_t)st * PLN;
#pragma unroll
      for (int j = 0; j < NSLOT; ++j) {
        if (!slot_ok(j)) continue;
        const int li = tid + j * NT;
        const cx<R> d = Ds[li];
#pragma unroll
        for (int r = 0; r < RB; ++r) sY1[(size_t)r * PLN + li] = om * (d * Xs[(size_t)r * PLN + li]);
      }
      __syncthreads();
    }

#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const cx<R>* P = (MODE == M_J2) ? sY1 + (size_t)r * PLN : Xs + (size_t)r * PLN;
      cx<R> v[3][NPX + 2];
#pragma unroll
      for (int row = 0; row < 3; ++row) {
        const cx<R>* q = P + (ty + row) * PWS + NPX * tx;
        if constexpr (NPX == 2 && sizeof(R) == 4) {
          const float4 u0 = *reinterpret_cast<const float4*>(q);
          const float4 u1 = *reinterpret_cast<const float4*>(q + 2);
          v[row][0] = mkc<R>(u0.x, u0.y);
          v[row][1] = mkc<R>(u0.z, u0.w);
          v[row][2] = mkc<R>(u1.x, u1.y);
          v[row][3] = mkc<R>(u1.z, u1.w);
        } else {
#pragma unroll
          for (int j = 0; j < NPX + 2; ++j) v[row][j] = q[j];
        }
      }
      cx<R> sv[NPX + 2];
#pragma unroll
      for (int j = 0; j < NPX + 2; ++j) sv[j] = v[0][j] + v[2][j];
#pragma unroll
      for (int i = 0; i < NPX; ++i) {
        const cx<R> c = v[1][i + 1];
        const cx<R> ex = v[1][i] + v[1][i + 2];
        const cx<R> e = ex + sv[i + 1];
        const cx<R> kk = sv[i] + sv[i + 2];
        cx<R> Ac = mkc<R>(0, 0), Bc = mkc<R>(0, 0);
        if constexpr (YC) {
          const cx<R> Up = v[2][i + 1] - c, Um = v[0][i + 1] - c;
          const cx<R> Vp = (v[2][i] + v[2][i + 2]) - ex, Vm = (v[0][i] + v[0][i + 2]) - ex;
          Ac = eyp * Up + eym * Um;
          Bc = eyp * Vp + eym * Vm;
        }
        if constexpr (XC) {
          const cx<R> Up = v[1][i + 2] - c, Um = v[1][i] - c;
          const cx<R> Vp = sv[i + 2] - sv[i + 1], Vm = sv[i] - sv[i + 1];
          cfma(Ac, exp_[i], Up);
          cfma(Ac, exm_[i], Um);
          cfma(Bc, exp_[i], Vp);
          cfma(Bc, exm_[i], Vm);
        }
        if (o3) {
          const cx<R> h = accM[r][i] + contrib<+1, CORR, ZP>(C[CM][i], T3[i], c, e, kk, Ac, Bc, zq3, ez3);
          if (act[i]) {
            const int idx = (p - 1) * plane_sz + col0 + i;
            cx<R> out;
            if constexpr (MODE == M_APPLY || MODE == M_AWIN) {
              out = h;
            } else if constexpr (MODE == M_RESID) {
              out = gq[r][i] - h;
              nrm2[r] += abs2(out);
            } else if constexpr (MODE == M_J2) {
              const cx<R> g0 = Xsp[(size_t)r * PLN + lc0 + i];
              const cx<R> d0 = sD[(size_t)stp * PLN + lc0 + i];
              out = om * (d0 * g0) + om * (d0 * (g0 - h));
              if (a.base) out += gq[r][i];
            } else {  // M_JSWEEP
              const cx<R> x0c = Xsp[(size_t)r * PLN + lc0 + i];
              const cx<R> d0 = a.dinv[idx];
              out = x0c + om * (d0 * (gq[r][i] - h));
            }
            a.y[(size_t)(rhs0 + r) * (size_t)ys + idx - (long long)zr0 * plane_sz] = out;
          }
        }
        if (o0) accP[r][i] += contrib<0, CORR, ZP>(C[CP][i], T0[i], c, e, kk, Ac, Bc, zq0, ez0);
        if (o1) accM[r][i] = contrib<-1, CORR, ZP>(C[CN][i], T1[i], c, e, kk, Ac, Bc, zq1, ez1);
      }
    }
    // row p+1 (now in accM) is next step's role-0 row; row p becomes its row to complete
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < NPX; ++i) {
        const cx<R> t = accP[r][i];
        accP[r][i] = accM[r][i];
        accM[r][i] = t;
      }
    stp = st;
    st = (st + 1 == NSTG) ? 0 : st + 1;
    sti = (sti + 1 == NSTG) ? 0 : sti + 1;
  };

  for (int k0 = 0; k0 < nplanes; k0 += 3) {
    // each step is skipped past the last plane (uniform across the block)
    if (k0 + 0 < nplanes) step(std::integral_constant<int, 0>{}, k0 + 0);
    if (k0 + 1 < nplanes) step(std::integral_constant<int, 1>{}, k0 + 1);
    if (k0 + 2 < nplanes) step(std::integral_constant<int, 2>{}, k0 + 2);
  }
  fcp_wait<0>();

  if constexpr (MODE == M_RESID) {
    if (a.red.out) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const unsigned rr = (unsigned)(rhs0 + r);
        double s = block_sum((double)nrm2[r], sRed, tid, NT);
        if (tid == 0) a.red.partial[(size_t)rr * nblk + bid] = s;
        if (last_block_arrive(a.red.count + rr, nblk, tid)) {
          double t = 0.0;
          for (unsigned b = tid; b < nblk; b += NT) t += __ldcg(a.red.partial + (size_t)rr * nblk + b);
          t = block_sum(t, sRed, tid, NT);
          if (tid == 0) {
            a.red.out[rr] = t;
            if (a.red.root) a.red.root[rr] = sqrt(t);
            if (a.red.inv_root) a.red.inv_root[rr] = t > 1e-300 ? 1.0 / sqrt(t) : 0.0;
            a.red.count[rr] = 0;
          }
        }
      }
    }
  }
}

// does any output row of z-block blockIdx.z (of the call's row window) lie in the z-PML?
template <int MODE, class R>
__device__ __forceinline__ bool block_in_zpml(const StencilCall<R>& a, int zblock) {
  const LevelView<R>& L = a.lv;
  constexpr bool WIN = MODE == M_AWIN;
  const int zr0 = WIN ? a.zr0 : 0, zr1 = (WIN && a.zr1 > 0) ? a.zr1 : L.nz;
  const int zb0 = zr0 + blockIdx.z * zblock, zb1 = min(zb0 + zblock, zr1);
  return zb0 < L.plain_lo[2] || zb1 - 1 > L.plain_hi[2];
}

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------
// resident blocks per SM the register allocation targets
template <class R, int RB, int NT, int NPX, int OPK>
struct FMinB {
  static constexpr int v = sizeof(R) == 8 ? 1 : (NT == 256 ? (NPX == 1 && RB == 1 && OPK != OPK_B ? 3 : 2) : 4);
};

// the PML-free rectangle (shell rows)
template <class R, int MODE, int OPK, int RB, int SS>
__global__ void __launch_bounds__(Shapes<SS>::Rect::NT,
                                  FMinB<R, RB, Shapes<SS>::Rect::NT, Shapes<SS>::Rect::NPX, OPK>::v)
    k_fwd_rect(StencilCall<R> a, int zblock, TileMap tm) {
  using ShRect = typename Shapes<SS>::Rect;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int ng = a.nrhs / RB;
  const int g = blockIdx.x % ng, t = blockIdx.x / ng;
  const unsigned bid = (unsigned)(tm.bid_offset + t + tm.ntx * (blockIdx.y + gridDim.y * blockIdx.z));
  const int x0 = tm.ox + t * ShRect::TWN, y0 = tm.oy + (int)blockIdx.y * ShRect::TYT;
  const unsigned nb = (unsigned)tm.nblk_total;
  if (block_in_zpml<MODE>(a, zblock))
    fwd_tile<R, MODE, OPK, 0, true, ShRect, RB>(a, fsm, zblock, x0, y0, tm.rx1, tm.ry1, g * RB, bid, nb);
  else
    fwd_tile<R, MODE, OPK, 0, false, ShRect, RB>(a, fsm, zblock, x0, y0, tm.rx1, tm.ry1, g * RB, bid, nb);
}

// the PML frame around it: strips below and above the rectangle (y stretched)
// and left and right of it (x stretched, y too in the corners)
template <class R, int MODE, int OPK, int RB, int SS>
__global__ void __launch_bounds__(Shapes<SS>::Wide::NT, FMinB<R, RB, Shapes<SS>::Wide::NT, 2, OPK>::v)
    k_fwd_frame(StencilCall<R> a, int zblock, TileMap tm) {
  using ShWide = typename Shapes<SS>::Wide;
  using ShTall = typename Shapes<SS>::Tall;
  static_assert(ShWide::NT == ShTall::NT, "one block size for both frame tile shapes");
  extern __shared__ __align__(16) unsigned char fsm[];
  const int ng = a.nrhs / RB;
  const int g = blockIdx.x % ng, t = blockIdx.x / ng;
  const FrameTile f = decode_frame(tm, t);
  const unsigned bid = (unsigned)(tm.bid_offset + t + tm.count * blockIdx.z);
  const unsigned nb = (unsigned)tm.nblk_total;
  const bool zp = block_in_zpml<MODE>(a, zblock);
  if (f.wide) {
    if (zp) fwd_tile<R, MODE, OPK, 3, true, ShWide, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
    else fwd_tile<R, MODE, OPK, 3, false, ShWide, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
  } else {
    if (zp) fwd_tile<R, MODE, OPK, 2, true, ShTall, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
    else fwd_tile<R, MODE, OPK, 2, false, ShTall, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
  }
}

// a whole (small) grid in one launch, the row form chosen per tile; Q_h (shell
// form everywhere) always takes this path
template <class R, int MODE, int OPK, int RB, int SS>
__global__ void __launch_bounds__(Shapes<SS>::Rect::NT, sizeof(R) == 8 ? 1 : 2) k_fwd_grid(StencilCall<R> a, int zblock,
                                                                                           TileMap tm) {
  using ShRect = typename Shapes<SS>::Rect;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int ng = a.nrhs / RB;
  const int g = blockIdx.x % ng, t = blockIdx.x / ng;
  const unsigned bid = (unsigned)(t + tm.ntx * (blockIdx.y + gridDim.y * blockIdx.z));
  const int x0 = t * ShRect::TWN, y0 = (int)blockIdx.y * ShRect::TYT;
  const int rx1 = a.lv.nx - 1, ry1 = a.lv.ny - 1;
  const unsigned nb = (unsigned)tm.nblk_total;
  if constexpr (OPK == OPK_Q) {
    fwd_tile<R, MODE, OPK, 0, false, ShRect, RB>(a, fsm, zblock, x0, y0, rx1, ry1, g * RB, bid, nb);
  } else {
    const bool zp = block_in_zpml<MODE>(a, zblock);
    if (grid_tile_form(x0, y0, ShRect::TWN, ShRect::TYT, a.lv.nx, a.lv.ny, a.lv.plain_lo, a.lv.plain_hi) == 0) {
      if (zp) fwd_tile<R, MODE, OPK, 0, true, ShRect, RB>(a, fsm, zblock, x0, y0, rx1, ry1, g * RB, bid, nb);
      else fwd_tile<R, MODE, OPK, 0, false, ShRect, RB>(a, fsm, zblock, x0, y0, rx1, ry1, g * RB, bid, nb);
    } else {
      fwd_tile<R, MODE, OPK, 2, true, ShRect, RB>(a, fsm, zblock, x0, y0, rx1, ry1, g * RB, bid, nb);
    }
  }
}

// rectangle and frame tiles of a small grid in one launch (tile set 2): block t
// < RW * RH (tm.ntx * tm.rows) is a rectangle tile, the rest frame tiles
template <class R, int MODE, int OPK, int RB>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 1 : 2) k_fwd_fused(StencilCall<R> a, int zblock, TileMap tm) {
  using SRect = Shapes<2>::Rect;
  using SWide = Shapes<2>::Wide;
  using STall = Shapes<2>::Tall;
  static_assert(SRect::NT == 256 && SWide::NT == 256 && STall::NT == 256, "one block size");
  extern __shared__ __align__(16) unsigned char fsm[];
  const int ng = a.nrhs / RB;
  const int g = blockIdx.x % ng, t = blockIdx.x / ng;
  const int nrect = tm.ntx * tm.nrow;
  const unsigned bid = (unsigned)(t + (nrect + tm.count) * blockIdx.z);
  const unsigned nb = (unsigned)tm.nblk_total;
  const bool zp = block_in_zpml<MODE>(a, zblock);
  if (t < nrect) {
    const int x0 = tm.px0 + (t % tm.ntx) * SRect::TWN, y0 = tm.py0 + (t / tm.ntx) * SRect::TYT;
    if (zp) fwd_tile<R, MODE, OPK, 0, true, SRect, RB>(a, fsm, zblock, x0, y0, tm.px1, tm.py1, g * RB, bid, nb);
    else fwd_tile<R, MODE, OPK, 0, false, SRect, RB>(a, fsm, zblock, x0, y0, tm.px1, tm.py1, g * RB, bid, nb);
    return;
  }
  const FrameTile f = decode_frame(tm, t - nrect);
  if (f.wide) {
    if (zp) fwd_tile<R, MODE, OPK, 3, true, SWide, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
    else fwd_tile<R, MODE, OPK, 3, false, SWide, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
  } else {
    fwd_tile<R, MODE, OPK, 2, true, STall, RB>(a, fsm, zblock, f.x0, f.y0, f.rx1, f.ry1, g * RB, bid, nb);
  }
}

template <class R, int MODE, int OPK, int RB>
constexpr size_t fwd_smem_fused() {
  return std::max(std::max(FLayout<R, MODE, OPK, Shapes<2>::Rect, RB>::bytes,
                           FLayout<R, MODE, OPK, Shapes<2>::Wide, RB>::bytes),
                  FLayout<R, MODE, OPK, Shapes<2>::Tall, RB>::bytes);
}

template <class R, int MODE, int OPK, int RB, int SS>
constexpr size_t fwd_smem_rect() { return FLayout<R, MODE, OPK, typename Shapes<SS>::Rect, RB>::bytes; }
template <class R, int MODE, int OPK, int RB, int SS>
constexpr size_t fwd_smem_frame() {
  return std::max(FLayout<R, MODE, OPK, typename Shapes<SS>::Wide, RB>::bytes,
                  FLayout<R, MODE, OPK, typename Shapes<SS>::Tall, RB>::bytes);
}

}  // namespace hz
