// Gather-form forward stencil of the coarse levels (2h, 4h) for sm_103a.
//
// Operator as in hz_fwd.cuh (Sec. 2.2, Eq. iofd-shell-form / Eq.
// pml-second-difference).  Design for small, L2-resident grids, where latency
// and parallelism matter more than instructions per node: one column per
// thread, a CTA of 256 threads marching in z over a block of planes that
// stream through a 6-stage cp.async ring; each thread keeps three planes of
// in-plane partial sums (centre, face ring, corner ring, and on PML tiles the
// first differences) in registers and evaluates the row's five Hermite alpha's
// (Eq. iofd-clamped-coordinate) per row.  Large coarse levels run the
// PML-free rectangle (32 x 8 tiles, shell rows) and the PML frame (64 x 4 /
// 4 x 64 tiles, tensor-product rows) as two launches on two streams; small
// ones one launch of 16 x 16 tiles choosing the row form per tile.  One CTA
// serves one right-hand side.  Epilogues: residual with its norm, the
// two-sweep Jacobi map from zero, one further Jacobi sweep.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "hz_gram_solve.cuh"
#include "hz_kernels.h"

namespace hz {
namespace gather {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int PW = TX + 2, PH = TY + 2, PLANE = PW * PH;

// Column-tile shapes of the forward kernel (NT threads, one column each).  A
// plane of a tile plus its one-node halo is TX_ + 2 by TY_ + 2 nodes and is
// loaded with at most two cp.async per thread.
template <int TX_, int TY_>
struct TileShape {
  static constexpr int TXS = TX_, TYS = TY_, PWS = TX_ + 2, PLN = (TX_ + 2) * (TY_ + 2);
  static_assert(TX_ * TY_ == NT, "one column per thread");
  static_assert(PLN <= 2 * NT, "two load slots per thread");
};
using TileSq = TileShape<TX, TY>;   // the PML-free rectangle; whole small grids
using TileW = TileShape<64, 4>;     // PML strips below and above the rectangle (all x)
using TileT = TileShape<4, 64>;     // PML strips left and right of it (its y range)
using TileG = TileShape<16, 16>;    // whole small grids (coarse levels): fewer idle columns
constexpr int NSTAGE = 6;   // shared-memory plane ring
constexpr int PREF = 5;     // planes in flight ahead of the one consumed (NSTAGE - 1)

// ----------------------------------------------------------------------------
// cp.async (zero fill when pred is false; the source address is then unused)
// ----------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool pred) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  int sz = pred ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES), "r"(sz));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ----------------------------------------------------------------------------
// per-plane partial sums of the 3x3 in-plane neighbourhood
// ----------------------------------------------------------------------------
template <class R, bool GEN> struct Part;
template <class R> struct Part<R, false> { cx<R> c, e, k; };
// PML tiles: e = ex + ey and d = ex - ey (x and y neighbours), k corners, g* and k*
// antisymmetric first differences along x and y
template <class R> struct Part<R, true> { cx<R> c, e, d, k, gx, gy, kx, ky; };

template <class R>
__device__ __forceinline__ void zero_part(Part<R, false>& o) {
  o.c = o.e = o.k = mkc<R>(0, 0);
}
template <class R>
__device__ __forceinline__ void zero_part(Part<R, true>& o) {
  o.c = o.e = o.d = o.k = o.gx = o.gy = o.kx = o.ky = mkc<R>(0, 0);
}

template <int PWS, class R>
__device__ __forceinline__ void partials(const cx<R>* P, int lx, int ly, Part<R, false>& o) {
  const cx<R>* r0 = P + (ly - 1) * PWS + lx;
  const cx<R>* r1 = r0 + PWS;
  const cx<R>* r2 = r1 + PWS;
  cx<R> m0 = r0[-1], c0 = r0[0], p0 = r0[1];
  cx<R> m1 = r1[-1], c1 = r1[0], p1 = r1[1];
  cx<R> m2 = r2[-1], c2 = r2[0], p2 = r2[1];
  o.c = c1;
  o.e = (m1 + p1) + (c0 + c2);
  o.k = (m0 + p0) + (m2 + p2);
}
template <int PWS, class R>
__device__ __forceinline__ void partials(const cx<R>* P, int lx, int ly, Part<R, true>& o) {
  const cx<R>* r0 = P + (ly - 1) * PWS + lx;
  const cx<R>* r1 = r0 + PWS;
  const cx<R>* r2 = r1 + PWS;
  cx<R> m0 = r0[-1], c0 = r0[0], p0 = r0[1];
  cx<R> m1 = r1[-1], c1 = r1[0], p1 = r1[1];
  cx<R> m2 = r2[-1], c2 = r2[0], p2 = r2[1];
  o.c = c1;
  const cx<R> ex = m1 + p1, ey = c0 + c2;
  o.e = ex + ey;
  o.d = ex - ey;
  o.k = (m0 + p0) + (m2 + p2);
  o.gx = p1 - m1;
  o.gy = c2 - c0;
  o.kx = (p0 + p2) - (m0 + m2);
  o.ky = (m2 + p2) - (m0 + p0);
}

// ----------------------------------------------------------------------------
// row application from three planes of partials
// ----------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ cx<R> stiff_mass(const Part<R, false>& m, const Part<R, false>& o, const Part<R, false>& p,
                                            const R* a, cx<R> abz, cx<R> acz, cx<R>& Mv) {
  const R a1 = a[0], a2 = a[1], a3 = a[2], a4 = a[3], a5 = a[4];
  const R q5 = a5 * (R)0.25, qb = ((R)1 - a4 - a5) * (R)0.25;
  const R w1 = a2 * (R)(1.0 / 6.0), w2 = a3 * (R)(1.0 / 12.0), w3 = ((R)1 - a1 - a2 - a3) * (R)0.125;
  cx<R> T3m = a4 * m.c + q5 * m.e + qb * m.k;
  cx<R> T30 = a4 * o.c + q5 * o.e + qb * o.k;
  cx<R> T3p = a4 * p.c + q5 * p.e + qb * p.k;
  cx<R> S3 = (T3p + T3m) - (R)2 * T30;
  cx<R> D3 = T3p - T3m;
  cx<R> S12 = a4 * (o.e - (R)4 * o.c) + q5 * ((R)2 * (o.k - o.e)) + q5 * ((m.e + p.e) - (R)4 * (m.c + p.c)) +
              qb * ((R)2 * ((m.k + p.k) - (m.e + p.e)));
  Mv = a1 * o.c + w1 * (o.e + m.c + p.c) + w2 * (o.k + m.e + p.e) + w3 * (m.k + p.k);
  return S12 + abz * S3 + acz * D3;
}

// General row (PML tiles).  With sb = (abar_x + abar_y)/2 and db = (abar_x - abar_y)/2,
// abar_x S_1 + abar_y S_2 = sb (S_1 + S_2) + db (S_1 - S_2), where S_1 + S_2 is the
// shell combination of e and S_1 - S_2 = (a4 + 2 a5/4) d_0 + (a5/4 + 2 b/4)(d_- + d_+).
template <int FORM, class R>
__device__ __forceinline__ cx<R> stiff_mass(const Part<R, true>& m, const Part<R, true>& o, const Part<R, true>& p,
                                            const R* a, cx<R> sb, cx<R> db, cx<R> acx, cx<R> acy, cx<R> abz,
                                            cx<R> acz, cx<R>& Mv) {
  const R a1 = a[0], a2 = a[1], a3 = a[2], a4 = a[3], a5 = a[4];
  const R q5 = a5 * (R)0.25, qb = ((R)1 - a4 - a5) * (R)0.25;
  const R w1 = a2 * (R)(1.0 / 6.0), w2 = a3 * (R)(1.0 / 12.0), w3 = ((R)1 - a1 - a2 - a3) * (R)0.125;
  cx<R> T3m = a4 * m.c + q5 * m.e + qb * m.k;
  cx<R> T30 = a4 * o.c + q5 * o.e + qb * o.k;
  cx<R> T3p = a4 * p.c + q5 * p.e + qb * p.k;
  cx<R> S3 = (T3p + T3m) - (R)2 * T30;
  cx<R> D3 = T3p - T3m;
  cx<R> S12 = a4 * (o.e - (R)4 * o.c) + q5 * ((R)2 * (o.k - o.e)) + q5 * ((m.e + p.e) - (R)4 * (m.c + p.c)) +
              qb * ((R)2 * ((m.k + p.k) - (m.e + p.e)));
  cx<R> Sd = (a4 + (R)2 * q5) * o.d + (q5 + (R)2 * qb) * (m.d + p.d);
  Mv = a1 * o.c + w1 * (o.e + m.c + p.c) + w2 * (o.k + m.e + p.e) + w3 * (m.k + p.k);
  cx<R> r = sb * S12 + db * Sd + abz * S3 + acz * D3;
  if constexpr (FORM != 3) r += acx * (a4 * o.gx + q5 * o.kx + q5 * (m.gx + p.gx) + qb * (m.kx + p.kx));
  if constexpr (FORM != 1) r += acy * (a4 * o.gy + q5 * o.ky + q5 * (m.gy + p.gy) + qb * (m.ky + p.ky));
  return r;
}

// Q_h row (Eq. q-operator) from the shell partials.
template <class R>
__device__ __forceinline__ cx<R> q_row(const Part<R, false>& m, const Part<R, false>& o, const Part<R, false>& p,
                                       const R* b) {
  const R q0 = b[0], q1 = b[1] * (R)(1.0 / 6.0), q2 = b[2] * (R)(1.0 / 12.0);
  const R q3 = ((R)1 - b[0] - b[1] - b[2]) * (R)0.125;
  return q0 * o.c + q1 * (o.e + m.c + p.c) + q2 * (o.k + m.e + p.e) + q3 * (m.k + p.k);
}

template <class R>
__device__ __forceinline__ cx<R> ldc(const cx<R>* p) { return *p; }

// ----------------------------------------------------------------------------
// forward kernel body
// ----------------------------------------------------------------------------
// alpha_1 and alpha_4 only (the diagonal needs no more)
template <class R>
__device__ __forceinline__ void table_a1a4(const R* __restrict__ tab, int nseg, R ds, R inv_ds, R eta, R& a1, R& a4) {
  int seg = (int)(eta * inv_ds);
  seg = seg < 0 ? 0 : (seg > nseg - 1 ? nseg - 1 : seg);
  R u = eta - (R)seg * ds;
  const R* c = tab + seg * kNumFn * 4;
  a1 = c[0] + u * (c[1] + u * (c[2] + u * c[3]));
  a4 = c[12] + u * (c[13] + u * (c[14] + u * c[15]));
}

// Which tiles a launch covers.  Rectangle launches (PATH 0: 32 x 8 tiles,
// PATH 2: 16 x 16): tile (t, blockIdx.y) has its origin at (ox + TXS t,
// oy + TYS blockIdx.y) and writes the columns up to (rx1, ry1).  Frame launches (PATH 1): the PML
// frame around the PML-free rectangle [px0, px1] x [py0, py1], as rows of
// 64 x 4 tiles below and above it (full x range) followed by rows of 4 x 64
// tiles left and right of it (its y range).  The blocks of all the launches of
// one operator application share one numbering (bid_offset, nblk_total) so
// that a fused grid reduction spans them.
struct TileMap {
  int ox = 0, oy = 0, ntx = 1, rx1 = 0, ry1 = 0;
  int nx = 0, ny = 0, px0 = 0, px1 = -1, py0 = 0, py1 = -1;
  int nwx = 0, nw_lo = 0, nw_hi = 0;  // 64 x 4 tiles per strip row; tile rows below / above
  int nty = 0, nt_lo = 0, nt_hi = 0;  // rows of 4 x 64 tiles; tiles left / right per row
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
    f.x0 = c * TileW::TXS;
    f.rx1 = m.nx - 1;
    if (r < m.nw_lo) {
      f.y0 = r * TileW::TYS;
      f.ry1 = m.py0 - 1;
    } else {
      f.y0 = m.py1 + 1 + (r - m.nw_lo) * TileW::TYS;
      f.ry1 = m.ny - 1;
    }
    f.wide = true;
  } else {
    const int u = t - nw, per = m.nt_lo + m.nt_hi;
    const int r = u / per, c = u - r * per;
    f.y0 = m.py0 + r * TileT::TYS;
    f.ry1 = m.py1;
    if (c < m.nt_lo) {
      f.x0 = c * TileT::TXS;
      f.rx1 = m.px0 - 1;
    } else {
      f.x0 = m.px1 + 1 + (c - m.nt_lo) * TileT::TXS;
      f.rx1 = m.nx - 1;
    }
    f.wide = false;
  }
  return f;
}

// One CTA: the tile of shape TL with origin (x0, y0), writing the columns up to
// (rx1, ry1) (both inside the grid), over z-block bz.
// Row forms: 0 shell (x and y outside the PML), 1 PML along x only, 2 general,
// 3 PML along y only.  Forms 1 and 3 drop the first-difference term of the
// PML-free axis, whose achk is exactly zero.
template <class R, int MODE, int OP, int FORM, class TL>
__device__ __forceinline__ void fwd_body(const StencilCall<R>& a, int zblock, int bz, const TileMap& tm, int rhs, int x0,
                                         int y0, int rx1, int ry1, unsigned bid, cx<R>* sX, cx<R>* sD, cx<R>* sY1,
                                         const R* sTab, double* sRed, R (*sKc)[NT], cx<R> (*sGc)[NT]) {
  constexpr int PWS = TL::PWS, PLN = TL::PLN;
  constexpr bool GEN = FORM != 0;
  const LevelView<R>& L = a.lv;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int tx = tid % TL::TXS, ty = tid / TL::TXS;
  const int zb0 = bz * zblock;
  const int zb1 = min(zb0 + zblock, L.nz);
  const int nplanes = zb1 - zb0 + 2;
  const long long N = L.N;
  const cx<R>* X = a.x + rhs * N;
  cx<R>* Y = a.y + rhs * N;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = (gx <= rx1) && (gy <= ry1);
  // fields have fewer than 2^31 nodes (checked at creation): 32-bit offsets
  const int col = gy * L.nx + gx;
  const int plane_sz = L.nx * L.ny;
  const R inv_ell2 = L.inv_ell2;
  const cx<R> shift = a.mass_shift;
  const int nseg = a.tab.nseg;
  const R ds = a.tab.ds, inv_ds = a.tab.inv_ds;
  const int zpl_lo = L.plain_lo[2], zpl_hi = L.plain_hi[2];

  // per-thread PML factors of its column (x, y fixed during the march)
  cx<R> abx = mkc<R>(1, 0), acx = mkc<R>(0, 0), aby = mkc<R>(1, 0), acy = mkc<R>(0, 0);
  if (GEN && OP == OP_AB) {
    int cxi = min(gx, L.nx - 1), cyi = min(gy, L.ny - 1);
    abx = L.abar[0][cxi];
    acx = L.achk[0][cxi];
    aby = L.abar[1][cyi];
    acy = L.achk[1][cyi];
  }
  const cx<R> sbxy = (R)0.5 * (abx + aby), dbxy = (R)0.5 * (abx - aby);

  // this thread's (at most two) load slots in every plane, fixed for the march
  const bool has1 = tid + NT < PLN;
  const int li0 = tid, li1 = tid + NT;
  int go0 = 0, go1 = 0;
  bool in0, in1 = false;
  {
    int ly = li0 / PWS, lx = li0 - ly * PWS;
    int qx = x0 - 1 + lx, qy = y0 - 1 + ly;
    in0 = qx >= 0 && qx < L.nx && qy >= 0 && qy < L.ny;
    go0 = in0 ? qy * L.nx + qx : 0;
    if (has1) {
      ly = li1 / PWS;
      lx = li1 - ly * PWS;
      qx = x0 - 1 + lx;
      qy = y0 - 1 + ly;
      in1 = qx >= 0 && qx < L.nx && qy >= 0 && qy < L.ny;
      go1 = in1 ? qy * L.nx + qx : 0;
    }
  }
  const cx<R>* G = (MODE == M_RESID || MODE == M_JSWEEP) ? a.g + rhs * N : nullptr;
  const cx<R>* DI = a.dinv;  // shared by all right-hand sides
  // shared-memory addresses of this thread's load slots in stage 0
  const unsigned sx0 = (unsigned)__cvta_generic_to_shared(sX + li0);
  const unsigned sx1 = (unsigned)__cvta_generic_to_shared(sX + li1);
  constexpr unsigned kStageBytes = PLN * sizeof(cx<R>);
  auto issue = [&](int z, int st) {
    const bool zin = (unsigned)z < (unsigned)L.nz;
    const int zo = zin ? z * plane_sz : 0;
    const bool p0 = zin && in0, p1 = zin && in1;
    const unsigned so = (unsigned)st * kStageBytes;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sx0 + so), "l"(X + (zo + go0)),
                 "n"(sizeof(cx<R>)), "r"(p0 ? (int)sizeof(cx<R>) : 0));
    if (has1)
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sx1 + so), "l"(X + (zo + go1)),
                   "n"(sizeof(cx<R>)), "r"(p1 ? (int)sizeof(cx<R>) : 0));
    if (MODE == M_J2) {
      // precomputed 1/diag of every loaded node (zero outside the grid)
      cp_async<sizeof(cx<R>)>(sD + st * PLN + li0, DI + (zo + go0), p0);
      if (has1) cp_async<sizeof(cx<R>)>(sD + st * PLN + li1, DI + (zo + go1), p1);
    }
    {
      // the own row's kappa (and right-hand side) ride the same pipeline
      const bool pc = zin && active;
      cp_async<sizeof(R)>(&sKc[st][tid], L.kappa + (pc ? zo + col : 0), pc);
      if (MODE == M_RESID || MODE == M_JSWEEP)
        cp_async<sizeof(cx<R>)>(&sGc[st][tid], G + (pc ? zo + col : 0), pc);
    }
    cp_commit();
  };

  // prologue: PREF planes in flight (zb0-1 ...)
#pragma unroll
  for (int k = 0; k < PREF; ++k) {
    if (k < nplanes) issue(zb0 - 1 + k, k);
    else cp_commit();
  }

  // Three planes of partial sums and two planes of per-row values live in
  // registers; the z-march is unrolled by NSTAGE so that the ring stage, the
  // window slot and the previous/current slot of every step are compile-time
  // constants (no register moves, no modulo).
  Part<R, GEN> w[3];
  zero_part(w[0]);
  zero_part(w[1]);
  zero_part(w[2]);
  R kapv[2] = {0, 0};
  cx<R> gv[2] = {mkc<R>(0, 0), mkc<R>(0, 0)};      // RESID/JSWEEP rhs, J2 raw g
  cx<R> xcv[2] = {mkc<R>(0, 0), mkc<R>(0, 0)};     // JSWEEP iterate / J2 y1 at the centre
  cx<R> dinvv[2] = {mkc<R>(0, 0), mkc<R>(0, 0)};
  // per-thread sum of |r|^2 in the working precision (one FP64 add per node
  // would cost more than the rest of the row on this GPU's FP64 rate)
  R nrm2 = 0;
  const bool want_norm = MODE == M_RESID && a.red.out != nullptr;
  const cx<R>* Bs = a.base ? a.base + rhs * N : nullptr;

  auto step = [&](auto Sc, int k) {
    constexpr int S = decltype(Sc)::value;    // k % NSTAGE
    constexpr int CUR = S % 3, PRV = (S + 2) % 3, PP = (S + 1) % 3;
    constexpr int C2 = S % 2, P2 = (S + 1) % 2;
    const int zk = zb0 - 1 + k;
    cp_wait<PREF - 1>();
    __syncthreads();
    // plane k + PREF goes to the stage plane k - 1 used (PREF = NSTAGE - 1)
    if (k + PREF < nplanes) issue(zk + PREF, (S + PREF) % NSTAGE);
    else cp_commit();
    const bool zin = (unsigned)zk < (unsigned)L.nz;
    const cx<R>* P = sX + S * PLN;
    if (MODE == M_J2) {
      // y1 = omega D^-1 g on every loaded node of the plane (Eq. jacobi-map, first
      // sweep), each thread on its own load slots; g and D^-1 are zero-filled
      // outside the grid, so is y1
      sY1[li0] = a.omega_j * (sD[S * PLN + li0] * P[li0]);
      if (has1) sY1[li1] = a.omega_j * (sD[S * PLN + li1] * P[li1]);
      const int lc = (ty + 1) * PWS + tx + 1;
      gv[C2] = P[lc];
      dinvv[C2] = sD[S * PLN + lc];
      __syncthreads();
      xcv[C2] = sY1[lc];
      P = sY1;
    } else {
      if (MODE == M_RESID || MODE == M_JSWEEP) gv[C2] = sGc[S][tid];
      if (MODE == M_JSWEEP) xcv[C2] = P[(ty + 1) * PWS + tx + 1];
    }
    kapv[C2] = sKc[S][tid];
    partials<PWS>(P, tx + 1, ty + 1, w[CUR]);

    if (k >= 2 && active) {
      const Part<R, GEN>& wm = w[PP];
      const Part<R, GEN>& w0 = w[PRV];
      const Part<R, GEN>& wp = w[CUR];
      const R kap_prev = kapv[P2];
      const int z = zk - 1;
      const int idx = z * plane_sz + col;
      cx<R> out;
      if constexpr (OP == OP_Q) {
        R bv[3];
        table_eval<R, 5, 3>(sTab, nseg, ds, inv_ds, eta_star(kap_prev), bv);
        if constexpr (!GEN) out = q_row(wm, w0, wp, bv);
        else out = mkc<R>(0, 0);
      } else {
        R av[5];
        table_eval<R, 0, 5>(sTab, nseg, ds, inv_ds, eta_star(kap_prev), av);
        const R mk = inv_ell2 * kap_prev * kap_prev;
        cx<R> Hx, sab;
        bool shell_row = false;
        if constexpr (!GEN) {
          if (z >= zpl_lo && z <= zpl_hi) {
            // interior row: shell form of Eq. iofd-shell-form, stiffness and mass parts
            const R a1 = av[0], a2 = av[1], a3 = av[2], a4 = av[3], a5 = av[4];
            const R b = (R)1 - a4 - a5;
            const cx<R> N1 = w0.e + (wm.c + wp.c);
            const cx<R> N2 = w0.k + (wm.e + wp.e);
            const cx<R> N3 = wm.k + wp.k;
            const cx<R> Ls =
                ((R)6 * a4) * w0.c + (a5 - a4) * N1 + ((R)0.5 * (b - a5)) * N2 + ((R)(-0.75) * b) * N3;
            const cx<R> Ms = a1 * w0.c + (a2 * (R)(1.0 / 6.0)) * N1 + (a3 * (R)(1.0 / 12.0)) * N2 +
                             (((R)1 - a1 - a2 - a3) * (R)0.125) * N3;
            Hx = inv_ell2 * Ls - (mk * shift) * Ms;
            sab = mkc<R>(3, 0);
            shell_row = true;
          }
        }
        if (!shell_row) {
          const cx<R> abz = L.abar[2][z], acz = L.achk[2][z];
          cx<R> Mv, Ls;
          if constexpr (GEN) Ls = stiff_mass<FORM>(wm, w0, wp, av, sbxy, dbxy, acx, acy, abz, acz, Mv);
          else Ls = stiff_mass(wm, w0, wp, av, abz, acz, Mv);
          Hx = (-inv_ell2) * Ls - (mk * shift) * Mv;
          sab = abx + aby + abz;
        }
        if (MODE == M_APPLY) {
          out = Hx;
        } else if (MODE == M_RESID) {
          out = gv[P2] - Hx;
        } else if (MODE == M_J2) {
          out = xcv[P2] + a.omega_j * (dinvv[P2] * (gv[P2] - Hx));
          if (Bs) out += Bs[idx];
        } else {  // M_JSWEEP
          const cx<R> D = inv_ell2 * ((R)2 * av[3] * sab) - (mk * av[0]) * shift;
          out = xcv[P2] + a.omega_j * cdiv(gv[P2] - Hx, D);
        }
      }
      Y[idx] = out;
      if (MODE == M_RESID && want_norm) nrm2 += abs2(out);
    }
  };

  for (int k0 = 0; k0 < nplanes; k0 += NSTAGE) {
    // each step returns early past the last plane (uniform across the CTA)
    if (k0 + 0 < nplanes) step(std::integral_constant<int, 0>{}, k0 + 0);
    if (k0 + 1 < nplanes) step(std::integral_constant<int, 1>{}, k0 + 1);
    if (k0 + 2 < nplanes) step(std::integral_constant<int, 2>{}, k0 + 2);
    if (k0 + 3 < nplanes) step(std::integral_constant<int, 3>{}, k0 + 3);
    if (k0 + 4 < nplanes) step(std::integral_constant<int, 4>{}, k0 + 4);
    if (k0 + 5 < nplanes) step(std::integral_constant<int, 5>{}, k0 + 5);
  }
  cp_wait<0>();

  if (MODE == M_RESID && a.red.out) {
    double s = block_sum((double)nrm2, sRed, tid, NT);
    const unsigned nblk = (unsigned)tm.nblk_total;
    if (tid == 0) a.red.partial[(size_t)rhs * nblk + bid] = s;
    if (last_block_arrive(a.red.count + rhs, nblk, tid)) {
      double t = 0.0;
      for (unsigned b = tid; b < nblk; b += NT) t += __ldcg(a.red.partial + (size_t)rhs * nblk + b);
      // fixed-order combine: per-thread strided sums then the block tree
      t = block_sum(t, sRed, tid, NT);
      if (tid == 0) {
        a.red.out[rhs] = t;
        if (a.red.root) a.red.root[rhs] = sqrt(t);
        if (a.red.inv_root) a.red.inv_root[rhs] = t > 1e-300 ? 1.0 / sqrt(t) : 0.0;
        a.red.count[rhs] = 0;
      }
    }
  }
}

// PATH 0: the PML-free rectangle (shell rows); 1: the PML frame around it
// (general rows); 2: a whole (small) grid, the row form chosen per tile.
template <class R, int MODE, int OP, int PATH>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? (PATH == 0 ? 4 : 2) : 1) k_fwd(StencilCall<R> a, int zblock,
                                                                                      TileMap tm) {
  constexpr int PL = (PATH == 1) ? (TileW::PLN > TileT::PLN ? TileW::PLN : TileT::PLN) : TileSq::PLN;
  __shared__ __align__(16) cx<R> sX[NSTAGE * PL];
  __shared__ __align__(16) cx<R> sD[(MODE == M_J2) ? NSTAGE * PL : 1];
  __shared__ cx<R> sY1[(MODE == M_J2) ? PL : 1];
  __shared__ __align__(16) R sTab[kMaxSeg * kNumFn * 4];
  __shared__ R sKc[NSTAGE][NT];                                              // kappa of the own column
  __shared__ cx<R> sGc[(MODE == M_RESID || MODE == M_JSWEEP) ? NSTAGE : 1][NT];  // rhs of the own column
  __shared__ double sRed[32];
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int i = tid; i < a.tab.nseg * kNumFn * 4; i += NT) sTab[i] = a.tab.coef[i];
  // (visibility of sTab is ensured by the first __syncthreads of the march)
  const int rhs = blockIdx.x % a.nrhs;
  const int t = blockIdx.x / a.nrhs;
  if constexpr (PATH == 1 && OP != OP_Q) {
    const FrameTile f = decode_frame(tm, t);
    const unsigned bid = (unsigned)(tm.bid_offset + t + tm.count * blockIdx.z);
    if (f.wide) {
      // strips below / above the rectangle: PML along y only away from the corners
      const bool xplain = f.x0 >= a.lv.plain_lo[0] && f.x0 + TileW::TXS - 1 <= a.lv.plain_hi[0];
      if (xplain)
        fwd_body<R, MODE, OP, 3, TileW>(a, zblock, (int)blockIdx.z, tm, rhs, f.x0, f.y0, f.rx1, f.ry1, bid, sX, sD, sY1, sTab, sRed,
                                        sKc, sGc);
      else
        fwd_body<R, MODE, OP, 2, TileW>(a, zblock, (int)blockIdx.z, tm, rhs, f.x0, f.y0, f.rx1, f.ry1, bid, sX, sD, sY1, sTab, sRed,
                                        sKc, sGc);
    } else {
      // strips left / right of the rectangle lie in its y range: PML along x only
      fwd_body<R, MODE, OP, 1, TileT>(a, zblock, (int)blockIdx.z, tm, rhs, f.x0, f.y0, f.rx1, f.ry1, bid, sX, sD, sY1, sTab, sRed,
                                      sKc, sGc);
    }
  } else {
    const unsigned bid = (unsigned)(tm.bid_offset + t + tm.ntx * (blockIdx.y + gridDim.y * blockIdx.z));
    if constexpr (OP == OP_Q || PATH == 0) {
      const int x0 = tm.ox + t * TX, y0 = tm.oy + (int)blockIdx.y * TY;
      fwd_body<R, MODE, OP, 0, TileSq>(a, zblock, (int)blockIdx.z, tm, rhs, x0, y0, tm.rx1, tm.ry1, bid, sX, sD, sY1, sTab, sRed,
                                       sKc, sGc);
    } else {
      constexpr int GX = TileG::TXS, GY = TileG::TYS;
      const int x0 = tm.ox + t * GX, y0 = tm.oy + (int)blockIdx.y * GY;
      const LevelView<R>& L = a.lv;
      const bool plain = (x0 >= L.plain_lo[0]) && (x0 + GX - 1 <= L.plain_hi[0]) && (y0 >= L.plain_lo[1]) &&
                         (y0 + GY - 1 <= L.plain_hi[1]);
      if (plain)
        fwd_body<R, MODE, OP, 0, TileG>(a, zblock, (int)blockIdx.z, tm, rhs, x0, y0, tm.rx1, tm.ry1, bid, sX, sD, sY1, sTab, sRed,
                                        sKc, sGc);
      else
        fwd_body<R, MODE, OP, 2, TileG>(a, zblock, (int)blockIdx.z, tm, rhs, x0, y0, tm.rx1, tm.ry1, bid, sX, sD, sY1, sTab, sRed,
                                        sKc, sGc);
    }
  }
}


// ----------------------------------------------------------------------------
// launcher
// ----------------------------------------------------------------------------
static int choose_zblock(int nx, int ny, int nz, int nrhs) {
  long long tiles = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * nrhs;
  // aim for about 4 waves of 2 CTAs on 152 SMs, with at least 4 planes per CTA
  long long want = 152LL * 2 * 4;
  long long nzb = (want + tiles - 1) / tiles;
  int zb = (int)((nz + nzb - 1) / nzb);
  if (zb < 4) zb = 4;
  if (zb > 64) zb = 64;
  return zb;
}

// Grids of at least this many nodes split interior and PML tiles into two
// launches (each kernel then carries only its own path's registers); smaller
// grids, where launch latency dominates, use one launch choosing per tile.
constexpr long long kSplitNodes = 1LL << 20;

static int cdiv_i(int a, int b) { return a > 0 ? (a + b - 1) / b : 0; }

// Launch layout of a forward operator application: one rectangle launch over
// the whole grid, or (large grids, A/B) the PML-free rectangle of shell rows
// plus the PML frame around it.
struct FwdPlan {
  int zb = 4, nzb = 1;     // whole grid or PML-free rectangle
  int zbf = 4, nzbf = 1;   // PML frame
  bool split = false;
  int TXT = 1, TYT = 1;  // whole-grid tiling (16 x 16 for A/B, 32 x 8 for Q)
  int RW = 0, RH = 0;    // 32 x 8 tiling of the PML-free rectangle
  TileMap frame;         // frame tiling (count = frame tiles per z-block)
  long long blocks() const {
    return split ? (long long)RW * RH * nzb + (long long)frame.count * nzbf : (long long)TXT * TYT * nzb;
  }
};

static FwdPlan plan_layout(int nx, int ny, int nz, const int* plo, const int* phi, int op, int zb, int zbf) {
  FwdPlan p;
  p.zb = std::min(zb, nz);
  p.nzb = (nz + p.zb - 1) / p.zb;
  p.zbf = std::min(zbf > 0 ? zbf : zb, nz);
  p.nzbf = (nz + p.zbf - 1) / p.zbf;
  p.TXT = (nx + TX - 1) / TX;
  p.TYT = (ny + TY - 1) / TY;
  const int px0 = std::max(plo[0], 0), px1 = std::min(phi[0], nx - 1);
  const int py0 = std::max(plo[1], 0), py1 = std::min(phi[1], ny - 1);
  p.split = (op == OP_AB) && (long long)nx * ny * nz >= kSplitNodes && px1 >= px0 && py1 >= py0;
  if (!p.split) {
    if (op == OP_AB) {  // whole-grid launch of the A/B operators: 16 x 16 tiles
      p.TXT = (nx + TileG::TXS - 1) / TileG::TXS;
      p.TYT = (ny + TileG::TYS - 1) / TileG::TYS;
    }
    return p;
  }
  p.RW = cdiv_i(px1 - px0 + 1, TX);
  p.RH = cdiv_i(py1 - py0 + 1, TY);
  TileMap& f = p.frame;
  f.nx = nx;
  f.ny = ny;
  f.px0 = px0;
  f.px1 = px1;
  f.py0 = py0;
  f.py1 = py1;
  f.nwx = cdiv_i(nx, TileW::TXS);
  f.nw_lo = cdiv_i(py0, TileW::TYS);
  f.nw_hi = cdiv_i(ny - 1 - py1, TileW::TYS);
  f.nty = cdiv_i(py1 - py0 + 1, TileT::TYS);
  f.nt_lo = cdiv_i(px0, TileT::TXS);
  f.nt_hi = cdiv_i(nx - 1 - px1, TileT::TXS);
  f.count = f.nwx * (f.nw_lo + f.nw_hi) + f.nty * (f.nt_lo + f.nt_hi);
  return p;
}

template <class R>
static FwdPlan plan_fwd(const LevelView<R>& L, int nrhs, int op) {
  const int zb = L.zblock > 0 ? L.zblock : choose_zblock(L.nx, L.ny, L.nz, nrhs);
  return plan_layout(L.nx, L.ny, L.nz, L.plain_lo, L.plain_hi, op, zb, L.zblock_f);
}

template <class R, int MODE, int OP>
static void launch_fwd_t(const StencilCall<R>& c, cudaStream_t s) {
  const LevelView<R>& L = c.lv;
  const FwdPlan p = plan_fwd(L, c.nrhs, OP);
  const int nblk_total = (int)p.blocks();
  if (!p.split) {
    TileMap tm;
    tm.ntx = p.TXT;
    tm.rx1 = L.nx - 1;
    tm.ry1 = L.ny - 1;
    tm.nblk_total = nblk_total;
    dim3 grid(p.TXT * c.nrhs, p.TYT, p.nzb);
    count_launch();
    k_fwd<R, MODE, OP, (OP == OP_Q) ? 0 : 2><<<grid, dim3(TX, TY), 0, s>>>(c, p.zb, tm);
    return;
  }
  TileMap ti;
  ti.ox = p.frame.px0;
  ti.oy = p.frame.py0;
  ti.ntx = p.RW;
  ti.rx1 = p.frame.px1;
  ti.ry1 = p.frame.py1;
  ti.bid_offset = 0;
  ti.nblk_total = nblk_total;
  TileMap tp = p.frame;
  tp.bid_offset = p.RW * p.RH * p.nzb;
  tp.nblk_total = nblk_total;
  // the two launches are independent (disjoint outputs; a fused norm combines
  // through its arrival counter): with a side stream they run concurrently
  const bool fork = c.side && c.fork && c.join && tp.count > 0;
  cudaStream_t s2 = fork ? c.side : s;
  if (fork) {
    cudaEventRecord(c.fork, s);
    cudaStreamWaitEvent(s2, c.fork, 0);
  }
  count_launch();
  k_fwd<R, MODE, OP, 0><<<dim3(p.RW * c.nrhs, p.RH, p.nzb), dim3(TX, TY), 0, s>>>(c, p.zb, ti);
  if (tp.count > 0) {
    count_launch();
    k_fwd<R, MODE, OP, 1><<<dim3(tp.count * c.nrhs, 1, p.nzbf), dim3(TX, TY), 0, s2>>>(c, p.zbf, tp);
  }
  if (fork) {
    cudaEventRecord(c.join, s2);
    cudaStreamWaitEvent(s, c.join, 0);
  }
}

// Blocks per right-hand side of a forward stencil launch on this grid (the
// size of the per-block partial-sum array its reductions need).
long long gather_blocks_per_rhs(int nx, int ny, int nz, const int* plain_lo, const int* plain_hi, int nrhs,
                                int zblock, int zblock_f) {
  const int zb = zblock > 0 ? zblock : choose_zblock(nx, ny, nz, nrhs);
  const FwdPlan p = plan_layout(nx, ny, nz, plain_lo, plain_hi, OP_AB, zb, zblock_f);
  return p.blocks();
}

// Host replay of launch_fwd_t and k_fwd's block and thread decode (the plan,
// the frame tile decode, the thread-to-column map, the z-block of every CTA,
// the row form each tile takes and its block id for fused reductions).
// Violations counted: a written column outside the grid, a column outside the
// PML-free range on a row form that drops that axis's PML terms (form 0 both
// axes, form 1 y, form 3 x), a block id out of range or repeated.  counts
// (nx * ny * nz bytes, or null) receives how often each node of right-hand
// side 0 is written, saturating at 255.
long long replay_gather_layout(int nx, int ny, int nz, const int* plo, const int* phi, int op, int nrhs,
                               int zblock, int zblock_f, unsigned char* counts, long long* blocks) {
  const int zb = zblock > 0 ? zblock : choose_zblock(nx, ny, nz, nrhs);
  const FwdPlan p = plan_layout(nx, ny, nz, plo, phi, op, zb, zblock_f);
  const long long nblk = p.blocks();
  if (blocks) *blocks = nblk;
  std::vector<unsigned char> seen((size_t)nblk, 0);
  long long bad = 0;
  const bool ab = op == OP_AB;
  auto plain_x = [&](int x) { return x >= plo[0] && x <= phi[0]; };
  auto plain_y = [&](int y) { return y >= plo[1] && y <= phi[1]; };
  auto cta = [&](int TXS, int x0, int y0, int rx1, int ry1, int form, int zbk, int bz, long long bid) {
    if (bid < 0 || bid >= nblk || seen[(size_t)bid]++) ++bad;
    const int zb0 = bz * zbk, zb1 = std::min(zb0 + zbk, nz);
    for (int tid = 0; tid < NT; ++tid) {
      const int gx = x0 + tid % TXS, gy = y0 + tid / TXS;
      if (!(gx <= rx1 && gy <= ry1)) continue;  // inactive thread
      if (gx < 0 || gy < 0 || gx >= nx || gy >= ny) {
        ++bad;
        continue;
      }
      if (ab && ((form == 0 && !(plain_x(gx) && plain_y(gy))) || (form == 1 && !plain_y(gy)) ||
                 (form == 3 && !plain_x(gx))))
        ++bad;
      if (counts)
        for (int z = zb0; z < zb1; ++z) {
          unsigned char& c = counts[((size_t)z * ny + gy) * nx + gx];
          if (c < 255) ++c;
        }
    }
  };
  if (!p.split) {
    const int TXS = ab ? TileG::TXS : TileSq::TXS, TYS = ab ? TileG::TYS : TileSq::TYS;
    for (int bz = 0; bz < p.nzb; ++bz)
      for (int by = 0; by < p.TYT; ++by)
        for (int bx = 0; bx < p.TXT * nrhs; ++bx) {
          if (bx % nrhs) continue;  // right-hand side 0
          const int t = bx / nrhs, x0 = t * TXS, y0 = by * TYS;
          const bool plain = x0 >= plo[0] && x0 + TXS - 1 <= phi[0] && y0 >= plo[1] && y0 + TYS - 1 <= phi[1];
          cta(TXS, x0, y0, nx - 1, ny - 1, (!ab || plain) ? 0 : 2, p.zb, bz, t + (long long)p.TXT * (by + p.TYT * bz));
        }
  } else {
    const int px0 = p.frame.px0, py0 = p.frame.py0;
    for (int bz = 0; bz < p.nzb; ++bz)
      for (int by = 0; by < p.RH; ++by)
        for (int bx = 0; bx < p.RW * nrhs; ++bx) {
          if (bx % nrhs) continue;
          const int t = bx / nrhs;
          cta(TileSq::TXS, px0 + t * TileSq::TXS, py0 + by * TileSq::TYS, p.frame.px1, p.frame.py1, 0, p.zb, bz,
              t + (long long)p.RW * (by + p.RH * bz));
        }
    const long long off = (long long)p.RW * p.RH * p.nzb;
    for (int bz = 0; bz < p.nzbf; ++bz)
      for (int bx = 0; bx < p.frame.count * nrhs; ++bx) {
        if (bx % nrhs) continue;
        const int t = bx / nrhs;
        const FrameTile f = decode_frame(p.frame, t);
        const long long bid = off + t + (long long)p.frame.count * bz;
        if (f.wide) {
          const bool xplain = f.x0 >= plo[0] && f.x0 + TileW::TXS - 1 <= phi[0];
          cta(TileW::TXS, f.x0, f.y0, f.rx1, f.ry1, xplain ? 3 : 2, p.zbf, bz, bid);
        } else {
          cta(TileT::TXS, f.x0, f.y0, f.rx1, f.ry1, 1, p.zbf, bz, bid);
        }
      }
  }
  for (unsigned char v : seen)
    if (v != 1) ++bad;
  return bad;
}

template <class R>
void launch_fwd_gather(const StencilCall<R>& c, int mode, int op, cudaStream_t s) {
  if (op == OP_Q) {
    launch_fwd_t<R, M_APPLY, OP_Q>(c, s);
    return;
  }
  switch (mode) {
    case M_APPLY: launch_fwd_t<R, M_APPLY, OP_AB>(c, s); break;
    case M_RESID: launch_fwd_t<R, M_RESID, OP_AB>(c, s); break;
    case M_J2: launch_fwd_t<R, M_J2, OP_AB>(c, s); break;
    case M_JSWEEP: launch_fwd_t<R, M_JSWEEP, OP_AB>(c, s); break;
  }
}

template void launch_fwd_gather<float>(const StencilCall<float>&, int, int, cudaStream_t);
template void launch_fwd_gather<double>(const StencilCall<double>&, int, int, cudaStream_t);


// ----------------------------------------------------------------------------
// The bottom solve C_4h (Sec. 3.2) as one persistent cooperative kernel
// ----------------------------------------------------------------------------
// The s-step CA-GMRES of the 4h level is a chain of short, latency-bound
// steps on an L2-resident grid: p_{k+1} = B J(p_k) for k < s (a two-sweep
// Jacobi map and a B apply per step), the Gram matrix of p_0 .. p_s with the
// normal-equation solve, and e = sum_k y_k J(p_k).  As separate launches each
// step pays a launch and a ramp; here every block of one cooperative launch
// (all blocks resident) takes work items of each sweep in turn and waits at a
// grid barrier between dependent steps.  The sweeps run the same tile bodies
// as the separate launches (the 16 x 16 whole-grid tiles of small grids).
//
// Grid barrier: arrival counter bar[0] (never reset inside a launch) and
// released generation bar[1], both zeroed before the launch; the last block
// to arrive at barrier g releases generation g + 1.  Every wait is bounded:
// after b.spins polls (about a second by default) the block records the
// failure in *err and goes on (its results are then wrong, the host reports
// HZ_ETIMEOUT, and no wait can hang the device).  b.extra > 0 (a test of that
// path) makes the barrier expect arrivals that never come.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned& gen, int* err, unsigned spins, unsigned extra) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    const unsigned target = (gen + 1) * (gridDim.x + extra);
    if (atomicAdd(bar, 1u) + 1u == target) {
      atomicExch(bar + 1, gen + 1);
    } else {
      unsigned it = 0;
      while (*reinterpret_cast<volatile unsigned*>(bar + 1) < gen + 1) {
        if (++it > spins) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  ++gen;
  __syncthreads();
}

// one sweep of the 4h operator over all work items (tile, z-block, right-hand side)
template <class R, int MODE>
__device__ __forceinline__ void bottom_sweep(const StencilCall<R>& c, const BottomArgs<R>& b, cx<R>* sX, cx<R>* sD,
                                             cx<R>* sY1, const R* sTab, double* sRed, R (*sKc)[NT],
                                             cx<R> (*sGc)[NT]) {
  const LevelView<R>& L = c.lv;
  TileMap tm;
  tm.rx1 = L.nx - 1;
  tm.ry1 = L.ny - 1;
  const int items = b.ntx * b.nty * b.nzb * c.nrhs;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int rhs = it % c.nrhs, t = it / c.nrhs;
    const int tx = t % b.ntx, r = t / b.ntx, ty = r % b.nty, bz = r / b.nty;
    const int x0 = tx * TileG::TXS, y0 = ty * TileG::TYS;
    const bool plain = (x0 >= L.plain_lo[0]) && (x0 + TileG::TXS - 1 <= L.plain_hi[0]) && (y0 >= L.plain_lo[1]) &&
                       (y0 + TileG::TYS - 1 <= L.plain_hi[1]);
    if (plain)
      fwd_body<R, MODE, OP_AB, 0, TileG>(c, b.zblock, bz, tm, rhs, x0, y0, tm.rx1, tm.ry1, 0u, sX, sD, sY1, sTab,
                                         sRed, sKc, sGc);
    else
      fwd_body<R, MODE, OP_AB, 2, TileG>(c, b.zblock, bz, tm, rhs, x0, y0, tm.rx1, tm.ry1, 0u, sX, sD, sY1, sTab,
                                         sRed, sKc, sGc);
    __syncthreads();  // the next item refills the plane ring
  }
}

template <class R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) k_bottom4h(BottomArgs<R> b) {
  constexpr int KN = kBottomSteps + 1, NV = KN * (KN + 1);  // Gram entries a <= b, re and im
  constexpr int PL = TileSq::PLN;
  __shared__ __align__(16) cx<R> sX[NSTAGE * PL];
  __shared__ __align__(16) cx<R> sD[NSTAGE * PL];
  __shared__ cx<R> sY1[PL];
  __shared__ __align__(16) R sTab[kMaxSeg * kNumFn * 4];
  __shared__ R sKc[NSTAGE][NT];
  __shared__ cx<R> sGc[1][NT];
  __shared__ double sRed[32];
  __shared__ double sG[NT / 32][NV];
  __shared__ double sres[NV];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < b.c.tab.nseg * kNumFn * 4; i += NT) sTab[i] = b.c.tab.coef[i];
  __syncthreads();
  unsigned gen = 0;
  const int nrhs = b.c.nrhs;
  const long long N = b.c.lv.N;
  // basis: p_{k+1} = B J(p_k)
  for (int k = 0; k < kBottomSteps; ++k) {
    StencilCall<R> cj = b.c;
    cj.x = b.P + k * b.vs;
    cj.y = b.Zc + k * b.vs;
    cj.base = nullptr;
    bottom_sweep<R, M_J2>(cj, b, sX, sD, sY1, sTab, sRed, sKc, sGc);
    grid_barrier(b.bar, gen, b.err, b.spins, b.extra);
    StencilCall<R> ca = b.c;
    ca.x = b.Zc + k * b.vs;
    ca.y = b.P + (k + 1) * b.vs;
    bottom_sweep<R, M_APPLY>(ca, b, sX, sD, sY1, sTab, sRed, sKc, sGc);
    grid_barrier(b.bar, gen, b.err, b.spins, b.extra);
  }
  // Gram entries <p_a, p_b> (a <= b) per right-hand side: per-block partial sums
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    R acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0;
    const cx<R>* Pr = b.P + (long long)rhs * N;
    for (long long i = blockIdx.x * (long long)NT + tid; i < N; i += (long long)gridDim.x * NT) {
      cx<R> p[KN];
#pragma unroll
      for (int a = 0; a < KN; ++a) p[a] = Pr[a * b.vs + i];
      int q = 0;
#pragma unroll
      for (int a = 0; a < KN; ++a)
#pragma unroll
        for (int c2 = a; c2 < KN; ++c2) {
          const cx<R> t = cjmul(p[a], p[c2]);
          acc[2 * q] += t.x;
          acc[2 * q + 1] += t.y;
          ++q;
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double x = warp_sum((double)acc[v]);
      if (lane == 0) sG[w][v] = x;
    }
    __syncthreads();
    if (tid < NV) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < NT / 32; ++k) t += sG[k][tid];
      b.partial[((size_t)blockIdx.x * nrhs + rhs) * NV + tid] = t;
    }
    __syncthreads();
  }
  grid_barrier(b.bar, gen, b.err, b.spins, b.extra);
  // one block per right-hand side: sum the partials in block order, solve for y
  for (int rhs = blockIdx.x; rhs < nrhs; rhs += gridDim.x) {
    if (tid < NV) {
      double t = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) t += __ldcg(b.partial + ((size_t)k * nrhs + rhs) * NV + tid);
      sres[tid] = t;
    }
    __syncthreads();
    if (tid == 0) gram_lsq_solve<KN>(sres, b.y + (size_t)rhs * b.ld * 2);
    __syncthreads();
  }
  grid_barrier(b.bar, gen, b.err, b.spins, b.extra);
  // e = sum_k y_k J(p_k)
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    cx<R> yk[kBottomSteps];
#pragma unroll
    for (int k = 0; k < kBottomSteps; ++k) {
      const double* yr = b.y + (size_t)rhs * b.ld * 2;
      yk[k] = mkc<R>((R)__ldcg(yr + 2 * k), (R)__ldcg(yr + 2 * k + 1));
    }
    for (long long i = blockIdx.x * (long long)NT + tid; i < N; i += (long long)gridDim.x * NT) {
      cx<R> acc = mkc<R>(0, 0);
#pragma unroll
      for (int k = 0; k < kBottomSteps; ++k) acc += yk[k] * b.Zc[k * b.vs + (long long)rhs * N + i];
      b.e[(long long)rhs * N + i] = acc;
    }
  }
}

__global__ void k_coop_probe(int* p) {
  if (p && blockIdx.x == 0 && threadIdx.x == 0) *p = 1;
}

// per-device caches of the probes below (every thread that races on a first
// probe stores the same answer)
constexpr int kProbeDevices = 64;

// Cooperative launches captured into a CUDA graph (the preconditioner is
// replayed as one graph): probed once per process and device on a trivial kernel.
bool coop_capture_supported() {
  static int cache[kProbeDevices];  // 0 unknown, 1 yes, 2 no
  int dev = 0, coop = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kProbeDevices) return false;
  if (cache[dev]) return cache[dev] == 1;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  bool ok = coop != 0;
  if (ok) {
    cudaStream_t s = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ex = nullptr;
      int* nullp = nullptr;
      void* args[] = {&nullp};
      ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bool launched = cudaLaunchCooperativeKernel((void*)k_coop_probe, dim3(1), dim3(32), args, 0, s) ==
                              cudaSuccess;
        const bool ended = cudaStreamEndCapture(s, &g) == cudaSuccess;
        ok = launched && ended && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
      }
      if (ex) cudaGraphExecDestroy(ex);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(s);
    }
    cudaGetLastError();  // clear any error of a refused capture
  }
  cache[dev] = ok ? 1 : 2;
  return ok;
}

// Blocks of one cooperative launch of k_bottom4h<R> that fit on the device at once.
template <class R>
int bottom_max_blocks() {
  static int cache[kProbeDevices];  // 0 unknown, else blocks + 1
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kProbeDevices) return 0;
  if (!cache[dev]) {
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bottom4h<R>, NT, 0);
    cache[dev] = per * nsm + 1;
  }
  return cache[dev] - 1;
}

template <class R>
size_t bottom_partial_doubles(int nrhs) {
  return (size_t)bottom_max_blocks<R>() * nrhs * (kBottomSteps + 1) * (kBottomSteps + 2);
}

template <class R>
bool launch_bottom4h(BottomArgs<R> b, cudaStream_t s) {
  const int maxb = bottom_max_blocks<R>();
  if (maxb < 1) return false;
  const LevelView<R>& L = b.c.lv;
  b.ntx = (L.nx + TileG::TXS - 1) / TileG::TXS;
  b.nty = (L.ny + TileG::TYS - 1) / TileG::TYS;
  // z-blocks: about one work item per resident block, at most 64 planes each
  const int tiles = b.ntx * b.nty * b.c.nrhs;
  const int want = std::max(1, maxb / std::max(1, tiles));
  b.zblock = std::min(64, std::max(2, (L.nz + want - 1) / want));
  b.nzb = (L.nz + b.zblock - 1) / b.zblock;
  const int grid = std::min(maxb, tiles * b.nzb);
  if (cudaMemsetAsync(b.bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return false;
  void* args[] = {&b};
  count_launch();
  return cudaLaunchCooperativeKernel((void*)k_bottom4h<R>, dim3(grid), dim3(TX, TY), args, 0, s) == cudaSuccess;
}

template bool launch_bottom4h<float>(BottomArgs<float>, cudaStream_t);
template bool launch_bottom4h<double>(BottomArgs<double>, cudaStream_t);
template size_t bottom_partial_doubles<float>(int);
template size_t bottom_partial_doubles<double>(int);

}  // namespace gather
}  // namespace hz
