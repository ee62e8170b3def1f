// Launch layout and launchers of the forward stencil (hz_fwd.cuh).
#pragma once

#include <algorithm>

#include "hz_fwd.cuh"

namespace hz {

// tile set of a grid (hz_fwd.cuh)
inline int tile_set(int nx, int ny, int nz) {
  const long long n = (long long)nx * ny * nz;
  return n < kFusedNodes ? 2 : (n < kCoarseNodes ? 1 : 0);
}
inline int rect_w(int ss) { return ss ? Shapes<1>::Rect::TWN : Shapes<0>::Rect::TWN; }
inline int rect_h(int ss) { return ss ? Shapes<1>::Rect::TYT : Shapes<0>::Rect::TYT; }

// Planes per block when neither the caller nor the tuner chose: about four
// waves of two blocks on 152 SMs, at least kMinZblock planes.
inline int choose_zblock(int nx, int ny, int nz, int nrhs) {
  const int ss = tile_set(nx, ny, nz);
  const long long tiles =
      (long long)((nx + rect_w(ss) - 1) / rect_w(ss)) * ((ny + rect_h(ss) - 1) / rect_h(ss)) * nrhs;
  const long long want = 152LL * 2 * 4;
  const long long nzb = (want + tiles - 1) / tiles;
  int zb = (int)((nz + nzb - 1) / nzb);
  zb = std::max(zb, 4);
  zb = std::min(zb, kMaxZb);
  return zb;
}

inline int cdiv_i(int a, int b) { return a > 0 ? (a + b - 1) / b : 0; }

// An A/B application with a PML-free core runs as two launches, the
// PML-free rectangle (shell rows) and the PML frame around it, each carrying
// only its own row forms (and run side by side on two streams); Q_h, and
// grids whose PML leaves no core, use one launch choosing the form per tile.
struct FwdPlan {
  int ss = 0;             // tile set
  int zb = 4, nzb = 1;    // whole grid or rectangle
  int zbf = 4, nzbf = 1;  // frame
  bool split = false;
  bool fused = false;     // split tiles in one launch (tile set 2; one z-block)
  int GW = 1, GH = 1;     // whole-grid tiles
  int RW = 0, RH = 0;     // tiles of the PML-free rectangle
  TileMap frame;          // frame tiling (count = frame tiles per z-block)
  long long blocks() const {
    if (fused) return ((long long)RW * RH + frame.count) * nzb;
    return split ? (long long)RW * RH * nzb + (long long)frame.count * nzbf : (long long)GW * GH * nzb;
  }
};

// nzr: rows of a z-window (0: all nz); the tile set stays that of the whole grid
inline FwdPlan plan_layout(int nx, int ny, int nz, const int* plo, const int* phi, bool ab, int zb, int zbf,
                           int nzr = 0) {
  FwdPlan p;
  const int nzw = nzr > 0 ? nzr : nz;
  p.zb = std::min(std::min(zb, kMaxZb), nzw);
  p.nzb = (nzw + p.zb - 1) / p.zb;
  p.zbf = std::min(std::min(zbf > 0 ? zbf : zb, kMaxZb), nzw);
  p.nzbf = (nzw + p.zbf - 1) / p.zbf;
  p.ss = tile_set(nx, ny, nz);
  TileMap& f = p.frame;
  f.rw = rect_w(p.ss);
  f.rh = rect_h(p.ss);
  f.ww = p.ss == 2 ? Shapes<2>::Wide::TWN : (p.ss ? Shapes<1>::Wide::TWN : Shapes<0>::Wide::TWN);
  f.wh = p.ss == 2 ? Shapes<2>::Wide::TYT : (p.ss ? Shapes<1>::Wide::TYT : Shapes<0>::Wide::TYT);
  f.tw = p.ss == 2 ? Shapes<2>::Tall::TWN : Shapes<0>::Tall::TWN;
  f.th = p.ss == 2 ? Shapes<2>::Tall::TYT : Shapes<0>::Tall::TYT;
  p.GW = cdiv_i(nx, f.rw);
  p.GH = cdiv_i(ny, f.rh);
  const int px0 = std::max(plo[0], 0), px1 = std::min(phi[0], nx - 1);
  const int py0 = std::max(plo[1], 0), py1 = std::min(phi[1], ny - 1);
  p.split = ab && px1 >= px0 && py1 >= py0;
  if (!p.split) return p;
  p.RW = cdiv_i(px1 - px0 + 1, f.rw);
  p.RH = cdiv_i(py1 - py0 + 1, f.rh);
  f.nx = nx;
  f.ny = ny;
  f.px0 = px0;
  f.px1 = px1;
  f.py0 = py0;
  f.py1 = py1;
  f.nwx = cdiv_i(px1 - px0 + 1, f.ww);
  f.nw_lo = cdiv_i(py0, f.wh);
  f.nw_hi = cdiv_i(ny - 1 - py1, f.wh);
  f.nty = cdiv_i(ny, f.th);
  f.nt_lo = cdiv_i(px0, f.tw);
  f.nt_hi = cdiv_i(nx - 1 - px1, f.tw);
  f.count = f.nwx * (f.nw_lo + f.nw_hi) + f.nty * (f.nt_lo + f.nt_hi);
  f.ntx = p.RW;
  f.nrow = p.RH;
  if (p.ss == 2) {  // one launch, one z-block for every tile
    p.fused = true;
    p.zbf = p.zb;
    p.nzbf = p.nzb;
  }
  return p;
}

template <class R>
inline FwdPlan plan_fwd(const StencilCall<R>& c, bool ab) {
  const LevelView<R>& L = c.lv;
  const int zb = L.zblock > 0 ? L.zblock : choose_zblock(L.nx, L.ny, L.nz, c.nrhs);
  return plan_layout(L.nx, L.ny, L.nz, L.plain_lo, L.plain_hi, ab, zb, L.zblock_f,
                     c.zr1 > 0 ? c.zr1 - c.zr0 : 0);
}
// (the row window applies to M_AWIN launches only: other modes plan all rows)
template <class R, int MODE>
inline FwdPlan plan_fwd_mode(StencilCall<R> c, bool ab) {
  if (MODE != M_AWIN) c.zr0 = c.zr1 = 0;
  return plan_fwd(c, ab);
}

template <class R, int MODE, int OPK, int RB, int SS>
void launch_fwd_split(const StencilCall<R>& c, const FwdPlan& p, int ng, int nblk_total, cudaStream_t s);

template <class R, int MODE, int OPK, int RB, int SS>
void launch_fwd_ss(const StencilCall<R>& c, const FwdPlan& p, cudaStream_t s) {
  const int ng = c.nrhs / RB;
  const int nblk_total = (int)p.blocks();
  if (OPK == OPK_Q || !p.split) {
    TileMap tm = p.frame;
    tm.ntx = p.GW;
    tm.nblk_total = nblk_total;
    count_launch();
    k_fwd_grid<R, MODE, OPK, RB, SS><<<dim3(p.GW * ng, p.GH, p.nzb), Shapes<SS>::Rect::NT,
                                       fwd_smem_rect<R, MODE, OPK, RB, SS>(), s>>>(c, p.zb, tm);
    return;
  }
  if constexpr (OPK != OPK_Q) launch_fwd_split<R, MODE, OPK, RB, SS>(c, p, ng, nblk_total, s);
}

template <class R, int MODE, int OPK, int RB>
void launch_fwd_rb(const StencilCall<R>& c, cudaStream_t s) {
  const FwdPlan p = plan_fwd_mode<R, MODE>(c, OPK != OPK_Q);
  if constexpr (OPK != OPK_Q) {
    if (p.fused) {
      TileMap tm = p.frame;
      tm.nblk_total = (int)p.blocks();
      const int ng = c.nrhs / RB;
      count_launch();
      k_fwd_fused<R, MODE, OPK, RB><<<dim3((p.RW * p.RH + tm.count) * ng, 1, p.nzb), 256,
                                      fwd_smem_fused<R, MODE, OPK, RB>(), s>>>(c, p.zb, tm);
      return;
    }
  }
  if (p.ss == 0) launch_fwd_ss<R, MODE, OPK, RB, 0>(c, p, s);
  else launch_fwd_ss<R, MODE, OPK, RB, 1>(c, p, s);
}

// the rectangle and frame launches of a split application
template <class R, int MODE, int OPK, int RB, int SS>
void launch_fwd_split(const StencilCall<R>& c, const FwdPlan& p, int ng, int nblk_total, cudaStream_t s) {
  TileMap ti = p.frame;
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
  k_fwd_rect<R, MODE, OPK, RB, SS><<<dim3(p.RW * ng, p.RH, p.nzb), Shapes<SS>::Rect::NT,
                                     fwd_smem_rect<R, MODE, OPK, RB, SS>(), s>>>(c, p.zb, ti);
  if (tp.count > 0) {
    count_launch();
    k_fwd_frame<R, MODE, OPK, RB, SS><<<dim3(tp.count * ng, 1, p.nzbf), Shapes<SS>::Wide::NT,
                                        fwd_smem_frame<R, MODE, OPK, RB, SS>(), s2>>>(c, p.zbf, tp);
  }
  if (fork) {
    cudaEventRecord(c.join, s2);
    cudaStreamWaitEvent(s, c.join, 0);
  }
}

// right-hand sides per block: two for complex64 (the coefficients of three
// rows and two accumulators per right-hand side stay in registers), one for
// complex128 (its kernels are bound by the FP64 rate)
template <class R, int MODE>
constexpr int fwd_rb_max() {
  return sizeof(R) == 8 ? 1 : 2;
}
inline int fwd_pick_rb(int nrhs, int rbmax) { return (rbmax >= 2 && nrhs % 2 == 0) ? 2 : 1; }

template <class R, int MODE, int OPK>
void launch_fwd_opk(const StencilCall<R>& c, cudaStream_t s) {
  constexpr int RBM = fwd_rb_max<R, MODE>();
  if constexpr (RBM >= 2) {
    if (fwd_pick_rb(c.nrhs, RBM) == 2) {
      launch_fwd_rb<R, MODE, OPK, 2>(c, s);
      return;
    }
  }
  launch_fwd_rb<R, MODE, OPK, 1>(c, s);
}

template <class R, int MODE, int OPK, int RB, int SS>
void fwd_attrs_ss() {
  cudaFuncSetAttribute(k_fwd_grid<R, MODE, OPK, RB, SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fwd_smem_rect<R, MODE, OPK, RB, SS>());
  if constexpr (OPK != OPK_Q) {
    cudaFuncSetAttribute(k_fwd_rect<R, MODE, OPK, RB, SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fwd_smem_rect<R, MODE, OPK, RB, SS>());
    cudaFuncSetAttribute(k_fwd_frame<R, MODE, OPK, RB, SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fwd_smem_frame<R, MODE, OPK, RB, SS>());
  }
}
template <class R, int MODE, int OPK, int RB>
void fwd_attrs_rb() {
  fwd_attrs_ss<R, MODE, OPK, RB, 0>();
  fwd_attrs_ss<R, MODE, OPK, RB, 1>();
  if constexpr (OPK != OPK_Q)
    cudaFuncSetAttribute(k_fwd_fused<R, MODE, OPK, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fwd_smem_fused<R, MODE, OPK, RB>());
}
template <class R, int MODE, int OPK>
void fwd_attrs_opk() {
  fwd_attrs_rb<R, MODE, OPK, 1>();
  if constexpr (fwd_rb_max<R, MODE>() >= 2) fwd_attrs_rb<R, MODE, OPK, 2>();
}

// Entry points of one (precision, mode): instantiated in hz_fwd.cu, one
// translation unit per pair.
template <class R, int MODE>
void launch_fwd(const StencilCall<R>& c, int opk, cudaStream_t s) {
  if constexpr (MODE == M_APPLY) {
    if (opk == OPK_Q) {
      launch_fwd_opk<R, MODE, OPK_Q>(c, s);
      return;
    }
  }
  if (opk == OPK_B) launch_fwd_opk<R, MODE, OPK_B>(c, s);
  else launch_fwd_opk<R, MODE, OPK_A>(c, s);
}

template <class R, int MODE>
void fwd_init_attrs() {
  fwd_attrs_opk<R, MODE, OPK_A>();
  fwd_attrs_opk<R, MODE, OPK_B>();
  if constexpr (MODE == M_APPLY) fwd_attrs_opk<R, MODE, OPK_Q>();
}

}  // namespace hz
