// Adjoint 27-point IOFD stencil, the one-sweep Jacobi map, and the dispatch
// of every stencil application (the forward kernels live in hz_fwd.cuh).
//
// Operator (paper Sec. 2.2, Eq. iofd-shell-form / Eq. pml-second-difference):
//   (H x)_i = -ell^-2 sum_j [ abar_j S_j + achk_j D_j ] - s kappa_i^2 ell^-2 (M x)_i
// where, with the transverse weights a4, a5/4, (1-a4-a5)/4 of the row i,
//   T_j(s)  = transverse-weighted sum of x over the plane at offset s along j,
//   S_j     = T_j(+1) + T_j(-1) - 2 T_j(0),   D_j = T_j(+1) - T_j(-1),
//   M x     = a1 N0 + a2/6 N1 + a3/12 N2 + (1-a1-a2-a3)/8 N3 (shell sums N_m),
//   abar_j, achk_j = half sum / half difference of the two PML second-
//   difference weights of row i along j (1 and 0 outside the PML),
//   s = 1 (A_ell) or 1 + i sigma (B_ell, Eq. shifted-iofd-levels).
// Coefficients are evaluated per row from kappa = k ell through the cubic
// Hermite tables at eta* = min(kappa / 2 pi, 0.4) (Eq. iofd-clamped-coordinate).
//
// The adjoint kernel applies (H^H x)_i = sum_delta conj(H_{i+delta}(-delta)) x_{i+delta};
// it needs the neighbours' own coefficients, which it evaluates once per
// loaded node into shared memory.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "hz_fwd_launch.cuh"

namespace hz {

// the forward kernels are instantiated in hz_fwd.cu
extern template void launch_fwd<float, M_APPLY>(const StencilCall<float>&, int, cudaStream_t);
extern template void launch_fwd<float, M_RESID>(const StencilCall<float>&, int, cudaStream_t);
extern template void launch_fwd<float, M_J2>(const StencilCall<float>&, int, cudaStream_t);
extern template void launch_fwd<float, M_JSWEEP>(const StencilCall<float>&, int, cudaStream_t);
extern template void launch_fwd<double, M_APPLY>(const StencilCall<double>&, int, cudaStream_t);
extern template void launch_fwd<double, M_RESID>(const StencilCall<double>&, int, cudaStream_t);
extern template void launch_fwd<double, M_J2>(const StencilCall<double>&, int, cudaStream_t);
extern template void launch_fwd<double, M_JSWEEP>(const StencilCall<double>&, int, cudaStream_t);
extern template void launch_fwd<float, M_AWIN>(const StencilCall<float>&, int, cudaStream_t);
extern template void launch_fwd<double, M_AWIN>(const StencilCall<double>&, int, cudaStream_t);
extern template void fwd_init_attrs<float, M_APPLY>();
extern template void fwd_init_attrs<float, M_RESID>();
extern template void fwd_init_attrs<float, M_J2>();
extern template void fwd_init_attrs<float, M_JSWEEP>();
extern template void fwd_init_attrs<double, M_APPLY>();
extern template void fwd_init_attrs<double, M_RESID>();
extern template void fwd_init_attrs<double, M_J2>();
extern template void fwd_init_attrs<double, M_JSWEEP>();
extern template void fwd_init_attrs<float, M_AWIN>();
extern template void fwd_init_attrs<double, M_AWIN>();

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int PW = TX + 2, PH = TY + 2, PLANE = PW * PH;

// ----------------------------------------------------------------------------
// adjoint kernel: generic 27-neighbour gather with neighbour coefficients
// ----------------------------------------------------------------------------
template <int OP> struct AdjNP { static constexpr int v = 8; };
template <> struct AdjNP<OP_Q> { static constexpr int v = 4; };

template <class R, int MODE, int OP>
__global__ void __launch_bounds__(NT) k_adj(StencilCall<R> a, int zblock, int tiles_x) {
  constexpr int NP = AdjNP<OP>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* sV = reinterpret_cast<cx<R>*>(smem_raw);            // [3][PLANE]
  R* sP = reinterpret_cast<R*>(sV + 3 * PLANE);                // [3][PLANE][NP]
  R* sTab = sP + 3 * PLANE * NP;                               // table
  __shared__ double sRed[32];
  const LevelView<R>& L = a.lv;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  for (int i = tid; i < a.tab.nseg * kNumFn * 4; i += NT) sTab[i] = a.tab.coef[i];
  __syncthreads();
  const int rhs = blockIdx.x % a.nrhs, tile_x = blockIdx.x / a.nrhs;
  const int x0 = tile_x * TX, y0 = blockIdx.y * TY;
  const int zb0 = blockIdx.z * zblock;
  const int zb1 = min(zb0 + zblock, L.nz);
  const long long N = L.N;
  const long long plane_sz = (long long)L.nx * L.ny;
  const cx<R>* X = a.x + rhs * N;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = (gx < L.nx) && (gy < L.ny);
  const R inv_ell2 = L.inv_ell2;
  const cx<R> shift = a.mass_shift;
  const cx<R> cshift = conjc(shift);
  const int nseg = a.tab.nseg;
  const R ds = a.tab.ds, inv_ds = a.tab.inv_ds;

  cx<R> abx[3], acx[3], aby[3], acy[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int ix = min(max(gx + d - 1, 0), L.nx - 1), iy = min(max(gy + d - 1, 0), L.ny - 1);
    abx[d] = L.abar[0][ix];
    acx[d] = L.achk[0][ix];
    aby[d] = L.abar[1][iy];
    acy[d] = L.achk[1][iy];
  }

  auto load = [&](int z, int slot) {
    cx<R> abz = (z >= 0 && z < L.nz) ? L.abar[2][z] : mkc<R>(1, 0);
    for (int i = tid; i < PLANE; i += NT) {
      int ly = i / PW, lx = i - ly * PW;
      int qx = x0 - 1 + lx, qy = y0 - 1 + ly;
      bool in = (z >= 0) && (z < L.nz) && (qx >= 0) && (qx < L.nx) && (qy >= 0) && (qy < L.ny);
      cx<R> v = mkc<R>(0, 0);
      R prm[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) prm[j] = 0;
      if (in) {
        long long off = (long long)z * plane_sz + (long long)qy * L.nx + qx;
        v = X[off];
        R kap = L.kappa[off];
        if (OP == OP_Q) {
          R b[3];
          table_eval<R, 5, 3>(sTab, nseg, ds, inv_ds, eta_star(kap), b);
          prm[0] = b[0];
          prm[1] = b[1] * (R)(1.0 / 6.0);
          prm[2] = b[2] * (R)(1.0 / 12.0);
          prm[3] = ((R)1 - b[0] - b[1] - b[2]) * (R)0.125;
        } else {
          R av[5];
          table_eval<R, 0, 5>(sTab, nseg, ds, inv_ds, eta_star(kap), av);
          prm[0] = av[3];
          prm[1] = av[4] * (R)0.25;
          prm[2] = ((R)1 - av[3] - av[4]) * (R)0.25;
          prm[3] = av[0];
          prm[4] = av[1] * (R)(1.0 / 6.0);
          prm[5] = av[2] * (R)(1.0 / 12.0);
          prm[6] = ((R)1 - av[0] - av[1] - av[2]) * (R)0.125;
          prm[7] = inv_ell2 * kap * kap;
          if (MODE == M_J2) {
            cx<R> sab = L.abar[0][qx] + L.abar[1][qy] + abz;
            cx<R> D = inv_ell2 * ((R)2 * prm[0] * sab) - (prm[7] * prm[3]) * shift;
            v = a.omega_j * cdiv(v, conjc(D));   // y1 = omega D^-H g
          }
        }
      }
      sV[slot * PLANE + i] = v;
#pragma unroll
      for (int j = 0; j < NP; ++j) sP[(slot * PLANE + i) * NP + j] = prm[j];
    }
  };

  R nrm2 = 0;
  const bool want_norm = MODE == M_RESID && a.red.out != nullptr;
  load(zb0 - 1, (zb0 + 2) % 3);
  load(zb0, zb0 % 3);
  for (int z = zb0; z < zb1; ++z) {
    load(z + 1, (z + 1) % 3);
    __syncthreads();
    if (active) {
      cx<R> abz[3], acz[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int iz = min(max(z + d - 1, 0), L.nz - 1);
        abz[d] = L.abar[2][iz];
        acz[d] = L.achk[2][iz];
      }
      cx<R> acc = mkc<R>(0, 0);
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        const int slot = (z + dz + 3) % 3;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int li = slot * PLANE + (ty + 1 + dy) * PW + (tx + 1 + dx);
            const cx<R> v = sV[li];
            const R* p = sP + li * NP;
            const int sh = (dx != 0) + (dy != 0) + (dz != 0);
            if (OP == OP_Q) {
              acc += p[sh] * v;
            } else {
              // row j = i + delta reaches i at offset -delta
              auto dval = [&](cx<R> ab, cx<R> ac, int off) -> cx<R> {
                return off == 0 ? (R)(-2) * ab : (off > 0 ? ab + ac : ab - ac);
              };
              cx<R> st = p[(dy != 0) + (dz != 0)] * dval(abx[dx + 1], acx[dx + 1], -dx) +
                         p[(dx != 0) + (dz != 0)] * dval(aby[dy + 1], acy[dy + 1], -dy) +
                         p[(dx != 0) + (dy != 0)] * dval(abz[dz + 1], acz[dz + 1], -dz);
              cx<R> coef = (-inv_ell2) * conjc(st) - (p[7] * p[3 + sh]) * cshift;
              acc += coef * v;
            }
          }
        }
      }
      const long long idx = (long long)z * plane_sz + (long long)gy * L.nx + gx;
      cx<R> out;
      if (MODE == M_APPLY) {
        out = acc;
      } else if (MODE == M_RESID) {
        out = a.g[rhs * N + idx] - acc;
        if (want_norm) nrm2 += abs2(out);
      } else {
        const int li = (z % 3) * PLANE + (ty + 1) * PW + (tx + 1);
        const R* p = sP + li * NP;
        cx<R> sab = abx[1] + aby[1] + abz[1];
        cx<R> Dh = conjc(inv_ell2 * ((R)2 * p[0] * sab) - (p[7] * p[3]) * shift);
        if (MODE == M_J2) {
          cx<R> g = X[idx];
          out = sV[li] + a.omega_j * cdiv(g - acc, Dh);
          if (a.base) out += a.base[rhs * N + idx];
        } else {  // JSWEEP
          out = sV[li] + a.omega_j * cdiv(a.g[rhs * N + idx] - acc, Dh);
        }
      }
      a.y[rhs * N + idx] = out;
    }
    __syncthreads();
  }
  if (MODE == M_RESID && a.red.out) {
    double s = block_sum((double)nrm2, sRed, tid, NT);
    const unsigned nblk = (unsigned)(tiles_x * gridDim.y * gridDim.z);
    const unsigned bid = (unsigned)(tile_x + tiles_x * (blockIdx.y + gridDim.y * blockIdx.z));
    if (tid == 0) a.red.partial[(size_t)rhs * nblk + bid] = s;
    if (last_block_arrive(a.red.count + rhs, nblk, tid)) {
      double t = 0.0;
      for (unsigned b = tid; b < nblk; b += NT) t += __ldcg(a.red.partial + (size_t)rhs * nblk + b);
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

// One Jacobi sweep from zero: y = omega D^-1 g (pointwise; forward or adjoint).
template <class R>
__global__ void k_j1(StencilCall<R> a, int adjoint) {
  const LevelView<R>& L = a.lv;
  const long long n = L.N * a.nrhs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    long long i = t % L.N;
    int x = (int)(i % L.nx);
    int y = (int)((i / L.nx) % L.ny);
    int z = (int)(i / ((long long)L.nx * L.ny));
    R kap = L.kappa[i];
    R av[5];
    table_eval<R, 0, 5>(a.tab.coef, a.tab.nseg, a.tab.ds, a.tab.inv_ds, eta_star(kap), av);
    cx<R> sab = L.abar[0][x] + L.abar[1][y] + L.abar[2][z];
    cx<R> D = L.inv_ell2 * ((R)2 * av[3] * sab) - (L.inv_ell2 * kap * kap * av[0]) * a.mass_shift;
    if (adjoint) D = conjc(D);
    cx<R> out = a.omega_j * cdiv(a.x[t], D);
    if (a.base) out += a.base[t];
    a.y[t] = out;
  }
}


// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
// z-block of the adjoint kernel (32 x 8 tiles over the whole grid)
static int adj_zblock(int nx, int ny, int nz, int nrhs) {
  const long long tiles = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * nrhs;
  const long long want = 152LL * 2 * 4;
  const long long nzb = (want + tiles - 1) / tiles;
  int zb = (int)((nz + nzb - 1) / nzb);
  return std::min(std::max(zb, 4), kMaxZb);
}

template <class R, int MODE, int OP>
static void launch_adj_t(const StencilCall<R>& c, cudaStream_t s) {
  constexpr int NP = AdjNP<OP>::v;
  const LevelView<R>& L = c.lv;
  const int zb = adj_zblock(L.nx, L.ny, L.nz, c.nrhs);
  const int tiles_x = (L.nx + TX - 1) / TX;
  dim3 grid(tiles_x * c.nrhs, (L.ny + TY - 1) / TY, (L.nz + zb - 1) / zb);
  size_t smem = 3 * PLANE * (sizeof(cx<R>) + NP * sizeof(R)) + kMaxSeg * kNumFn * 4 * sizeof(R);
  count_launch();
  k_adj<R, MODE, OP><<<grid, dim3(TX, TY), smem, s>>>(c, zb, tiles_x);
}

// forward operator kind of a call: A (real shell coefficients) unless the mass
// is shifted, B otherwise
template <class R>
static int fwd_opk(const StencilCall<R>& c, int op) {
  if (op == OP_Q) return OPK_Q;
  return (c.mass_shift.x == (R)1 && c.mass_shift.y == (R)0) ? OPK_A : OPK_B;
}

template <class R>
void launch_stencil(const StencilCall<R>& c, int mode, int op, bool adjoint, cudaStream_t s) {
  if (mode == M_J1) {
    long long n = c.lv.N * c.nrhs;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    count_launch();
    k_j1<R><<<blocks, 256, 0, s>>>(c, adjoint ? 1 : 0);
    return;
  }
  if (!adjoint && c.lv.level > 0) {
    gather::launch_fwd_gather<R>(c, mode, op, s);
    return;
  }
  if (!adjoint) {
    const int opk = fwd_opk(c, op);
    if (op == OP_Q) {
      launch_fwd<R, M_APPLY>(c, opk, s);
      return;
    }
    switch (mode) {
      case M_APPLY: launch_fwd<R, M_APPLY>(c, opk, s); break;
      case M_RESID: launch_fwd<R, M_RESID>(c, opk, s); break;
      case M_J2: launch_fwd<R, M_J2>(c, opk, s); break;
      case M_JSWEEP: launch_fwd<R, M_JSWEEP>(c, opk, s); break;
      case M_AWIN: launch_fwd<R, M_AWIN>(c, opk, s); break;
    }
  } else {
    if (op == OP_Q) {
      launch_adj_t<R, M_APPLY, OP_Q>(c, s);
      return;
    }
    switch (mode) {
      case M_APPLY: launch_adj_t<R, M_APPLY, OP_AB>(c, s); break;
      case M_RESID: launch_adj_t<R, M_RESID, OP_AB>(c, s); break;
      case M_J2: launch_adj_t<R, M_J2, OP_AB>(c, s); break;
      case M_JSWEEP: launch_adj_t<R, M_JSWEEP, OP_AB>(c, s); break;
    }
  }
}

// Blocks per right-hand side of a forward stencil launch on this grid (the
// size of the per-block partial-sum array its fused reductions need).
long long stencil_blocks_per_rhs(int level, int nx, int ny, int nz, const int* plain_lo, const int* plain_hi,
                                 int nrhs, int zblock, int zblock_f) {
  if (level > 0) return gather::gather_blocks_per_rhs(nx, ny, nz, plain_lo, plain_hi, nrhs, zblock, zblock_f);
  const int zb = zblock > 0 ? zblock : choose_zblock(nx, ny, nz, nrhs);
  const FwdPlan p = plan_layout(nx, ny, nz, plain_lo, plain_hi, true, zb, zblock_f);
  return p.blocks();
}

// Blocks per right-hand side of an adjoint stencil launch with nrhs
// right-hand sides (zblock > 0: that z-block instead of the launch's own).
long long adj_blocks_per_rhs(int nx, int ny, int nz, int nrhs, int zblock) {
  const int zb = zblock > 0 ? zblock : adj_zblock(nx, ny, nz, nrhs);
  return (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + zb - 1) / zb);
}

// Host replay of the forward launch layout and of the kernels' block and
// thread decode (the plan, the frame tile decode, the thread-to-column map of
// each tile shape, the z-block of every block, the row form each tile takes
// and its block id for fused reductions).  Violations counted: a written
// column outside the grid, a column outside the PML-free range on a row form
// that drops that axis's PML corrections (form 0 both axes, form 1 y, form 3
// x), a block id out of range or repeated.  (The kernels use forms 0, 2, 3.)  counts (nx * ny * nz bytes, or
// null) receives how often each node of right-hand side 0 is written,
// saturating at 255.
long long replay_fwd_layout(int level, int nx, int ny, int nz, const int* plo, const int* phi, int op, int nrhs,
                            int zblock, int zblock_f, unsigned char* counts, long long* blocks) {
  if (level > 0) return gather::replay_gather_layout(nx, ny, nz, plo, phi, op, nrhs, zblock, zblock_f, counts, blocks);
  const bool ab = op == OP_AB;
  const int zb = zblock > 0 ? zblock : choose_zblock(nx, ny, nz, nrhs);
  const FwdPlan p = plan_layout(nx, ny, nz, plo, phi, ab, zb, zblock_f);
  const long long nblk = p.blocks();
  if (blocks) *blocks = nblk;
  std::vector<unsigned char> seen((size_t)nblk, 0);
  long long bad = 0;
  auto plain_x = [&](int x) { return x >= plo[0] && x <= phi[0]; };
  auto plain_y = [&](int y) { return y >= plo[1] && y <= phi[1]; };
  // one block of a tile shape (npx columns per thread, txt x tyt threads)
  auto cta = [&](int npx, int txt, int tyt, int x0, int y0, int rx1, int ry1, int form, int zbk, int bz,
                 long long bid) {
    if (bid < 0 || bid >= nblk || seen[(size_t)bid]++) ++bad;
    const int zb0 = bz * zbk, zb1 = std::min(zb0 + zbk, nz);
    for (int tid = 0; tid < txt * tyt; ++tid) {
      const int tx = tid % txt, ty = tid / txt;
      for (int i = 0; i < npx; ++i) {
        const int gx = x0 + npx * tx + i, gy = y0 + ty;
        if (!(gx <= rx1 && gy <= ry1)) continue;  // inactive column
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
    }
  };
  const TileMap& m = p.frame;
  const int rnpx = p.ss ? Shapes<1>::Rect::NPX : Shapes<0>::Rect::NPX;
  const int wnpx = p.ss == 2 ? Shapes<2>::Wide::NPX : (p.ss ? Shapes<1>::Wide::NPX : Shapes<0>::Wide::NPX);
  const int tnpx = p.ss == 2 ? Shapes<2>::Tall::NPX : Shapes<0>::Tall::NPX;
  if (!p.split) {
    for (int bz = 0; bz < p.nzb; ++bz)
      for (int by = 0; by < p.GH; ++by)
        for (int t = 0; t < p.GW; ++t) {
          const int x0 = t * m.rw, y0 = by * m.rh;
          const int form = ab ? (grid_tile_form(x0, y0, m.rw, m.rh, nx, ny, plo, phi) == 0 ? 0 : 2) : 0;
          cta(rnpx, m.rw / rnpx, m.rh, x0, y0, nx - 1, ny - 1, form, p.zb, bz, t + (long long)p.GW * (by + p.GH * bz));
        }
  } else {
    // split: rectangle blocks numbered first, then the frame's; fused (one
    // launch): per z-block, the rectangle tiles and then the frame tiles
    const int px0 = p.frame.px0, py0 = p.frame.py0;
    const long long nrect = (long long)p.RW * p.RH, per_z = nrect + p.frame.count;
    for (int bz = 0; bz < p.nzb; ++bz)
      for (int by = 0; by < p.RH; ++by)
        for (int t = 0; t < p.RW; ++t)
          cta(rnpx, m.rw / rnpx, m.rh, px0 + t * m.rw, py0 + by * m.rh, p.frame.px1, p.frame.py1, 0, p.zb, bz,
              p.fused ? t + (long long)p.RW * by + per_z * bz : t + (long long)p.RW * (by + p.RH * bz));
    const long long off = (long long)p.RW * p.RH * p.nzb;
    for (int bz = 0; bz < p.nzbf; ++bz)
      for (int t = 0; t < p.frame.count; ++t) {
        const FrameTile f = decode_frame(p.frame, t);
        const long long bid = p.fused ? nrect + t + per_z * bz : off + t + (long long)p.frame.count * bz;
        if (f.wide)
          cta(wnpx, m.ww / wnpx, m.wh, f.x0, f.y0, f.rx1, f.ry1, 3, p.zbf, bz, bid);
        else
          cta(tnpx, m.tw / tnpx, m.th, f.x0, f.y0, f.rx1, f.ry1, 2, p.zbf, bz, bid);
      }
  }
  for (unsigned char v : seen)
    if (v != 1) ++bad;
  return bad;
}

// Host replay of the adjoint launch layout (32 x 8 tiles over the whole grid,
// adj_zblock planes per block unless zblock > 0): per-node write counts of
// right-hand side 0 (or null) and the blocks per right-hand side.
long long replay_adj_layout(int nx, int ny, int nz, int nrhs, int zblock, unsigned char* counts, long long* blocks) {
  const int zb = zblock > 0 ? zblock : adj_zblock(nx, ny, nz, nrhs);
  const int tx = (nx + TX - 1) / TX, ty = (ny + TY - 1) / TY, tz = (nz + zb - 1) / zb;
  if (blocks) *blocks = (long long)tx * ty * tz;
  if (counts)
    for (int bz = 0; bz < tz; ++bz)
      for (int by = 0; by < ty; ++by)
        for (int bx = 0; bx < tx; ++bx)
          for (int t = 0; t < NT; ++t) {
            const int gx = bx * TX + t % TX, gy = by * TY + t / TX;
            if (gx >= nx || gy >= ny) continue;
            for (int z = bz * zb; z < std::min(bz * zb + zb, nz); ++z) {
              unsigned char& c = counts[((size_t)z * ny + gy) * nx + gx];
              if (c < 255) ++c;
            }
          }
  return 0;
}

template <class R, int MODE, int OP>
static void set_adj_attr() {
  constexpr int NP = AdjNP<OP>::v;
  size_t smem = 3 * PLANE * (sizeof(cx<R>) + NP * sizeof(R)) + kMaxSeg * kNumFn * 4 * sizeof(R);
  cudaFuncSetAttribute(k_adj<R, MODE, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Opt the stencil kernels into more than 48 KB of dynamic shared memory where
// they need it.  Called before any launch and outside stream capture.
void init_kernel_attributes() {
  set_adj_attr<float, M_APPLY, OP_AB>();
  set_adj_attr<float, M_RESID, OP_AB>();
  set_adj_attr<float, M_J2, OP_AB>();
  set_adj_attr<float, M_JSWEEP, OP_AB>();
  set_adj_attr<float, M_APPLY, OP_Q>();
  set_adj_attr<double, M_APPLY, OP_AB>();
  set_adj_attr<double, M_RESID, OP_AB>();
  set_adj_attr<double, M_J2, OP_AB>();
  set_adj_attr<double, M_JSWEEP, OP_AB>();
  set_adj_attr<double, M_APPLY, OP_Q>();
  fwd_init_attrs<float, M_APPLY>();
  fwd_init_attrs<float, M_RESID>();
  fwd_init_attrs<float, M_J2>();
  fwd_init_attrs<float, M_JSWEEP>();
  fwd_init_attrs<double, M_APPLY>();
  fwd_init_attrs<double, M_RESID>();
  fwd_init_attrs<double, M_J2>();
  fwd_init_attrs<double, M_JSWEEP>();
  fwd_init_attrs<float, M_AWIN>();
  fwd_init_attrs<double, M_AWIN>();
}

template void launch_stencil<float>(const StencilCall<float>&, int, int, bool, cudaStream_t);
template void launch_stencil<double>(const StencilCall<double>&, int, int, bool, cudaStream_t);

}  // namespace hz
