// The small solve of the bottom Krylov method C_4h (Sec. 3.2): from the Gram
// entries of the basis p_0 .. p_S, the normal equations of
// min || p_0 - sum_k y_k p_{k+1} || solved with a Cholesky factor in FP64.
// Shared by the Gram kernel of the launch chain and the persistent bottom
// kernel.
#pragma once

namespace hz {

// sres: Gram entries <p_a, p_b> (a <= b, row by row; re, im interleaved);
// yo: y_0 .. y_{S-1} (re, im).  Called by one thread of the block.
template <int KN>
__device__ __forceinline__ void gram_lsq_solve(const double* sres, double* yo) {
  constexpr int S = KN - 1;
  // index of G[a][b] = <p_a, p_b>, a <= b, in sres (rows a = 0 .. KN - 1, b = a .. KN - 1)
  auto gidx = [](int a, int b) { return a * KN - a * (a - 1) / 2 + (b - a); };
  // normal equations of min || p_0 - sum_k y_k p_{k+1} ||:  G_rr y = g_r0 with
  // G_rr = [<p_a, p_b>]_{a,b>=1}, g_r0 = [<p_a, p_0>]_{a>=1}; Cholesky G_rr = U^H U.
  // One thread, small arrays in shared memory and rolled loops: the solve must
  // not raise the register count of the streaming loop above.
  __shared__ double sUr[S * S], sUi[S * S], szr[S], szi[S], syr[S], syi[S];
  for (int a = 0; a < S * S; ++a) sUr[a] = sUi[a] = 0.0;
  double dmax = 0.0;
  for (int a = 1; a < KN; ++a) dmax = fmax(dmax, sres[2 * gidx(a, a)]);
  int rank = S;
#pragma unroll 1
  for (int j = 0; j < rank; ++j) {
    double d = sres[2 * gidx(j + 1, j + 1)];
    for (int k = 0; k < j; ++k) d -= sUr[k * S + j] * sUr[k * S + j] + sUi[k * S + j] * sUi[k * S + j];
    if (!(d > 1e-13 * dmax)) {
      rank = j;  // drop the remaining (numerically dependent) directions
      break;
    }
    const double ujj = sqrt(d), inv = 1.0 / ujj;
    sUr[j * S + j] = ujj;
#pragma unroll 1
    for (int b = j + 1; b < S; ++b) {
      double tr = sres[2 * gidx(j + 1, b + 1)], ti = sres[2 * gidx(j + 1, b + 1) + 1];
      for (int k = 0; k < j; ++k) {  // t -= conj(U[k][j]) U[k][b]
        tr -= sUr[k * S + j] * sUr[k * S + b] + sUi[k * S + j] * sUi[k * S + b];
        ti -= sUr[k * S + j] * sUi[k * S + b] - sUi[k * S + j] * sUr[k * S + b];
      }
      sUr[j * S + b] = tr * inv;
      sUi[j * S + b] = ti * inv;
    }
  }
  // U^H z = g_r0 (forward), then U y = z (backward); g_r0[a] = <p_{a+1}, p_0> = conj(G[0][a+1])
  for (int a = 0; a < S; ++a) szr[a] = szi[a] = syr[a] = syi[a] = 0.0;
#pragma unroll 1
  for (int a = 0; a < rank; ++a) {
    double tr = sres[2 * gidx(0, a + 1)], ti = -sres[2 * gidx(0, a + 1) + 1];
    for (int k = 0; k < a; ++k) {  // t -= conj(U[k][a]) z_k
      tr -= sUr[k * S + a] * szr[k] + sUi[k * S + a] * szi[k];
      ti -= sUr[k * S + a] * szi[k] - sUi[k * S + a] * szr[k];
    }
    szr[a] = tr / sUr[a * S + a];
    szi[a] = ti / sUr[a * S + a];
  }
#pragma unroll 1
  for (int a = rank - 1; a >= 0; --a) {
    double tr = szr[a], ti = szi[a];
    for (int k = a + 1; k < rank; ++k) {
      tr -= sUr[a * S + k] * syr[k] - sUi[a * S + k] * syi[k];
      ti -= sUr[a * S + k] * syi[k] + sUi[a * S + k] * syr[k];
    }
    syr[a] = tr / sUr[a * S + a];
    syi[a] = ti / sUr[a * S + a];
  }
  for (int a = 0; a < S; ++a) {
    yo[2 * a] = syr[a];
    yo[2 * a + 1] = syi[a];
  }
}

}  // namespace hz
