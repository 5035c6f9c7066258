// Normal equations of the CA-GCR(s) smoother (Sec. 3.2, Table 1): with the
// power basis W_i = A^i V0 (i = 1..s), minimise |V0 - sum_i a_i W_i| by
//   (W^dag W) a = W^dag V0.
// The Gram matrix is scaled to unit diagonal, factored by Cholesky, and a
// basis vector whose pivot falls below 1e-12 (numerically dependent on the
// earlier ones) is dropped (its coefficient is 0).
//
// One warp solves one system: lane i owns row i of the factor, the factor
// lives in shared memory, and each column / substitution step is one
// parallel update.  GB300 runs FP64 at a small fraction of its FP32 rate, so
// the dependent chain of a one-thread factorisation is what this avoids.
#pragma once
#include "common.cuh"

namespace smg {

constexpr int kCaMaxS = 10;

// g: the Gram pairs <W_i, W_j> for i <= j in row order of the upper triangle,
// then <W_i, V0> for i = 0..s-1 (FP64).  Ls: shared scratch [kCaMaxS][kCaMaxS]
// for this warp.  Lane i < s writes coef[i].  All 32 lanes must call.
__device__ __forceinline__ void ca_solve_warp(const double2* g, int s, double2* coef,
                                              double2 (*Ls)[kCaMaxS]) {
  const unsigned full = 0xffffffffu;
  const int i = threadIdx.x & 31;
  const bool own = i < s;
  // row i of the lower factor: L[i][j] = conj(G[j][i]), j <= i
  double2 c = make_double2(0, 0);
  if (own) {
    for (int j = 0; j <= i; ++j) {
      const int p = j * s - j * (j - 1) / 2 + (i - j);
      Ls[i][j] = make_double2(g[p].x, -g[p].y);
    }
    c = g[s * (s + 1) / 2 + i];
  }
  const double dii = own ? Ls[i][i].x : 0.0;
  const double dsc = dii > 0 ? 1.0 / sqrt(dii) : 0.0;
  c = cscale(c, dsc);
  for (int j = 0; j < s; ++j) {
    const double dj = __shfl_sync(full, dsc, j);
    if (own && j <= i) Ls[i][j] = cscale(Ls[i][j], dsc * dj);
  }
  __syncwarp();
  // left-looking Cholesky, one column per step
  bool drop = false;
  for (int j = 0; j < s; ++j) {
    double ljj = 1.0;
    int dj = 0;
    if (i == j) {
      double d = Ls[j][j].x;
      for (int k = 0; k < j; ++k) d -= Ls[j][k].x * Ls[j][k].x + Ls[j][k].y * Ls[j][k].y;
      drop = !(d > 1e-12) || dsc == 0.0;
      ljj = drop ? 1.0 : sqrt(d);
      Ls[j][j] = make_double2(ljj, 0);
      dj = drop ? 1 : 0;
    }
    ljj = __shfl_sync(full, ljj, j);
    dj = __shfl_sync(full, dj, j);
    if (own && i > j) {
      if (dj) {
        Ls[i][j] = make_double2(0, 0);
      } else {
        double2 v = Ls[i][j];
        for (int k = 0; k < j; ++k) {
          const double2 x = Ls[i][k], y = Ls[j][k];   // v -= x * conj(y)
          v.x -= x.x * y.x + x.y * y.y;
          v.y -= x.y * y.x - x.x * y.y;
        }
        Ls[i][j] = make_double2(v.x / ljj, v.y / ljj);
      }
    }
    __syncwarp();
  }
  const double lii = own ? Ls[i][i].x : 1.0;
  // L y = c, column by column
  for (int k = 0; k < s; ++k) {
    if (i == k) c = drop ? make_double2(0, 0) : make_double2(c.x / lii, c.y / lii);
    const double2 ck = make_double2(__shfl_sync(full, c.x, k), __shfl_sync(full, c.y, k));
    if (own && i > k) {
      const double2 x = Ls[i][k];
      c.x -= x.x * ck.x - x.y * ck.y;
      c.y -= x.x * ck.y + x.y * ck.x;
    }
  }
  // L^dag a = y, from the last row up
  for (int k = s - 1; k >= 0; --k) {
    if (i == k) c = drop ? make_double2(0, 0) : make_double2(c.x / lii, c.y / lii);
    const double2 ck = make_double2(__shfl_sync(full, c.x, k), __shfl_sync(full, c.y, k));
    if (own && i < k) {
      const double2 l = Ls[k][i];                      // c_i -= conj(L[k][i]) c_k
      c.x -= l.x * ck.x + l.y * ck.y;
      c.y -= l.x * ck.y - l.y * ck.x;
    }
  }
  if (own) {
    const double2 v = cscale(c, dsc);
    coef[i] = (isfinite(v.x) && isfinite(v.y)) ? v : make_double2(0, 0);
  }
  __syncwarp();
}

}  // namespace smg
