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

__device__ __forceinline__ float ca_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double ca_rsqrt(double x) { return rsqrt(x); }

// g: the Gram pairs <W_i, W_j> for i <= j in row order of the upper triangle,
// then <W_i, V0> for i = 0..s-1.  R is the arithmetic (double for FP64
// vectors; float for FP32 vectors, whose Gram entries carry FP32 rounding
// anyway): a pivot of the unit-diagonal matrix at or below 1e-12 (double) or
// 1e-5 (float) marks a dependent basis vector.  Ls: shared scratch
// [kCaMaxS][kCaMaxS] for this warp.  Lane i < s writes coef[i].  All 32 lanes
// must call.
template <typename R, typename GIn, typename COut>
__device__ __forceinline__ void ca_solve_warp(const GIn* g, int s, COut* coef,
                                              typename cplx<R>::T (*Ls)[kCaMaxS]) {
  using C = typename cplx<R>::T;
  const unsigned full = 0xffffffffu;
  const R dtol = sizeof(R) == 8 ? R(1e-12) : R(1e-5);
  const int i = threadIdx.x & 31;
  const bool own = i < s;
  // row i of the lower factor: L[i][j] = conj(G[j][i]), j <= i
  C c = C{0, 0};
  if (own) {
    for (int j = 0; j <= i; ++j) {
      const int p = j * s - j * (j - 1) / 2 + (i - j);
      Ls[i][j] = C{(R)g[p].x, (R)-g[p].y};
    }
    c = C{(R)g[s * (s + 1) / 2 + i].x, (R)g[s * (s + 1) / 2 + i].y};
  }
  const R dii = own ? Ls[i][i].x : R(0);
  const R dsc = dii > R(0) ? ca_rsqrt(dii) : R(0);
  c = cscale(c, dsc);
  for (int j = 0; j < s; ++j) {
    const R dj = __shfl_sync(full, dsc, j);
    if (own && j <= i) Ls[i][j] = cscale(Ls[i][j], dsc * dj);
  }
  __syncwarp();
  // left-looking Cholesky, one column per step; each pivot is inverted once
  bool drop = false;
  R inv = R(1);   // 1 / L[i][i] of this lane's row
  for (int j = 0; j < s; ++j) {
    R ij = R(1);
    int dj = 0;
    if (i == j) {
      R d = Ls[j][j].x;
      for (int k = 0; k < j; ++k) d -= Ls[j][k].x * Ls[j][k].x + Ls[j][k].y * Ls[j][k].y;
      drop = !(d > dtol) || dsc == R(0);
      inv = drop ? R(1) : ca_rsqrt(d);
      Ls[j][j] = C{drop ? R(1) : d * inv, R(0)};
      ij = inv;
      dj = drop ? 1 : 0;
    }
    ij = __shfl_sync(full, ij, j);
    dj = __shfl_sync(full, dj, j);
    if (own && i > j) {
      if (dj) {
        Ls[i][j] = C{0, 0};
      } else {
        C v = Ls[i][j];
        for (int k = 0; k < j; ++k) {
          const C x = Ls[i][k], y = Ls[j][k];   // v -= x * conj(y)
          v.x -= x.x * y.x + x.y * y.y;
          v.y -= x.y * y.x - x.x * y.y;
        }
        Ls[i][j] = C{v.x * ij, v.y * ij};
      }
    }
    __syncwarp();
  }
  // L y = c, column by column
  for (int k = 0; k < s; ++k) {
    if (i == k) c = drop ? C{0, 0} : C{c.x * inv, c.y * inv};
    const C ck = C{__shfl_sync(full, c.x, k), __shfl_sync(full, c.y, k)};
    if (own && i > k) {
      const C x = Ls[i][k];
      c.x -= x.x * ck.x - x.y * ck.y;
      c.y -= x.x * ck.y + x.y * ck.x;
    }
  }
  // L^dag a = y, from the last row up
  for (int k = s - 1; k >= 0; --k) {
    if (i == k) c = drop ? C{0, 0} : C{c.x * inv, c.y * inv};
    const C ck = C{__shfl_sync(full, c.x, k), __shfl_sync(full, c.y, k)};
    if (own && i < k) {
      const C l = Ls[k][i];                      // c_i -= conj(L[k][i]) c_k
      c.x -= l.x * ck.x + l.y * ck.y;
      c.y -= l.x * ck.y - l.y * ck.x;
    }
  }
  if (own) {
    const C v = cscale(c, dsc);
    const bool fin = isfinite(v.x) && isfinite(v.y);
    coef[i] = COut{fin ? v.x : R(0), fin ? v.y : R(0)};
  }
  __syncwarp();
}

}  // namespace smg
