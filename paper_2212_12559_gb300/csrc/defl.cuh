// Coarsest-level deflation (Table 1: SVD-deflated Chebyshev-basis CA-GCR):
// block inner products and combinations of vector blocks, and the one-CTA
// Rayleigh-Ritz step of the Chebyshev-filtered subspace iteration that finds
// the lowest singular triplets of the coarsest operator (see defl.cu).
#pragma once
#include "blas.cuh"

namespace smg {

constexpr int kDeflMaxBlock = 64;   // vectors in one deflation block (k + guard)

// Guard vectors iterated beside the k wanted ones (they take the slowest
// convergence of the subspace iteration): max(4, k / 4).
inline int defl_guard(int k) { return k / 4 > 4 ? k / 4 : 4; }

// out[i * kb + j] = <A_i, B_j> = sum_r conj(A_i[r]) B_j[r] (FP64 sums) for the
// ka vectors of block A and kb of block B, each of length n, vector-major
// (A.nsys = ka, B.nsys = kb); ka, kb <= kDeflMaxBlock.
void block_gram(const Vec& A, const Vec& B, double2* out, Workspace& ws, cudaStream_t st, const int* run = nullptr);
// out_j = sum_{i < X.nsys} X_i Y[i * ldy + j] for j < out.nsys; out must not alias X.
void block_combine(const Vec& out, const Vec& X, const double2* Y, int ldy, cudaStream_t st,
                   const int* run = nullptr);
// Rayleigh-Ritz of a block V with W = A V: from G = V^dag V and H = W^dag W
// (k x k, Hermitian, row-major) the coefficients Y (k x k; new vector j =
// sum_m V_m Y[m][j], orthonormal) and the Ritz values lam (ascending) of
// A^dag A on span(V).  Directions of V with Gram eigenvalue <= 1e-13 of the
// largest are dropped (their Ritz value is returned as 1e300, their column of
// Y is zero).  scratch: 3 k^2 double2.  One CTA.
void rayleigh_ritz(const double2* G, const double2* H, int k, double2* Y, double* lam, double2* scratch,
                   cudaStream_t st);
// Convergence flags of the deflated coarsest solve, per system s:
// active[s] = (first || active[s]) && rr[s].x > tol2 * bb[s].x; *drun = any.
// When run_outer is set and 0, only *drun = 0.
void defl_active(const double2* rr, const double2* bb, double tol2, int* active, int* drun, int nsys, bool first,
                 cudaStream_t st, const int* run_outer);

constexpr int kCaBasisMax = 16;      // Chebyshev-basis CA-GCR length on the coarsest level (Table 1: 16)

// Per-system Gram sums of a vector list: out[s][p] = <vs[i], vs[j]> for the
// pairs i <= j in row order of the upper triangle (p = i nv - i (i - 1) / 2 +
// j - i), FP64 sums; nv <= kCaBasisMax + 1.  All vectors batched alike.
void multi_gram(const Vec* vs, int nv, double2* out, Workspace& ws, cudaStream_t st, const int* run = nullptr);
// Minimum-residual coefficients of CA-GCR(m) from multi_gram over the list
// [r, W_0 .. W_{m-1}]: a = argmin |r - sum_i a_i W_i| through the
// eigen-decomposition of the Gram matrix W^dag W (one CTA per system, cyclic
// Jacobi in FP64), eigenvalues at or below drop x the largest left out (the
// minimum-norm least-squares solution).  coef[s * m + i]; 0 for systems with
// active[s] == 0.  scratch: 2 m^2 double2 per system.
void cagcr_coef(const double2* gram, int m, double drop, const int* active, double2* coef, double2* scratch,
                int nsys, cudaStream_t st, const int* run = nullptr);

}  // namespace smg
