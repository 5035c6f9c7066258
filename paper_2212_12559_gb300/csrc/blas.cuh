// Batched vectors and the BLAS-1 / reduction launchers (see blas.cu).
#pragma once
#include "common.cuh"

namespace smg {

constexpr int kMaxVecs = 20;
constexpr int kMaxPairs = 64;

// A batched complex vector: nsys systems of n complex numbers each, system-major.
struct Vec {
  void* p = nullptr;
  long long n = 0;
  int nsys = 1;
  Prec prec = P64;
  size_t bytes() const { return (size_t)n * nsys * prec_bytes(prec); }
  void* sys(int s) const { return (char*)p + (size_t)s * n * prec_bytes(prec); }
};

struct MultiPtr { const void* p[kMaxVecs]; };

struct PairDotArgs {
  MultiPtr v;
  int nv, npairs;
  long long n;
  int pi[kMaxPairs], pj[kMaxPairs];
};

// Grow-only device scratch for reduction partials, plus the arrival counter
// of the single-kernel reductions (the last CTA to arrive finishes the sum).
struct Workspace {
  void* ptr = nullptr;
  size_t cap = 0;
  unsigned* counter = nullptr;
  void* get(size_t bytes);
  ~Workspace();
};

// Scalar work done by the last CTA of a reduction, once the sums are final.
// Which pointers a kind uses is listed beside it; all arrays are per system.
enum EpiKind {
  EPI_NONE = 0,
  EPI_GCR_INIT,    // sums: |r|^2.  r02=da, r2=db, thr2=dc, active=ia, nk=ib, run; tol2 or abs_target
  EPI_GCR_BETA1,   // sums: <w_j, w_k>, j<k (first CGS pass).  beta=d2a [K][K]
  EPI_GCR_STEP,    // sums: <w_j, w_k> (second pass), |w_k|^2, <w_k, r>, |r|^2.  beta=d2a, gamma=d2b,
                   //   alpha=d2c, ginv=d2d, na=d2e, r2=db, thr2=dc, active=ia, nk=ib, run, run_outer
  EPI_CA,          // sums: CA-GCR Gram pairs.  coef=d2a [s]
  EPI_CGNE_INIT,   // sums: |r|^2.  rr_prev=da, rr0=db, active=ia, iters=ib, run
  EPI_CGNE_ALPHA,  // sums: |p|^2.  rr_prev=da, active=ia, alpha=d2a, nalpha=d2b
  EPI_CGNE_BETA    // sums: |r|^2.  rr_prev=da, rr0=db, tol2, active=ia, iters=ib, bcoef=d2a [2], run
};

struct Epilogue {
  int kind = EPI_NONE;
  int k = 0, K = 0, s = 0, it = 0;
  double tol2 = 0.0;
  const double* abs_target = nullptr;
  double2 *d2a = nullptr, *d2b = nullptr, *d2c = nullptr, *d2d = nullptr, *d2e = nullptr;
  double *da = nullptr, *db = nullptr, *dc = nullptr;
  int *ia = nullptr, *ib = nullptr, *run = nullptr;
  const int* run_outer = nullptr;
};

void blas_copy(const Vec& dst, const Vec& src, cudaStream_t st, const int* run = nullptr);
void blas_zero(const Vec& x, cudaStream_t st, const int* run = nullptr);
// y = (accumulate ? y : 0) + sign * sum_j c[s*ldc + j] x_j
void blas_maxpy(const Vec& y, const Vec* xs, int nx, const double2* c, int ldc, double sign, bool accumulate,
                cudaStream_t st, const int* run = nullptr);
// x *= c[s], or x *= 1/c[s].x when inv_real
void blas_scale(const Vec& x, const double2* c, bool inv_real, cudaStream_t st, const int* run = nullptr);
// z = x - y
void blas_sub(const Vec& z, const Vec& x, const Vec& y, cudaStream_t st, const int* run = nullptr);
// out[s*ldo + p] = <vs[pi[p]], vs[pj[p]]> (conjugate-linear in the first slot), FP64,
// one kernel; `epi` runs in the last CTA on the finished sums.
void blas_pair_dots(const Vec* vs, int nv, const int* pi, const int* pj, int np, double2* out, int ldo,
                    Workspace& ws, cudaStream_t st, const int* run = nullptr, const Epilogue& epi = Epilogue());
// GCR step update: w_k <- (w_k - sum_{j<k} c[s*ldc+j] w_j) * ginv[s];  r <- r + na[s] * w_k
void blas_gcr_update(const Vec* W, int k, const double2* c, int ldc, const double2* ginv, const Vec& r,
                     const double2* na, cudaStream_t st, const int* run);
// GCR solution: y from gamma_j y_j + sum_{k>j} beta[k][j] y_k = alpha_j (j < nk), then x += sum_k y_k z_k
void blas_gcr_finish(const Vec& x, const Vec* Z, int K, const double2* alpha, const double2* gamma,
                     const double2* beta, const int* nk, cudaStream_t st, const int* run);

// Multi-shift CG update (FP64): X[s] += coef[s] P[s]; P[s] = coef[nshift+s] r + coef[2 nshift+s] P[s]
void blas_shift_update(const Vec& X, const Vec& P, const Vec& r, const double* coef, cudaStream_t st);

}  // namespace smg
