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

// Grow-only device scratch for reduction partials.
struct Workspace {
  void* ptr = nullptr;
  size_t cap = 0;
  void* get(size_t bytes);
  ~Workspace();
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
// out[s*ldo + p] = <vs[pi[p]], vs[pj[p]]> (conjugate-linear in the first slot), FP64
void blas_pair_dots(const Vec* vs, int nv, const int* pi, const int* pj, int np, double2* out, int ldo,
                    Workspace& ws, cudaStream_t st, const int* run = nullptr);

}  // namespace smg
