// The Galerkin coarse operator A_hat = R A P as a 9-point stencil
// (Sec. 2.1, 3.1): (A_hat v)(X) = X v(X) + sum_mu Y_{+mu} v(X+mu) + Y_{-mu} v(X-mu).
//
// Stencil layout [Vc][N rows][9 dirs][N cols] (dir 0 self, 1+2mu forward,
// 2+2mu backward): for one output row the nine N-long rows are one
// contiguous "super-row" of 9N complex numbers, which a warp streams with
// consecutive lanes on consecutive entries while the nine neighbour vectors
// sit in shared memory.  FP16 storage keeps one FP32 scale per (site, row),
// the 16-bit analogue of the paper's fixed-point coarse links with a norm.
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "ops.cuh"
#include "stencil_row.cuh"
#include "tune.cuh"

namespace smg {
namespace {

__device__ __forceinline__ int nbr(const Geom& g, const int c[4], int dir) {
  if (dir == 0) return g.index(c);
  const int mu = (dir - 1) >> 1;
  const int k = ((dir - 1) & 1) ? -1 : 1;
  return g.shift(c, mu, k);
}

// Whether direction `dir` contributes to operator part `part` at coarse coords c.
__device__ __forceinline__ bool dir_in_part(int dir, int part, const int c[4], const int agg[4]) {
  if (part < 0) return true;
  if (dir == 0) return part == 0;
  const int mu = (dir - 1) >> 1;
  const int r = c[mu] % agg[mu];
  const bool cross = ((dir - 1) & 1) ? (r - 1 < 0) : (r + 1 >= agg[mu]);
  return part == 0 ? !cross : (part == dir && cross);
}

template <typename R, typename SL>
__global__ void __launch_bounds__(256) coarse_apply_kernel(typename cplx<R>::T* __restrict__ out,
                                                           const typename cplx<R>::T* __restrict__ in,
                                                           const SL* __restrict__ S, const float* __restrict__ rs,
                                                           Geom g, int N, int part, int4 agg4,
                                                           const typename cplx<R>::T* __restrict__ sub_from,
                                                           const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* vin = (C*)smem_raw;   // [9][N]
  const int X = blockIdx.x, s = blockIdx.y;
  const int agg[4] = {agg4.x, agg4.y, agg4.z, agg4.w};
  int c[4];
  g.coords(X, c);
  const long long n = (long long)g.V * N;
  for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
    const int dir = e / N, j = e % N;
    C v = C{0, 0};
    if (dir_in_part(dir, part, c, agg)) v = in[(size_t)s * n + (size_t)nbr(g, c, dir) * N + j];
    vin[e] = v;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = w; i < N; i += nw) {
    const SL* row = S + ((size_t)X * N + i) * 9 * N;
    C acc = C{0, 0};
    if constexpr (sizeof(R) == 4 && sizeof(SL) <= 8) {
      if (N % 4 == 0) {
        acc = stencil_row_dot<SL>(row, N, lane, [&](int dir, int j) { return vin + dir * N + j; });
      } else {
        for (int e = lane; e < 9 * N; e += 32) cfma(acc, ld<R>(row, e), vin[e]);
      }
    } else {
      for (int e = lane; e < 9 * N; e += 32) cfma(acc, ld<R>(row, e), vin[e]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      if (rs != nullptr) acc = cscale(acc, (R)rs[(size_t)X * N + i]);
      const size_t oi = (size_t)s * n + (size_t)X * N + i;
      if (sub_from != nullptr) acc = csub(sub_from[oi], acc);
      out[oi] = acc;
    }
  }
}

// The same operator with the V*N output rows of system blockIdx.y split into
// gridDim.x contiguous ranges that differ by at most one row.  A CTA walks its
// range site by site, staging each site's nine neighbour vectors in shared
// memory once, and gives each half warp one row; the grid is sized to the
// resident CTAs of the GPU, so every SM streams the same share of the stencil.
template <typename R, typename SL>
__global__ void __launch_bounds__(256) coarse_apply_rows_kernel(typename cplx<R>::T* __restrict__ out,
                                                                const typename cplx<R>::T* __restrict__ in,
                                                                const SL* __restrict__ S,
                                                                const float* __restrict__ rs, Geom g, int N,
                                                                int part, int4 agg4,
                                                                const typename cplx<R>::T* __restrict__ sub_from,
                                                                const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* vin = (C*)smem_raw;   // [9][N]
  const int s = blockIdx.y;
  const int agg[4] = {agg4.x, agg4.y, agg4.z, agg4.w};
  const long long n = (long long)g.V * N;
  const long long r0 = n * blockIdx.x / gridDim.x, r1 = n * (blockIdx.x + 1) / gridDim.x;
  const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15, nhw = blockDim.x >> 4;
  const unsigned hmask = 0xffffu << (threadIdx.x & 16);
  for (long long row = r0; row < r1;) {
    const int X = (int)(row / N);
    const long long rend = min(r1, (long long)(X + 1) * N);
    int c[4];
    g.coords(X, c);
    __syncthreads();   // the previous site's rows are done with vin
    for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
      const int dir = e / N, j = e % N;
      C v = C{0, 0};
      if (dir_in_part(dir, part, c, agg)) v = in[(size_t)s * n + (size_t)nbr(g, c, dir) * N + j];
      vin[e] = v;
    }
    __syncthreads();
    for (long long rr = row + hw; rr < rend; rr += nhw) {
      const int i = (int)(rr - (long long)X * N);
      const SL* srow = S + ((size_t)X * N + i) * 9 * N;
      C acc = C{0, 0};
      if constexpr (sizeof(R) == 4 && sizeof(SL) <= 8) {
        if (N % 4 == 0) {
          acc = stencil_row_dot_lanes<16, SL>(srow, N, hl, [&](int dir, int j) { return vin + dir * N + j; });
        } else {
          for (int e = hl; e < 9 * N; e += 16) cfma(acc, ld<R>(srow, e), vin[e]);
        }
      } else {
        for (int e = hl; e < 9 * N; e += 16) cfma(acc, ld<R>(srow, e), vin[e]);
      }
      for (int o = 8; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(hmask, acc.x, o);
        acc.y += __shfl_xor_sync(hmask, acc.y, o);
      }
      if (hl == 0) {
        if (rs != nullptr) acc = cscale(acc, (R)rs[(size_t)X * N + i]);
        const size_t oi = (size_t)s * n + (size_t)X * N + i;
        if (sub_from != nullptr) acc = csub(sub_from[oi], acc);
        out[oi] = acc;
      }
    }
    row = rend;
  }
}

// The row-balanced apply for up to SB systems per CTA (FP32 vectors, FP16 or
// FP32 stencil): each stencil chunk is loaded once and multiplied into every
// system of the group, in FP32 without rounding the vectors (the kernel of
// batched applies that must keep FP32 inputs, as the near-null CGNE does).
template <typename SL, int SB>
__global__ void __launch_bounds__(256) coarse_apply_rows_multi_kernel(float2* __restrict__ out,
                                                                      const float2* __restrict__ in,
                                                                      const SL* __restrict__ S,
                                                                      const float* __restrict__ rs, Geom g, int N,
                                                                      int part, int4 agg4,
                                                                      const float2* __restrict__ sub_from, int nsys,
                                                                      const int* run) {
  constexpr int C = Chunk<SL>::C;
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* vin = (float2*)smem_raw;   // [SB][9][N]
  const int s0 = blockIdx.y * SB, ns = min(SB, nsys - s0);
  const int agg[4] = {agg4.x, agg4.y, agg4.z, agg4.w};
  const long long n = (long long)g.V * N;
  const long long r0 = n * blockIdx.x / gridDim.x, r1 = n * (blockIdx.x + 1) / gridDim.x;
  const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15, nhw = blockDim.x >> 4;
  const unsigned hmask = 0xffffu << (threadIdx.x & 16);
  const int nine = 9 * N, nchunk = 9 * N / C;
  for (long long row = r0; row < r1;) {
    const int X = (int)(row / N);
    const long long rend = min(r1, (long long)(X + 1) * N);
    int c[4];
    g.coords(X, c);
    __syncthreads();
    for (int e = threadIdx.x; e < SB * nine; e += blockDim.x) {
      const int sb = e / nine, q = e - sb * nine;
      const int dir = q / N, j = q - dir * N;
      float2 v = make_float2(0.f, 0.f);
      if (sb < ns && dir_in_part(dir, part, c, agg)) v = in[(size_t)(s0 + sb) * n + (size_t)nbr(g, c, dir) * N + j];
      vin[e] = v;
    }
    __syncthreads();
    for (long long rr = row + hw; rr < rend; rr += nhw) {
      const int i = (int)(rr - (long long)X * N);
      const SL* srow = S + ((size_t)X * N + i) * 9 * N;
      float2 acc[SB];
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) acc[sb] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int q = hl; q < nchunk; q += 16) {
        const int e = q * C;
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(srow + e));
        const SL* m = reinterpret_cast<const SL*>(&raw);
        float2 mf[C];
#pragma unroll
        for (int u = 0; u < C; ++u) mf[u] = ld<float>(m, u);
#pragma unroll
        for (int sb = 0; sb < SB; ++sb) {
          const float4* v = reinterpret_cast<const float4*>(vin + sb * nine + e);
#pragma unroll
          for (int u = 0; u < C; u += 2) {
            const float4 vv = v[u / 2];
            cfma(acc[sb], mf[u], make_float2(vv.x, vv.y));
            cfma(acc[sb], mf[u + 1], make_float2(vv.z, vv.w));
          }
        }
      }
#pragma unroll
      for (int sb = 0; sb < SB; ++sb)
        for (int o = 8; o > 0; o >>= 1) {
          acc[sb].x += __shfl_xor_sync(hmask, acc[sb].x, o);
          acc[sb].y += __shfl_xor_sync(hmask, acc[sb].y, o);
        }
      const float sc = rs != nullptr ? rs[(size_t)X * N + i] : 1.f;
#pragma unroll
      for (int sb = 0; sb < SB; ++sb)
        if (hl == sb && sb < ns) {
          float2 a = cscale(acc[sb], sc);
          const size_t oi = (size_t)(s0 + sb) * n + (size_t)X * N + i;
          if (sub_from != nullptr) a = csub(sub_from[oi], a);
          out[oi] = a;
        }
    }
    row = rend;
  }
}

template <typename SL>
__global__ void coarse_pack_kernel(SL* __restrict__ dst, float* __restrict__ rs, const double2* __restrict__ S,
                                   long long rows, int N) {
  const long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const double2* src = S + (size_t)row * 9 * N;
  float sc = 1.0f;
  if (rs != nullptr) {
    double mx = 0.0;
    for (int e = lane; e < 9 * N; e += 32) mx = fmax(mx, fmax(fabs(src[e].x), fabs(src[e].y)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sc = mx > 0 ? (float)mx : 1.0f;
    if (lane == 0) rs[row] = sc;
  }
  const double isc = 1.0 / sc;
  for (int e = lane; e < 9 * N; e += 32) {
    const double2 v = src[e];
    SL* o = dst + (size_t)row * 9 * N + e;
    if constexpr (sizeof(SL) == 16) *o = SL{v.x, v.y};
    else if constexpr (sizeof(SL) == 8) *o = SL{(float)v.x, (float)v.y};
    else *o = __floats2half2_rn((float)(v.x * isc), (float)(v.y * isc));
  }
}

__global__ void coarse_dagger_kernel(double2* __restrict__ dst, const double2* __restrict__ src, Geom g, int N) {
  const long long total = (long long)g.V * N * 9 * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % N);
    long long q = e / N;
    const int dir = (int)(q % 9);
    q /= 9;
    const int i = (int)(q % N);
    const int X = (int)(q / N);
    int c[4];
    g.coords(X, c);
    int Xs = X, sdir = 0;
    if (dir > 0) {
      const int mu = (dir - 1) >> 1;
      const bool fwd = ((dir - 1) & 1) == 0;
      Xs = g.shift(c, mu, fwd ? 1 : -1);
      sdir = fwd ? dir + 1 : dir - 1;
    }
    const double2 v = src[(((size_t)Xs * N + j) * 9 + sdir) * N + i];
    dst[e] = make_double2(v.x, -v.y);
  }
}

__global__ void galerkin_scatter_kernel(double2* __restrict__ S, const double2* __restrict__ Cm, long long Vc,
                                        int N, int dir, int j0, int ncol) {
  const long long total = (long long)ncol * Vc * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % N);
    const long long q = e / N;
    const long long X = q % Vc;
    const int s = (int)(q / Vc);
    S[(((size_t)X * N + i) * 9 + dir) * N + j0 + s] = Cm[e];
  }
}

__global__ void unit_probes_kernel(double2* __restrict__ E, long long Vc, int N, int j0, int ncol) {
  const long long total = (long long)ncol * Vc * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % N);
    const int s = (int)(e / ((long long)Vc * N));
    E[e] = make_double2(i == j0 + s ? 1.0 : 0.0, 0.0);
  }
}

// ------------------------------------------------------------ dense coarsest
__global__ void dense_from_stencil_kernel(double2* __restrict__ D, const double2* __restrict__ S, Geom g, int N) {
  const long long n = (long long)g.V * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / n, col = e % n;
    const int X = (int)(row / N), i = (int)(row % N);
    const int Xp = (int)(col / N), j = (int)(col % N);
    int c[4];
    g.coords(X, c);
    double2 acc = make_double2(0, 0);
    for (int dir = 0; dir < 9; ++dir)
      if (nbr(g, c, dir) == Xp) acc = cadd(acc, S[(((size_t)X * N + i) * 9 + dir) * N + j]);
    D[e] = acc;
  }
}

// pivot search, row swap and pivot-row scaling for column k (one CTA)
__global__ void __launch_bounds__(1024) gj_pivot_kernel(double2* __restrict__ A, int n, int k,
                                                        double2* __restrict__ fac, int* __restrict__ perm) {
  __shared__ double bm[32];
  __shared__ int bi[32];
  __shared__ int prow;
  const int t = threadIdx.x;
  double best = -1.0;
  int idx = k;
  for (int i = k + t; i < n; i += blockDim.x) {
    const double2 v = A[(size_t)i * n + k];
    const double m2 = v.x * v.x + v.y * v.y;
    if (m2 > best) { best = m2; idx = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
  }
  if ((t & 31) == 0) { bm[t >> 5] = best; bi[t >> 5] = idx; }
  __syncthreads();
  if (t == 0) {
    double b = -1.0; int p = k;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (bm[w] > b || (bm[w] == b && bi[w] < p)) { b = bm[w]; p = bi[w]; }
    prow = p;
    perm[k] = p;
    if (!(b > 0.0)) perm[n] = 1;   // singular flag
  }
  __syncthreads();
  const int p = prow;
  if (p != k)
    for (int j = t; j < n; j += blockDim.x) {
      const double2 tmp = A[(size_t)k * n + j];
      A[(size_t)k * n + j] = A[(size_t)p * n + j];
      A[(size_t)p * n + j] = tmp;
    }
  __syncthreads();
  const double2 pv = A[(size_t)k * n + k];
  const double d = pv.x * pv.x + pv.y * pv.y;
  const double2 ip = d > 0 ? make_double2(pv.x / d, -pv.y / d) : make_double2(0, 0);
  __syncthreads();
  for (int j = t; j < n; j += blockDim.x) {
    const double2 v = (j == k) ? make_double2(1, 0) : A[(size_t)k * n + j];
    A[(size_t)k * n + j] = cmul(v, ip);
  }
  for (int i = t; i < n; i += blockDim.x) fac[i] = (i == k) ? make_double2(0, 0) : A[(size_t)i * n + k];
}

__global__ void gj_eliminate_kernel(double2* __restrict__ A, int n, int k, const double2* __restrict__ fac) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i == k) continue;
    const double2 f = fac[i];
    double2 v = (j == k) ? make_double2(0, 0) : A[e];
    const double2 w = A[(size_t)k * n + j];
    v.x -= f.x * w.x - f.y * w.y;
    v.y -= f.x * w.y + f.y * w.x;
    A[e] = v;
  }
}

__global__ void gj_unpermute_kernel(double2* __restrict__ A, int n, const int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      const double2 tmp = A[(size_t)i * n + k];
      A[(size_t)i * n + k] = A[(size_t)i * n + p];
      A[(size_t)i * n + p] = tmp;
    }
  }
}

// ------------------------------------------------ block-preconditioned stencil
// X^{-1} A_hat (Sec. 2.3) by Gauss-Jordan elimination with partial pivoting
// on the augmented rows [X | Y_1 .. Y_8 | 1] of one coarse site, one CTA per
// site, in place in global memory.  A super-row of the stencil layout is an
// augmented row without its identity part, which is kept in Xinv; the
// elimination leaves [1 | X^{-1} Y_1 .. X^{-1} Y_8 | X^{-1}].  Row swaps act
// on whole augmented rows, so no column unpermutation is needed.
constexpr int kBlockPrecThreads = 256;

__global__ void __launch_bounds__(kBlockPrecThreads) block_precondition_kernel(double2* __restrict__ S,
                                                                               double2* __restrict__ Xinv, int N,
                                                                               int* __restrict__ err) {
  constexpr int NW = kBlockPrecThreads / 32;
  __shared__ double bm[NW];
  __shared__ int bi[NW];
  __shared__ int prow;
  __shared__ double2 ipiv;
  extern __shared__ double2 fac[];          // elimination factors, N
  const int t = threadIdx.x;
  const int W = 10 * N;                     // augmented row length
  double2* Sx = S + (size_t)blockIdx.x * N * 9 * N;
  double2* Ix = Xinv + (size_t)blockIdx.x * N * N;
  auto at = [&](int i, int j) -> double2& {
    return j < 9 * N ? Sx[(size_t)i * 9 * N + j] : Ix[(size_t)i * N + (j - 9 * N)];
  };
  for (int e = t; e < N * N; e += kBlockPrecThreads) Ix[e] = make_double2(e / N == e % N ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    // pivot: the largest |X_ik| over rows i >= k (the first one on ties)
    double best = -1.0;
    int idx = k;
    for (int i = k + t; i < N; i += kBlockPrecThreads) {
      const double2 v = Sx[(size_t)i * 9 * N + k];
      const double m2 = v.x * v.x + v.y * v.y;
      if (m2 > best) { best = m2; idx = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, idx, o);
      if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
    }
    if ((t & 31) == 0) { bm[t >> 5] = best; bi[t >> 5] = idx; }
    __syncthreads();
    if (t == 0) {
      double b = -1.0;
      int p = k;
      for (int w = 0; w < NW; ++w)
        if (bm[w] > b || (bm[w] == b && bi[w] < p)) { b = bm[w]; p = bi[w]; }
      prow = p;
      const double2 pv = Sx[(size_t)p * 9 * N + k];
      const double d = pv.x * pv.x + pv.y * pv.y;
      if (d > 0.0) {
        ipiv = make_double2(pv.x / d, -pv.y / d);
      } else {
        ipiv = make_double2(0.0, 0.0);
        atomicExch(err, 1);                 // singular self block
      }
    }
    __syncthreads();
    const int p = prow;
    if (p != k)
      for (int j = t; j < W; j += kBlockPrecThreads) {
        const double2 tmp = at(k, j);
        at(k, j) = at(p, j);
        at(p, j) = tmp;
      }
    __syncthreads();
    const double2 ip = ipiv;
    for (int j = t; j < W; j += kBlockPrecThreads) at(k, j) = (j == k) ? make_double2(1.0, 0.0) : cmul(at(k, j), ip);
    for (int i = t; i < N; i += kBlockPrecThreads) fac[i] = (i == k) ? make_double2(0.0, 0.0) : at(i, k);
    __syncthreads();
    // eliminate column k from the other rows; the X columns j < k are unit
    // columns already (row k is zero there), so the row update starts at k
    const int Wk = W - k;
    for (int e = t; e < N * Wk; e += kBlockPrecThreads) {
      const int i = e / Wk, j = k + e % Wk;
      if (i == k) continue;
      const double2 f = fac[i];
      if (j == k) { at(i, j) = make_double2(0.0, 0.0); continue; }
      double2 v = at(i, j);
      const double2 w = at(k, j);
      v.x -= f.x * w.x - f.y * w.y;
      v.y -= f.x * w.y + f.y * w.x;
      at(i, j) = v;
    }
    __syncthreads();
  }
}

// out(X) = even(X) on even coarse sites, odd(X) on odd ones (a null source
// gives zeros), per system; in place when out is one of the sources.
template <typename C>
__global__ void parity_pick_kernel(C* out, const C* even, const C* odd, Geom g, int N, long long n,
                                   long long total, const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int X = (int)((e % n) / N);
    int c[4];
    g.coords(X, c);
    const C* src = ((c[0] + c[1] + c[2] + c[3]) & 1) ? odd : even;
    C v;
    v.x = 0;
    v.y = 0;
    if (src != nullptr) v = src[e];
    out[e] = v;
  }
}

// v[s](X) <- Xinv(X) v[s](X) in place, one CTA per (site, system): the site's
// N entries are staged in shared memory, each warp takes rows with its lanes
// on consecutive columns of X^{-1}.
template <typename C>
__global__ void __launch_bounds__(128) block_diag_kernel(C* __restrict__ v, const C* __restrict__ Xinv, int V, int N,
                                                         const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  extern __shared__ unsigned char bd_smem[];
  C* vin = reinterpret_cast<C*>(bd_smem);
  C* vx = v + ((size_t)blockIdx.y * V + blockIdx.x) * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) vin[j] = vx[j];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const C* Xr = Xinv + (size_t)blockIdx.x * N * N;
  for (int i = threadIdx.x >> 5; i < N; i += nw) {
    C acc;
    acc.x = 0;
    acc.y = 0;
    for (int j = lane; j < N; j += 32) cfma(acc, Xr[(size_t)i * N + j], vin[j]);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) vx[i] = acc;
  }
}

template <typename R, typename DT>
__global__ void __launch_bounds__(256) dense_apply_kernel(typename cplx<R>::T* __restrict__ out,
                                                          const typename cplx<R>::T* __restrict__ in,
                                                          const DT* __restrict__ D, int n, const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  const int s = blockIdx.y;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + w;
  if (row >= n) return;
  const C* v = in + (size_t)s * n;
  const DT* Dr = D + (size_t)row * n;
  C acc = C{0, 0};
  for (int j = lane; j < n; j += 32) cfma(acc, ld<R>(Dr, j), v[j]);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) out[(size_t)s * n + row] = acc;
}

// Synthetic stencil values in [-1, 1) from a hash of the index (timing only).
template <typename SL>
__global__ void synth_fill_kernel(SL* __restrict__ dst, long long n, unsigned seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)(e * 2654435761ull) ^ seed;
    h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
    const float a = (float)(h & 0xffff) / 32768.f - 1.f, b = (float)(h >> 16) / 32768.f - 1.f;
    if constexpr (sizeof(SL) == 4) dst[e] = __floats2half2_rn(a, b);
    else if constexpr (sizeof(SL) == 8) dst[e] = SL{a, b};
    else dst[e] = SL{(double)a, (double)b};
  }
}


// ---------------------------------------------------------- multi-RHS, tensor cores
// For nsys right-hand sides the stencil is read once per site: per site the
// apply is the real GEMM  D[N][2 nsys] = A[N][18N] * B[18N][2 nsys]  with
// A the FP16 stencil rows as stored (complex entries = (re, im) pairs along K)
// and B the gathered neighbour vectors embedded as real 2x2 blocks
// (B[2j][2r] = Re v, B[2j+1][2r] = -Im v, B[2j][2r+1] = Im v, B[2j+1][2r+1] = Re v),
// so D[i][2r] = Re (A v_r)_i and D[i][2r+1] = Im (A v_r)_i.
// Each warp owns 16 rows and issues m16n8k16 FP16 MMAs with FP32 accumulation.
// A is loaded straight from global memory, 16 bytes (4 complex) per thread;
// the K order inside each 16-complex block is permuted identically in A and B
// (slot t <- complex 4t + 2ks, slot t+4 <- 4t + 2ks + 1 for k-step ks).  B is
// built once per site in shared memory, in fragment order, scaled per system
// by a power of two sigma_r that puts the site's largest gathered entry in
// [0.5, 1) (FP16 range), and the scale is undone in the FP32 epilogue.
constexpr int kMmaMaxRhs = 16;

__device__ __forceinline__ unsigned h2u(__half2 h) { return *reinterpret_cast<unsigned*>(&h); }

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
               "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int NT>
__global__ void __launch_bounds__(256) coarse_apply_mma_kernel(float2* __restrict__ out, const float2* __restrict__ in,
                                                              const __half2* __restrict__ S,
                                                              const float* __restrict__ rs, Geom g, int N,
                                                              int nsys, int s0, long long sys_stride,
                                                              const float2* __restrict__ sub_from,
                                                              const int* run) {
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char mma_smem[];
  uint2* Bf = reinterpret_cast<uint2*>(mma_smem);   // [kb][NT][ks][lane]
  __shared__ unsigned vmax[kMmaMaxRhs];
  __shared__ float sig[kMmaMaxRhs];
  __shared__ int nb[9];
  const int X = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nrhs = min(kMmaMaxRhs, nsys - s0);
  const int nkb = 9 * N / 16;
  const long long n = (long long)g.V * N;
  if (tid < 9) {
    int c[4];
    g.coords(X, c);
    nb[tid] = tid == 0 ? X : g.shift(c, (tid - 1) >> 1, ((tid - 1) & 1) ? -1 : 1);
  }
  if (tid < kMmaMaxRhs) vmax[tid] = 0u;
  __syncthreads();
  // pass 1: largest |re|, |im| of the gathered entries per system
  for (int e = tid; e < nrhs * 9 * N; e += blockDim.x) {
    const int r = e / (9 * N), q = e - r * 9 * N;
    const int dir = q / N, j = q - dir * N;
    const float2 v = in[(size_t)(s0 + r) * sys_stride + (size_t)nb[dir] * N + j];
    const float m = fmaxf(fabsf(v.x), fabsf(v.y));
    atomicMax(&vmax[r], __float_as_uint(m));
  }
  __syncthreads();
  if (tid < kMmaMaxRhs) {
    const float m = tid < nrhs ? __uint_as_float(vmax[tid]) : 0.f;
    int e2 = 0;
    if (m > 0.f) frexpf(m, &e2);
    sig[tid] = ldexpf(1.f, -e2);
  }
  __syncthreads();
  // pass 2: B fragments in shared memory
  const int nfrag = nkb * NT * 2 * 32;
  for (int f = tid; f < nfrag; f += blockDim.x) {
    const int ln = f & 31, ks = (f >> 5) & 1;
    const int nt = (f >> 6) % NT, kb = (f >> 6) / NT;
    const int gg = ln >> 2, tt = ln & 3;
    const int col = nt * 8 + gg, r = col >> 1, im_out = col & 1;
    unsigned h[2] = {0u, 0u};
    if (r < nrhs) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int jj = kb * 16 + 4 * tt + 2 * ks + q;        // complex index along K
        const int dir = jj / N, j = jj - dir * N;
        float2 v = in[(size_t)(s0 + r) * sys_stride + (size_t)nb[dir] * N + j];
        v.x *= sig[r];
        v.y *= sig[r];
        h[q] = im_out ? h2u(__floats2half2_rn(v.y, v.x)) : h2u(__floats2half2_rn(v.x, -v.y));
      }
    }
    Bf[f] = make_uint2(h[0], h[1]);
  }
  __syncthreads();
  // MMA: warp w owns rows 16w .. 16w+15
  const int rows_w = 16 * w;
  if (rows_w >= N) return;
  const int gq = lane >> 2, tq = lane & 3;
  const __half2* A0 = S + ((size_t)X * N + rows_w + gq) * 9 * N + 4 * tq;
  const __half2* A1 = A0 + (size_t)8 * 9 * N;
  float acc[NT][4];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
#pragma unroll 4
  for (int kb = 0; kb < nkb; ++kb) {
    const uint4 r0 = __ldg(reinterpret_cast<const uint4*>(A0 + kb * 16));
    const uint4 r1 = __ldg(reinterpret_cast<const uint4*>(A1 + kb * 16));
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      unsigned a[4];
      a[0] = ks ? r0.z : r0.x;   // row g,   slot t
      a[1] = ks ? r1.z : r1.x;   // row g+8, slot t
      a[2] = ks ? r0.w : r0.y;   // row g,   slot t+4
      a[3] = ks ? r1.w : r1.y;   // row g+8, slot t+4
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const uint2 b = Bf[((kb * NT + nt) * 2 + ks) * 32 + lane];
        mma16816(acc[nt], a, b.x, b.y);
      }
    }
  }
  // epilogue: D fragment (row g / g+8, columns 2t, 2t+1 of tile nt) = (Re, Im) of system nt*4 + t
  const float sc0 = rs[(size_t)X * N + rows_w + gq], sc1 = rs[(size_t)X * N + rows_w + gq + 8];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int r = nt * 4 + tq;
    if (r >= nrhs) continue;
    const float inv = 1.f / sig[r];
    const size_t o0 = (size_t)(s0 + r) * sys_stride + (size_t)X * N + rows_w + gq;
    const size_t o1 = o0 + 8;
    float2 v0 = make_float2(acc[nt][0] * sc0 * inv, acc[nt][1] * sc0 * inv);
    float2 v1 = make_float2(acc[nt][2] * sc1 * inv, acc[nt][3] * sc1 * inv);
    if (sub_from != nullptr) {
      v0 = csub(sub_from[o0], v0);
      v1 = csub(sub_from[o1], v1);
    }
    out[o0] = v0;
    out[o1] = v1;
  }
  (void)n;
}

unsigned grid_cap(long long total, int threads) {
  long long g = (total + threads - 1) / threads;
  if (g > 16384) g = 16384;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

template <int NT>
void launch_mma(const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S, cudaStream_t st,
                const int* run, int s0) {
  const int nkb = 9 * p.N / 16;
  const size_t smem = (size_t)nkb * NT * 2 * 32 * sizeof(uint2);
  static size_t set = 0;
  if (smem > 48 * 1024 && smem > set) {
    SMG_CUDA_OK(cudaFuncSetAttribute(coarse_apply_mma_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    set = smem;
  }
  const int threads = 32 * (p.N / 16);
  launch_k(coarse_apply_mma_kernel<NT>, dim3(p.g.V), dim3(threads), smem, st, (float2*)out.p, (const float2*)in.p,
                                                            (const __half2*)S.p, S.scale, p.g, p.N, in.nsys, s0,
                                                            in.n, (const float2*)p.sub_from, run);
  SMG_LAUNCH_OK();
}

namespace {
constexpr int kRowsMultiSys = 8;   // systems per CTA of the multi-system row-balanced kernel
size_t rows_multi_smem(int N) { return (size_t)kRowsMultiSys * 9 * N * sizeof(float2); }
}  // namespace

bool coarse_path_ok(int path, int N, int nsys, Prec vp, Store s, bool full_op) {
  const bool multi16 = vp == P32 && s == S16 && nsys >= 2 && full_op;
  switch (path) {
    case CPATH_CORES:
    case CPATH_ROWS: return 9 * (size_t)N * prec_bytes(vp) <= 48 * 1024;
    case CPATH_ROWS_MULTI: return vp == P32 && s != S64 && nsys >= 2 && N % 4 == 0 && rows_multi_smem(N) <= 200 * 1024;
    case CPATH_MMA: return multi16 && N % 16 == 0 && N <= 128;
    case CPATH_UMMA_1x4:
    case CPATH_UMMA_2x4:
    case CPATH_UMMA_1x6: return multi16 && N == 128;
    default: return false;
  }
}

int coarse_path_list(int N, int nsys, Prec vp, Store s, bool full_op, int* out, int cap) {
  int n = 0;
  for (int path : {CPATH_UMMA_2x4, CPATH_UMMA_1x4, CPATH_UMMA_1x6, CPATH_MMA, CPATH_CORES, CPATH_ROWS,
                   CPATH_ROWS_MULTI})
    if (coarse_path_ok(path, N, nsys, vp, s, full_op)) {
      if (out != nullptr && n < cap) out[n] = path;
      ++n;
    }
  return n;
}

namespace {
const char* path_name(int path) {
  switch (path) {
    case CPATH_CORES: return "cuda-cores warp/row";
    case CPATH_MMA: return "mma.sync m16n8k16";
    case CPATH_UMMA_1x4: return "tcgen05 1 CTA/SM 4 stages";
    case CPATH_UMMA_2x4: return "tcgen05 2 CTA/SM 4 stages";
    case CPATH_UMMA_1x6: return "tcgen05 1 CTA/SM 6 stages";
    case CPATH_ROWS: return "cuda-cores half-warp/row, balanced grid";
    case CPATH_ROWS_MULTI: return "cuda-cores half-warp/row, balanced grid, 8 systems/CTA";
    default: return "?";
  }
}

// Candidate paths of a shape, the untuned default first.
std::vector<TuneCandidate> coarse_candidates(int N, int nsys, Prec vp, Store s, bool full_op) {
  int ids[CPATH_COUNT];
  const int n = coarse_path_list(N, nsys, vp, s, full_op, ids, CPATH_COUNT);
  std::vector<TuneCandidate> c;
  for (int i = 0; i < n; ++i) c.push_back({ids[i], path_name(ids[i])});
  return c;
}

void coarse_launch(int path, const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S, cudaStream_t st,
                   const int* run) {
  switch (path) {
    case CPATH_UMMA_1x4: coarse_apply_umma(out, in, p, S, coarse_umma_err(), st, run, 1, 4); return;
    case CPATH_UMMA_2x4: coarse_apply_umma(out, in, p, S, coarse_umma_err(), st, run, 2, 4); return;
    case CPATH_UMMA_1x6: coarse_apply_umma(out, in, p, S, coarse_umma_err(), st, run, 1, 6); return;
    case CPATH_MMA:
      for (int s0 = 0; s0 < in.nsys; s0 += kMmaMaxRhs) {
        const int nr = std::min(kMmaMaxRhs, in.nsys - s0);
        const int nt = (2 * nr + 7) / 8;
        if (nt <= 1) launch_mma<1>(out, in, p, S, st, run, s0);
        else if (nt == 2) launch_mma<2>(out, in, p, S, st, run, s0);
        else if (nt == 3) launch_mma<3>(out, in, p, S, st, run, s0);
        else launch_mma<4>(out, in, p, S, st, run, s0);
      }
      return;
    case CPATH_ROWS: {
      const size_t smem = (size_t)9 * p.N * prec_bytes(in.prec);
      SMG_REQUIRE(smem <= 48 * 1024, "coarse_apply: N too large");
      int4 agg = make_int4(p.agg[0], p.agg[1], p.agg[2], p.agg[3]);
      const long long rows = (long long)p.g.V * p.N;
      auto grid_of = [&](auto kernel) {
        // resident CTAs of this kernel on the whole GPU (host queries, not stream operations)
        static int per_gpu = 0;
        if (per_gpu == 0) {
          int dev = 0, sms = 0, per_sm = 0;
          SMG_CUDA_OK(cudaGetDevice(&dev));
          SMG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
          SMG_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 48 * 1024));
          per_gpu = std::max(1, sms * std::max(1, per_sm));
        }
        return dim3((unsigned)std::max(1LL, std::min<long long>(per_gpu, (rows + 15) / 16)), in.nsys);
      };
      if (in.prec == P64) {
        SMG_REQUIRE(S.s == S64, "coarse_apply: FP64 vectors need FP64 stencil");
        auto k = coarse_apply_rows_kernel<double, double2>;
        launch_k(k, grid_of(k), dim3(256), smem, st, (double2*)out.p, (const double2*)in.p, (const double2*)S.p,
                 nullptr, p.g, p.N, p.part, agg, (const double2*)p.sub_from, run);
      } else if (S.s == S32) {
        auto k = coarse_apply_rows_kernel<float, float2>;
        launch_k(k, grid_of(k), dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const float2*)S.p,
                 nullptr, p.g, p.N, p.part, agg, (const float2*)p.sub_from, run);
      } else {
        SMG_REQUIRE(S.s == S16, "coarse_apply: unsupported storage");
        auto k = coarse_apply_rows_kernel<float, __half2>;
        launch_k(k, grid_of(k), dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const __half2*)S.p,
                 S.scale, p.g, p.N, p.part, agg, (const float2*)p.sub_from, run);
      }
      SMG_LAUNCH_OK();
      return;
    }
    case CPATH_ROWS_MULTI: {
      const size_t smem = rows_multi_smem(p.N);
      int4 agg = make_int4(p.agg[0], p.agg[1], p.agg[2], p.agg[3]);
      const long long rows = (long long)p.g.V * p.N;
      const dim3 block(256);
      auto go = [&](auto kernel, auto* S_p) {
        static int per_sm = -1;
        static size_t smem_set = 0;
        if (smem > 48 * 1024 && smem > smem_set) {
          SMG_CUDA_OK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          smem_set = smem;
          per_sm = -1;
        }
        static int sms = 0;
        if (per_sm < 0) {
          int dev = 0;
          SMG_CUDA_OK(cudaGetDevice(&dev));
          SMG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
          SMG_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem));
        }
        const long long per_gpu = std::max(1, sms * std::max(1, per_sm));
        const dim3 grid((unsigned)std::max(1LL, std::min<long long>(per_gpu, (rows + 15) / 16)),
                        ceil_div(in.nsys, kRowsMultiSys));
        launch_k(kernel, grid, block, smem, st, (float2*)out.p, (const float2*)in.p, S_p,
                 S.s == S16 ? S.scale : nullptr, p.g, p.N, p.part, agg, (const float2*)p.sub_from, in.nsys, run);
      };
      if (S.s == S32) go(coarse_apply_rows_multi_kernel<float2, kRowsMultiSys>, (const float2*)S.p);
      else go(coarse_apply_rows_multi_kernel<__half2, kRowsMultiSys>, (const __half2*)S.p);
      SMG_LAUNCH_OK();
      return;
    }
    default: break;
  }
  const size_t smem = (size_t)9 * p.N * prec_bytes(in.prec);
  SMG_REQUIRE(smem <= 48 * 1024, "coarse_apply: N too large");
  dim3 grid(p.g.V, in.nsys);
  int4 agg = make_int4(p.agg[0], p.agg[1], p.agg[2], p.agg[3]);
  if (in.prec == P64) {
    SMG_REQUIRE(S.s == S64, "coarse_apply: FP64 vectors need FP64 stencil");
    launch_k(coarse_apply_kernel<double, double2>, dim3(grid), dim3(256), smem, st, (double2*)out.p,
             (const double2*)in.p, (const double2*)S.p, nullptr, p.g, p.N, p.part, agg, (const double2*)p.sub_from,
             run);
  } else if (S.s == S32) {
    launch_k(coarse_apply_kernel<float, float2>, dim3(grid), dim3(256), smem, st, (float2*)out.p, (const float2*)in.p,
             (const float2*)S.p, nullptr, p.g, p.N, p.part, agg, (const float2*)p.sub_from, run);
  } else {
    SMG_REQUIRE(S.s == S16, "coarse_apply: unsupported storage");
    launch_k(coarse_apply_kernel<float, __half2>, dim3(grid), dim3(256), smem, st, (float2*)out.p,
             (const float2*)in.p, (const __half2*)S.p, S.scale, p.g, p.N, p.part, agg, (const float2*)p.sub_from,
             run);
  }
  SMG_LAUNCH_OK();
}
}  // namespace

// The kernel is CoarseParams::path when given; otherwise the autotuner's
// choice for the shape (timed once on this stencil and these inputs into a
// scratch output), CUDA cores when allow_tc = 0.
void coarse_apply(const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S, cudaStream_t st,
                  const int* run) {
  SMG_REQUIRE(in.n == (long long)p.g.V * p.N && out.n == in.n && in.nsys == out.nsys && in.prec == out.prec,
              "coarse_apply: shape mismatch");
  const bool full = p.part < 0;
  auto is_tc = [](int id) { return id == CPATH_MMA || id == CPATH_UMMA_1x4 || id == CPATH_UMMA_2x4 || id == CPATH_UMMA_1x6; };
  int path = p.path;
  if (!p.allow_tc && is_tc(path)) path = CPATH_AUTO;
  if (path == CPATH_AUTO) {
    std::vector<TuneCandidate> cands = coarse_candidates(p.N, in.nsys, in.prec, S.s, full);
    if (!p.allow_tc) {
      std::vector<TuneCandidate> keep;
      for (const auto& cd : cands)
        if (!is_tc(cd.id)) keep.push_back(cd);
      cands.swap(keep);
    }
    SMG_REQUIRE(!cands.empty(), "coarse_apply: no kernel serves this shape");
    if (cands.size() == 1) {
      path = cands[0].id;
    } else {
      char key[160];
      std::snprintf(key, sizeof(key), "coarse_apply V=%d N=%d nsys=%d vec=%s store=%s sub=%d%s%s", p.g.V, p.N,
                    in.nsys, in.prec == P64 ? "f64" : "f32", S.s == S16 ? "f16" : (S.s == S32 ? "f32" : "f64"),
                    p.sub_from != nullptr ? 1 : 0, p.allow_tc ? "" : " fp32-inputs", full ? "" : " part");
      // candidates write a scratch output (freed after tuning)
      struct Scratch {
        void* p = nullptr;
        ~Scratch() { if (p) cudaFree(p); }
      } scratch;
      path = tune_pick(key, cands, st, [&](int id) {
        if (scratch.p == nullptr) {
          SMG_CUDA_OK(cudaMalloc(&scratch.p, out.bytes()));
        }
        Vec o = out;
        o.p = scratch.p;
        coarse_launch(id, o, in, p, S, st, nullptr);
      });
    }
  } else {
    SMG_REQUIRE(coarse_path_ok(path, p.N, in.nsys, in.prec, S.s, full),
                "coarse_apply: the requested kernel does not serve this shape");
  }
  coarse_launch(path, out, in, p, S, st, run);
}

void synth_fill(void* dst, Store s, long long n, unsigned seed, cudaStream_t st) {
  const unsigned g = grid_cap(n, 256);
  if (s == S16) synth_fill_kernel<__half2><<<g, 256, 0, st>>>((__half2*)dst, n, seed);
  else if (s == S32) synth_fill_kernel<float2><<<g, 256, 0, st>>>((float2*)dst, n, seed);
  else synth_fill_kernel<double2><<<g, 256, 0, st>>>((double2*)dst, n, seed);
  SMG_LAUNCH_OK();
}

void coarse_pack(Stored& dst, const double2* S64src, const Geom& g, int N, cudaStream_t st) {
  const long long rows = (long long)g.V * N;
  const unsigned grid = ceil_div(rows, 8);
  if (dst.s == S64) coarse_pack_kernel<double2><<<grid, 256, 0, st>>>((double2*)dst.p, nullptr, S64src, rows, N);
  else if (dst.s == S32) coarse_pack_kernel<float2><<<grid, 256, 0, st>>>((float2*)dst.p, nullptr, S64src, rows, N);
  else coarse_pack_kernel<__half2><<<grid, 256, 0, st>>>((__half2*)dst.p, dst.scale, S64src, rows, N);
  SMG_LAUNCH_OK();
}

void coarse_dagger(double2* dst, const double2* src, const Geom& g, int N, cudaStream_t st) {
  coarse_dagger_kernel<<<grid_cap((long long)g.V * N * 9 * N, 256), 256, 0, st>>>(dst, src, g, N);
  SMG_LAUNCH_OK();
}

void galerkin_scatter(double2* Sdst, const double2* C, const Geom& g, int N, int dir, int j0, int ncol,
                      cudaStream_t st) {
  galerkin_scatter_kernel<<<grid_cap((long long)ncol * g.V * N, 256), 256, 0, st>>>(Sdst, C, g.V, N, dir, j0, ncol);
  SMG_LAUNCH_OK();
}

void unit_probes(double2* E, long long Vc, int N, int j0, int ncol, cudaStream_t st) {
  unit_probes_kernel<<<grid_cap((long long)ncol * Vc * N, 256), 256, 0, st>>>(E, Vc, N, j0, ncol);
  SMG_LAUNCH_OK();
}

void dense_from_stencil(double2* Dn, const double2* Ssrc, const Geom& g, int N, cudaStream_t st) {
  const long long n = (long long)g.V * N;
  dense_from_stencil_kernel<<<grid_cap(n * n, 256), 256, 0, st>>>(Dn, Ssrc, g, N);
  SMG_LAUNCH_OK();
}

void dense_invert(double2* Dn, int n, double2* fac, int* perm, cudaStream_t st) {
  SMG_CUDA_OK(cudaMemsetAsync(perm, 0, sizeof(int) * (n + 1), st));
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, st>>>(Dn, n, k, fac, perm);
    gj_eliminate_kernel<<<grid_cap((long long)n * n, 256), 256, 0, st>>>(Dn, n, k, fac);
  }
  gj_unpermute_kernel<<<ceil_div(n, 128), 128, 0, st>>>(Dn, n, perm);
  SMG_LAUNCH_OK();
}

void block_precondition(double2* S64, double2* Xinv, const Geom& g, int N, int* err, cudaStream_t st) {
  SMG_REQUIRE(N >= 1 && N <= 256, "block_precondition: N out of range");
  block_precondition_kernel<<<(unsigned)g.V, kBlockPrecThreads, sizeof(double2) * N, st>>>(S64, Xinv, N, err);
  SMG_LAUNCH_OK();
}

void block_diag_apply(const Vec& v, const void* Xinv, Prec xprec, int N, cudaStream_t st, const int* run) {
  SMG_REQUIRE(N >= 1 && N <= 1024 && v.n % N == 0 && v.nsys >= 1 && v.nsys <= 65535 && xprec == v.prec,
              "block_diag_apply: shape or precision mismatch");
  const int V = (int)(v.n / N);
  const dim3 grid(V, v.nsys);
  if (v.prec == P64)
    launch_k(block_diag_kernel<double2>, grid, dim3(128), sizeof(double2) * N, st, (double2*)v.p,
             (const double2*)Xinv, V, N, run);
  else
    launch_k(block_diag_kernel<float2>, grid, dim3(128), sizeof(float2) * N, st, (float2*)v.p,
             (const float2*)Xinv, V, N, run);
  SMG_LAUNCH_OK();
}

void parity_pick(const Vec& out, const Vec* even, const Vec* odd, const Geom& g, int N, cudaStream_t st,
                 const int* run) {
  SMG_REQUIRE(out.n == (long long)g.V * N, "parity_pick: shape mismatch");
  for (const Vec* v : {even, odd})
    SMG_REQUIRE(v == nullptr || (v->n == out.n && v->nsys == out.nsys && v->prec == out.prec),
                "parity_pick: source shape mismatch");
  const long long total = out.n * out.nsys;
  const unsigned grid = grid_cap(total, 256);
  if (out.prec == P64)
    launch_k(parity_pick_kernel<double2>, dim3(grid), dim3(256), 0, st, (double2*)out.p,
             (const double2*)(even ? even->p : nullptr), (const double2*)(odd ? odd->p : nullptr), g, N, out.n,
             total, run);
  else
    launch_k(parity_pick_kernel<float2>, dim3(grid), dim3(256), 0, st, (float2*)out.p,
             (const float2*)(even ? even->p : nullptr), (const float2*)(odd ? odd->p : nullptr), g, N, out.n,
             total, run);
  SMG_LAUNCH_OK();
}

// Even/odd Schur complement of a block-preconditioned coarse operator
// A = 1 + K (self blocks exactly 1, every hop changes the site parity):
// with R(u) = u - A u = -K u,  S v = v - K_eo K_oe v = mask_e(v - R(mask_o(R(v))))
// for v that vanishes on odd sites.  The masks also drop what the rounding of
// stored (FP16 / FP32) identity self blocks leaves on the wrong parity.  With
// the adjoint stencil the same steps give S^dag.  t1, t2: scratch like v.
void schur_apply(const Vec& out, const Vec& in, const CoarseParams& cp0, const Stored& S, const Vec& t1,
                 const Vec& t2, cudaStream_t st, const int* run) {
  CoarseParams cp = cp0;
  cp.sub_from = in.p;
  coarse_apply(t1, in, cp, S, st, run);                  // t1 = R(in)
  parity_pick(t1, nullptr, &t1, cp.g, cp.N, st, run);    // its odd part
  cp.sub_from = t1.p;
  coarse_apply(t2, t1, cp, S, st, run);                  // t2 = R(t1)
  blas_sub(t1, in, t2, st, run);                         // in - t2
  parity_pick(out, &t1, nullptr, cp.g, cp.N, st, run);   // its even part
}

void dense_apply(const Vec& out, const Vec& in, const void* Dinv, Prec dprec, int n, cudaStream_t st,
                 const int* run) {
  SMG_REQUIRE(in.n == n && out.n == n && in.nsys == out.nsys && in.prec == out.prec, "dense_apply: shape mismatch");
  dim3 grid(ceil_div(n, 8), in.nsys);
  if (in.prec == P64) {
    SMG_REQUIRE(dprec == P64, "dense_apply: FP64 vectors need the FP64 inverse");
    launch_k(dense_apply_kernel<double, double2>, dim3(grid), dim3(256), 0, st, (double2*)out.p, (const double2*)in.p,
                                                              (const double2*)Dinv, n, run);
  } else {
    SMG_REQUIRE(dprec == P32, "dense_apply: FP32 vectors need the FP32 inverse");
    launch_k(dense_apply_kernel<float, float2>, dim3(grid), dim3(256), 0, st, (float2*)out.p, (const float2*)in.p,
                                                            (const float2*)Dinv, n, run);
  }
  SMG_LAUNCH_OK();
}

}  // namespace smg
