// Coarsest-level deflation (Table 1: SVD-deflated Chebyshev-basis CA-GCR).
//
// The k lowest singular triplets of the coarsest operator A come from a
// Chebyshev-filtered subspace iteration on A^dag A (the polynomial
// acceleration of Table 1's deflation setup): a block of k + guard vectors is
// filtered by a Chebyshev polynomial that damps [a, b] (a = the block's
// largest Ritz value, b >= lambda_max(A^dag A)) and amplifies the low end,
// then Rayleigh-Ritz makes it orthonormal and sorts it.  The host drives the
// loop (solver.cu); this file holds the block kernels it needs:
//
// * block_gram: all inner products between two vector blocks, tiled through
//   shared memory (every vector read once per call), FP64 sums;
// * block_combine: a vector block times a small coefficient matrix;
// * rayleigh_ritz: one CTA, two cyclic Jacobi eigen-decompositions (of the
//   Gram matrix G = V^dag V, then of G^{-1/2} H G^{-1/2}), in FP64;
// * the per-system Gram sums and minimum-residual coefficients of the
//   coarsest Chebyshev-basis CA-GCR, and the flags of its 0.25 / cycle-cap rule.
#include <algorithm>

#include "defl.cuh"

namespace smg {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramRows = 16;                                               // rows per tile
constexpr int kGramPerThread = kDeflMaxBlock * kDeflMaxBlock / kGramThreads;   // pair accumulators
constexpr int kRRThreads = 256;

// partial[b][i * kb + j] = this CTA's share of sum_r conj(A_i[r]) B_j[r]
template <typename C>
__global__ void __launch_bounds__(kGramThreads) gram_partial_kernel(const C* __restrict__ A, int ka,
                                                                    const C* __restrict__ B, int kb, long long n,
                                                                    double2* __restrict__ partial,
                                                                    const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  __shared__ C ta[kDeflMaxBlock][kGramRows];
  __shared__ C tb[kDeflMaxBlock][kGramRows];
  const int t = threadIdx.x;
  const int np = ka * kb;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * per;
  const long long r1 = r0 + per < n ? r0 + per : n;
  double2 acc[kGramPerThread];
#pragma unroll
  for (int m = 0; m < kGramPerThread; ++m) acc[m] = make_double2(0.0, 0.0);
  for (long long base = r0; base < r1; base += kGramRows) {
    const int cnt = (int)(r1 - base < kGramRows ? r1 - base : kGramRows);
    for (int e = t; e < (ka + kb) * kGramRows; e += kGramThreads) {
      const int v = e / kGramRows, r = e % kGramRows;
      C val;
      val.x = 0;
      val.y = 0;
      if (r < cnt) val = v < ka ? A[(size_t)v * n + base + r] : B[(size_t)(v - ka) * n + base + r];
      if (v < ka) ta[v][r] = val;
      else tb[v - ka][r] = val;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kGramPerThread; ++m) {
      const int q = t + m * kGramThreads;
      if (q < np) {
        const int i = q / kb, j = q % kb;
        for (int r = 0; r < cnt; ++r) {
          const C a = ta[i][r], b = tb[j][r];
          acc[m].x += (double)a.x * b.x + (double)a.y * b.y;
          acc[m].y += (double)a.x * b.y - (double)a.y * b.x;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < kGramPerThread; ++m) {
    const int q = t + m * kGramThreads;
    if (q < np) partial[(size_t)blockIdx.x * np + q] = acc[m];
  }
}

// out[q] = sum_b partial[b][q] in a fixed order
__global__ void gram_final_kernel(const double2* __restrict__ partial, int nb, int np, double2* __restrict__ out,
                                  const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nb; ++b) s = cadd(s, partial[(size_t)b * np + q]);
  out[q] = s;
}

template <typename C>
__global__ void block_combine_kernel(C* __restrict__ out, int kout, const C* __restrict__ X, int kx,
                                     const double2* __restrict__ Y, int ldy, long long n,
                                     const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  const long long total = (long long)kout * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n);
    const long long r = e % n;
    double ax = 0.0, ay = 0.0;
    for (int i = 0; i < kx; ++i) {
      const C x = X[(size_t)i * n + r];
      const double2 y = Y[(size_t)i * ldy + j];
      ax += (double)x.x * y.x - (double)x.y * y.y;
      ay += (double)x.x * y.y + (double)x.y * y.x;
    }
    C o;
    o.x = ax;
    o.y = ay;
    out[e] = o;
  }
}

// sum of v over the CTA; every thread calls and gets the sum
__device__ double cta_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int h = kRRThreads / 2; h > 0; h >>= 1) {
    if (t < h) red[t] += red[t + h];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// Cyclic Jacobi eigen-decomposition of the Hermitian k x k matrix H (global,
// row-major) by one CTA: H becomes diagonal (the eigenvalues), Z (global) the
// unitary matrix of eigenvectors (columns).  The rotation of pivot (p, q):
// with H_pq = |b| e, tau = (H_qq - H_pp) / (2 |b|), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)) (the smaller root of t^2 + 2 tau t - 1 = 0), c = 1 /
// sqrt(1 + t^2), s = t c, the unitary J = [[c, s e], [-s conj(e), c]] on
// coordinates (p, q) makes (J^dag H J)_pq vanish; H <- J^dag H J, Z <- Z J.
// Sweeps stop when the off-diagonal norm is below 1e-15 of the full norm.
__device__ void cta_jacobi(double2* H, double2* Z, int k, double* red) {
  const int t = threadIdx.x;
  for (int e = t; e < k * k; e += kRRThreads) Z[e] = make_double2(e / k == e % k ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int e = t; e < k * k; e += kRRThreads) {
      const double2 h = H[e];
      const double m = h.x * h.x + h.y * h.y;
      all += m;
      if (e / k != e % k) off += m;
    }
    off = cta_sum(off, red);
    all = cta_sum(all, red);
    if (!(off > 1e-30 * all)) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double2 b = H[(size_t)p * k + q];
        const double a = H[(size_t)p * k + p].x, d = H[(size_t)q * k + q].x;
        __syncthreads();   // all pivot reads happen before the entries change
        const double ab = sqrt(b.x * b.x + b.y * b.y);
        if (ab == 0.0) continue;   // the same decision in every thread
        const double2 ee = make_double2(b.x / ab, b.y / ab);
        const double tau = (d - a) / (2.0 * ab);
        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
        const double2 se = make_double2(s * ee.x, s * ee.y);     // s e
        const double2 sc = make_double2(s * ee.x, -s * ee.y);    // s conj(e)
        for (int r = t; r < k; r += kRRThreads) {
          const double2 hp = H[(size_t)r * k + p], hq = H[(size_t)r * k + q];
          H[(size_t)r * k + p] = csub(cscale(hp, c), cmul(sc, hq));
          H[(size_t)r * k + q] = cadd(cmul(se, hp), cscale(hq, c));
          const double2 zp = Z[(size_t)r * k + p], zq = Z[(size_t)r * k + q];
          Z[(size_t)r * k + p] = csub(cscale(zp, c), cmul(sc, zq));
          Z[(size_t)r * k + q] = cadd(cmul(se, zp), cscale(zq, c));
        }
        __syncthreads();
        for (int col = t; col < k; col += kRRThreads) {
          const double2 hp = H[(size_t)p * k + col], hq = H[(size_t)q * k + col];
          H[(size_t)p * k + col] = col == q ? make_double2(0.0, 0.0) : csub(cscale(hp, c), cmul(se, hq));
          H[(size_t)q * k + col] = col == p ? make_double2(0.0, 0.0) : cadd(cmul(sc, hp), cscale(hq, c));
        }
        __syncthreads();
      }
  }
}

__global__ void __launch_bounds__(kRRThreads) rayleigh_ritz_kernel(const double2* __restrict__ G,
                                                                   const double2* __restrict__ H, int k,
                                                                   double2* __restrict__ Y, double* __restrict__ lam,
                                                                   double2* S0, double2* S1, double2* S2) {
  __shared__ double red[kRRThreads];
  __shared__ double isq[kDeflMaxBlock];
  __shared__ double lv[kDeflMaxBlock];
  __shared__ int perm[kDeflMaxBlock];
  const int t = threadIdx.x;
  const int kk = k * k;
  // G = Q diag(g) Q^dag
  for (int e = t; e < kk; e += kRRThreads) S0[e] = G[e];
  __syncthreads();
  cta_jacobi(S0, S1, k, red);
  if (t == 0) {
    double gmax = 0.0;
    for (int i = 0; i < k; ++i) gmax = fmax(gmax, S0[(size_t)i * k + i].x);
    for (int i = 0; i < k; ++i) {
      const double g = S0[(size_t)i * k + i].x;
      isq[i] = (gmax > 0.0 && g > 1e-13 * gmax) ? 1.0 / sqrt(g) : 0.0;
    }
  }
  __syncthreads();
  // P = Q diag(g)^{-1/2} (S1), T = H P (S2), B = P^dag T (S0)
  for (int e = t; e < kk; e += kRRThreads) S1[e] = cscale(S1[e], isq[e % k]);
  __syncthreads();
  for (int e = t; e < kk; e += kRRThreads) {
    const int r = e / k, j = e % k;
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < k; ++m) cfma(acc, H[(size_t)r * k + m], S1[(size_t)m * k + j]);
    S2[e] = acc;
  }
  __syncthreads();
  for (int e = t; e < kk; e += kRRThreads) {
    const int i = e / k, j = e % k;
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < k; ++r) cfmac(acc, S1[(size_t)r * k + i], S2[(size_t)r * k + j]);
    S0[e] = acc;
  }
  __syncthreads();
  // B = Z diag(lam) Z^dag (Z in S2), Ritz vectors' coefficients P Z (S0)
  cta_jacobi(S0, S2, k, red);
  for (int i = t; i < k; i += kRRThreads) lv[i] = S0[(size_t)i * k + i].x;
  __syncthreads();
  for (int e = t; e < kk; e += kRRThreads) {
    const int r = e / k, j = e % k;
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < k; ++m) cfma(acc, S1[(size_t)r * k + m], S2[(size_t)m * k + j]);
    S0[e] = acc;
  }
  __syncthreads();
  for (int j = t; j < k; j += kRRThreads) {
    double nrm = 0.0;
    for (int r = 0; r < k; ++r) {
      const double2 y = S0[(size_t)r * k + j];
      nrm += y.x * y.x + y.y * y.y;
    }
    if (nrm == 0.0) lv[j] = 1e300;   // a dropped direction
  }
  __syncthreads();
  if (t == 0) {
    for (int j = 0; j < k; ++j) perm[j] = j;
    for (int j = 1; j < k; ++j) {
      const int pj = perm[j];
      int i = j - 1;
      while (i >= 0 && lv[perm[i]] > lv[pj]) { perm[i + 1] = perm[i]; --i; }
      perm[i + 1] = pj;
    }
  }
  __syncthreads();
  for (int e = t; e < kk; e += kRRThreads) {
    const int r = e / k, j = e % k;
    Y[e] = S0[(size_t)r * k + perm[j]];
  }
  for (int j = t; j < k; j += kRRThreads) lam[j] = lv[perm[j]];
}

// partial[s][b][p] = this CTA's share of the upper-triangle pair sums of system s
template <typename C>
__global__ void __launch_bounds__(kGramThreads) multi_gram_kernel(MultiPtr v, int nv, long long n,
                                                                  double2* __restrict__ partial,
                                                                  const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  constexpr int TR = 32;
  __shared__ C tile[kCaBasisMax + 1][TR];
  const int t = threadIdx.x;
  const int s = blockIdx.y;
  const int np = nv * (nv + 1) / 2;
  int pi = 0, pj = 0;
  if (t < np) {                       // pair t -> (i, j), i <= j, row order
    int rem = t;
    while (rem >= nv - pi) { rem -= nv - pi; ++pi; }
    pj = pi + rem;
  }
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * per;
  const long long r1 = r0 + per < n ? r0 + per : n;
  double2 acc = make_double2(0.0, 0.0);
  for (long long base = r0; base < r1; base += TR) {
    const int cnt = (int)(r1 - base < TR ? r1 - base : TR);
    for (int e = t; e < nv * TR; e += kGramThreads) {
      const int vi = e / TR, r = e % TR;
      C val;
      val.x = 0;
      val.y = 0;
      if (r < cnt) val = ((const C*)v.p[vi])[(size_t)s * n + base + r];
      tile[vi][r] = val;
    }
    __syncthreads();
    if (t < np)
      for (int r = 0; r < cnt; ++r) {
        const C a = tile[pi][r], b = tile[pj][r];
        acc.x += (double)a.x * b.x + (double)a.y * b.y;
        acc.y += (double)a.x * b.y - (double)a.y * b.x;
      }
    __syncthreads();
  }
  if (t < np) partial[((size_t)s * gridDim.x + blockIdx.x) * np + t] = acc;
}

// out[s][p] = sum_b partial[s][b][p]
__global__ void multi_gram_final_kernel(const double2* __restrict__ partial, int nb, int np, int nsys,
                                        double2* __restrict__ out, const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np * nsys) return;
  const int s = q / np, p = q % np;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < nb; ++b) acc = cadd(acc, partial[((size_t)s * nb + b) * np + p]);
  out[q] = acc;
}

// One CTA per system: H = W^dag W (m x m) from the pair sums over [r, W_0..],
// H = Q diag(lam) Q^dag by cyclic Jacobi, a = Q diag(1/lam) Q^dag (W^dag r)
// over the eigenvalues above drop x max.
__global__ void __launch_bounds__(kRRThreads) cagcr_coef_kernel(const double2* __restrict__ gram, int m,
                                                                double drop, const int* __restrict__ active,
                                                                double2* __restrict__ coef, double2* scratch,
                                                                const int* __restrict__ run) {
  if (run != nullptr && *run == 0) return;
  __shared__ double red[kRRThreads];
  __shared__ double2 gq[kCaBasisMax];    // Q^dag g / lam
  __shared__ double lv[kCaBasisMax];
  const int s = blockIdx.x;
  const int t = threadIdx.x;
  const int nv = m + 1;
  const int np = nv * (nv + 1) / 2;
  const double2* g = gram + (size_t)s * np;
  double2* H = scratch + (size_t)s * 2 * m * m;
  double2* Q = H + (size_t)m * m;
  // vector list index 0 is r, 1 + i is W_i; pair (a, b), a <= b, sits at a nv - a (a - 1) / 2 + b - a
  auto pidx = [&](int a, int b) { return a * nv - a * (a - 1) / 2 + (b - a); };
  for (int e = t; e < m * m; e += kRRThreads) {
    const int i = e / m, j = e % m;
    const double2 v = i <= j ? g[pidx(1 + i, 1 + j)] : g[pidx(1 + j, 1 + i)];
    H[e] = i <= j ? v : make_double2(v.x, -v.y);   // <W_i, W_j> = conj(<W_j, W_i>)
  }
  __syncthreads();
  cta_jacobi(H, Q, m, red);
  if (t == 0) {
    double lmax = 0.0;
    for (int i = 0; i < m; ++i) lmax = fmax(lmax, H[(size_t)i * m + i].x);
    for (int i = 0; i < m; ++i) {
      const double l = H[(size_t)i * m + i].x;
      lv[i] = (lmax > 0.0 && l > drop * lmax) ? 1.0 / l : 0.0;
    }
  }
  __syncthreads();
  // gq_k = (sum_i conj(Q_ik) <W_i, r>) / lam_k ; <W_i, r> is pair (0, 1 + i) conjugated
  for (int k = t; k < m; k += kRRThreads) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < m; ++i) {
      const double2 wr0 = g[pidx(0, 1 + i)];             // <r, W_i>
      cfmac(acc, Q[(size_t)i * m + k], make_double2(wr0.x, -wr0.y));
    }
    gq[k] = cscale(acc, lv[k]);
  }
  __syncthreads();
  const bool on = active == nullptr || active[s] != 0;
  for (int i = t; i < m; i += kRRThreads) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < m; ++k) cfma(acc, Q[(size_t)i * m + k], gq[k]);
    coef[(size_t)s * m + i] = on ? acc : make_double2(0.0, 0.0);
  }
}

__global__ void defl_active_kernel(const double2* __restrict__ rr, const double2* __restrict__ bb, double tol2,
                                   int* __restrict__ active, int* __restrict__ drun, int nsys, int first,
                                   const int* __restrict__ run_outer) {
  if (run_outer != nullptr && *run_outer == 0) {
    if (threadIdx.x == 0) *drun = 0;
    return;
  }
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    const int a = ((first != 0 || active[s] != 0) && rr[s].x > tol2 * bb[s].x) ? 1 : 0;
    active[s] = a;
    if (a) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *drun = any;
}

}  // namespace

void block_gram(const Vec& A, const Vec& B, double2* out, Workspace& ws, cudaStream_t st, const int* run) {
  SMG_REQUIRE(A.n == B.n && A.prec == B.prec && A.n > 0, "block_gram: shape mismatch");
  SMG_REQUIRE(A.nsys >= 1 && A.nsys <= kDeflMaxBlock && B.nsys >= 1 && B.nsys <= kDeflMaxBlock,
              "block_gram: at most 64 vectors per block");
  const int np = A.nsys * B.nsys;
  const int nb = (int)std::min<long long>(2 * 152, (A.n + 255) / 256);
  double2* partial = (double2*)ws.get(sizeof(double2) * (size_t)nb * np);
  if (A.prec == P64)
    launch_k(gram_partial_kernel<double2>, dim3(nb), dim3(kGramThreads), 0, st, (const double2*)A.p, A.nsys,
             (const double2*)B.p, B.nsys, A.n, partial, run);
  else
    launch_k(gram_partial_kernel<float2>, dim3(nb), dim3(kGramThreads), 0, st, (const float2*)A.p, A.nsys,
             (const float2*)B.p, B.nsys, A.n, partial, run);
  launch_k(gram_final_kernel, dim3(ceil_div(np, 256)), dim3(256), 0, st, (const double2*)partial, nb, np, out, run);
  SMG_LAUNCH_OK();
}

void block_combine(const Vec& out, const Vec& X, const double2* Y, int ldy, cudaStream_t st, const int* run) {
  SMG_REQUIRE(out.n == X.n && out.prec == X.prec && out.p != X.p, "block_combine: shape mismatch or aliasing");
  SMG_REQUIRE(X.nsys >= 1 && X.nsys <= kDeflMaxBlock && out.nsys >= 1 && out.nsys <= ldy,
              "block_combine: bad block sizes");
  const unsigned grid = (unsigned)std::min<long long>(4 * 152, ((long long)out.nsys * out.n + 255) / 256);
  if (X.prec == P64)
    launch_k(block_combine_kernel<double2>, dim3(grid), dim3(256), 0, st, (double2*)out.p, out.nsys,
             (const double2*)X.p, X.nsys, Y, ldy, X.n, run);
  else
    launch_k(block_combine_kernel<float2>, dim3(grid), dim3(256), 0, st, (float2*)out.p, out.nsys,
             (const float2*)X.p, X.nsys, Y, ldy, X.n, run);
  SMG_LAUNCH_OK();
}

void rayleigh_ritz(const double2* G, const double2* H, int k, double2* Y, double* lam, double2* scratch,
                   cudaStream_t st) {
  SMG_REQUIRE(k >= 1 && k <= kDeflMaxBlock, "rayleigh_ritz: 1 <= k <= 64");
  const size_t kk = (size_t)k * k;
  rayleigh_ritz_kernel<<<1, kRRThreads, 0, st>>>(G, H, k, Y, lam, scratch, scratch + kk, scratch + 2 * kk);
  SMG_LAUNCH_OK();
}

void multi_gram(const Vec* vs, int nv, double2* out, Workspace& ws, cudaStream_t st, const int* run) {
  SMG_REQUIRE(nv >= 1 && nv <= kCaBasisMax + 1 && nv <= kMaxVecs, "multi_gram: 1 <= nv <= 17");
  MultiPtr mp{};
  for (int i = 0; i < nv; ++i) {
    SMG_REQUIRE(vs[i].n == vs[0].n && vs[i].nsys == vs[0].nsys && vs[i].prec == vs[0].prec,
                "multi_gram: vector shapes differ");
    mp.p[i] = vs[i].p;
  }
  const int np = nv * (nv + 1) / 2;
  const long long n = vs[0].n;
  const int nsys = vs[0].nsys;
  const int nb = (int)std::min<long long>(2 * 152 / std::max(1, nsys) + 1, (n + 255) / 256);
  double2* partial = (double2*)ws.get(sizeof(double2) * (size_t)nb * np * nsys);
  const dim3 grid(nb, nsys);
  if (vs[0].prec == P64)
    launch_k(multi_gram_kernel<double2>, grid, dim3(kGramThreads), 0, st, mp, nv, n, partial, run);
  else
    launch_k(multi_gram_kernel<float2>, grid, dim3(kGramThreads), 0, st, mp, nv, n, partial, run);
  launch_k(multi_gram_final_kernel, dim3(ceil_div((long long)np * nsys, 256)), dim3(256), 0, st,
           (const double2*)partial, nb, np, nsys, out, run);
  SMG_LAUNCH_OK();
}

void cagcr_coef(const double2* gram, int m, double drop, const int* active, double2* coef, double2* scratch,
                int nsys, cudaStream_t st, const int* run) {
  SMG_REQUIRE(m >= 1 && m <= kCaBasisMax && nsys >= 1, "cagcr_coef: 1 <= m <= 16");
  launch_k(cagcr_coef_kernel, dim3(nsys), dim3(kRRThreads), 0, st, gram, m, drop, active, coef, scratch, run);
  SMG_LAUNCH_OK();
}

void defl_active(const double2* rr, const double2* bb, double tol2, int* active, int* drun, int nsys, bool first,
                 cudaStream_t st, const int* run_outer) {
  launch_k(defl_active_kernel, dim3(1), dim3(128), 0, st, rr, bb, tol2, active, drun, nsys, first ? 1 : 0,
           run_outer);
  SMG_LAUNCH_OK();
}

}  // namespace smg
