// Batched BLAS-1 kernels and reductions for the Krylov solvers.
//
// Every kernel works on nsys systems at once (blockIdx.y = system) and takes
// its coefficients from device memory, one per system, so that whole solver
// iterations run without a host round trip.  Each kernel also takes an
// optional `run` flag: when it points at 0 the kernel returns at once, which
// lets a fixed launch sequence (and a CUDA graph of it) stop early once an
// inner solve has converged.
//
// Reductions are deterministic: per-CTA partial sums, then one finishing pass
// in a fixed order.  FP64 vectors reduce in FP64; FP32 vectors in FP32 (the
// sums are returned as FP64 for the solvers' scalar steps).
#include "blas.cuh"
#include "ca_solve.cuh"

namespace smg {

namespace {

constexpr int kThreads = 256;

template <typename C> struct RealOf;
template <> struct RealOf<double2> { using R = double; };
template <> struct RealOf<float2> { using R = float; };

__device__ __forceinline__ bool skip(const int* run) { return run != nullptr && *run == 0; }

__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }

// --------------------------------------------------------------- elementwise
template <typename CD, typename CS>
__global__ void copy_kernel(CD* __restrict__ dst, const CS* __restrict__ src, long long n,
                            long long dstride, long long sstride, const int* run) {
  if (skip(run)) return;
  const int s = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 v = to_d(src[s * sstride + i]);
    st(dst, s * dstride + i, v);
  }
}

template <typename C>
__global__ void zero_kernel(C* __restrict__ dst, long long n, const int* run) {
  if (skip(run)) return;
  const int s = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    dst[s * n + i] = C{0, 0};
  }
}

// y = a*y + sign * sum_j c[s*ldc + j] * x_j  (a = 0 or 1)
template <typename C>
__global__ void maxpy_kernel(C* __restrict__ y, MultiPtr xs, int nx, const double2* __restrict__ c,
                             int ldc, double sign, int accumulate, long long n, const int* run) {
  if (skip(run)) return;
  using R = typename RealOf<C>::R;
  const int s = blockIdx.y;
  __shared__ C coef[kMaxVecs];
  if (threadIdx.x < nx) {
    double2 v = c[(long long)s * ldc + threadIdx.x];
    coef[threadIdx.x] = C{(R)(sign * v.x), (R)(sign * v.y)};
  }
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    C acc = accumulate ? y[s * n + i] : C{0, 0};
    for (int j = 0; j < nx; ++j) {
      // a zero coefficient contributes nothing, whatever the vector holds
      // (slots a converged solver never wrote may hold any bit pattern)
      if (coef[j].x == R(0) && coef[j].y == R(0)) continue;
      const C* xj = (const C*)xs.p[j];
      cfma(acc, coef[j], xj[s * n + i]);
    }
    y[s * n + i] = acc;
  }
}

// x *= c[s] (complex coefficient), or x *= 1/|c[s]| when `inv_real`.
template <typename C>
__global__ void scale_kernel(C* __restrict__ x, const double2* __restrict__ c, int inv_real, long long n,
                             const int* run) {
  if (skip(run)) return;
  using R = typename RealOf<C>::R;
  const int s = blockIdx.y;
  double2 cv = c[s];
  C f;
  if (inv_real) {
    double v = cv.x > 0 ? 1.0 / cv.x : 0.0;
    f = C{(R)v, (R)0};
  } else {
    f = C{(R)cv.x, (R)cv.y};
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[s * n + i] = cmul(x[s * n + i], f);
  }
}

// z = x - y  (residual update r = b - A x)
template <typename C>
__global__ void sub_kernel(C* __restrict__ z, const C* __restrict__ x, const C* __restrict__ y, long long n,
                           const int* run) {
  if (skip(run)) return;
  const int s = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    z[s * n + i] = csub(x[s * n + i], y[s * n + i]);
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ bool off_flag(const int* run) { return run != nullptr && *run == 0; }

// Per-system scalar logic of the solvers, on the finished sums `o` (row ldo).
__device__ void epilogue_system(const Epilogue& e, int s, const double2* o) {
  switch (e.kind) {
    case EPI_GCR_INIT: {
      const double b2 = o[0].x;
      const double thr = e.abs_target != nullptr ? e.abs_target[s] : e.tol2 * b2;
      e.da[s] = b2;
      e.db[s] = b2;
      e.dc[s] = thr;
      e.ia[s] = (!off_flag(e.run_outer) && b2 > thr && b2 > 0.0) ? 1 : 0;
      e.ib[s] = 0;
      break;
    }
    case EPI_GCR_BETA1: {
      for (int j = 0; j < e.k; ++j) e.d2a[((size_t)s * e.K + e.k) * e.K + j] = o[j];
      break;
    }
    case EPI_GCR_STEP: {
      const int k = e.k, K = e.K;
      double sumc = 0.0;
      for (int j = 0; j < k; ++j) {
        double2& b = e.d2a[((size_t)s * K + k) * K + j];
        b = cadd(b, o[j]);
        sumc += o[j].x * o[j].x + o[j].y * o[j].y;
      }
      const double ww = o[k].x - sumc;
      const double2 wr = o[k + 1];
      const double rr = o[k + 2].x;      // |r|^2 before this step
      const double g = sqrt(fmax(ww, 0.0));
      const bool gfin = g > 0.0 && isfinite(g);
      const bool ok = e.ia[s] && gfin;
      const double2 a = ok ? make_double2(wr.x / g, wr.y / g) : make_double2(0, 0);
      e.d2b[(size_t)s * K + k] = make_double2(ok ? g : 0.0, 0);
      e.d2c[(size_t)s * K + k] = a;
      e.d2d[s] = make_double2(gfin ? 1.0 / g : 0.0, 0);
      e.d2e[s] = make_double2(-a.x, -a.y);
      if (e.ia[s]) {
        e.ib[s] = k + 1;
        // |r - a w_k|^2 = |r|^2 - |a|^2 from this step's own |r|^2: a running
        // difference from |b|^2 carries a rounding error of about 1e-16 |b|^2,
        // which hides residuals below 1e-8 |b| from a 1e-10 test
        const double r2 = rr - (a.x * a.x + a.y * a.y);
        e.db[s] = r2;
        // converged, stagnated (w_k in the span of w_0..w_{k-1}) or non-finite
        if (!(r2 > e.dc[s]) || !gfin) e.ia[s] = 0;
      }
      break;
    }
    case EPI_CA: break;   // one warp per system, see pair_dot_kernel
    case EPI_CGNE_INIT: {
      e.da[s] = o[0].x;
      e.db[s] = o[0].x;
      e.ia[s] = o[0].x > 0.0 ? 1 : 0;
      e.ib[s] = 0;
      break;
    }
    case EPI_CGNE_ALPHA: {
      const double d = o[0].x;
      const double a = (e.ia[s] && d > 0.0) ? e.da[s] / d : 0.0;
      e.d2a[s] = make_double2(a, 0);
      e.d2b[s] = make_double2(-a, 0);
      break;
    }
    case EPI_CGNE_BETA: {
      const double v = o[0].x;
      double b = 0.0;
      if (e.ia[s]) {
        b = e.da[s] > 0 ? v / e.da[s] : 0.0;
        e.da[s] = v;
        e.ib[s] = e.it + 1;
        if (!(v > e.tol2 * e.db[s])) e.ia[s] = 0;
      }
      e.d2a[2 * s] = make_double2(e.ia[s] ? b : 0.0, 0);
      e.d2a[2 * s + 1] = make_double2(1.0, 0);
      break;
    }
    default: break;
  }
}

// partial[s][block][p] = this CTA's share of conj(v[pi[p]]) * v[pj[p]]; the
// last CTA to arrive adds the partials in a fixed order and runs the epilogue.
// Accumulator type of a reduction: FP64 for FP64 vectors, FP32 for FP32
// vectors (threads, CTA tree and grid sum; the inner solvers that use FP32
// vectors only need their inner products to FP32 accuracy).  GB300's FP64
// rate is a small fraction of its FP32 rate.
template <typename C> struct AccOf;
template <> struct AccOf<double2> { using T = double2; };
template <> struct AccOf<float2> { using T = float2; };

// partial[s][block][p] = this CTA's share of conj(v[pi[p]]) * v[pj[p]]; the
// last CTA to arrive adds the partials in a fixed order and runs the epilogue.
template <typename C>
__global__ void __launch_bounds__(kThreads) pair_dot_kernel(PairDotArgs a, double2* __restrict__ partial,
                                                            double2* __restrict__ out, int ldo,
                                                            unsigned* __restrict__ counter, Epilogue epi,
                                                            const int* run) {
  using A = typename AccOf<C>::T;
  if (skip(run)) return;
  constexpr int TR = 128;   // rows per tile
  // one padding entry per vector row: the pairs of one row (same r, different
  // vectors) then fall in different shared-memory banks
  __shared__ __align__(16) C tile[kMaxVecs][TR + 1];
  __shared__ A red[kThreads];
  __shared__ bool last;
  const int s = blockIdx.y;
  const int np = a.npairs;
  const int groups = kThreads / np;               // row groups per pair
  const int t = threadIdx.x;
  const int p = t % np;
  const int grp = t / np;
  const bool active = grp < groups;
  A acc = A{0, 0};
  const long long n = a.n;
  const long long rows_per_block = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * rows_per_block;
  const long long r1 = min(n, r0 + rows_per_block);
  // the next tile's loads are issued before the current tile is used
  constexpr int PF = (kMaxVecs * TR + kThreads - 1) / kThreads;
  C buf[PF];
  const int nload = a.nv * TR;
  auto fetch = [&](long long base) {
    const int cnt = (int)min((long long)TR, r1 - base);
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int e = t + m * kThreads;
      const int v = e / TR, r = e % TR;
      buf[m] = (e < nload && r < cnt) ? ((const C*)a.v.p[v])[s * n + base + r] : C{0, 0};
    }
  };
  if (r0 < r1) fetch(r0);
  for (long long base = r0; base < r1; base += TR) {
    const int cnt = (int)min((long long)TR, r1 - base);
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int e = t + m * kThreads;
      if (e < nload) tile[e / TR][e % TR] = buf[m];
    }
    __syncthreads();
    if (base + TR < r1) fetch(base + TR);
    if (active) {
      const int vi = a.pi[p], vj = a.pj[p];
      for (int r = grp; r < cnt; r += groups) cfmac(acc, tile[vi][r], tile[vj][r]);
    }
    __syncthreads();
  }
  red[t] = active ? acc : A{0, 0};
  __syncthreads();
  const int nb = gridDim.x, nsys = gridDim.y;
  // partial sums in the accumulator type (FP32 for FP32 vectors: this part
  // runs FP64 at a small fraction of the FP32 rate)
  A* part = reinterpret_cast<A*>(partial);
  // fixed-order tree over the row groups
  for (int gc = groups; gc > 1;) {
    const int half = (gc + 1) / 2;
    for (int e = t; e < (gc - half) * np; e += kThreads) red[e] = cadd(red[e], red[e + half * np]);
    gc = half;
    __syncthreads();
  }
  if (t < np) part[((long long)s * nb + blockIdx.x) * np + t] = red[t];
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned ticket = atomicAdd(counter, 1u);
    last = (ticket == (unsigned)(nb * nsys) - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // one warp per output: lanes take every 32nd partial, then a fixed-order
  // shuffle tree (deterministic, and the loads of a lane are independent)
  {
    const int warp = t >> 5, lane = t & 31;
    for (int o = warp; o < nsys * np; o += kThreads / 32) {
      const int ss = o / np, pp = o % np;
      A sum = A{0, 0};
      for (int b = lane; b < nb; b += 32) sum = cadd(sum, __ldcg(&part[((long long)ss * nb + b) * np + pp]));
      for (int off = 16; off > 0; off >>= 1) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
      }
      if (lane == 0) out[(long long)ss * ldo + pp] = make_double2(sum.x, sum.y);
    }
  }
  if (t == 0) *counter = 0;
  if (epi.kind == EPI_NONE) return;
  __threadfence_block();
  __syncthreads();
  if (epi.kind == EPI_CA) {
    // the reduction tiles are free now: one factor scratch per warp, in the
    // arithmetic of the vectors
    using R = typename RealOf<C>::R;
    using CR = typename cplx<R>::T;
    static_assert(sizeof(tile) >= sizeof(CR) * kCaMaxS * kCaMaxS * (kThreads / 32), "CA scratch");
    CR(*Ls)[kCaMaxS] = reinterpret_cast<CR(*)[kCaMaxS]>(&tile[0][0]) + (t >> 5) * kCaMaxS;
    for (int ss = t >> 5; ss < nsys; ss += kThreads / 32)
      ca_solve_warp<R>(out + (long long)ss * ldo, epi.s, epi.d2a + (size_t)ss * epi.s, Ls);
  } else {
    for (int ss = t; ss < nsys; ss += kThreads) epilogue_system(epi, ss, out + (long long)ss * ldo);
  }
  __syncthreads();
  if (t == 0 && epi.run != nullptr &&
      (epi.kind == EPI_GCR_INIT || epi.kind == EPI_GCR_STEP || epi.kind == EPI_CGNE_INIT ||
       epi.kind == EPI_CGNE_BETA)) {
    int any = 0;
    for (int ss = 0; ss < nsys; ++ss) any |= epi.ia[ss];
    *epi.run = (any && !off_flag(epi.run_outer)) ? 1 : 0;
  }
}

template <typename C>
__global__ void gcr_update_kernel(MultiPtr W, int k, const double2* __restrict__ c, int ldc,
                                  const double2* __restrict__ ginv, C* __restrict__ r, const double2* __restrict__ na,
                                  long long n, const int* run) {
  if (skip(run)) return;
  using R = typename RealOf<C>::R;
  const int s = blockIdx.y;
  __shared__ C coef[kMaxVecs];
  __shared__ C gi, nal;
  if (threadIdx.x < k) {
    const double2 v = c[(long long)s * ldc + threadIdx.x];
    coef[threadIdx.x] = C{(R)(-v.x), (R)(-v.y)};
  }
  if (threadIdx.x == 0) {
    gi = C{(R)ginv[s].x, (R)0};
    nal = C{(R)na[s].x, (R)na[s].y};
  }
  __syncthreads();
  C* wk = (C*)W.p[k];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    C acc = wk[s * n + i];
    for (int j = 0; j < k; ++j) cfma(acc, coef[j], ((const C*)W.p[j])[s * n + i]);
    acc = cmul(acc, gi);
    wk[s * n + i] = acc;
    C rv = r[s * n + i];
    cfma(rv, nal, acc);
    r[s * n + i] = rv;
  }
}

template <typename C>
__global__ void gcr_finish_kernel(C* __restrict__ x, MultiPtr Z, int K, const double2* __restrict__ alpha,
                                  const double2* __restrict__ gamma, const double2* __restrict__ beta,
                                  const int* __restrict__ nk, long long n, const int* run) {
  if (skip(run)) return;
  using R = typename RealOf<C>::R;
  const int s = blockIdx.y;
  __shared__ C yc[kMaxVecs];
  __shared__ int nks;
  if (threadIdx.x == 0) {
    const int m = nk[s];
    nks = m;
    double2 y[kMaxVecs];
    for (int j = K - 1; j >= 0; --j) {
      double2 v = make_double2(0, 0);
      if (j < m) {
        v = alpha[(size_t)s * K + j];
        for (int q = j + 1; q < m; ++q) {
          const double2 b = beta[((size_t)s * K + q) * K + j];
          v.x -= b.x * y[q].x - b.y * y[q].y;
          v.y -= b.x * y[q].y + b.y * y[q].x;
        }
        const double g = gamma[(size_t)s * K + j].x;
        v = g > 0 ? make_double2(v.x / g, v.y / g) : make_double2(0, 0);
      }
      y[j] = v;
      yc[j] = C{(R)v.x, (R)v.y};
    }
  }
  __syncthreads();
  const int m = nks;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    C acc = x[s * n + i];
    for (int j = 0; j < m; ++j) cfma(acc, yc[j], ((const C*)Z.p[j])[s * n + i]);
    x[s * n + i] = acc;
  }
}

unsigned grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// Multi-shift CG step for shift s (coef = [alpha | zeta | beta] per shift,
// real): x[s] += alpha[s] p[s] (skipped when alpha is 0), then
// p[s] = zeta[s] r + beta[s] p[s] with one base residual r for every shift.
__global__ void shift_update_kernel(double2* __restrict__ x, double2* __restrict__ p, const double2* __restrict__ r,
                                    const double* __restrict__ coef, int nshift, long long n) {
  const int s = blockIdx.y;
  const double a = coef[s], z = coef[nshift + s], b = coef[2 * nshift + s];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const size_t o = (size_t)s * n + i;
    const double2 pv = p[o];
    if (a != 0.0) {
      double2 xv = x[o];
      xv.x = fma(a, pv.x, xv.x);
      xv.y = fma(a, pv.y, xv.y);
      x[o] = xv;
    }
    const double2 rv = r[i];
    p[o] = make_double2(fma(z, rv.x, b * pv.x), fma(z, rv.y, b * pv.y));
  }
}

// ------------------------------------------------------------------- host API
void blas_copy(const Vec& dst, const Vec& src, cudaStream_t st, const int* run) {
  SMG_REQUIRE(dst.n == src.n && dst.nsys == src.nsys, "copy: shape mismatch");
  dim3 grid(grid_for(dst.n), dst.nsys);
  if (dst.prec == P64 && src.prec == P64)
    launch_k(copy_kernel<double2, double2>, dim3(grid), dim3(kThreads), 0, st, (double2*)dst.p, (const double2*)src.p, dst.n, dst.n, src.n, run);
  else if (dst.prec == P64)
    launch_k(copy_kernel<double2, float2>, dim3(grid), dim3(kThreads), 0, st, (double2*)dst.p, (const float2*)src.p, dst.n, dst.n, src.n, run);
  else if (src.prec == P64)
    launch_k(copy_kernel<float2, double2>, dim3(grid), dim3(kThreads), 0, st, (float2*)dst.p, (const double2*)src.p, dst.n, dst.n, src.n, run);
  else
    launch_k(copy_kernel<float2, float2>, dim3(grid), dim3(kThreads), 0, st, (float2*)dst.p, (const float2*)src.p, dst.n, dst.n, src.n, run);
  SMG_LAUNCH_OK();
}

void blas_zero(const Vec& x, cudaStream_t st, const int* run) {
  dim3 grid(grid_for(x.n), x.nsys);
  if (x.prec == P64) launch_k(zero_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, (double2*)x.p, x.n, run);
  else launch_k(zero_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, (float2*)x.p, x.n, run);
  SMG_LAUNCH_OK();
}

void blas_maxpy(const Vec& y, const Vec* xs, int nx, const double2* c, int ldc, double sign, bool accumulate,
                cudaStream_t st, const int* run) {
  SMG_REQUIRE(nx >= 0 && nx <= kMaxVecs, "maxpy: too many vectors");
  if (nx == 0 && accumulate) return;
  MultiPtr mp{};
  for (int j = 0; j < nx; ++j) {
    SMG_REQUIRE(xs[j].n == y.n && xs[j].nsys == y.nsys && xs[j].prec == y.prec, "maxpy: shape mismatch");
    mp.p[j] = xs[j].p;
  }
  dim3 grid(grid_for(y.n), y.nsys);
  if (y.prec == P64)
    launch_k(maxpy_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, (double2*)y.p, mp, nx, c, ldc, sign, accumulate ? 1 : 0, y.n, run);
  else
    launch_k(maxpy_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, (float2*)y.p, mp, nx, c, ldc, sign, accumulate ? 1 : 0, y.n, run);
  SMG_LAUNCH_OK();
}

void blas_scale(const Vec& x, const double2* c, bool inv_real, cudaStream_t st, const int* run) {
  dim3 grid(grid_for(x.n), x.nsys);
  if (x.prec == P64) launch_k(scale_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, (double2*)x.p, c, inv_real ? 1 : 0, x.n, run);
  else launch_k(scale_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, (float2*)x.p, c, inv_real ? 1 : 0, x.n, run);
  SMG_LAUNCH_OK();
}

void blas_sub(const Vec& z, const Vec& x, const Vec& y, cudaStream_t st, const int* run) {
  SMG_REQUIRE(z.n == x.n && x.n == y.n && z.prec == x.prec && x.prec == y.prec, "sub: shape mismatch");
  dim3 grid(grid_for(z.n), z.nsys);
  if (z.prec == P64)
    launch_k(sub_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, (double2*)z.p, (const double2*)x.p, (const double2*)y.p, z.n, run);
  else
    launch_k(sub_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, (float2*)z.p, (const float2*)x.p, (const float2*)y.p, z.n, run);
  SMG_LAUNCH_OK();
}

void blas_pair_dots(const Vec* vs, int nv, const int* pi, const int* pj, int np, double2* out, int ldo,
                    Workspace& ws, cudaStream_t st, const int* run, const Epilogue& epi) {
  SMG_REQUIRE(nv >= 1 && nv <= kMaxVecs && np >= 1 && np <= kMaxPairs, "pair_dots: bad sizes");
  PairDotArgs a{};
  a.nv = nv; a.npairs = np; a.n = vs[0].n;
  for (int v = 0; v < nv; ++v) {
    SMG_REQUIRE(vs[v].n == a.n && vs[v].prec == vs[0].prec && vs[v].nsys == vs[0].nsys, "pair_dots: mismatch");
    a.v.p[v] = vs[v].p;
  }
  for (int p = 0; p < np; ++p) { a.pi[p] = pi[p]; a.pj[p] = pj[p]; }
  const int nsys = vs[0].nsys;
  // two or more 128-row tiles per CTA, at most two CTAs per SM
  long long nb = (a.n + 2 * 128 - 1) / (2 * 128);
  if (nb > 2 * 152) nb = 2 * 152;
  if (nb < 1) nb = 1;
  double2* partial = (double2*)ws.get(sizeof(double2) * (size_t)nb * np * nsys);
  dim3 grid((unsigned)nb, nsys);
  if (vs[0].prec == P64)
    launch_k(pair_dot_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, a, partial, out, ldo, ws.counter, epi, run);
  else
    launch_k(pair_dot_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, a, partial, out, ldo, ws.counter, epi, run);
  SMG_LAUNCH_OK();
}

void blas_gcr_update(const Vec* W, int k, const double2* c, int ldc, const double2* ginv, const Vec& r,
                     const double2* na, cudaStream_t st, const int* run) {
  SMG_REQUIRE(k >= 0 && k < kMaxVecs, "gcr_update: bad k");
  MultiPtr mp{};
  for (int j = 0; j <= k; ++j) {
    SMG_REQUIRE(W[j].n == r.n && W[j].prec == r.prec && W[j].nsys == r.nsys, "gcr_update: mismatch");
    mp.p[j] = W[j].p;
  }
  dim3 grid(grid_for(r.n), r.nsys);
  if (r.prec == P64)
    launch_k(gcr_update_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, mp, k, c, ldc, ginv, (double2*)r.p, na, r.n, run);
  else
    launch_k(gcr_update_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, mp, k, c, ldc, ginv, (float2*)r.p, na, r.n, run);
  SMG_LAUNCH_OK();
}

void blas_gcr_finish(const Vec& x, const Vec* Z, int K, const double2* alpha, const double2* gamma,
                     const double2* beta, const int* nk, cudaStream_t st, const int* run) {
  SMG_REQUIRE(K >= 1 && K <= kMaxVecs, "gcr_finish: bad K");
  MultiPtr mp{};
  for (int j = 0; j < K; ++j) mp.p[j] = Z[j].p;
  dim3 grid(grid_for(x.n), x.nsys);
  if (x.prec == P64)
    launch_k(gcr_finish_kernel<double2>, dim3(grid), dim3(kThreads), 0, st, (double2*)x.p, mp, K, alpha, gamma, beta, nk, x.n, run);
  else
    launch_k(gcr_finish_kernel<float2>, dim3(grid), dim3(kThreads), 0, st, (float2*)x.p, mp, K, alpha, gamma, beta, nk, x.n, run);
  SMG_LAUNCH_OK();
}

void* Workspace::get(size_t bytes) {
  if (counter == nullptr) {
    SMG_CUDA_OK(cudaMalloc(&counter, sizeof(unsigned)));
    SMG_CUDA_OK(cudaMemset(counter, 0, sizeof(unsigned)));
    SMG_CUDA_OK(cudaDeviceSynchronize());
  }
  if (bytes > cap) {
    if (ptr) SMG_CUDA_OK(cudaFree(ptr));
    ptr = nullptr;
    size_t nb = bytes < (1u << 20) ? (1u << 20) : bytes;
    SMG_CUDA_OK(cudaMalloc(&ptr, nb));
    cap = nb;
  }
  return ptr;
}

Workspace::~Workspace() {
  if (ptr) cudaFree(ptr);
  if (counter) cudaFree(counter);
}

void blas_shift_update(const Vec& X, const Vec& P, const Vec& r, const double* coef, cudaStream_t st) {
  SMG_REQUIRE(X.prec == P64 && P.prec == P64 && r.prec == P64 && X.n == r.n && P.n == r.n && X.nsys == P.nsys &&
                  r.nsys == 1,
              "shift_update: FP64 batch with one base residual");
  dim3 grid(grid_for(r.n), X.nsys);
  launch_k(shift_update_kernel, grid, dim3(kThreads), 0, st, (double2*)X.p, (double2*)P.p, (const double2*)r.p, coef,
           X.nsys, r.n);
  SMG_LAUNCH_OK();
}

}  // namespace smg
