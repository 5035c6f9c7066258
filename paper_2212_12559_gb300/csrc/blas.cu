// Batched BLAS-1 kernels and reductions for the Krylov solvers.
//
// Every kernel works on nsys systems at once (blockIdx.y = system) and takes
// its coefficients from device memory, one per system, so that whole solver
// iterations run without a host round trip.  Each kernel also takes an
// optional `run` flag: when it points at 0 the kernel returns at once, which
// lets a fixed launch sequence (and a CUDA graph of it) stop early once an
// inner solve has converged.
//
// Reductions accumulate in FP64 whatever the vector precision and are
// deterministic: per-CTA partial sums, then one finishing pass.
#include "blas.cuh"

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
// partial[s][block][p] = sum over this CTA's rows of conj(v[pi[p]]) * v[pj[p]]
template <typename C>
__global__ void __launch_bounds__(kThreads) pair_dot_kernel(PairDotArgs a, double2* __restrict__ partial,
                                                            const int* run) {
  if (skip(run)) return;
  constexpr int TR = 128;   // rows per tile
  __shared__ double2 tile[kMaxVecs][TR];
  __shared__ double2 red[kThreads];
  const int s = blockIdx.y;
  const int np = a.npairs;
  const int groups = kThreads / np;               // row groups per pair
  const int t = threadIdx.x;
  const int p = t % np;
  const int grp = t / np;
  const bool active = grp < groups;
  double2 acc = make_double2(0, 0);
  const long long n = a.n;
  const long long rows_per_block = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * rows_per_block;
  const long long r1 = min(n, r0 + rows_per_block);
  for (long long base = r0; base < r1; base += TR) {
    const int cnt = (int)min((long long)TR, r1 - base);
    for (int e = t; e < a.nv * TR; e += kThreads) {
      const int v = e / TR, r = e % TR;
      double2 val = make_double2(0, 0);
      if (r < cnt) val = to_d(((const C*)a.v.p[v])[s * n + base + r]);
      tile[v][r] = val;
    }
    __syncthreads();
    if (active) {
      const int vi = a.pi[p], vj = a.pj[p];
      for (int r = grp; r < cnt; r += groups) cfmac(acc, tile[vi][r], tile[vj][r]);
    }
    __syncthreads();
  }
  red[t] = active ? acc : make_double2(0, 0);
  __syncthreads();
  if (t < np) {
    double2 sum = make_double2(0, 0);
    for (int g = 0; g < groups; ++g) sum = cadd(sum, red[g * np + t]);
    partial[((long long)s * gridDim.x + blockIdx.x) * np + t] = sum;
  }
}

__global__ void pair_dot_finish(const double2* __restrict__ partial, int nblocks, int np, double2* __restrict__ out,
                                int ldo, const int* run) {
  if (skip(run)) return;
  const int s = blockIdx.x;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    double2 sum = make_double2(0, 0);
    for (int b = 0; b < nblocks; ++b) sum = cadd(sum, partial[((long long)s * nblocks + b) * np + p]);
    out[(long long)s * ldo + p] = sum;
  }
}

unsigned grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// ------------------------------------------------------------------- host API
void blas_copy(const Vec& dst, const Vec& src, cudaStream_t st, const int* run) {
  SMG_REQUIRE(dst.n == src.n && dst.nsys == src.nsys, "copy: shape mismatch");
  dim3 grid(grid_for(dst.n), dst.nsys);
  if (dst.prec == P64 && src.prec == P64)
    copy_kernel<<<grid, kThreads, 0, st>>>((double2*)dst.p, (const double2*)src.p, dst.n, dst.n, src.n, run);
  else if (dst.prec == P64)
    copy_kernel<<<grid, kThreads, 0, st>>>((double2*)dst.p, (const float2*)src.p, dst.n, dst.n, src.n, run);
  else if (src.prec == P64)
    copy_kernel<<<grid, kThreads, 0, st>>>((float2*)dst.p, (const double2*)src.p, dst.n, dst.n, src.n, run);
  else
    copy_kernel<<<grid, kThreads, 0, st>>>((float2*)dst.p, (const float2*)src.p, dst.n, dst.n, src.n, run);
  SMG_LAUNCH_OK();
}

void blas_zero(const Vec& x, cudaStream_t st, const int* run) {
  dim3 grid(grid_for(x.n), x.nsys);
  if (x.prec == P64) zero_kernel<<<grid, kThreads, 0, st>>>((double2*)x.p, x.n, run);
  else zero_kernel<<<grid, kThreads, 0, st>>>((float2*)x.p, x.n, run);
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
    maxpy_kernel<<<grid, kThreads, 0, st>>>((double2*)y.p, mp, nx, c, ldc, sign, accumulate ? 1 : 0, y.n, run);
  else
    maxpy_kernel<<<grid, kThreads, 0, st>>>((float2*)y.p, mp, nx, c, ldc, sign, accumulate ? 1 : 0, y.n, run);
  SMG_LAUNCH_OK();
}

void blas_scale(const Vec& x, const double2* c, bool inv_real, cudaStream_t st, const int* run) {
  dim3 grid(grid_for(x.n), x.nsys);
  if (x.prec == P64) scale_kernel<<<grid, kThreads, 0, st>>>((double2*)x.p, c, inv_real ? 1 : 0, x.n, run);
  else scale_kernel<<<grid, kThreads, 0, st>>>((float2*)x.p, c, inv_real ? 1 : 0, x.n, run);
  SMG_LAUNCH_OK();
}

void blas_sub(const Vec& z, const Vec& x, const Vec& y, cudaStream_t st, const int* run) {
  SMG_REQUIRE(z.n == x.n && x.n == y.n && z.prec == x.prec && x.prec == y.prec, "sub: shape mismatch");
  dim3 grid(grid_for(z.n), z.nsys);
  if (z.prec == P64)
    sub_kernel<<<grid, kThreads, 0, st>>>((double2*)z.p, (const double2*)x.p, (const double2*)y.p, z.n, run);
  else
    sub_kernel<<<grid, kThreads, 0, st>>>((float2*)z.p, (const float2*)x.p, (const float2*)y.p, z.n, run);
  SMG_LAUNCH_OK();
}

void blas_pair_dots(const Vec* vs, int nv, const int* pi, const int* pj, int np, double2* out, int ldo,
                    Workspace& ws, cudaStream_t st, const int* run) {
  SMG_REQUIRE(nv >= 1 && nv <= kMaxVecs && np >= 1 && np <= kMaxPairs, "pair_dots: bad sizes");
  PairDotArgs a{};
  a.nv = nv; a.npairs = np; a.n = vs[0].n;
  for (int v = 0; v < nv; ++v) {
    SMG_REQUIRE(vs[v].n == a.n && vs[v].prec == vs[0].prec && vs[v].nsys == vs[0].nsys, "pair_dots: mismatch");
    a.v.p[v] = vs[v].p;
  }
  for (int p = 0; p < np; ++p) { a.pi[p] = pi[p]; a.pj[p] = pj[p]; }
  const int nsys = vs[0].nsys;
  long long nb = (a.n + 4 * 128 - 1) / (4 * 128);
  if (nb > 152 * 4) nb = 152 * 4;
  if (nb < 1) nb = 1;
  double2* partial = (double2*)ws.get(sizeof(double2) * (size_t)nb * np * nsys);
  dim3 grid((unsigned)nb, nsys);
  if (vs[0].prec == P64) pair_dot_kernel<double2><<<grid, kThreads, 0, st>>>(a, partial, run);
  else pair_dot_kernel<float2><<<grid, kThreads, 0, st>>>(a, partial, run);
  SMG_LAUNCH_OK();
  pair_dot_finish<<<nsys, 64, 0, st>>>(partial, (int)nb, np, out, ldo, run);
  SMG_LAUNCH_OK();
}

void* Workspace::get(size_t bytes) {
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
}

}  // namespace smg
