// Persistent coarse-level solver: the whole GCR solve of one coarse level
// (Sec. 2.1 "iterate on the coarser level linear system to some fixed
// tolerance"; Table 1: GCR to 0.25 or 8 iterations with CA-GCR(s)
// post-smoothing and an exact coarsest solve) in ONE cooperative launch.
//
// On one GPU the coarse levels are latency bound: a 256-site level holds
// 12k unknowns per vector, and launching each stencil apply, reduction and
// axpy separately costs more than the work.  Here every CTA of a grid that
// fills the GPU walks the same sequence of phases:
//   restrict -> dense coarsest solve -> prolong -> residual -> s smoother
//   applies -> Gram reduction -> correction -> operator apply -> two
//   Gram-Schmidt reductions -> update
// separated by grid barriers.  Reduction partials are written per CTA and
// every CTA adds them in the same order, so all CTAs hold bit-identical
// solver scalars in shared memory and no broadcast is needed.  Elementwise
// work uses the same contiguous per-CTA row ranges as the reductions, so it
// needs no grid barrier before the next reduction.
//
// Every barrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// sets an error word that the host reads, and returns.
#include "persist.cuh"
#include "stencil_row.cuh"

namespace smg {
namespace {

constexpr int PT = 512;          // threads per CTA
constexpr int TR = 64;           // rows per reduction tile
constexpr int kMaxP = 12;        // vectors per reduction

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier: arrival counter + generation word.  Returns false (and sets
// *err) when the wait exceeds the time limit.
__device__ bool grid_sync(unsigned* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else {
      const unsigned long long t0 = gtime();
      while (*gen == g) {
        if (*(volatile int*)err != 0 || gtime() - t0 > 2000000000ull) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ float2 ldh(const __half2* p, size_t i) { return __half22float2(p[i]); }
__device__ __forceinline__ float2 ldh(const float2* p, size_t i) { return p[i]; }

struct Shared {
  float2 tile[kMaxP][TR + 1];   // padded: the pairs of one row sit in different banks
  double2 red[PT];
  // per-system solver state (identical in every CTA)
  double2 alpha[kPersistMaxSys][kPersistMaxK];
  double2 gamma[kPersistMaxSys][kPersistMaxK];
  double2 beta[kPersistMaxSys][kPersistMaxK][kPersistMaxK];
  double2 sums[kPersistMaxSys][kMaxP + kPersistMaxK];
  double2 coef[kPersistMaxSys][16];
  double r2[kPersistMaxSys], thr2[kPersistMaxSys];
  int active[kPersistMaxSys], nk[kPersistMaxSys];
  int any;
  int xs[256];                  // aggregate sites (restriction)
};

// ------------------------------------------------------------------ phases
// This CTA's contiguous share [r0, r1) of a per-system vector of length n.
__device__ __forceinline__ void my_rows(long long n, long long& r0, long long& r1) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  r0 = blockIdx.x * per;
  r1 = min(n, r0 + per);
}

// out = A_hat in (or sub - A_hat in): one warp per (system, site, row)
template <typename SL>
__device__ void stencil_phase(const PersistArgs& a, float2* out, const float2* in, const float2* sub) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int N = a.N;
  const long long n = (long long)a.g.V * N;
  const long long rows = (long long)a.nsys * n;
  const SL* S = (const SL*)a.S;
  for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nw) {
    const int s = (int)(row / n);
    const long long rem = row - (long long)s * n;
    const int X = (int)(rem / N), i = (int)(rem % N);
    int c[4];
    a.g.coords(X, c);
    int nb[9];
    nb[0] = X;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      nb[1 + 2 * mu] = a.g.shift(c, mu, 1);
      nb[2 + 2 * mu] = a.g.shift(c, mu, -1);
    }
    const SL* sr = S + ((size_t)X * N + i) * 9 * N;
    const float2* vin = in + (size_t)s * n;
    float2 acc;
    if (N % 4 == 0) {
      acc = stencil_row_dot<SL>(sr, N, lane,
                                [&](int dir, int j) { return vin + (size_t)pick_site(nb, dir) * N + j; });
    } else {
      acc = make_float2(0.f, 0.f);
      for (int e = lane; e < 9 * N; e += 32) {
        const int dir = e / N, j = e - dir * N;
        cfma(acc, ldh(sr, e), vin[(size_t)pick_site(nb, dir) * N + j]);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      if (a.Srs != nullptr) acc = cscale(acc, a.Srs[(size_t)X * N + i]);
      const size_t oi = (size_t)s * n + rem;
      if (sub != nullptr) acc = csub(sub[oi], acc);
      out[oi] = acc;
    }
  }
}

// rc = R r : one CTA per (system, coarse site) at a time; thread t owns vector
// k = t % nvec and a strided set of the aggregate's rows (prolongator layout
// [site][dof][vector], so the nvec threads of a row read consecutive entries).
template <typename SL>
__device__ void restrict_phase(const PersistArgs& a, Shared& sh, float2* rc, const float2* r) {
  const TransferGeom& t = a.tg;
  const int nv = t.nvec, Nc = 2 * nv, half = t.ndof / 2;
  const int k = threadIdx.x % nv, grp = threadIdx.x / nv, groups = PT / nv;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int rows = npos * t.ndof;
  const long long nf = (long long)t.fine.V * t.ndof;
  const SL* P = (const SL*)a.P;
  double2* part = &sh.red[0];   // reused: [2][PT] FP32 pairs fit in PT double2
  float2* pf = reinterpret_cast<float2*>(part);
  int* xs = sh.xs;              // fine site of each aggregate position
  for (long long job = blockIdx.x; job < (long long)a.nsys * t.coarse.V; job += gridDim.x) {
    const int s = (int)(job / t.coarse.V), X = (int)(job % t.coarse.V);
    int Xc[4];
    t.coarse.coords(X, Xc);
    for (int p = threadIdx.x; p < npos; p += PT) {
      int q = p, cc[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) { cc[mu] = Xc[mu] * t.agg[mu] + q % t.agg[mu]; q /= t.agg[mu]; }
      xs[p] = t.fine.index(cc);
    }
    __syncthreads();
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    if (grp < groups) {
#pragma unroll 8
      for (int rr = grp; rr < rows; rr += groups) {
        const int p = rr / t.ndof, d = rr - p * t.ndof;
        const size_t row = (size_t)xs[p] * t.ndof + d;
        const float2 v = r[(size_t)s * nf + row];
        const float2 pv = ldh(P, row * nv + k);
        if (d < half) cfmac(acc0, pv, v);
        else cfmac(acc1, pv, v);
      }
    }
    __syncthreads();
    pf[threadIdx.x] = acc0;
    pf[PT + threadIdx.x] = acc1;
    __syncthreads();
    for (int i = threadIdx.x; i < Nc; i += PT) {
      const int chi = i / nv, kk = i % nv;
      float2 sum = make_float2(0.f, 0.f);
      for (int g = 0; g < groups; ++g) sum = cadd(sum, pf[chi * PT + g * nv + kk]);
      rc[(size_t)s * t.coarse.V * Nc + (size_t)X * Nc + i] = sum;
    }
    __syncthreads();
  }
}

// ec = D rc : one warp per (system, row) of the dense coarsest inverse
__device__ void dense_phase(const PersistArgs& a, float2* ec, const float2* rc) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int nd = a.nd;
  for (long long o = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < (long long)a.nsys * nd; o += nw) {
    const int s = (int)(o / nd), row = (int)(o % nd);
    const float2* Dr = a.D + (size_t)row * nd;
    const float2* v = rc + (size_t)s * nd;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = lane; j < nd; j += 32) cfma(acc, Dr[j], v[j]);
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) ec[o] = acc;
  }
}

// z = P ec : one thread per (system, site, component), contiguous prolongator run
template <typename SL>
__device__ void prolong_phase(const PersistArgs& a, float2* z, const float2* ec) {
  const TransferGeom& t = a.tg;
  const long long nf = (long long)t.fine.V * t.ndof;
  const int Nc = 2 * t.nvec, half = t.ndof / 2;
  const SL* P = (const SL*)a.P;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)a.nsys * nf;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / nf);
    const long long rem = e - (long long)s * nf;
    const int x = (int)(rem / t.ndof), d = (int)(rem % t.ndof);
    int c[4];
    t.fine.coords(x, c);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) c[mu] /= t.agg[mu];
    const int X = t.coarse.index(c);
    const int chi = d >= half ? 1 : 0;
    const float2* v = ec + (size_t)s * t.coarse.V * Nc + (size_t)X * Nc + chi * t.nvec;
    const SL* Px = P + (size_t)rem * t.nvec;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < t.nvec; ++k) cfma(acc, ldh(Px, k), v[k]);
    z[e] = acc;
  }
}

// Per-CTA partial sums of conj(v[pi[p]]) v[pj[p]] over this CTA's rows, for
// every system, accumulated in FP32 per thread and FP64 across threads;
// written to partial[cta][s][p].
__device__ void dots_partial(const PersistArgs& a, Shared& sh, float2* const* v, int nv, const int* pi,
                             const int* pj, int np) {
  const int t = threadIdx.x;
  const int groups = PT / np;
  const int p = t % np, grp = t / np;
  const bool act = grp < groups;
  const long long n = a.n;
  long long r0, r1;
  my_rows(n, r0, r1);
  for (int s = 0; s < a.nsys; ++s) {
    float2 acc = make_float2(0.f, 0.f);
    for (long long base = r0; base < r1; base += TR) {
      const int cnt = (int)min((long long)TR, r1 - base);
      for (int e = t; e < nv * TR; e += PT) {
        const int vi = e / TR, r = e % TR;
        float2 val = make_float2(0.f, 0.f);
        if (r < cnt) val = v[vi][(size_t)s * n + base + r];
        sh.tile[vi][r] = val;
      }
      __syncthreads();
      if (act)
        for (int r = grp; r < cnt; r += groups) cfmac(acc, sh.tile[pi[p]][r], sh.tile[pj[p]][r]);
      __syncthreads();
    }
    sh.red[t] = act ? make_double2(acc.x, acc.y) : make_double2(0, 0);
    __syncthreads();
    if (t < np) {
      double2 sum = make_double2(0, 0);
      for (int g = 0; g < groups; ++g) sum = cadd(sum, sh.red[g * np + t]);
      a.partial[((size_t)blockIdx.x * kPersistMaxSys + s) * 64 + t] = sum;
    }
    __syncthreads();
  }
}

// After a barrier: every CTA adds all CTAs' partials in the same order.
__device__ void dots_final(const PersistArgs& a, Shared& sh, int np) {
  for (int e = threadIdx.x; e < a.nsys * np; e += PT) {
    const int s = e / np, p = e % np;
    double2 sum = make_double2(0, 0);
    for (int b = 0; b < (int)gridDim.x; ++b)
      sum = cadd(sum, __ldcg(&a.partial[((size_t)b * kPersistMaxSys + s) * 64 + p]));
    sh.sums[s][p] = sum;
  }
  __syncthreads();
}

// CA-GCR normal equations (same algorithm as the launch-based path)
__device__ void ca_solve_sh(const double2* g, int s, double2* coef) {
  constexpr int MS = 10;
  double2 L[MS][MS], c[MS];
  double dsc[MS];
  bool drop[MS];
  int p = 0;
  for (int i = 0; i < s; ++i)
    for (int j = i; j < s; ++j) { L[j][i] = make_double2(g[p].x, -g[p].y); ++p; }
  for (int i = 0; i < s; ++i) c[i] = g[p++];
  for (int i = 0; i < s; ++i) dsc[i] = L[i][i].x > 0 ? 1.0 / sqrt(L[i][i].x) : 0.0;
  for (int i = 0; i < s; ++i) {
    c[i] = cscale(c[i], dsc[i]);
    for (int j = 0; j <= i; ++j) L[i][j] = cscale(L[i][j], dsc[i] * dsc[j]);
  }
  for (int j = 0; j < s; ++j) {
    double d = L[j][j].x;
    for (int k = 0; k < j; ++k) d -= L[j][k].x * L[j][k].x + L[j][k].y * L[j][k].y;
    drop[j] = !(d > 1e-12) || dsc[j] == 0.0;
    const double ljj = drop[j] ? 1.0 : sqrt(d);
    L[j][j] = make_double2(ljj, 0);
    for (int i = j + 1; i < s; ++i) {
      if (drop[j]) { L[i][j] = make_double2(0, 0); continue; }
      double2 v = L[i][j];
      for (int k = 0; k < j; ++k) {
        const double2 x = L[i][k], y = L[j][k];
        v.x -= x.x * y.x + x.y * y.y;
        v.y -= x.y * y.x - x.x * y.y;
      }
      L[i][j] = make_double2(v.x / ljj, v.y / ljj);
    }
  }
  for (int i = 0; i < s; ++i) {
    if (drop[i]) { c[i] = make_double2(0, 0); continue; }
    double2 v = c[i];
    for (int k = 0; k < i; ++k) { const double2 x = L[i][k], y = c[k]; v.x -= x.x * y.x - x.y * y.y; v.y -= x.x * y.y + x.y * y.x; }
    c[i] = make_double2(v.x / L[i][i].x, v.y / L[i][i].x);
  }
  for (int i = s - 1; i >= 0; --i) {
    if (drop[i]) { c[i] = make_double2(0, 0); continue; }
    double2 v = c[i];
    for (int k = i + 1; k < s; ++k) { const double2 l = L[k][i], b = c[k]; v.x -= l.x * b.x + l.y * b.y; v.y -= l.x * b.y - l.y * b.x; }
    c[i] = make_double2(v.x / L[i][i].x, v.y / L[i][i].x);
  }
  for (int i = 0; i < s; ++i) {
    const double2 v = cscale(c[i], dsc[i]);
    coef[i] = (isfinite(v.x) && isfinite(v.y)) ? v : make_double2(0, 0);
  }
}

// ------------------------------------------------------------------ kernel
template <typename SL>
__global__ void __launch_bounds__(PT, 1) persist_gcr_kernel(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Shared& sh = *reinterpret_cast<Shared*>(smem);
  if (a.run != nullptr && *a.run == 0) return;   // uniform across the grid
  const long long n = a.n;
  const int K = a.K, S = a.s, nsys = a.nsys;
  long long r0, r1;
  my_rows(n, r0, r1);
  const int t = threadIdx.x;
#define BARRIER() do { if (!grid_sync(a.bar, a.err)) return; } while (0)

  // r = b, x = 0 on this CTA's rows; |r|^2
  for (int s = 0; s < nsys; ++s)
    for (long long i = r0 + t; i < r1; i += PT) {
      a.r[(size_t)s * n + i] = a.b[(size_t)s * n + i];
      a.x[(size_t)s * n + i] = make_float2(0.f, 0.f);
    }
  __syncthreads();
  {
    float2* vv[1] = {a.r};
    const int pi[1] = {0}, pj[1] = {0};
    dots_partial(a, sh, vv, 1, pi, pj, 1);
  }
  BARRIER();
  dots_final(a, sh, 1);
  if (t == 0) {
    int any = 0;
    for (int s = 0; s < nsys; ++s) {
      const double b2 = sh.sums[s][0].x;
      sh.r2[s] = b2;
      sh.thr2[s] = a.tol2 * b2;
      sh.active[s] = b2 > sh.thr2[s] && b2 > 0.0;
      sh.nk[s] = 0;
      any |= sh.active[s];
    }
    sh.any = any;
  }
  __syncthreads();

  for (int k = 0; k < K && sh.any; ++k) {
    float2* zk = a.z[k];
    float2* wk = a.w[k];
    // ---- preconditioner z_k = K(r)
    if (a.has_pre) {
      restrict_phase<SL>(a, sh, a.rc, a.r);
      BARRIER();
      dense_phase(a, a.ec, a.rc);
      BARRIER();
      prolong_phase<SL>(a, zk, a.ec);
      BARRIER();
      stencil_phase<SL>(a, a.V[0], zk, a.r);          // V0 = r - A z
      BARRIER();
      for (int i = 1; i <= S; ++i) {
        stencil_phase<SL>(a, a.V[i], a.V[i - 1], nullptr);
        BARRIER();
      }
      {
        int pi[kMaxP * kMaxP], pj[kMaxP * kMaxP], np = 0;
        for (int i = 0; i < S; ++i)
          for (int j = i; j < S; ++j) { pi[np] = i + 1; pj[np] = j + 1; ++np; }
        for (int i = 0; i < S; ++i) { pi[np] = i + 1; pj[np] = 0; ++np; }
        dots_partial(a, sh, a.V, S + 1, pi, pj, np);
        BARRIER();
        dots_final(a, sh, np);
      }
      if (t < nsys) ca_solve_sh(sh.sums[t], S, sh.coef[t]);
      __syncthreads();
      for (int s = 0; s < nsys; ++s)
        for (long long i = r0 + t; i < r1; i += PT) {
          const size_t o = (size_t)s * n + i;
          float2 acc = zk[o];
          for (int q = 0; q < S; ++q) {
            const double2 cq = sh.coef[s][q];
            cfma(acc, make_float2((float)cq.x, (float)cq.y), a.V[q][o]);
          }
          zk[o] = acc;
        }
      BARRIER();
    } else {
      for (int s = 0; s < nsys; ++s)
        for (long long i = r0 + t; i < r1; i += PT) zk[(size_t)s * n + i] = a.r[(size_t)s * n + i];
      BARRIER();
    }
    // ---- w_k = A z_k
    stencil_phase<SL>(a, wk, zk, nullptr);
    BARRIER();
    // ---- classical Gram-Schmidt, pass 1
    if (k > 0) {
      int pi[kPersistMaxK], pj[kPersistMaxK];
      for (int j = 0; j < k; ++j) { pi[j] = j; pj[j] = k; }
      dots_partial(a, sh, a.w, k + 1, pi, pj, k);
      BARRIER();
      dots_final(a, sh, k);
      if (t < nsys)
        for (int j = 0; j < k; ++j) sh.beta[t][k][j] = sh.sums[t][j];
      __syncthreads();
      for (int s = 0; s < nsys; ++s)
        for (long long i = r0 + t; i < r1; i += PT) {
          const size_t o = (size_t)s * n + i;
          float2 acc = wk[o];
          for (int j = 0; j < k; ++j) {
            const double2 b = sh.beta[s][k][j];
            cfma(acc, make_float2((float)-b.x, (float)-b.y), a.w[j][o]);
          }
          wk[o] = acc;
        }
      __syncthreads();
    }
    // ---- pass 2 with |w_k|^2 and <w_k, r>
    {
      float2* vv[kPersistMaxK + 1];
      int pi[kPersistMaxK + 2], pj[kPersistMaxK + 2];
      for (int j = 0; j <= k; ++j) vv[j] = a.w[j];
      vv[k + 1] = a.r;
      for (int j = 0; j < k; ++j) { pi[j] = j; pj[j] = k; }
      pi[k] = k; pj[k] = k;
      pi[k + 1] = k; pj[k + 1] = k + 1;
      dots_partial(a, sh, vv, k + 2, pi, pj, k + 2);
      BARRIER();
      dots_final(a, sh, k + 2);
    }
    if (t < nsys) {
      const int s = t;
      double sumc = 0.0;
      for (int j = 0; j < k; ++j) {
        const double2 c2 = sh.sums[s][j];
        sh.beta[s][k][j] = cadd(sh.beta[s][k][j], c2);
        sumc += c2.x * c2.x + c2.y * c2.y;
      }
      const double ww = sh.sums[s][k].x - sumc;
      const double2 wr = sh.sums[s][k + 1];
      const double g = sqrt(fmax(ww, 0.0));
      const bool gfin = g > 0.0 && isfinite(g);
      const bool ok = sh.active[s] && gfin;
      const double2 al = ok ? make_double2(wr.x / g, wr.y / g) : make_double2(0, 0);
      sh.gamma[s][k] = make_double2(ok ? g : 0.0, 0);
      sh.alpha[s][k] = al;
      sh.coef[s][0] = make_double2(gfin ? 1.0 / g : 0.0, 0);   // 1/gamma for the update
      if (sh.active[s]) {
        sh.nk[s] = k + 1;
        const double r2 = sh.r2[s] - (al.x * al.x + al.y * al.y);
        sh.r2[s] = r2;
        if (!(r2 > sh.thr2[s]) || !gfin) sh.active[s] = 0;
      }
    }
    __syncthreads();
    if (t == 0) {
      int any = 0;
      for (int s = 0; s < nsys; ++s) any |= sh.active[s];
      sh.any = any;
    }
    // ---- w_k <- (w_k - sum c2_j w_j) / gamma ; r <- r - alpha w_k
    for (int s = 0; s < nsys; ++s) {
      const float gi = (float)sh.coef[s][0].x;
      const double2 al = sh.alpha[s][k];
      const float2 na = make_float2((float)-al.x, (float)-al.y);
      for (long long i = r0 + t; i < r1; i += PT) {
        const size_t o = (size_t)s * n + i;
        float2 acc = wk[o];
        for (int j = 0; j < k; ++j) {
          const double2 c2 = sh.sums[s][j];
          cfma(acc, make_float2((float)-c2.x, (float)-c2.y), a.w[j][o]);
        }
        acc = make_float2(acc.x * gi, acc.y * gi);
        wk[o] = acc;
        float2 rv = a.r[o];
        cfma(rv, na, acc);
        a.r[o] = rv;
      }
    }
    __syncthreads();
    BARRIER();
  }
  // ---- x = sum_k y_k z_k with gamma_j y_j + sum_{q>j} beta[q][j] y_q = alpha_j
  if (t < nsys) {
    const int s = t, m = sh.nk[s];
    for (int j = K - 1; j >= 0; --j) {
      double2 v = make_double2(0, 0);
      if (j < m) {
        v = sh.alpha[s][j];
        for (int q = j + 1; q < m; ++q) {
          const double2 b = sh.beta[s][q][j], y = sh.coef[s][q];
          v.x -= b.x * y.x - b.y * y.y;
          v.y -= b.x * y.y + b.y * y.x;
        }
        const double g = sh.gamma[s][j].x;
        v = g > 0 ? make_double2(v.x / g, v.y / g) : make_double2(0, 0);
      }
      sh.coef[s][j] = v;
    }
  }
  __syncthreads();
  for (int s = 0; s < nsys; ++s) {
    const int m = sh.nk[s];
    for (long long i = r0 + t; i < r1; i += PT) {
      const size_t o = (size_t)s * n + i;
      float2 acc = make_float2(0.f, 0.f);
      for (int q = 0; q < m; ++q) {
        const double2 y = sh.coef[s][q];
        cfma(acc, make_float2((float)y.x, (float)y.y), a.z[q][o]);
      }
      a.x[o] = acc;
    }
  }
#undef BARRIER
}

template <typename SL>
int occupancy_grid(int dev_sms) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist_gcr_kernel<SL>, PT, sizeof(Shared));
  return per >= 1 ? dev_sms : 0;
}

}  // namespace

size_t persist_smem_bytes() { return sizeof(Shared); }

bool persist_supported(int nsys, int K, int s, int N, Store st, int npos) {
  return (st == S16 || st == S32) && nsys >= 1 && nsys <= kPersistMaxSys && K >= 1 && K <= kPersistMaxK &&
         s >= 1 && s + 1 <= kMaxP && K + 2 <= kMaxP && N >= 2 && npos <= 256;
}

void persist_gcr(const PersistArgs& a, Store st, cudaStream_t stream) {
  static int sms = 0;
  static bool attr16 = false, attr32 = false;
  if (sms == 0) {
    int dev = 0;
    SMG_CUDA_OK(cudaGetDevice(&dev));
    SMG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const size_t smem = sizeof(Shared);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.blockDim = dim3(PT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (st == S16) {
    if (!attr16) {
      SMG_CUDA_OK(cudaFuncSetAttribute(persist_gcr_kernel<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
      attr16 = true;
    }
    const int g = occupancy_grid<__half2>(sms);
    SMG_REQUIRE(g > 0, "persistent coarse solver does not fit on an SM");
    cfg.gridDim = dim3(g);
    SMG_CUDA_OK(cudaLaunchKernelEx(&cfg, persist_gcr_kernel<__half2>, a));
  } else {
    if (!attr32) {
      SMG_CUDA_OK(cudaFuncSetAttribute(persist_gcr_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
      attr32 = true;
    }
    const int g = occupancy_grid<float2>(sms);
    SMG_REQUIRE(g > 0, "persistent coarse solver does not fit on an SM");
    cfg.gridDim = dim3(g);
    SMG_CUDA_OK(cudaLaunchKernelEx(&cfg, persist_gcr_kernel<float2>, a));
  }
  SMG_LAUNCH_OK();
}

int persist_grid_size() {
  int dev = 0, sms = 0;
  SMG_CUDA_OK(cudaGetDevice(&dev));
  SMG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

}  // namespace smg
