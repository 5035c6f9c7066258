// Persistent coarse-level solver: the whole GCR solve of one coarse level
// (Sec. 2.1: the coarse system is iterated to a fixed tolerance; Table 1:
// GCR to 0.25 or 8 iterations with CA-GCR(s) post-smoothing and an exact
// coarsest solve) in ONE cooperative launch.
//
// On one GPU the coarse levels are latency bound: a 256-site level holds 12k
// unknowns per vector, and launching each stencil apply, reduction and axpy
// separately costs more than the work.  Here every CTA of a grid of one CTA
// per SM owns the same contiguous range of rows [c*per, (c+1)*per) of every
// vector, and all CTAs walk the same sequence of phases separated by grid
// barriers.  Per GCR iteration k (with the K-cycle preconditioner):
//
//   assemble R r from the CTAs' partial restrictions | dense coarsest solve |
//   prolong z = P e (own rows) | V0 = r - A z | V_i = A V_{i-1}, i = 1..s,
//   with the smoother's Gram partials after V_s | smoother correction
//   z += sum c_q V_q and w = A z = r - V0 + sum c_q V_{q+1} (no apply) |
//   Gram-Schmidt pass 1 | pass 2 | update w, r and the partial restriction of
//   the new r (own rows).
//
// Reduction partials are written per CTA and every CTA adds them in the same
// order, so all CTAs hold bit-identical solver scalars in shared memory and
// no broadcast is needed.  Elementwise work and reduction partials use the
// CTA's own rows, so they need no barrier between them.
//
// Resident mode (when it fits): the CTA's rows of the stencil (FP16 with row
// scales, or FP32) and of the prolongator are copied into shared memory once
// per launch; a stencil apply then stages the neighbour entries of its input
// in shared memory (one round trip to L2) and reads everything else on chip.
// Otherwise the stencil rows stream from global memory, each row once for all
// systems of the batch.
//
// Grid barriers use one 64-bit arrival counter that only grows during a
// launch (barrier b completes when it reaches b * gridDim); the last CTA to
// exit clears it.  Every wait is bounded (2 s of %globaltimer by default); on
// expiry the kernel sets an error word that the host reads, and returns.
#include "ca_solve.cuh"
#include "persist.cuh"
#include "stencil_row.cuh"

#include <algorithm>

namespace smg {
namespace {

constexpr int PT = 512;          // threads per CTA
constexpr int NW = PT / 32;      // warps per CTA
constexpr int TR = 64;           // rows per reduction tile
constexpr int kMaxP = 12;        // vectors per reduction
constexpr int kCaWarps = 8;      // warps that solve the smoother's normal equations

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ float2 ldh(const __half2* p, size_t i) { return __half22float2(p[i]); }
__device__ __forceinline__ float2 ldh(const float2* p, size_t i) { return p[i]; }

// Solver scalars of this level are FP32: the level's GCR only has to reduce
// its residual by a fixed factor (0.25) and its inner products come from FP32
// vectors; GB300's FP64 pipe is a small fraction of its FP32 rate, and these
// scalars sit on the critical path of every phase.
struct Shared {
  union {
    struct {
      float2 tile[kMaxP][TR + 1];   // padded: the pairs of one row sit in different banks
      float2 red[PT];
    } d;
    float2 ca[kCaWarps][kCaMaxS][kCaMaxS];   // CA-GCR factor scratch, one per warp
  } u;
  // per-system solver state (identical in every CTA)
  float2 alpha[kPersistMaxSys][kPersistMaxK];
  float2 gamma[kPersistMaxSys][kPersistMaxK];
  float2 beta[kPersistMaxSys][kPersistMaxK][kPersistMaxK];
  float2 sums[kPersistMaxSys][kPersistSums];
  float2 coef[kPersistMaxSys][16];
  float r2[kPersistMaxSys], thr2[kPersistMaxSys];
  int active[kPersistMaxSys], nk[kPersistMaxSys];
  int any;
  int ok;
  int nbt[kPersistMaxTouch][9];   // neighbour sites of the touched sites (resident mode)
  unsigned long long mbar;        // completion of the resident-data bulk copy
};

// This CTA's rows and the lattice sites they touch.
struct Own {
  int r0, r1;   // every index of a level fits in 32 bits (checked by persist_supported)
  int xs0, nts;
};

__device__ __forceinline__ Own own_rows(const PersistArgs& a) {
  Own o;
  const int per = (int)a.plan.per, n = (int)a.n;
  o.r0 = min(n, (int)blockIdx.x * per);
  o.r1 = min(n, o.r0 + per);
  o.xs0 = o.r0 / a.N;
  o.nts = o.r1 > o.r0 ? (o.r1 - 1) / a.N - o.xs0 + 1 : 0;
  return o;
}

// Optional phase trace (CTA 0, thread 0): (phase id, %globaltimer) pairs
// after trace[0] = count; the host turns consecutive marks into durations.
__device__ __forceinline__ void trace_mark(const PersistArgs& a, int id) {
  if (a.trace == nullptr || blockIdx.x != 0) return;
  const unsigned long long i = a.trace[0];
  if (i < (unsigned long long)a.trace_cap) {
    a.trace[1 + 2 * i] = (unsigned long long)id;
    a.trace[2 + 2 * i] = gtime();
  }
  a.trace[0] = i + 1;
}

// Grid barrier.  `target` (thread 0's copy) counts the arrivals expected so
// far.  Returns false (and sets *err) when the wait exceeds the time limit or
// another CTA already gave up.  `id` names the phase it ends (trace only).
__device__ bool grid_sync(const PersistArgs& a, Shared& sh, unsigned long long& target, int id) {
  __syncthreads();
  if (threadIdx.x == 0) {
    sh.ok = 1;
    target += gridDim.x;
    __threadfence();
    atomicAdd(a.bar, 1ull);
    const unsigned long long t0 = gtime();
    while (ld_acquire(a.bar) < target + (unsigned long long)a.bar_extra) {
      if (*(volatile int*)a.err != 0 || gtime() - t0 > a.bar_limit_ns) {
        atomicExch(a.err, 1);
        sh.ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    trace_mark(a, id);
  }
  __syncthreads();
  return sh.ok != 0;
}

// acc += S chunk (C entries) . v[0..C)
__device__ __forceinline__ void fma_chunk(float2& acc, const uint4& raw, const __half2*, const float2* v) {
  const __half2* h = reinterpret_cast<const __half2*>(&raw);
  const float4 v01 = *reinterpret_cast<const float4*>(v);
  const float4 v23 = *reinterpret_cast<const float4*>(v + 2);
  cfma(acc, __half22float2(h[0]), make_float2(v01.x, v01.y));
  cfma(acc, __half22float2(h[1]), make_float2(v01.z, v01.w));
  cfma(acc, __half22float2(h[2]), make_float2(v23.x, v23.y));
  cfma(acc, __half22float2(h[3]), make_float2(v23.z, v23.w));
}
__device__ __forceinline__ void fma_chunk(float2& acc, const uint4& raw, const float2*, const float2* v) {
  const float2* f = reinterpret_cast<const float2*>(&raw);
  const float4 v01 = *reinterpret_cast<const float4*>(v);
  cfma(acc, f[0], make_float2(v01.x, v01.y));
  cfma(acc, f[1], make_float2(v01.z, v01.w));
}

__device__ __forceinline__ float2 warp_sum(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// ------------------------------------------------------------------ phases
// The own rows of one staging round of ns <= NS systems (NS a compile-time
// bound, so the per-system accumulators stay in registers without issuing
// work for systems that are not there).
template <typename SL, int NS>
__device__ __forceinline__ void resident_rows(const PersistArgs& a, const Own& o, const SL* Sres, const float* Ssc,
                                              const float2* stg, float2* out, const float2* sub, int s0, int ns,
                                              int warp, int lane) {
  constexpr int C = Chunk<SL>::C;
  const int N = a.N, W = 9 * N, nq = W / C;
  for (int row = o.r0 + warp; row < o.r1; row += NW) {
    const int x = row / N, xl = x - o.xs0;
    const SL* sr = Sres + (size_t)(row - o.r0) * W;
    float2 acc[NS];
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) acc[sl] = make_float2(0.f, 0.f);
    for (int q = lane; q < nq; q += 32) {
      const int e = q * C;
      const uint4 raw = *reinterpret_cast<const uint4*>(sr + e);
#pragma unroll
      for (int sl = 0; sl < NS; ++sl)
        if (NS == 1 || sl < ns) fma_chunk(acc[sl], raw, sr, stg + ((size_t)sl * o.nts + xl) * W + e);
    }
    const float sc = a.Srs != nullptr ? Ssc[row - o.r0] : 1.0f;
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      if (NS > 1 && sl >= ns) break;
      float2 v = warp_sum(acc[sl]);
      if (lane == 0) {
        v = make_float2(v.x * sc, v.y * sc);
        const size_t oi = (size_t)(s0 + sl) * a.n + row;
        if (sub != nullptr) v = csub(sub[oi], v);
        out[oi] = v;
      }
    }
  }
}

// One system, up to RW rows per warp at once (rows warp, warp + NW, ...):
// the rows' loads and FMA chains interleave and their shuffle trees run side
// by side, instead of one row's latency after another.
template <typename SL, int RW>
__device__ __forceinline__ void resident_rows_multi(const PersistArgs& a, const Own& o, const SL* Sres,
                                                    const float* Ssc, const float2* stg, float2* out,
                                                    const float2* sub, int s0, int warp, int lane) {
  constexpr int C = Chunk<SL>::C;
  const int N = a.N, W = 9 * N, nq = W / C;
  const int nrows = o.r1 - o.r0;
  for (int base = warp; base < nrows; base += NW * RW) {
    int xl[RW];
    float2 acc[RW];
#pragma unroll
    for (int u = 0; u < RW; ++u) {
      const int lr = base + u * NW;
      xl[u] = lr < nrows ? (o.r0 + lr) / N - o.xs0 : 0;
      acc[u] = make_float2(0.f, 0.f);
    }
    for (int q = lane; q < nq; q += 32) {
      const int e = q * C;
#pragma unroll
      for (int u = 0; u < RW; ++u) {
        const int lr = base + u * NW;
        if (lr < nrows) {
          const uint4 raw = *reinterpret_cast<const uint4*>(Sres + (size_t)lr * W + e);
          fma_chunk(acc[u], raw, Sres, stg + (size_t)xl[u] * W + e);
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int u = 0; u < RW; ++u) {
        acc[u].x += __shfl_xor_sync(0xffffffffu, acc[u].x, off);
        acc[u].y += __shfl_xor_sync(0xffffffffu, acc[u].y, off);
      }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < RW; ++u) {
        const int lr = base + u * NW;
        if (lr < nrows) {
          const float sc = a.Srs != nullptr ? Ssc[lr] : 1.0f;
          float2 v = make_float2(acc[u].x * sc, acc[u].y * sc);
          const size_t oi = (size_t)s0 * a.n + o.r0 + lr;
          if (sub != nullptr) v = csub(sub[oi], v);
          out[oi] = v;
        }
      }
    }
  }
}

// out = A_hat in (or sub - A_hat in) on the CTA's own rows, stencil rows in
// shared memory.  Inputs of the touched sites' nine neighbours are staged in
// shared memory in the stencil's own [dir][col] order, so a row is one
// contiguous dot product of 9N entries.  N is a multiple of 4.
template <typename SL>
__device__ void stencil_resident(const PersistArgs& a, Shared& sh, const Own& o, unsigned char* smem,
                                 float2* out, const float2* in, const float2* sub) {
  const int N = a.N, W = 9 * N;
  const SL* Sres = reinterpret_cast<const SL*>(smem + a.plan.off_S);
  const float* Ssc = reinterpret_cast<const float*>(smem + a.plan.off_sc);
  float2* stg = reinterpret_cast<float2*>(smem + a.plan.off_stg);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int per_sys = o.nts * W;
  for (int s0 = 0; s0 < a.nsys; s0 += a.plan.sg) {
    const int ns = min(a.plan.sg, a.nsys - s0);
    for (int e = 2 * t; e < ns * per_sys; e += 2 * PT) {
      const int sl = e / per_sys, rem = e - sl * per_sys;
      const int xl = rem / W, rr = rem - xl * W;
      const int dir = rr / N, j = rr - dir * N;
      const float2* src = in + (size_t)(s0 + sl) * a.n + (size_t)sh.nbt[xl][dir] * N + j;
      *reinterpret_cast<float4*>(stg + e) = *reinterpret_cast<const float4*>(src);
    }
    __syncthreads();
    if (t == 0) trace_mark(a, 13);
    if (ns == 1) resident_rows_multi<SL, 6>(a, o, Sres, Ssc, stg, out, sub, s0, warp, lane);
    else if (ns == 2) resident_rows<SL, 2>(a, o, Sres, Ssc, stg, out, sub, s0, ns, warp, lane);
    else if (ns <= 4) resident_rows<SL, 4>(a, o, Sres, Ssc, stg, out, sub, s0, ns, warp, lane);
    else if (ns <= 8) resident_rows<SL, 8>(a, o, Sres, Ssc, stg, out, sub, s0, ns, warp, lane);
    else resident_rows<SL, kPersistMaxSys>(a, o, Sres, Ssc, stg, out, sub, s0, ns, warp, lane);
    __syncthreads();
    if (t == 0) trace_mark(a, 14);
  }
}

// The same from global memory: each stencil row is read once for all systems.
template <typename SL, int NS>
__device__ void stencil_stream_ns(const PersistArgs& a, const Own& o, float2* out, const float2* in,
                                  const float2* sub) {
  constexpr int C = Chunk<SL>::C;
  const int N = a.N, W = 9 * N, ns = a.nsys;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SL* S = reinterpret_cast<const SL*>(a.S);
  for (int row = o.r0 + warp; row < o.r1; row += NW) {
    const int X = row / N;
    int c[4];
    a.g.coords(X, c);
    int nb[9];
    nb[0] = X;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      nb[1 + 2 * mu] = a.g.shift(c, mu, 1);
      nb[2 + 2 * mu] = a.g.shift(c, mu, -1);
    }
    const SL* sr = S + (size_t)row * W;
    float2 acc[NS];
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) acc[sl] = make_float2(0.f, 0.f);
    if (N % 4 == 0) {
      for (int q = lane; q < W / C; q += 32) {
        const int e = q * C;
        const int dir = e / N, j = e - dir * N;
        const size_t off = (size_t)pick_site(nb, dir) * N + j;
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(sr + e));
#pragma unroll
        for (int sl = 0; sl < NS; ++sl)
          if (NS == 1 || sl < ns) fma_chunk(acc[sl], raw, sr, in + (size_t)sl * a.n + off);
      }
    } else {
      for (int e = lane; e < W; e += 32) {
        const int dir = e / N, j = e - dir * N;
        const size_t off = (size_t)pick_site(nb, dir) * N + j;
        const float2 sv = ldh(sr, e);
#pragma unroll
        for (int sl = 0; sl < NS; ++sl)
          if (NS == 1 || sl < ns) cfma(acc[sl], sv, in[(size_t)sl * a.n + off]);
      }
    }
    const float sc = a.Srs != nullptr ? a.Srs[row] : 1.0f;
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      if (NS > 1 && sl >= ns) break;
      float2 v = warp_sum(acc[sl]);
      if (lane == 0) {
        v = make_float2(v.x * sc, v.y * sc);
        const size_t oi = (size_t)sl * a.n + row;
        if (sub != nullptr) v = csub(sub[oi], v);
        out[oi] = v;
      }
    }
  }
  __syncthreads();
}

template <typename SL>
__device__ void stencil_stream(const PersistArgs& a, const Own& o, float2* out, const float2* in,
                               const float2* sub) {
  const int ns = a.nsys;
  if (ns == 1) stencil_stream_ns<SL, 1>(a, o, out, in, sub);
  else if (ns == 2) stencil_stream_ns<SL, 2>(a, o, out, in, sub);
  else if (ns <= 4) stencil_stream_ns<SL, 4>(a, o, out, in, sub);
  else if (ns <= 8) stencil_stream_ns<SL, 8>(a, o, out, in, sub);
  else stencil_stream_ns<SL, kPersistMaxSys>(a, o, out, in, sub);
}

template <typename SL>
__device__ __forceinline__ void stencil_phase(const PersistArgs& a, Shared& sh, const Own& o, unsigned char* smem,
                                              float2* out, const float2* in, const float2* sub) {
  if (a.plan.resident) stencil_resident<SL>(a, sh, o, smem, out, in, sub);
  else stencil_stream<SL>(a, o, out, in, sub);
}

// Prolongator row `row` of this level (resident copy or global).
template <typename SL>
__device__ __forceinline__ const SL* prolongator_row(const PersistArgs& a, const Own& o, unsigned char* smem,
                                                     int row) {
  const int nv = a.tg.nvec;
  if (a.plan.resident) return reinterpret_cast<const SL*>(smem + a.plan.off_P) + (size_t)(row - o.r0) * nv;
  return reinterpret_cast<const SL*>(a.P) + (size_t)row * nv;
}

// rpart[c][xl][s][i] = sum over this CTA's rows of touched site xs0 + xl of
// conj(P[row][k]) r[s][row], i = chi * nvec + k, chirality chi = (d >= N/2).
template <typename SL>
__device__ void restrict_partial(const PersistArgs& a, const Own& o, unsigned char* smem, const float2* r) {
  const int N = a.N, nv = a.tg.nvec, Nc = 2 * nv, half = N / 2;
  const int total = a.nsys * o.nts * Nc;
  for (int e = threadIdx.x; e < total; e += PT) {
    const int s = e / (o.nts * Nc), rem = e - s * (o.nts * Nc);
    const int xl = rem / Nc, i = rem - xl * Nc;
    const int chi = i / nv, k = i - chi * nv;
    const int x0 = (o.xs0 + xl) * N;
    const int lo = max(o.r0, x0 + chi * half), hi = min(o.r1, x0 + chi * half + half);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int row = lo; row < hi; ++row)
      cfmac(acc, ldh(prolongator_row<SL>(a, o, smem, row), k), r[(size_t)s * a.n + row]);
    a.rpart[(((size_t)blockIdx.x * a.plan.nslot + xl) * kPersistMaxSys + s) * Nc + i] = acc;
  }
}

// rc = R r: each entry adds the partials of the CTAs that own rows of the
// aggregate's sites.  P2 lanes (a power of two <= 32) share one entry, each
// taking every P2-th aggregate position, then a fixed shuffle tree.
__device__ void assemble_rc(const PersistArgs& a, float2* rc) {
  const TransferGeom& t = a.tg;
  const int N = a.N, Nc = 2 * t.nvec;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  int P2 = 1;
  while (P2 < npos && P2 < 32) P2 <<= 1;
  const int per = (int)a.plan.per;
  const int outs = a.nsys * t.coarse.V * Nc;
  const int nwarp_work = (outs * P2 + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (PT / 32);
  for (int w = blockIdx.x * (PT / 32) + (threadIdx.x >> 5); w < nwarp_work; w += nw) {
    const int e = w * 32 + lane;
    const int o = e / P2;
    const int sub = e % P2;
    float2 sum = make_float2(0.f, 0.f);
    if (o < outs) {
      const int s = o / (t.coarse.V * Nc);
      const int rem = o - s * t.coarse.V * Nc;
      const int X = rem / Nc, i = rem - X * Nc;
      int Xc[4];
      t.coarse.coords(X, Xc);
      for (int p = sub; p < npos; p += P2) {
        int q = p, cc[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) { cc[mu] = Xc[mu] * t.agg[mu] + q % t.agg[mu]; q /= t.agg[mu]; }
        const int x = t.fine.index(cc);
        const int c_lo = x * N / per, c_hi = (x * N + N - 1) / per;
        for (int c = c_lo; c <= c_hi; ++c) {
          const int slot = x - c * per / N;
          sum = cadd(sum, a.rpart[(((size_t)c * a.plan.nslot + slot) * kPersistMaxSys + s) * Nc + i]);
        }
      }
    }
    for (int off = P2 / 2; off > 0; off >>= 1) {
      sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
      sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
    }
    if (o < outs && sub == 0) rc[o] = sum;
  }
}

// ec = D rc : one warp per (system, row) of the dense coarsest inverse
__device__ void dense_phase(const PersistArgs& a, float2* ec, const float2* rc) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nd = a.nd;
  for (int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < a.nsys * nd; o += nw) {
    const int s = o / nd, row = o - s * nd;
    const float2* Dr = a.D + (size_t)row * nd;
    const float2* v = rc + (size_t)s * nd;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = lane; j < nd; j += 32) cfma(acc, Dr[j], v[j]);
    acc = warp_sum(acc);
    if (lane == 0) ec[o] = acc;
  }
}

// z = P ec on the CTA's own rows, one thread per (system, row)
template <typename SL>
__device__ void prolong_own(const PersistArgs& a, const Own& o, unsigned char* smem, float2* z, const float2* ec) {
  const TransferGeom& t = a.tg;
  const int N = a.N, nv = t.nvec, Nc = 2 * nv, half = N / 2;
  const int rows = o.r1 - o.r0;
  for (int e = threadIdx.x; e < a.nsys * rows; e += PT) {
    const int s = e / rows;
    const int row = o.r0 + (e - s * rows);
    const int x = row / N, d = row - x * N;
    int c[4];
    t.fine.coords(x, c);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) c[mu] /= t.agg[mu];
    const int chi = d >= half ? 1 : 0;
    const float2* v = ec + (size_t)s * t.coarse.V * Nc + (size_t)t.coarse.index(c) * Nc + chi * nv;
    const SL* Pr = prolongator_row<SL>(a, o, smem, row);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int k = 0; k < nv; ++k) cfma(acc, ldh(Pr, k), v[k]);
    z[(size_t)s * a.n + row] = acc;
  }
}

// Per-CTA partial sums of conj(v[pi[p]]) v[pj[p]] over the CTA's own rows,
// for every system (FP32); written to partial[cta][s][p].
__device__ void dots_partial(const PersistArgs& a, Shared& sh, const Own& o, float2* const* v, int nv,
                             const int* pi, const int* pj, int np) {
  const int t = threadIdx.x;
  const int groups = PT / np;
  const int p = t % np, grp = t / np;
  const bool act = grp < groups;
  const long long n = a.n;
  for (int s = 0; s < a.nsys; ++s) {
    float2 acc = make_float2(0.f, 0.f);
    for (int base = o.r0; base < o.r1; base += TR) {
      const int cnt = min(TR, o.r1 - base);
      for (int e = t; e < nv * TR; e += PT) {
        const int vi = e / TR, r = e % TR;
        float2 val = make_float2(0.f, 0.f);
        if (r < cnt) val = v[vi][(size_t)s * n + base + r];
        sh.u.d.tile[vi][r] = val;
      }
      __syncthreads();
      if (act)
        for (int r = grp; r < cnt; r += groups) cfmac(acc, sh.u.d.tile[pi[p]][r], sh.u.d.tile[pj[p]][r]);
      __syncthreads();
    }
    sh.u.d.red[t] = act ? acc : make_float2(0.f, 0.f);
    __syncthreads();
    // fixed-order tree over the row groups
    for (int gc = groups; gc > 1;) {
      const int half = (gc + 1) / 2;
      for (int e = t; e < (gc - half) * np; e += PT) sh.u.d.red[e] = cadd(sh.u.d.red[e], sh.u.d.red[e + half * np]);
      gc = half;
      __syncthreads();
    }
    if (t < np) a.partial[((size_t)blockIdx.x * kPersistMaxSys + s) * kPersistSums + t] = sh.u.d.red[t];
    __syncthreads();
  }
}

// After a barrier: every CTA adds all CTAs' partials in the same order (one
// warp per output, lanes over the CTAs, fixed shuffle tree).  A warp takes
// four outputs at once so that their loads are in flight together.
__device__ void dots_final(const PersistArgs& a, Shared& sh, int np) {
  constexpr int U = 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = a.nsys * np;
  for (int e0 = warp; e0 < total; e0 += NW * U) {
    float2 sum[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      sum[u] = make_float2(0.f, 0.f);
      const int e = e0 + u * NW;
      if (e < total) {
        const int s = e / np, p = e - (e / np) * np;
        for (int b = lane; b < (int)gridDim.x; b += 32)
          sum[u] = cadd(sum[u], __ldcg(&a.partial[((size_t)b * kPersistMaxSys + s) * kPersistSums + p]));
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        sum[u].x += __shfl_xor_sync(0xffffffffu, sum[u].x, off);
        sum[u].y += __shfl_xor_sync(0xffffffffu, sum[u].y, off);
      }
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NW;
        if (e < total) sh.sums[e / np][e % np] = sum[u];
      }
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Bounded wait for phase 0 of the CTA's mbarrier.
__device__ __forceinline__ bool mbar_wait0(unsigned long long* b, unsigned long long limit_ns) {
  const unsigned addr = smem_u32(b);
  const unsigned long long t0 = gtime();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr)
        : "memory");
    if (done) return true;
    if (gtime() - t0 > limit_ns) return false;
  }
}

// Resident mode: the CTA's stencil rows (and prolongator rows, when their
// byte offsets are 16-byte multiples) arrive by bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on one mbarrier); row scales,
// unaligned prolongator rows and the neighbour table of the touched sites are
// filled by the other threads meanwhile.  Returns false when the copy does
// not complete within the time limit.
template <typename SL>
__device__ bool load_resident(const PersistArgs& a, Shared& sh, const Own& o, unsigned char* smem) {
  const int t = threadIdx.x;
  const int N = a.N, W = 9 * N;
  const int rows = o.r1 - o.r0;
  const int nv = a.tg.nvec;
  const size_t sbytes = (size_t)rows * W * sizeof(SL);
  const size_t pbytes = a.has_pre ? (size_t)rows * nv * sizeof(SL) : 0;
  const bool p_bulk = a.has_pre && (nv * sizeof(SL)) % 16 == 0;
  const size_t total = sbytes + (p_bulk ? pbytes : 0);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     smem_u32(&sh.mbar)),
                 "r"((unsigned)total)
                 : "memory");
    auto bulk = [&](unsigned char* dst, const unsigned char* src, size_t bytes) {
      constexpr size_t kChunk = 32768;
      for (size_t off = 0; off < bytes; off += kChunk) {
        const unsigned sz = (unsigned)(bytes - off < kChunk ? bytes - off : kChunk);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst + off)),
            "l"(src + off), "r"(sz), "r"(smem_u32(&sh.mbar))
            : "memory");
      }
    };
    if (sbytes > 0)
      bulk(smem + a.plan.off_S,
           reinterpret_cast<const unsigned char*>(reinterpret_cast<const SL*>(a.S) + (size_t)o.r0 * W), sbytes);
    if (p_bulk && pbytes > 0)
      bulk(smem + a.plan.off_P,
           reinterpret_cast<const unsigned char*>(reinterpret_cast<const SL*>(a.P) + (size_t)o.r0 * nv), pbytes);
  }
  if (a.Srs != nullptr) {
    float* dst = reinterpret_cast<float*>(smem + a.plan.off_sc);
    for (int i = t; i < rows; i += PT) dst[i] = a.Srs[o.r0 + i];
  }
  if (a.has_pre && !p_bulk) {
    const SL* src = reinterpret_cast<const SL*>(a.P) + (size_t)o.r0 * nv;
    SL* dst = reinterpret_cast<SL*>(smem + a.plan.off_P);
    for (int i = t; i < rows * nv; i += PT) dst[i] = src[i];
  }
  for (int e = t; e < o.nts * 9; e += PT) {
    const int xl = e / 9, dir = e % 9;
    const int X = o.xs0 + xl;
    int c[4];
    a.g.coords(X, c);
    int site = X;
    if (dir > 0) site = a.g.shift(c, (dir - 1) / 2, (dir & 1) ? 1 : -1);
    sh.nbt[xl][dir] = site;
  }
  if (t == 0) {
    sh.ok = 1;
    if (!mbar_wait0(&sh.mbar, 1000000000ull)) {
      atomicExch(a.err, 1);
      sh.ok = 0;
      mbar_wait0(&sh.mbar, 1000000000ull);   // let a copy still in flight land before the CTA exits
    }
  }
  __syncthreads();
  return sh.ok != 0;
}

// ------------------------------------------------------------------ kernel
template <typename SL>
__device__ void persist_body(const PersistArgs& a, Shared& sh, unsigned char* smem) {
  const long long n = a.n;
  const int K = a.K, S = a.s, nsys = a.nsys;
  const Own o = own_rows(a);
  const int t = threadIdx.x, warp = t >> 5;
  unsigned long long target = 0;
#define BARRIER(id) do { if (!grid_sync(a, sh, target, id)) return; } while (0)

  if (t == 0) trace_mark(a, 0);
  if (a.plan.resident && !load_resident<SL>(a, sh, o, smem)) return;
  // r = b, x = 0 (z_0 = r without a preconditioner) on the own rows; |r|^2
  for (int s = 0; s < nsys; ++s)
    for (int i = o.r0 + t; i < o.r1; i += PT) {
      const float2 bv = a.b[(size_t)s * n + i];
      a.r[(size_t)s * n + i] = bv;
      a.x[(size_t)s * n + i] = make_float2(0.f, 0.f);
      if (!a.has_pre) a.z[0][(size_t)s * n + i] = bv;
    }
  __syncthreads();
  {
    float2* vv[1] = {a.r};
    const int pi[1] = {0}, pj[1] = {0};
    dots_partial(a, sh, o, vv, 1, pi, pj, 1);
  }
  if (a.has_pre) restrict_partial<SL>(a, o, smem, a.r);
  BARRIER(1);
  if (a.trace != nullptr) BARRIER(12);   // trace only: the cost of an empty phase
  dots_final(a, sh, 1);
  if (t == 0) {
    int any = 0;
    for (int s = 0; s < nsys; ++s) {
      const float b2 = sh.sums[s][0].x;
      sh.r2[s] = b2;
      sh.thr2[s] = (float)a.tol2 * b2;
      sh.active[s] = b2 > sh.thr2[s] && b2 > 0.f;
      sh.nk[s] = 0;
      any |= sh.active[s];
    }
    sh.any = any;
  }
  __syncthreads();

  for (int k = 0; k < K && sh.any; ++k) {
    float2* zk = a.z[k];
    float2* wk = a.w[k];
    if (a.has_pre) {
      // ---- z_k = K(r): coarse correction, then CA-GCR(s) on this level
      assemble_rc(a, a.rc);
      BARRIER(2);
      dense_phase(a, a.ec, a.rc);
      BARRIER(3);
      prolong_own<SL>(a, o, smem, zk, a.ec);
      BARRIER(4);
      stencil_phase<SL>(a, sh, o, smem, a.V[0], zk, a.r);          // V0 = r - A z
      for (int i = 1; i <= S; ++i) {
        BARRIER(i == 1 ? 5 : 6);
        stencil_phase<SL>(a, sh, o, smem, a.V[i], a.V[i - 1], nullptr);
      }
      {
        int pi[kPersistSums], pj[kPersistSums], np = 0;
        for (int i = 0; i < S; ++i)
          for (int j = i; j < S; ++j) { pi[np] = i + 1; pj[np] = j + 1; ++np; }
        for (int i = 0; i < S; ++i) { pi[np] = i + 1; pj[np] = 0; ++np; }
        dots_partial(a, sh, o, a.V, S + 1, pi, pj, np);
        BARRIER(7);
        dots_final(a, sh, np);
      }
      if (t == 0) trace_mark(a, 15);
      for (int s = warp; s < nsys && warp < kCaWarps; s += kCaWarps)
        ca_solve_warp<float>(sh.sums[s], S, sh.coef[s], sh.u.ca[warp]);
      __syncthreads();
      if (t == 0) trace_mark(a, 16);
      // z += sum_q c_q V_q ;  w = A z = (r - V0) + sum_q c_q V_{q+1}
      for (int s = 0; s < nsys; ++s)
        for (int i = o.r0 + t; i < o.r1; i += PT) {
          const size_t oi = (size_t)s * n + i;
          float2 zacc = zk[oi];
          float2 wacc = csub(a.r[oi], a.V[0][oi]);
          for (int q = 0; q < S; ++q) {
            const float2 cf = sh.coef[s][q];
            cfma(zacc, cf, a.V[q][oi]);
            cfma(wacc, cf, a.V[q + 1][oi]);
          }
          zk[oi] = zacc;
          wk[oi] = wacc;
        }
      __syncthreads();
      if (t == 0) trace_mark(a, 17);
    } else {
      // ---- z_k = r (set on the own rows before the last barrier); w_k = A z_k
      stencil_phase<SL>(a, sh, o, smem, wk, zk, nullptr);
    }
    // ---- classical Gram-Schmidt, pass 1
    if (k > 0) {
      int pi[kPersistMaxK], pj[kPersistMaxK];
      for (int j = 0; j < k; ++j) { pi[j] = j; pj[j] = k; }
      dots_partial(a, sh, o, a.w, k + 1, pi, pj, k);
      BARRIER(8);
      dots_final(a, sh, k);
      if (t < nsys)
        for (int j = 0; j < k; ++j) sh.beta[t][k][j] = sh.sums[t][j];
      __syncthreads();
      for (int s = 0; s < nsys; ++s)
        for (int i = o.r0 + t; i < o.r1; i += PT) {
          const size_t oi = (size_t)s * n + i;
          float2 acc = wk[oi];
          for (int j = 0; j < k; ++j) {
            const float2 b = sh.beta[s][k][j];
            cfma(acc, make_float2(-b.x, -b.y), a.w[j][oi]);
          }
          wk[oi] = acc;
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
      dots_partial(a, sh, o, vv, k + 2, pi, pj, k + 2);
      BARRIER(9);
      dots_final(a, sh, k + 2);
    }
    if (t < nsys) {
      const int s = t;
      float sumc = 0.f;
      for (int j = 0; j < k; ++j) {
        const float2 c2 = sh.sums[s][j];
        sh.beta[s][k][j] = cadd(sh.beta[s][k][j], c2);
        sumc += c2.x * c2.x + c2.y * c2.y;
      }
      const float ww = sh.sums[s][k].x - sumc;
      const float2 wr = sh.sums[s][k + 1];
      const float g = sqrtf(fmaxf(ww, 0.f));
      const bool gfin = g > 0.f && isfinite(g);
      const bool ok = sh.active[s] && gfin;
      const float gi = gfin ? 1.f / g : 0.f;
      const float2 al = ok ? make_float2(wr.x * gi, wr.y * gi) : make_float2(0.f, 0.f);
      sh.gamma[s][k] = make_float2(ok ? g : 0.f, 0.f);
      sh.alpha[s][k] = al;
      sh.coef[s][0] = make_float2(gi, 0.f);   // 1/gamma for the update
      if (sh.active[s]) {
        sh.nk[s] = k + 1;
        const float r2 = sh.r2[s] - (al.x * al.x + al.y * al.y);
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
    const bool next = k + 1 < K;
    for (int s = 0; s < nsys; ++s) {
      const float gi = sh.coef[s][0].x;
      const float2 al = sh.alpha[s][k];
      const float2 na = make_float2(-al.x, -al.y);
      for (int i = o.r0 + t; i < o.r1; i += PT) {
        const size_t oi = (size_t)s * n + i;
        float2 acc = wk[oi];
        for (int j = 0; j < k; ++j) {
          const float2 c2 = sh.sums[s][j];
          cfma(acc, make_float2(-c2.x, -c2.y), a.w[j][oi]);
        }
        acc = make_float2(acc.x * gi, acc.y * gi);
        wk[oi] = acc;
        float2 rv = a.r[oi];
        cfma(rv, na, acc);
        a.r[oi] = rv;
        if (!a.has_pre && next) a.z[k + 1][oi] = rv;
      }
    }
    __syncthreads();
    if (!sh.any || !next) break;
    if (a.has_pre) restrict_partial<SL>(a, o, smem, a.r);
    BARRIER(10);
  }
  // ---- x = sum_k y_k z_k with gamma_j y_j + sum_{q>j} beta[q][j] y_q = alpha_j
  if (t < nsys) {
    const int s = t, m = sh.nk[s];
    for (int j = K - 1; j >= 0; --j) {
      float2 v = make_float2(0.f, 0.f);
      if (j < m) {
        v = sh.alpha[s][j];
        for (int q = j + 1; q < m; ++q) {
          const float2 b = sh.beta[s][q][j], y = sh.coef[s][q];
          v.x -= b.x * y.x - b.y * y.y;
          v.y -= b.x * y.y + b.y * y.x;
        }
        const float g = sh.gamma[s][j].x;
        v = g > 0.f ? make_float2(v.x / g, v.y / g) : make_float2(0.f, 0.f);
      }
      sh.coef[s][j] = v;
    }
  }
  __syncthreads();
  for (int s = 0; s < nsys; ++s) {
    const int m = sh.nk[s];
    for (int i = o.r0 + t; i < o.r1; i += PT) {
      const size_t oi = (size_t)s * n + i;
      float2 acc = make_float2(0.f, 0.f);
      for (int q = 0; q < m; ++q) cfma(acc, sh.coef[s][q], a.z[q][oi]);
      a.x[oi] = acc;
    }
  }
  __syncthreads();
  if (t == 0) trace_mark(a, 11);
#undef BARRIER
}

template <typename SL>
__global__ void __launch_bounds__(PT, 1) persist_gcr_kernel(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Shared& sh = *reinterpret_cast<Shared*>(smem);
  if (a.run != nullptr && *a.run == 0) return;   // uniform across the grid
  persist_body<SL>(a, sh, smem);
  __syncthreads();
  if (threadIdx.x == 0) {
    // every arrival of this launch precedes its CTA's exit count, so the
    // last CTA out may clear the barrier for the next launch
    __threadfence();
    if (atomicAdd(a.exitc, 1u) == gridDim.x - 1) {
      atomicExch(a.bar, 0ull);
      atomicExch(a.exitc, 0u);
      __threadfence();
    }
  }
}

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    SMG_CUDA_OK(cudaGetDevice(&dev));
    SMG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

int smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    SMG_CUDA_OK(cudaGetDevice(&dev));
    SMG_CUDA_OK(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  }
  return v;
}

}  // namespace

const char* persist_phase_name(int id, bool has_pre) {
  static const char* pre[] = {"P.start", "P.init(|b|,Rb)", "P.assemble(Rr)", "P.dense", "P.prolong",
                              "P.V0=r-Az", "P.V_i=AV", "P.V_s+gram", "P.CA+corr+cgs1", "P.cgs2",
                              "P.update+Rr", "P.x", "P.empty_barrier", "P.stencil.stage", "P.stencil.rows",
                              "P.gram_final", "P.ca_solve", "P.correction"};
  static const char* nop[] = {"P.start", "P.init", "?", "?", "?", "?", "?", "?", "P.w=Az+cgs1", "P.cgs2",
                              "P.update", "P.x", "P.empty_barrier", "P.stencil.stage", "P.stencil.rows",
                              "?", "?", "?"};
  if (id < 0 || id > 17) return "?";
  return has_pre ? pre[id] : nop[id];
}

bool persist_supported(int nsys, int K, int s, int N, long long n, Store st) {
  return (st == S16 || st == S32) && n * nsys < (1LL << 30) && nsys >= 1 && nsys <= kPersistMaxSys && K >= 1 && K <= kPersistMaxK &&
         s >= 1 && s <= kCaMaxS && s + 1 <= kMaxP && K + 2 <= kMaxP && N >= 2 && N % 2 == 0;
}

PersistPlan persist_plan(const Geom& g, int N, int nsys, int nvec_next, Store st) {
  return persist_plan_for(g.V, N, nsys, nvec_next, st, device_sms(), (size_t)smem_optin());
}

PersistPlan persist_plan_for(int V, int N, int nsys, int nvec_next, Store st, int sms, size_t cap) {
  SMG_REQUIRE(V >= 1 && N >= 2 && nsys >= 1 && nvec_next >= 0 && sms >= 1, "persist plan: bad shape");
  PersistPlan p;
  const long long n = (long long)V * N;
  p.grid = std::min(sms, V);
  p.per = (n + p.grid - 1) / p.grid;
  p.nslot = (int)((p.per - 1 + N - 1) / N) + 1;
  const size_t sl = store_bytes(st);
  const size_t base = align16(sizeof(Shared));
  p.smem = base;
  p.resident = 0;
  p.sg = 0;
  if (N % 4 == 0 && p.nslot <= kPersistMaxTouch) {
    const size_t sres = align16((size_t)p.per * 9 * N * sl);
    const size_t scl = align16((size_t)p.per * sizeof(float));
    const size_t pres = nvec_next > 0 ? align16((size_t)p.per * nvec_next * sl) : 0;
    const size_t stage1 = (size_t)p.nslot * 9 * N * sizeof(float2);
    const size_t fixed = base + sres + scl + pres;
    if (fixed + stage1 <= cap) {
      p.resident = 1;
      p.sg = (int)std::min<size_t>((size_t)nsys, (cap - fixed) / stage1);
      p.off_S = base;
      p.off_sc = base + sres;
      p.off_P = base + sres + scl;
      p.off_stg = fixed;
      p.smem = fixed + (size_t)p.sg * stage1;
    }
  }
  return p;
}

size_t persist_buffer_bytes(const PersistPlan& p, int nvec_next) {
  const size_t part = (size_t)p.grid * kPersistMaxSys * kPersistSums * sizeof(float2);
  const size_t rp = nvec_next > 0 ? (size_t)p.grid * p.nslot * kPersistMaxSys * 2 * nvec_next * sizeof(float2) : 0;
  return align16(part) + align16(rp) + 64;
}

void persist_gcr(const PersistArgs& a, Store st, cudaStream_t stream) {
  static bool attr16 = false, attr32 = false;
  const PersistPlan& p = a.plan;
  SMG_REQUIRE(p.grid >= 1 && p.grid <= device_sms(), "persistent coarse solver: bad grid");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(p.grid);
  cfg.blockDim = dim3(PT);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int per = 0;
  if (st == S16) {
    if (!attr16) {
      SMG_CUDA_OK(cudaFuncSetAttribute(persist_gcr_kernel<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_optin()));
      attr16 = true;
    }
    SMG_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist_gcr_kernel<__half2>, PT, p.smem));
    SMG_REQUIRE(per >= 1, "persistent coarse solver does not fit on an SM");
    SMG_CUDA_OK(cudaLaunchKernelEx(&cfg, persist_gcr_kernel<__half2>, a));
  } else {
    if (!attr32) {
      SMG_CUDA_OK(cudaFuncSetAttribute(persist_gcr_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_optin()));
      attr32 = true;
    }
    SMG_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist_gcr_kernel<float2>, PT, p.smem));
    SMG_REQUIRE(per >= 1, "persistent coarse solver does not fit on an SM");
    SMG_CUDA_OK(cudaLaunchKernelEx(&cfg, persist_gcr_kernel<float2>, a));
  }
  SMG_LAUNCH_OK();
}

}  // namespace smg
