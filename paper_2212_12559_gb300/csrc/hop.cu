// Fine staggered operator M = m + D (Sec. 2.2) from phase-folded links:
// for every site x and direction mu one record
//
//   [ eta_mu(x) V_mu(x) | eta_mu(x) W_mu(x) ]     (W: Naik links, if any)
//
// padded to whole 16-byte chunks.  Because eta_mu depends only on the
// coordinates before mu, eta_mu(x - k mu) = eta_mu(x), so the backward hops
// read the folded record of the neighbour and apply its conjugate transpose:
//
//   (D psi)(x) = 1/2 sum_mu [ F_mu(x) psi(x+mu) - F_mu(x-mu)^dag psi(x-mu) ]
//              + c_N/2 sum_mu [ G_mu(x) psi(x+3mu) - G_mu(x-3mu)^dag psi(x-3mu) ].
//
// Four threads per site (one per mu) each load their own record and the
// needed halves of the two neighbour records with 16-byte loads and add the
// hops of their direction; a two-step shuffle adds the four directions.  Per
// site that is about 4 x (11 + 13) load instructions instead of the ~290 of
// a thread per (site, colour) reading link rows, and each link is stored once.
// The sign flip is exact in every storage precision.
#include <cstdio>
#include <vector>

#include "ops.cuh"
#include "tune.cuh"

namespace smg {
namespace {

// Record of (x, mu) in SL entries: fat at [0, 9), Naik at [9, 18), padded.
template <typename SL>
__host__ __device__ constexpr int record_entries(int K) {
  return (int)(((K * 9 * (int)sizeof(SL) + 15) / 16) * 16 / (int)sizeof(SL));
}
// 16-byte chunks that cover entries [e0, e0 + 9)
template <typename SL>
__host__ __device__ constexpr int chunk_lo(int e0) { return e0 * (int)sizeof(SL) / 16; }
template <typename SL>
__host__ __device__ constexpr int chunk_hi(int e0) { return ((e0 + 9) * (int)sizeof(SL) + 15) / 16; }

__device__ __forceinline__ float2 to_f2(__half2 h) { return __half22float2(h); }
__device__ __forceinline__ float2 to_f2(float2 f) { return f; }

template <typename SL>
__device__ __forceinline__ SL from_d2(double2 v, float inv_scale);
template <>
__device__ __forceinline__ __half2 from_d2<__half2>(double2 v, float inv_scale) {
  return __floats2half2_rn((float)v.x * inv_scale, (float)v.y * inv_scale);
}
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 v, float) {
  return make_float2((float)v.x, (float)v.y);
}

// One thread per (site, mu, entry).
template <typename SL, int K>
__global__ void build_hop_kernel(SL* __restrict__ H, const double2* __restrict__ fat, const double2* __restrict__ naik,
                                 Geom g, float inv_fat, float inv_naik) {
  constexpr int RE = record_entries<SL>(K);
  const long long total = (long long)g.V * 4 * RE;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % RE);
    const long long xm = e / RE;
    const int mu = (int)(xm % 4), x = (int)(xm / 4);
    const int kind = r / 9, ab = r % 9;
    if (kind >= K) {   // padding
      H[e] = from_d2<SL>(make_double2(0, 0), 1.f);
      continue;
    }
    int c[4];
    g.coords(x, c);
    int es = 0;
    for (int nu = 0; nu < mu; ++nu) es += c[nu];
    const double eta = (es & 1) ? -1.0 : 1.0;
    const double2 v = (kind == 0 ? fat : naik)[((size_t)mu * g.V + x) * 9 + ab];
    H[e] = from_d2<SL>(make_double2(eta * v.x, eta * v.y), kind == 0 ? inv_fat : inv_naik);
  }
}

// Loads the 16-byte chunks [lo, hi) of a record into raw[lo..hi).
template <int NCH>
__device__ __forceinline__ void load_chunks(uint4 (&raw)[NCH], const uint4* rec, int lo, int hi) {
#pragma unroll
  for (int q = 0; q < NCH; ++q)
    if (q >= lo && q < hi) raw[q] = __ldg(rec + q);
}

// acc += w * F psi (forward) or acc -= w * F^dag psi (backward), F = entries [e0, e0+9) of raw
template <typename SL, int NCH, bool DAG>
__device__ __forceinline__ void hop3(float2 (&acc)[3], const uint4 (&raw)[NCH], int e0, const float2* p, float w) {
  const SL* m = reinterpret_cast<const SL*>(raw);
  const float2 p0 = p[0], p1 = p[1], p2 = p[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 t = make_float2(0.f, 0.f);
    if (!DAG) {
      cfma(t, to_f2(m[e0 + a * 3 + 0]), p0);
      cfma(t, to_f2(m[e0 + a * 3 + 1]), p1);
      cfma(t, to_f2(m[e0 + a * 3 + 2]), p2);
      acc[a].x = fmaf(w, t.x, acc[a].x);
      acc[a].y = fmaf(w, t.y, acc[a].y);
    } else {
      cfmac(t, to_f2(m[e0 + 0 * 3 + a]), p0);
      cfmac(t, to_f2(m[e0 + 1 * 3 + a]), p1);
      cfmac(t, to_f2(m[e0 + 2 * 3 + a]), p2);
      acc[a].x = fmaf(-w, t.x, acc[a].x);
      acc[a].y = fmaf(-w, t.y, acc[a].y);
    }
  }
}

// The link records one (site, mu) thread needs: its own record and the
// needed chunks of the records of x - mu and x - 3mu, with the neighbour
// sites of the four hops.  Loaded once and reused for every system of the
// batch the thread handles.
template <typename SL, int K>
struct HopLinks {
  static constexpr int RE = record_entries<SL>(K);
  static constexpr int NCH = RE * (int)sizeof(SL) / 16;
  uint4 own[NCH], bf[NCH], bn[NCH];
  int xf1, xb1, xf3, xb3;
  __device__ __forceinline__ void load(const uint4* __restrict__ base, const Geom& g, int x, int mu,
                                       const int (&c)[4]) {
    xf1 = g.shift(c, mu, 1);
    xb1 = g.shift(c, mu, -1);
    xf3 = xb3 = 0;
    if constexpr (K == 2) { xf3 = g.shift(c, mu, 3); xb3 = g.shift(c, mu, -3); }
    load_chunks(own, base + ((size_t)x * 4 + mu) * NCH, 0, NCH);
    load_chunks(bf, base + ((size_t)xb1 * 4 + mu) * NCH, chunk_lo<SL>(0), chunk_hi<SL>(0));
    if constexpr (K == 2) load_chunks(bn, base + ((size_t)xb3 * 4 + mu) * NCH, chunk_lo<SL>(9), chunk_hi<SL>(9));
  }
};

// The hops of direction mu out of site x for one system: the neighbour
// spinor loads come first and are independent of each other (12 8-byte
// loads with Naik links), then the arithmetic.
template <typename SL, int K>
__device__ __forceinline__ void hop_dir(float2 (&acc)[3], const HopLinks<SL, K>& L, const float2* __restrict__ vin,
                                        float cf, float cn) {
  constexpr int NCH = HopLinks<SL, K>::NCH;
  float2 pf1[3], pb1[3], pf3[3], pb3[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    pf1[b] = vin[(size_t)L.xf1 * 3 + b];
    pb1[b] = vin[(size_t)L.xb1 * 3 + b];
    if constexpr (K == 2) {
      pf3[b] = vin[(size_t)L.xf3 * 3 + b];
      pb3[b] = vin[(size_t)L.xb3 * 3 + b];
    }
  }
  hop3<SL, NCH, false>(acc, L.own, 0, pf1, cf);
  hop3<SL, NCH, true>(acc, L.bf, 0, pb1, cf);
  if constexpr (K == 2) {
    hop3<SL, NCH, false>(acc, L.own, 9, pf3, cn);
    hop3<SL, NCH, true>(acc, L.bn, 9, pb3, cn);
  }
}

// add the four directions of a site held by lanes 4q .. 4q+3
__device__ __forceinline__ void sum_quad(float2 (&acc)[3]) {
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[a].x += __shfl_xor_sync(0xffffffffu, acc[a].x, o);
      acc[a].y += __shfl_xor_sync(0xffffffffu, acc[a].y, o);
    }
}

// out = m in + D in (or m in - D in with dagger; or sub_from - that).  Each
// CTA serves SB systems (blockIdx.y picks the group): the link records are
// loaded once per (site, mu) thread and applied to every system of the group.
template <typename SL, int K, int SB>
__global__ void __launch_bounds__(256) hop_dslash_kernel(float2* __restrict__ out, const float2* __restrict__ in,
                                                         const SL* __restrict__ H, float cf, float cn,
                                                         const double* __restrict__ mass, double mass0, int dagger,
                                                         Geom g, const float2* __restrict__ sub_from, int nsys,
                                                         const int* run) {
  if (run != nullptr && *run == 0) return;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = tid < g.V * 4;
  const int x = valid ? tid >> 2 : g.V - 1, mu = tid & 3;
  int c[4];
  g.coords(x, c);
  HopLinks<SL, K> L;
  L.load(reinterpret_cast<const uint4*>(H), g, x, mu, c);
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) {
    const int s = blockIdx.y * SB + sb;
    if (s >= nsys) break;                     // the same for the whole CTA
    const float2* vin = in + (size_t)s * g.V * 3;
    float2 acc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[a] = make_float2(0.f, 0.f);
    hop_dir<SL, K>(acc, L, vin, cf, cn);
    sum_quad(acc);
    if (valid && mu != 3) {
      // lane mu writes colour mu
      float2 v = mu == 0 ? acc[0] : (mu == 1 ? acc[1] : acc[2]);
      if (dagger) v = make_float2(-v.x, -v.y);
      const float m = (float)(mass != nullptr ? mass[s] : mass0);
      const size_t oi = (size_t)s * g.V * 3 + (size_t)x * 3 + mu;
      const float2 self = in[oi];
      v.x = fmaf(m, self.x, v.x);
      v.y = fmaf(m, self.y, v.y);
      if (sub_from != nullptr) v = csub(sub_from[oi], v);
      out[oi] = v;
    }
  }
}

template <typename SL, int K, int SB>
void launch_hop(const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run) {
  dim3 grid(ceil_div((long long)p.g.V * 4, 256), ceil_div(p.nsys, SB));
  const float cf = 0.5f * p.hop.gscale;
  const float cn = (float)(0.5 * p.c_naik) * p.hop_naik_scale;
  launch_k(hop_dslash_kernel<SL, K, SB>, dim3(grid), dim3(256), 0, st, (float2*)out.p, (const float2*)in.p,
           (const SL*)p.hop.p, cf, cn, p.mass, p.mass0, p.dagger, p.g, (const float2*)p.sub_from, p.nsys, run);
  SMG_LAUNCH_OK();
}

template <typename SL, int K>
void launch_hop_sb(int sb, const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run) {
  switch (sb) {
    case 1: launch_hop<SL, K, 1>(out, in, p, st, run); break;
    case 2: launch_hop<SL, K, 2>(out, in, p, st, run); break;
    case 4: launch_hop<SL, K, 4>(out, in, p, st, run); break;
    case 8: launch_hop<SL, K, 8>(out, in, p, st, run); break;
    default: launch_hop<SL, K, 16>(out, in, p, st, run); break;
  }
}

template <typename SL, int K>
void build_hop(void* H, const double2* fat, const double2* naik, const Geom& g, float sf, float sn, cudaStream_t st) {
  const long long total = (long long)g.V * 4 * record_entries<SL>(K);
  unsigned grid = ceil_div(total, 256);
  if (grid > 16384) grid = 16384;
  build_hop_kernel<SL, K><<<grid, 256, 0, st>>>((SL*)H, fat, naik, g, 1.0f / sf, 1.0f / sn);
  SMG_LAUNCH_OK();
}

}  // namespace

size_t hop_link_entries(const Geom& g, bool naik, Store s) {
  const int re = s == S16 ? (naik ? record_entries<__half2>(2) : record_entries<__half2>(1))
                          : (naik ? record_entries<float2>(2) : record_entries<float2>(1));
  return (size_t)g.V * 4 * re;
}

void build_hop_links(void* H, Store s, const double2* fat, const double2* naik, const Geom& g, float fat_scale,
                     float naik_scale, cudaStream_t st) {
  SMG_REQUIRE(s == S16 || s == S32, "hop links: FP16 or FP32 storage");
  if (s == S16) {
    if (naik != nullptr) build_hop<__half2, 2>(H, fat, naik, g, fat_scale, naik_scale, st);
    else build_hop<__half2, 1>(H, fat, nullptr, g, fat_scale, 1.f, st);
  } else {
    if (naik != nullptr) build_hop<float2, 2>(H, fat, naik, g, 1.f, 1.f, st);
    else build_hop<float2, 1>(H, fat, nullptr, g, 1.f, 1.f, st);
  }
}

bool hop_dslash_ok(const Vec& in, const DslashParams& p) {
  return p.hop.p != nullptr && p.part < 0 && in.prec == P32 && (p.hop.s == S16 || p.hop.s == S32);
}

// Systems per CTA of the phase-folded dslash: 1, 2, 4 or 8 (links read once
// per group); the autotuner times the ones that fit the batch.
void hop_dslash_sb(int sb, const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run) {
  SMG_REQUIRE(in.n == (long long)p.g.V * 3 && out.n == in.n, "dslash: field size does not match the lattice");
  SMG_REQUIRE(in.nsys == p.nsys && out.nsys == p.nsys && in.prec == P32 && out.prec == P32, "dslash: batch mismatch");
  SMG_REQUIRE(sb == 1 || sb == 2 || sb == 4 || sb == 8 || sb == 16, "dslash: 1, 2, 4, 8 or 16 systems per CTA");
  if (p.hop.s == S16) {
    if (p.hop_kinds == 2) launch_hop_sb<__half2, 2>(sb, out, in, p, st, run);
    else launch_hop_sb<__half2, 1>(sb, out, in, p, st, run);
  } else {
    if (p.hop_kinds == 2) launch_hop_sb<float2, 2>(sb, out, in, p, st, run);
    else launch_hop_sb<float2, 1>(sb, out, in, p, st, run);
  }
}

void hop_dslash(const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run) {
  if (p.nsys == 1) {
    hop_dslash_sb(1, out, in, p, st, run);
    return;
  }
  std::vector<TuneCandidate> cands;
  for (int sb : {1, 2, 4, 8, 16})
    if (sb == 1 || sb < 2 * p.nsys)
      cands.push_back({sb, sb == 1 ? "1 system/CTA" : sb == 2 ? "2 systems/CTA" : sb == 4 ? "4 systems/CTA"
                                                         : sb == 8 ? "8 systems/CTA" : "16 systems/CTA"});
  char key[160];
  std::snprintf(key, sizeof(key), "hop_dslash V=%d nsys=%d store=%s naik=%d sub=%d", p.g.V, p.nsys,
                p.hop.s == S16 ? "f16" : "f32", p.hop_kinds == 2 ? 1 : 0, p.sub_from != nullptr ? 1 : 0);
  struct Scratch {
    void* p = nullptr;
    ~Scratch() { if (p) cudaFree(p); }
  } scratch;
  const int sb = tune_pick(key, cands, st, [&](int id) {
    if (scratch.p == nullptr) SMG_CUDA_OK(cudaMalloc(&scratch.p, out.bytes()));
    Vec o = out;
    o.p = scratch.p;
    hop_dslash_sb(id, o, in, p, st, nullptr);
  });
  hop_dslash_sb(sb, out, in, p, st, run);
}

}  // namespace smg
