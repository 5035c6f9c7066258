// Restriction R = P^dag and prolongation P (Sec. 2.1) of FP32 vectors with an
// FP16 prolongator on the tensor cores, up to 16 systems per CTA.
//
// Per aggregate X and chirality chi the two transfers are small dense
// complex products over the aggregate's rows (site, d) of that chirality:
//   restriction   c[s][k]   = sum_r conj(P[r][k]) v[s][r]      (16 x R by R x nvec)
//   prolongation  e[s][r]   = sum_k P[r][k] c[s][chi][k]        (16 x nvec by nvec x R)
// Both run as real m16n8k16 MMAs (FP16 operands, FP32 accumulation) with the
// 16 systems as M.  The complex structure sits in the operand pairs: an A
// entry pair is (Re, Im) of a vector component, a B entry pair is one
// prolongator entry as stored, (Re P, Im P), or that pair conjugated or
// multiplied by -i (a half swap and a sign flip on the raw bits), which makes
// the two columns of a complex output its real and imaginary parts.  The
// rows of an aggregate are listed per chirality (sites of one parity on the
// fine lattice, the upper or lower half of the components on coarse ones),
// so one 8-row K step (restriction) or 4-row N tile (prolongation) never mixes
// chiralities.  The vector operand is rounded to FP16 after a per-(aggregate,
// system) power-of-two scale that maps its largest entry into [2^13, 2^14);
// the scale is undone in the FP32 epilogue.  The prolongator is streamed
// from global memory with 16-byte loads, each thread reading the run of
// entries its fragments need (the order of the vector index inside the
// contraction is permuted identically on both operands to make those runs
// contiguous), prefetched one step ahead.
#include <vector>

#include "ops.cuh"

namespace smg {
namespace {

constexpr int kTcSys = 16;       // systems per CTA: the MMA's M
constexpr int kTcThreads = 256;  // 8 warps
constexpr int kTcChunk = 128;    // restriction: rows per chirality staged per pass
constexpr int kTcRowWords = 24;  // staged row: 16 systems + 8 words of padding (conflict-free A loads)

__device__ __forceinline__ void mma_f16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
               "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (a, b) as an FP16 pair (a in the low half) -> (-b, a): the entry times i.
__device__ __forceinline__ unsigned pair_times_i(unsigned u) { return ((u >> 16) ^ 0x8000u) | (u << 16); }
// (a, b) -> (a, -b)
__device__ __forceinline__ unsigned pair_conj(unsigned u) { return u ^ 0x80000000u; }
// (a, b) -> (b, a)
__device__ __forceinline__ unsigned pair_swap(unsigned u) { return (u >> 16) | (u << 16); }

__device__ __forceinline__ unsigned to_h2(float2 v, float s) {
  __half2 h = __floats2half2_rn(v.x * s, v.y * s);
  return *reinterpret_cast<unsigned*>(&h);
}

__device__ __forceinline__ unsigned word_of(const uint4& u, int i) {
  return i == 0 ? u.x : i == 1 ? u.y : i == 2 ? u.z : u.w;
}

// rows[chi * R + i]: the aggregate's fine rows (site * ndof + d) of chirality
// chi, R = npos * ndof / 2 per chirality.  Fine lattice (chi_mode 0): the
// sites of each parity in position order, all d of a site together; coarse
// lattices: for each position the components of that chirality's half.
__device__ void tc_rows(int* rows, int* cnt, const TransferGeom& t, int X, int npos, int R) {
  const int nd = t.ndof, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int Xc[4];
  t.coarse.coords(X, Xc);
  auto site_of = [&](int p) {
    int c[4], q = p;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int lc = q % t.agg[mu];
      q /= t.agg[mu];
      c[mu] = Xc[mu] * t.agg[mu] + lc;
    }
    return t.fine.index(c);
  };
  if (t.chi_mode != 0) {
    const int h = nd / 2;
    for (int e = tid; e < npos * nd; e += blockDim.x) {
      const int p = e / nd, d = e - p * nd;
      const int chi = d >= h ? 1 : 0;
      rows[chi * R + p * h + (d - chi * h)] = site_of(p) * nd + d;
    }
    __syncthreads();
    return;
  }
  // fine lattice: rank every position among those of its parity (ballot prefix)
  int base0 = 0, base1 = 0;
  for (int p0 = 0; p0 < npos; p0 += blockDim.x) {
    const int p = p0 + tid;
    const bool valid = p < npos;
    int x = 0, par = 0;
    if (valid) {
      x = site_of(p);
      int c[4];
      t.fine.coords(x, c);
      par = (c[0] + c[1] + c[2] + c[3]) & 1;
    }
    const unsigned b0 = __ballot_sync(0xffffffffu, valid && par == 0);
    const unsigned b1 = __ballot_sync(0xffffffffu, valid && par == 1);
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) { cnt[2 * w] = __popc(b0); cnt[2 * w + 1] = __popc(b1); }
    __syncthreads();
    int pre0 = 0, pre1 = 0, tot0 = 0, tot1 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      if (i < w) { pre0 += cnt[2 * i]; pre1 += cnt[2 * i + 1]; }
      tot0 += cnt[2 * i];
      tot1 += cnt[2 * i + 1];
    }
    if (valid) {
      const int rank = par == 0 ? base0 + pre0 + __popc(b0 & lt) : base1 + pre1 + __popc(b1 & lt);
      for (int d = 0; d < nd; ++d) rows[par * R + rank * nd + d] = x * nd + d;
    }
    base0 += tot0;
    base1 += tot1;
    __syncthreads();
  }
}

// Power-of-two scale per system that maps the largest |Re|, |Im| into
// [2^13, 2^14) (1 for a zero system); NaN and Inf pass through to the output.
__device__ __forceinline__ float tc_scale(float m) {
  int e2 = 0;
  if (m > 0.f && m <= 3.0e38f) frexpf(m, &e2);
  return ldexpf(1.f, 14 - e2);
}

template <int NV>
__global__ void __launch_bounds__(kTcThreads) restrict_mma_kernel(float2* __restrict__ out,
                                                                  const float2* __restrict__ in,
                                                                  const __half2* __restrict__ P, float pscale,
                                                                  TransferGeom t, int nsys, int ngroups,
                                                                  const int* run) {
  constexpr int J = NV / 4;    // n8 tiles over (k, Re/Im) of one chirality
  constexpr int JW = J / 2;    // tiles per warp (the warp pair of one chirality splits k in halves)
  constexpr int LW = JW / 4;   // 16-byte prolongator loads per row and step
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char tc_smem[];
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int nd = t.ndof, R = npos * nd / 2;
  const int X = blockIdx.x / ngroups, s0 = (blockIdx.x % ngroups) * kTcSys;
  const int ns = min(kTcSys, nsys - s0);
  int* rows = reinterpret_cast<int*>(tc_smem);                          // [2][R]
  unsigned* vh = reinterpret_cast<unsigned*>(rows + 2 * R);             // [2][chunk][kTcRowWords]
  float* red = reinterpret_cast<float*>(vh + 2 * kTcChunk * kTcRowWords);   // [2 chi][2 half][32][JW * 4]
  __shared__ float sig[kTcSys];
  __shared__ int cnt[2 * kTcThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  tc_rows(rows, cnt, t, X, npos, R);
  const long long nf = (long long)t.fine.V * nd;
  // largest entry per system (warp w: systems w, w + 8)
  for (int s = w; s < kTcSys; s += kTcThreads / 32) {
    float m = 0.f;
    if (s < ns)
      for (int i = lane; i < 2 * R; i += 32) {
        const float2 v = in[(size_t)(s0 + s) * nf + rows[i]];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sig[s] = tc_scale(m);
  }
  const int chi = w >> 2, hk = (w >> 1) & 1, sub = w & 1;
  const int g = lane >> 2, tq = lane & 3, q = g >> 1;
  const bool im_col = (g & 1) != 0;
  const int kofs = q * J + hk * JW;
  float acc[JW][4];
#pragma unroll
  for (int j = 0; j < JW; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0.f;
  const int* crow = rows + chi * R;
  for (int c0 = 0; c0 < R; c0 += kTcChunk) {
    const int cr = min(kTcChunk, R - c0);
    __syncthreads();   // scales ready / the previous chunk's fragments consumed
    for (int e = tid; e < 2 * cr * kTcSys; e += kTcThreads) {
      const int s = e & (kTcSys - 1), ri = e >> 4;
      const int ch = ri / cr, i = ri - ch * cr;
      unsigned hv = 0u;
      if (s < ns) hv = to_h2(in[(size_t)(s0 + s) * nf + rows[ch * R + c0 + i]], sig[s]);
      vh[(ch * kTcChunk + i) * kTcRowWords + s] = hv;
    }
    __syncthreads();
    const int nst = cr / 8;
    const unsigned* vc = vh + chi * kTcChunk * kTcRowWords;
    uint4 u0[LW], u1[LW];
    int st = sub;
    if (st < nst) {
      const int rb = c0 + st * 8;
      const uint4* p0 = reinterpret_cast<const uint4*>(P + (size_t)crow[rb + tq] * NV + kofs);
      const uint4* p1 = reinterpret_cast<const uint4*>(P + (size_t)crow[rb + tq + 4] * NV + kofs);
#pragma unroll
      for (int l = 0; l < LW; ++l) { u0[l] = __ldg(p0 + l); u1[l] = __ldg(p1 + l); }
    }
    for (; st < nst; st += 2) {
      uint4 n0[LW], n1[LW];
      if (st + 2 < nst) {
        const int rb = c0 + (st + 2) * 8;
        const uint4* p0 = reinterpret_cast<const uint4*>(P + (size_t)crow[rb + tq] * NV + kofs);
        const uint4* p1 = reinterpret_cast<const uint4*>(P + (size_t)crow[rb + tq + 4] * NV + kofs);
#pragma unroll
        for (int l = 0; l < LW; ++l) { n0[l] = __ldg(p0 + l); n1[l] = __ldg(p1 + l); }
      }
      const unsigned* vr = vc + st * 8 * kTcRowWords;
      unsigned a[4];
      a[0] = vr[tq * kTcRowWords + g];
      a[1] = vr[tq * kTcRowWords + g + 8];
      a[2] = vr[(tq + 4) * kTcRowWords + g];
      a[3] = vr[(tq + 4) * kTcRowWords + g + 8];
#pragma unroll
      for (int j = 0; j < JW; ++j) {
        const unsigned w0 = word_of(u0[j >> 2], j & 3), w1 = word_of(u1[j >> 2], j & 3);
        mma_f16(acc[j], a, im_col ? pair_times_i(w0) : w0, im_col ? pair_times_i(w1) : w1);
      }
      if (st + 2 < nst) {
#pragma unroll
        for (int l = 0; l < LW; ++l) { u0[l] = n0[l]; u1[l] = n1[l]; }
      }
    }
  }
  // the odd-step warp of each (chirality, k half) parks its sums; the even one adds and writes
  float* myred = red + ((size_t)(chi * 2 + hk) * 32 + lane) * (JW * 4);
  if (sub == 1)
#pragma unroll
    for (int j = 0; j < JW; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) myred[j * 4 + c] = acc[j][c];
  __syncthreads();
  if (sub != 0) return;
  const int N = 2 * NV;
  const float f0 = g < ns ? pscale / sig[g] : 0.f, f1 = g + 8 < ns ? pscale / sig[g + 8] : 0.f;
#pragma unroll
  for (int j = 0; j < JW; ++j) {
    const int k = tq * J + hk * JW + j;
    const size_t o = (size_t)X * N + chi * NV + k;
    if (g < ns)
      out[(size_t)(s0 + g) * t.coarse.V * N + o] = make_float2((acc[j][0] + myred[j * 4 + 0]) * f0,
                                                               (acc[j][1] + myred[j * 4 + 1]) * f0);
    if (g + 8 < ns)
      out[(size_t)(s0 + g + 8) * t.coarse.V * N + o] = make_float2((acc[j][2] + myred[j * 4 + 2]) * f1,
                                                                   (acc[j][3] + myred[j * 4 + 3]) * f1);
  }
}

template <int NV>
__global__ void __launch_bounds__(kTcThreads) prolong_mma_kernel(float2* __restrict__ out,
                                                                 const float2* __restrict__ in,
                                                                 const __half2* __restrict__ P, float pscale,
                                                                 TransferGeom t, int nsys, int ngroups,
                                                                 const int* run) {
  constexpr int KS = NV / 8;   // k16 steps; K slot u of step m is vector k = u * KS + m
  constexpr int LW = KS / 4;   // 16-byte loads per run
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char tc_smem[];
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int nd = t.ndof, R = npos * nd / 2, N = 2 * NV;
  const int X = blockIdx.x / ngroups, s0 = (blockIdx.x % ngroups) * kTcSys;
  const int ns = min(kTcSys, nsys - s0);
  int* rows = reinterpret_cast<int*>(tc_smem);                 // [2][R]
  unsigned* ech = reinterpret_cast<unsigned*>(rows + 2 * R);   // [2 NV][16] FP16 pairs of the coarse components
  __shared__ float sig[kTcSys];
  __shared__ int cnt[2 * kTcThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  tc_rows(rows, cnt, t, X, npos, R);
  const size_t cstride = (size_t)t.coarse.V * N;
  for (int s = w; s < kTcSys; s += kTcThreads / 32) {
    float m = 0.f;
    if (s < ns)
      for (int i = lane; i < N; i += 32) {
        const float2 v = in[(size_t)(s0 + s) * cstride + (size_t)X * N + i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sig[s] = tc_scale(m);
  }
  __syncthreads();
  for (int e = tid; e < N * kTcSys; e += kTcThreads) {
    const int s = e & (kTcSys - 1), i = e >> 4;
    ech[e] = s < ns ? to_h2(in[(size_t)(s0 + s) * cstride + (size_t)X * N + i], sig[s]) : 0u;
  }
  __syncthreads();
  const int chi = w >> 2, sub = w & 3;
  const int g = lane >> 2, tq = lane & 3;
  const bool im_col = (g & 1) != 0;
  // A fragments of every k step (system g / g + 8, K slots tq and tq + 4)
  unsigned a[KS][4];
  const unsigned* ec = ech + chi * NV * kTcSys;
#pragma unroll
  for (int m = 0; m < KS; ++m) {
    a[m][0] = ec[(tq * KS + m) * kTcSys + g];
    a[m][1] = ec[(tq * KS + m) * kTcSys + g + 8];
    a[m][2] = ec[((tq + 4) * KS + m) * kTcSys + g];
    a[m][3] = ec[((tq + 4) * KS + m) * kTcSys + g + 8];
  }
  const int* crow = rows + chi * R;
  const int ntile = R / 4;
  const long long nf = (long long)t.fine.V * nd;
  const float f0 = g < ns ? pscale / sig[g] : 0.f, f1 = g + 8 < ns ? pscale / sig[g + 8] : 0.f;
  uint4 u0[LW], u1[LW];
  int nt = sub;
  if (nt < ntile) {
    const __half2* pr = P + (size_t)crow[nt * 4 + (g >> 1)] * NV;
#pragma unroll
    for (int l = 0; l < LW; ++l) {
      u0[l] = __ldg(reinterpret_cast<const uint4*>(pr + tq * KS) + l);
      u1[l] = __ldg(reinterpret_cast<const uint4*>(pr + (tq + 4) * KS) + l);
    }
  }
  for (; nt < ntile; nt += 4) {
    uint4 n0[LW], n1[LW];
    if (nt + 4 < ntile) {
      const __half2* pr = P + (size_t)crow[(nt + 4) * 4 + (g >> 1)] * NV;
#pragma unroll
      for (int l = 0; l < LW; ++l) {
        n0[l] = __ldg(reinterpret_cast<const uint4*>(pr + tq * KS) + l);
        n1[l] = __ldg(reinterpret_cast<const uint4*>(pr + (tq + 4) * KS) + l);
      }
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < KS; ++m) {
      const unsigned w0 = word_of(u0[m >> 2], m & 3), w1 = word_of(u1[m >> 2], m & 3);
      mma_f16(acc, a[m], im_col ? pair_swap(w0) : pair_conj(w0), im_col ? pair_swap(w1) : pair_conj(w1));
    }
    const int r = crow[nt * 4 + tq];
    if (g < ns) out[(size_t)(s0 + g) * nf + r] = make_float2(acc[0] * f0, acc[1] * f0);
    if (g + 8 < ns) out[(size_t)(s0 + g + 8) * nf + r] = make_float2(acc[2] * f1, acc[3] * f1);
    if (nt + 4 < ntile) {
#pragma unroll
      for (int l = 0; l < LW; ++l) { u0[l] = n0[l]; u1[l] = n1[l]; }
    }
  }
}

size_t restrict_mma_smem(int R, int nv) { return sizeof(int) * 2 * R + 4ull * 2 * kTcChunk * kTcRowWords + 4ull * 2 * 2 * 32 * (nv / 8) * 4; }
size_t prolong_mma_smem(int R, int nv) { return sizeof(int) * 2 * R + 4ull * 2 * nv * kTcSys; }

template <typename K>
void tc_ensure_smem(K kernel, size_t bytes) {
  static std::vector<std::pair<const void*, size_t>> set;
  if (bytes <= 48 * 1024) return;
  for (auto& e : set)
    if (e.first == (const void*)kernel && bytes <= e.second) return;
  SMG_CUDA_OK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  set.emplace_back((const void*)kernel, bytes);
}

}  // namespace

bool transfer_mma_ok(const TransferGeom& t, const Stored& P, Prec vp) {
  if (P.s != S16 || vp != P32) return false;
  if (t.nvec != 32 && t.nvec != 64) return false;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  if (t.chi_mode == 0) {
    // equal parity counts in every aggregate: one even extent suffices
    bool even = false;
    for (int mu = 0; mu < 4; ++mu) even = even || (t.agg[mu] % 2 == 0);
    if (!even) return false;
  } else if (t.ndof % 2 != 0) {
    return false;
  }
  const long long R = (long long)npos * t.ndof / 2;
  if (R % 8 != 0) return false;
  return restrict_mma_smem((int)R, t.nvec) <= 160 * 1024 && prolong_mma_smem((int)R, t.nvec) <= 160 * 1024;
}

void restrict_mma(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                  const int* run) {
  SMG_REQUIRE(transfer_mma_ok(t, P, in.prec), "restrict_mma: unsupported transfer shape");
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int R = npos * t.ndof / 2;
  const int ngroups = (int)ceil_div(in.nsys, kTcSys);
  const size_t smem = restrict_mma_smem(R, t.nvec);
  auto k = t.nvec == 64 ? restrict_mma_kernel<64> : restrict_mma_kernel<32>;
  tc_ensure_smem(k, smem);
  launch_k(k, dim3((unsigned)t.coarse.V * ngroups), dim3(kTcThreads), smem, st, (float2*)out.p,
           (const float2*)in.p, (const __half2*)P.p, P.gscale, t, in.nsys, ngroups, run);
  SMG_LAUNCH_OK();
}

void prolong_mma(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                 const int* run) {
  SMG_REQUIRE(transfer_mma_ok(t, P, in.prec), "prolong_mma: unsupported transfer shape");
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int R = npos * t.ndof / 2;
  const int ngroups = (int)ceil_div(in.nsys, kTcSys);
  const size_t smem = prolong_mma_smem(R, t.nvec);
  auto k = t.nvec == 64 ? prolong_mma_kernel<64> : prolong_mma_kernel<32>;
  tc_ensure_smem(k, smem);
  launch_k(k, dim3((unsigned)t.coarse.V * ngroups), dim3(kTcThreads), smem, st, (float2*)out.p,
           (const float2*)in.p, (const __half2*)P.p, P.gscale, t, in.nsys, ngroups, run);
  SMG_LAUNCH_OK();
}

}  // namespace smg
