// Kahler-Dirac block preconditioner (Eq. 1, Eq. 2, Sec. 3.1).
//
// B is the part of the distance-one hopping term that stays inside an
// aligned 2^4 hypercube, so B + m is block diagonal with one 48x48 complex
// block per hypercube (16 sites x 3 colours, ordered 3b + a with
// b = (x&1) + 2(y&1) + 4(z&1) + 8(t&1)).  kd_build assembles each block from
// the fat links and inverts it in FP64 (Gauss-Jordan with partial pivoting,
// one CTA per hypercube, the augmented 48x96 matrix in shared memory).
// kd_apply multiplies every hypercube of a batched field by its inverse.
#include <algorithm>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "ops.cuh"
#include "tune.cuh"

namespace smg {
namespace {

constexpr int NB = 48;

__global__ void __launch_bounds__(256) kd_build_kernel(double2* __restrict__ inv, const double2* __restrict__ fat,
                                                       double mass, Geom g) {
  extern __shared__ double2 aug[];   // [48][96]
  __shared__ double2 fac[NB];
  __shared__ int piv_row;
  const int blk = blockIdx.x;
  const int t = threadIdx.x;
  // assemble [B + m | 1]
  for (int e = t; e < NB * 2 * NB; e += blockDim.x) {
    const int row = e / (2 * NB), col = e % (2 * NB);
    double2 v = make_double2(0, 0);
    if (col >= NB) {
      if (col - NB == row) v.x = 1.0;
    } else {
      const int b = row / 3, a = row % 3, bp = col / 3, ap = col % 3;
      if (b == bp) {
        if (a == ap) v.x = mass;
      } else {
        const int diff = b ^ bp;
        if ((diff & (diff - 1)) == 0) {
          int mu = 0;
          while ((1 << mu) != diff) ++mu;
          const int xb = hypercube_site(g, blk, b);
          int c[4];
          g.coords(xb, c);
          int es = 0;
          for (int nu = 0; nu < mu; ++nu) es += c[nu];
          const double eta = (es & 1) ? -0.5 : 0.5;
          if (((b >> mu) & 1) == 0) {
            // forward hop inside the hypercube: +1/2 eta U_mu(x)[a][a']
            const double2 u = fat[((size_t)mu * g.V + xb) * 9 + a * 3 + ap];
            v = make_double2(eta * u.x, eta * u.y);
          } else {
            // backward hop: -1/2 eta conj(U_mu(x - mu)[a'][a])
            const int xn = hypercube_site(g, blk, bp);
            const double2 u = fat[((size_t)mu * g.V + xn) * 9 + ap * 3 + a];
            v = make_double2(-eta * u.x, eta * u.y);
          }
        }
      }
    }
    aug[e] = v;
  }
  __syncthreads();
  for (int k = 0; k < NB; ++k) {
    if (t < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + t; i < NB; i += 32) {
        const double2 v = aug[i * 2 * NB + k];
        const double m2 = v.x * v.x + v.y * v.y;
        if (m2 > best) { best = m2; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (t == 0) piv_row = bi;
    }
    __syncthreads();
    const int p = piv_row;
    if (p != k) {
      for (int j = t; j < 2 * NB; j += blockDim.x) {
        const double2 tmp = aug[k * 2 * NB + j];
        aug[k * 2 * NB + j] = aug[p * 2 * NB + j];
        aug[p * 2 * NB + j] = tmp;
      }
    }
    __syncthreads();
    const double2 pv = aug[k * 2 * NB + k];
    const double d = pv.x * pv.x + pv.y * pv.y;
    const double2 ip = make_double2(pv.x / d, -pv.y / d);
    __syncthreads();
    for (int j = t; j < 2 * NB; j += blockDim.x) aug[k * 2 * NB + j] = cmul(aug[k * 2 * NB + j], ip);
    if (t < NB) fac[t] = (t == k) ? make_double2(0, 0) : aug[t * 2 * NB + k];
    __syncthreads();
    for (int e = t; e < NB * 2 * NB; e += blockDim.x) {
      const int i = e / (2 * NB), j = e % (2 * NB);
      if (i == k) continue;
      const double2 f = fac[i];
      double2 v = aug[e];
      const double2 w = aug[k * 2 * NB + j];
      v.x -= f.x * w.x - f.y * w.y;
      v.y -= f.x * w.y + f.y * w.x;
      aug[e] = v;
    }
    __syncthreads();
  }
  for (int e = t; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    inv[(size_t)blk * NB * NB + e] = aug[i * 2 * NB + NB + j];
  }
}

// row-major FP64 -> column-major per block, in the requested storage
template <typename SL>
__global__ void kd_pack_kernel(SL* __restrict__ dst, float* __restrict__ scale, const double2* __restrict__ inv,
                               long long nblk) {
  const long long blk = blockIdx.x;
  const int r = threadIdx.x;   // one thread per row (48)
  if (r >= NB) return;
  const double2* row = inv + (size_t)blk * NB * NB + (size_t)r * NB;
  float sc = 1.0f;
  if (scale != nullptr) {
    double mx = 0.0;
    for (int c = 0; c < NB; ++c) mx = fmax(mx, fmax(fabs(row[c].x), fabs(row[c].y)));
    sc = mx > 0 ? (float)mx : 1.0f;
    scale[blk * NB + r] = sc;
  }
  const double isc = 1.0 / (double)sc;
  for (int c = 0; c < NB; ++c) {
    const double2 v = row[c];
    SL* o = dst + (size_t)blk * NB * NB + (size_t)c * NB + r;
    if constexpr (sizeof(SL) == 16) *o = SL{v.x, v.y};
    else if constexpr (sizeof(SL) == 8) *o = SL{(float)v.x, (float)v.y};
    else *o = __floats2half2_rn((float)(v.x * isc), (float)(v.y * isc));
  }
}

struct KdSet {
  const void* p[16];
  const float* scale[16];
};

// 4 hypercubes per CTA, one thread per output row; SB systems per CTA
// (blockIdx.y picks the group, which shares one block inverse), so each block
// entry is read once for the whole group.
// FP32 vectors, two rows per thread: eight hypercubes per CTA of 192
// threads, thread (hypercube lb, row pair rp) computes rows 2rp and 2rp + 1
// for SB systems.  The block entries of a column pair come in two 8-byte
// (FP16) or 16-byte (FP32) loads and each staged vector pair in one 16-byte
// shared load, which then feeds eight complex multiply-adds per system.
template <typename SL, int SB>
__global__ void __launch_bounds__(192) kd_apply2_kernel(float2* __restrict__ out, const float2* __restrict__ in,
                                                        KdSet kd, const int* __restrict__ sys_map, int dagger,
                                                        long long nblk, Geom g, const float2* __restrict__ sub_from,
                                                        int nsys, const int* run) {
  constexpr int PB = NB / 2;   // row pairs per hypercube
  using P2 = typename std::conditional<sizeof(SL) == 4, uint2, uint4>::type;   // two consecutive entries
  if (run != nullptr && *run == 0) return;
  __shared__ __align__(16) float2 vin[SB][8][NB];
  const int s0 = blockIdx.y * SB;
  const int ns = min(SB, nsys - s0);
  const int lb = threadIdx.x / PB, rp = threadIdx.x % PB;
  const int r0 = 2 * rp;
  const long long blk = (long long)blockIdx.x * 8 + lb;
  const long long vs = (long long)g.V * 3;
  const int kidx = sys_map != nullptr ? sys_map[s0] : 0;
  const SL* K = (const SL*)kd.p[kidx];
  const float* sc = kd.scale[kidx];
  int site0 = 0, site1 = 0;
  if (blk < nblk) {
    site0 = hypercube_site(g, (int)blk, r0 / 3);
    site1 = hypercube_site(g, (int)blk, (r0 + 1) / 3);
#pragma unroll
    for (int sb = 0; sb < SB; ++sb)
      if (sb < ns) {
        vin[sb][lb][r0] = in[(s0 + sb) * vs + (size_t)site0 * 3 + (r0 % 3)];
        vin[sb][lb][r0 + 1] = in[(s0 + sb) * vs + (size_t)site1 * 3 + ((r0 + 1) % 3)];
      }
  }
  __syncthreads();
  if (blk >= nblk) return;
  const SL* Kb = K + (size_t)blk * NB * NB;
  float2 a0[SB], a1[SB];
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) { a0[sb] = make_float2(0.f, 0.f); a1[sb] = a0[sb]; }
  auto pair = [](const SL* p, float2& x, float2& y) {
    const P2 raw = __ldg(reinterpret_cast<const P2*>(p));
    const SL* e = reinterpret_cast<const SL*>(&raw);
    x = ld<float>(e, 0);
    y = ld<float>(e, 1);
  };
  if (!dagger) {
    // out[r] = sum_c K[c][r] v[c], K stored column by column
#pragma unroll 4
    for (int c = 0; c < NB; c += 2) {
      float2 k00, k01, k10, k11;   // k<column><row>
      pair(Kb + (size_t)c * NB + r0, k00, k01);
      pair(Kb + (size_t)(c + 1) * NB + r0, k10, k11);
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) {
        const float4 v = *reinterpret_cast<const float4*>(&vin[sb][lb][c]);
        const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
        cfma(a0[sb], k00, v0);
        cfma(a0[sb], k10, v1);
        cfma(a1[sb], k01, v0);
        cfma(a1[sb], k11, v1);
      }
    }
    if (sc != nullptr) {
      const float f0 = sc[blk * NB + r0], f1 = sc[blk * NB + r0 + 1];
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) { a0[sb] = cscale(a0[sb], f0); a1[sb] = cscale(a1[sb], f1); }
    }
  } else {
    // out[r] = sum_c conj(K[r][c]) v[c] (K^dag), the scale of column c on each entry
#pragma unroll 4
    for (int c = 0; c < NB; c += 2) {
      float2 k00, k01, k10, k11;   // k<row><column>
      pair(Kb + (size_t)r0 * NB + c, k00, k01);
      pair(Kb + (size_t)(r0 + 1) * NB + c, k10, k11);
      if (sc != nullptr) {
        const float f0 = sc[blk * NB + c], f1 = sc[blk * NB + c + 1];
        k00 = cscale(k00, f0); k10 = cscale(k10, f0);
        k01 = cscale(k01, f1); k11 = cscale(k11, f1);
      }
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) {
        const float4 v = *reinterpret_cast<const float4*>(&vin[sb][lb][c]);
        const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
        cfmac(a0[sb], k00, v0);
        cfmac(a0[sb], k01, v1);
        cfmac(a1[sb], k10, v0);
        cfmac(a1[sb], k11, v1);
      }
    }
  }
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) {
    if (sb >= ns) break;
    const size_t o0 = (s0 + sb) * vs + (size_t)site0 * 3 + (r0 % 3);
    const size_t o1 = (s0 + sb) * vs + (size_t)site1 * 3 + ((r0 + 1) % 3);
    float2 v0 = a0[sb], v1 = a1[sb];
    if (sub_from != nullptr) { v0 = csub(sub_from[o0], v0); v1 = csub(sub_from[o1], v1); }
    out[o0] = v0;
    out[o1] = v1;
  }
}

template <typename R, typename SL, int SB>
__global__ void __launch_bounds__(192) kd_apply_kernel(typename cplx<R>::T* __restrict__ out,
                                                       const typename cplx<R>::T* __restrict__ in, KdSet kd,
                                                       const int* __restrict__ sys_map, int dagger, long long nblk,
                                                       Geom g, const typename cplx<R>::T* __restrict__ sub_from,
                                                       int nsys, const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  __shared__ C vin[SB][4][NB];
  const int s0 = blockIdx.y * SB;
  const int ns = min(SB, nsys - s0);
  const int lb = threadIdx.x / NB, r = threadIdx.x % NB;
  const long long blk = (long long)blockIdx.x * 4 + lb;
  const long long vs = (long long)g.V * 3;
  const int kidx = sys_map != nullptr ? sys_map[s0] : 0;
  const SL* K = (const SL*)kd.p[kidx];
  const float* sc = kd.scale[kidx];
  int site = 0;
  if (blk < nblk) {
    site = hypercube_site(g, (int)blk, r / 3);
#pragma unroll
    for (int sb = 0; sb < SB; ++sb)
      if (sb < ns) vin[sb][lb][r] = in[(s0 + sb) * vs + (size_t)site * 3 + (r % 3)];
  }
  __syncthreads();
  if (blk >= nblk) return;
  const SL* Kb = K + (size_t)blk * NB * NB;
  C acc[SB];
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) acc[sb] = C{0, 0};
  if (!dagger) {
#pragma unroll 8
    for (int c = 0; c < NB; ++c) {
      const C k = ld<R>(Kb, (size_t)c * NB + r);
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) cfma(acc[sb], k, vin[sb][lb][c]);
    }
    if (sc != nullptr) {
      const R f = (R)sc[blk * NB + r];
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) acc[sb] = cscale(acc[sb], f);
    }
  } else {
#pragma unroll 8
    for (int c = 0; c < NB; ++c) {
      C k = ld<R>(Kb, (size_t)r * NB + c);
      if (sc != nullptr) k = cscale(k, (R)sc[blk * NB + c]);
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) cfmac(acc[sb], k, vin[sb][lb][c]);
    }
  }
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) {
    if (sb >= ns) break;
    const size_t oi = (s0 + sb) * vs + (size_t)site * 3 + (r % 3);
    C v = acc[sb];
    if (sub_from != nullptr) v = csub(sub_from[oi], v);
    out[oi] = v;
  }
}

template <typename R, typename SL, int SB>
void launch_kd(const Vec& out, const Vec& in, const KdSet& set, const int* sys_map, int dagger, long long nblk,
               const Geom& g, const void* sub_from, cudaStream_t st, const int* run) {
  using C = typename cplx<R>::T;
  dim3 grid(ceil_div(nblk, 4), ceil_div(in.nsys, SB));
  launch_k(kd_apply_kernel<R, SL, SB>, grid, dim3(192), 0, st, (C*)out.p, (const C*)in.p, set, sys_map, dagger, nblk,
           g, (const C*)sub_from, in.nsys, run);
}

template <typename SL, int SB>
void launch_kd2(const Vec& out, const Vec& in, const KdSet& set, const int* sys_map, int dagger, long long nblk,
                const Geom& g, const void* sub_from, cudaStream_t st, const int* run) {
  dim3 grid(ceil_div(nblk, 8), ceil_div(in.nsys, SB));
  launch_k(kd_apply2_kernel<SL, SB>, grid, dim3(192), 0, st, (float2*)out.p, (const float2*)in.p, set, sys_map,
           dagger, nblk, g, (const float2*)sub_from, in.nsys, run);
}

template <typename SL>
void launch_kd2_sb(int sb, const Vec& out, const Vec& in, const KdSet& set, const int* sys_map, int dagger,
                   long long nblk, const Geom& g, const void* sub_from, cudaStream_t st, const int* run) {
  switch (sb) {
    case 1: launch_kd2<SL, 1>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    case 2: launch_kd2<SL, 2>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    case 4: launch_kd2<SL, 4>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    case 8: launch_kd2<SL, 8>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    default: launch_kd2<SL, 16>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
  }
}

template <typename R, typename SL>
void launch_kd_sb(int sb, const Vec& out, const Vec& in, const KdSet& set, const int* sys_map, int dagger,
                  long long nblk, const Geom& g, const void* sub_from, cudaStream_t st, const int* run) {
  switch (sb) {
    case 1: launch_kd<R, SL, 1>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    case 2: launch_kd<R, SL, 2>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    case 4: launch_kd<R, SL, 4>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
    default: launch_kd<R, SL, 8>(out, in, set, sys_map, dagger, nblk, g, sub_from, st, run); break;
  }
}

}  // namespace

void kd_build(double2* inv64, const Geom& g, const double2* fat64, double mass, cudaStream_t st) {
  for (int mu = 0; mu < 4; ++mu) SMG_REQUIRE(g.L[mu] % 2 == 0 && g.L[mu] >= 4, "kd_build: extents must be even and >= 4");
  const size_t smem = sizeof(double2) * NB * 2 * NB;
  static bool attr = false;
  if (!attr) {
    SMG_CUDA_OK(cudaFuncSetAttribute(kd_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  kd_build_kernel<<<g.V / 16, 256, smem, st>>>(inv64, fat64, mass, g);
  SMG_LAUNCH_OK();
}

void kd_pack(Stored& dst, const double2* inv64, long long nblk, cudaStream_t st) {
  if (dst.s == S64) kd_pack_kernel<double2><<<(unsigned)nblk, 64, 0, st>>>((double2*)dst.p, nullptr, inv64, nblk);
  else if (dst.s == S32) kd_pack_kernel<float2><<<(unsigned)nblk, 64, 0, st>>>((float2*)dst.p, nullptr, inv64, nblk);
  else kd_pack_kernel<__half2><<<(unsigned)nblk, 64, 0, st>>>((__half2*)dst.p, dst.scale, inv64, nblk);
  SMG_LAUNCH_OK();
}

void kd_apply(const Vec& out, const Vec& in, const Geom& g, const Stored* kd, const int* sys_map, int nkd,
              int dagger, cudaStream_t st, const int* run, const void* sub_from, int kd_run) {
  SMG_REQUIRE(in.n == (long long)g.V * 3 && out.n == in.n && in.nsys == out.nsys && in.prec == out.prec,
              "kd_apply: shape mismatch");
  SMG_REQUIRE(nkd >= 1 && nkd <= 16, "kd_apply: 1..16 block inverses");
  KdSet set{};
  for (int i = 0; i < nkd; ++i) {
    SMG_REQUIRE(kd[i].s == kd[0].s, "kd_apply: mixed storage");
    set.p[i] = kd[i].p;
    set.scale[i] = kd[i].s == S16 ? kd[i].scale : nullptr;
  }
  const long long nblk = g.V / 16;
  // with several inverses a group of systems may not straddle two masses:
  // kd_run consecutive systems share one inverse, and the group size must
  // divide it; with one inverse any group size serves
  const int run_len = (sys_map == nullptr) ? 0 : std::max(1, kd_run);
  // candidate ids: sb = systems per CTA of the one-row kernel, 32 + sb those of the two-row kernel
  const bool two_row = in.prec == P32 && (kd[0].s == S16 || kd[0].s == S32);
  auto go = [&](int sb, const Vec& o, const int* rr) {
    if (sb >= 32) {
      if (kd[0].s == S32) launch_kd2_sb<float2>(sb - 32, o, in, set, sys_map, dagger, nblk, g, sub_from, st, rr);
      else launch_kd2_sb<__half2>(sb - 32, o, in, set, sys_map, dagger, nblk, g, sub_from, st, rr);
      SMG_LAUNCH_OK();
      return;
    }
    if (in.prec == P64) {
      SMG_REQUIRE(kd[0].s == S64, "kd_apply: FP64 vectors need FP64 blocks");
      launch_kd_sb<double, double2>(sb, o, in, set, sys_map, dagger, nblk, g, sub_from, st, rr);
    } else if (kd[0].s == S32) {
      launch_kd_sb<float, float2>(sb, o, in, set, sys_map, dagger, nblk, g, sub_from, st, rr);
    } else if (kd[0].s == S16) {
      launch_kd_sb<float, __half2>(sb, o, in, set, sys_map, dagger, nblk, g, sub_from, st, rr);
    } else {
      SMG_REQUIRE(false, "kd_apply: unsupported precision pair");
    }
    SMG_LAUNCH_OK();
  };
  std::vector<TuneCandidate> cands;
  for (int sb : {1, 2, 4, 8})
    if (sb == 1 || (sb < 2 * in.nsys && (run_len == 0 || run_len % sb == 0)))
      cands.push_back({sb, sb == 1 ? "1 system/CTA" : sb == 2 ? "2 systems/CTA" : sb == 4 ? "4 systems/CTA"
                                                                                      : "8 systems/CTA"});
  if (two_row)
    for (int sb : {1, 2, 4, 8, 16})
      if (sb == 1 || (sb < 2 * in.nsys && (run_len == 0 || run_len % sb == 0)))
        cands.push_back({32 + sb, sb == 1 ? "2 rows/thread, 1 system/CTA" : sb == 2 ? "2 rows/thread, 2 systems/CTA"
                                  : sb == 4 ? "2 rows/thread, 4 systems/CTA" : sb == 8 ? "2 rows/thread, 8 systems/CTA"
                                                                                       : "2 rows/thread, 16 systems/CTA"});
  int sb = 1;
  if (cands.size() > 1) {
    char key[160];
    std::snprintf(key, sizeof(key), "kd_apply V=%d nsys=%d run=%d vec=%s store=%s dag=%d sub=%d", g.V, in.nsys,
                  run_len, in.prec == P64 ? "f64" : "f32", kd[0].s == S16 ? "f16" : (kd[0].s == S32 ? "f32" : "f64"),
                  dagger, sub_from != nullptr ? 1 : 0);
    struct Scratch {
      void* p = nullptr;
      ~Scratch() { if (p) cudaFree(p); }
    } scratch;
    sb = tune_pick(key, cands, st, [&](int id) {
      if (scratch.p == nullptr) SMG_CUDA_OK(cudaMalloc(&scratch.p, out.bytes()));
      Vec o = out;
      o.p = scratch.p;
      go(id, o, nullptr);
    });
  }
  go(sb, out, run);
}

}  // namespace smg
