// Restriction R, prolongation P = R^dag and block orthonormalisation of the
// chirally doubled near-null vectors (Sec. 2.1, 2.3).
//
// A level has `ndof` components per site; the chirality of component d at
// site x is parity(x) on the fine lattice and (d >= ndof/2) on coarse
// lattices.  Each near-null vector v_k yields two prolongator columns, its
// projections on the two chiralities, so the coarse site carries
// N = 2 nvec components, (s, k) -> s*nvec + k.  The prolongator is stored
// as [V][ndof][nvec] (vector index fastest): column (s, k) at (x, d) is
// P[x][d][k] if chi(x,d) == s and zero otherwise.  With k fastest the
// restriction's threads (one per k) read consecutive entries and each
// prolongation thread (one per (x, d)) reads one contiguous run.
#include <cstdio>
#include <vector>

#include "ops.cuh"
#include "tune.cuh"

namespace smg {
namespace {

__device__ __forceinline__ int agg_site(const TransferGeom& t, int X, int p) {
  int Xc[4], c[4];
  t.coarse.coords(X, Xc);
  int q = p;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int lc = q % t.agg[mu];
    q /= t.agg[mu];
    c[mu] = Xc[mu] * t.agg[mu] + lc;
  }
  return t.fine.index(c);
}

__device__ __forceinline__ int site_parity(const Geom& g, int x) {
  int c[4];
  g.coords(x, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

__device__ __forceinline__ int chirality(const TransferGeom& t, int x, int d) {
  return t.chi_mode == 0 ? site_parity(t.fine, x) : (d >= t.ndof / 2 ? 1 : 0);
}

__device__ __forceinline__ int coarse_of(const TransferGeom& t, int x) {
  int c[4];
  t.fine.coords(x, c);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) c[mu] /= t.agg[mu];
  return t.coarse.index(c);
}

template <int NT>
__device__ double2 block_sum(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double2 s = make_double2(0, 0);
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s = cadd(s, sh[i]);
  return s;
}

// One CTA per (aggregate, chirality): MGS in vector order, two passes.
__global__ void __launch_bounds__(256) orthonormalize_kernel(double2* __restrict__ raw, TransferGeom t) {
  __shared__ double2 sh[8];
  const int X = blockIdx.x, chi = blockIdx.y;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int nel = npos * t.ndof;
  const size_t vstride = (size_t)t.fine.V * t.ndof;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0; k < t.nvec; ++k) {
      double2* vk = raw + (size_t)k * vstride;
      for (int j = 0; j < k; ++j) {
        const double2* vj = raw + (size_t)j * vstride;
        double2 acc = make_double2(0, 0);
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
          const int p = e / t.ndof, d = e % t.ndof;
          const int x = agg_site(t, X, p);
          if (chirality(t, x, d) != chi) continue;
          const size_t i = (size_t)x * t.ndof + d;
          cfmac(acc, vj[i], vk[i]);
        }
        const double2 dot = block_sum<256>(acc, sh);
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
          const int p = e / t.ndof, d = e % t.ndof;
          const int x = agg_site(t, X, p);
          if (chirality(t, x, d) != chi) continue;
          const size_t i = (size_t)x * t.ndof + d;
          const double2 u = vj[i];
          double2 v = vk[i];
          v.x -= dot.x * u.x - dot.y * u.y;
          v.y -= dot.x * u.y + dot.y * u.x;
          vk[i] = v;
        }
        __syncthreads();
      }
      double2 acc = make_double2(0, 0);
      for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int p = e / t.ndof, d = e % t.ndof;
        const int x = agg_site(t, X, p);
        if (chirality(t, x, d) != chi) continue;
        const size_t i = (size_t)x * t.ndof + d;
        cfmac(acc, vk[i], vk[i]);
      }
      const double2 n2 = block_sum<256>(acc, sh);
      const double inv = n2.x > 0 ? 1.0 / sqrt(n2.x) : 0.0;
      for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int p = e / t.ndof, d = e % t.ndof;
        const int x = agg_site(t, X, p);
        if (chirality(t, x, d) != chi) continue;
        const size_t i = (size_t)x * t.ndof + d;
        vk[i] = cscale(vk[i], inv);
      }
      __syncthreads();
    }
  }
}

template <typename SL>
__global__ void transfer_pack_kernel(SL* __restrict__ dst, const double2* __restrict__ raw, TransferGeom t) {
  const long long total = (long long)t.fine.V * t.nvec * t.ndof;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % t.nvec);
    const long long q = e / t.nvec;
    const int d = (int)(q % t.ndof);
    const long long x = q / t.ndof;
    const double2 v = raw[(size_t)k * t.fine.V * t.ndof + (size_t)x * t.ndof + d];
    if constexpr (sizeof(SL) == 16) dst[e] = SL{v.x, v.y};
    else if constexpr (sizeof(SL) == 8) dst[e] = SL{(float)v.x, (float)v.y};
    else dst[e] = __floats2half2_rn((float)v.x, (float)v.y);
  }
}

// One CTA per (aggregate, system).  The aggregate's sites and input entries
// are staged in shared memory first; then thread t owns vector k = t % nvec
// and every (t / nvec)-th row (p, d) of the aggregate, with one accumulator
// per chirality, its prolongator loads independent across iterations; the
// CTA finally adds the row groups.
template <typename R, typename SL>
__global__ void __launch_bounds__(256) restrict_kernel(typename cplx<R>::T* __restrict__ out,
                                                       const typename cplx<R>::T* __restrict__ in,
                                                       const SL* __restrict__ P, R pscale, TransferGeom t,
                                                       const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char rs_smem[];
  C* part = reinterpret_cast<C*>(rs_smem);                    // [2][256]
  C* vx = part + 512;                                         // [npos][ndof]
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  int* xs = reinterpret_cast<int*>(vx + (size_t)t.ndof * npos);   // site of each position
  int* xpar = xs + npos;                                          // its parity
  const int X = blockIdx.x, s = blockIdx.y;
  const int nv = t.nvec;
  const int k = threadIdx.x % nv, grp = threadIdx.x / nv, groups = blockDim.x / nv;
  const int nd = t.ndof, half = nd / 2;
  const long long nf = (long long)t.fine.V * nd;
  const C* vin = in + (size_t)s * nf;
  for (int p = threadIdx.x; p < npos; p += blockDim.x) {
    const int x = agg_site(t, X, p);
    xs[p] = x;
    xpar[p] = site_parity(t.fine, x);
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < npos * nd; rr += blockDim.x) {
    const int p = rr / nd, d = rr - p * nd;
    vx[rr] = vin[(size_t)xs[p] * nd + d];
  }
  __syncthreads();
  C acc0 = C{0, 0}, acc1 = C{0, 0};
  if (grp < groups) {
    for (int p = grp; p < npos; p += groups) {
      const size_t base = (size_t)xs[p] * nd;
      const int par = xpar[p];
#pragma unroll 4
      for (int d = 0; d < nd; ++d) {
        const int chi = t.chi_mode == 0 ? par : (d >= half ? 1 : 0);
        const C pv = ld<R>(P, (base + d) * nv + k);
        if (chi == 0) cfmac(acc0, pv, vx[p * nd + d]);
        else cfmac(acc1, pv, vx[p * nd + d]);
      }
    }
  }
  part[threadIdx.x] = acc0;   // blockDim.x == 256 (see restrict_op)
  part[256 + threadIdx.x] = acc1;
  __syncthreads();
  const int N = 2 * nv;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int chi = i / nv, kk = i % nv;
    C sum = C{0, 0};
    for (int g = 0; g < groups; ++g) sum = cadd(sum, part[chi * 256 + g * nv + kk]);
    out[(size_t)s * t.coarse.V * N + (size_t)X * N + i] = cscale(sum, pscale);
  }
}

// The same with 16-byte prolongator loads (nvec a multiple of the entries per
// 16 bytes): thread t owns the chunk of vectors kc = t % (nvec / VPC) and
// every (t / (nvec / VPC))-th row of the aggregate, so a CTA of 512 threads
// keeps ~10 independent loads per thread in flight; the row groups are then
// added in two fixed-order passes.  A CTA serves SB systems (blockIdx.y picks
// the group): each prolongator chunk is loaded once and applied to all of
// them, and the partial sums of the systems are added one system after the
// other in the same shared-memory area.
template <typename R, typename SL, int SB>
__global__ void __launch_bounds__(512) restrict_vec_kernel(typename cplx<R>::T* __restrict__ out,
                                                           const typename cplx<R>::T* __restrict__ in,
                                                           const SL* __restrict__ P, R pscale, TransferGeom t,
                                                           int nsys, const int* run) {
  using C = typename cplx<R>::T;
  constexpr int VPC = 16 / (int)sizeof(SL);
  constexpr int kRed = 8;                                     // first-pass partial sums per output
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char rs_smem[];
  const int nv = t.nvec, nch = nv / VPC;
  const int groups = blockDim.x / nch;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const int nd = t.ndof, half = nd / 2;
  C* part = reinterpret_cast<C*>(rs_smem);                    // [groups][2][nv]
  C* red = part + (size_t)groups * 2 * nv;                    // [kRed][2][nv]
  C* vx = red + (size_t)kRed * 2 * nv;                        // [SB][npos][nd]
  int* xs = reinterpret_cast<int*>(vx + (size_t)SB * npos * nd);   // site of each position
  int* xpar = xs + npos;                                          // its parity
  const int X = blockIdx.x, s0 = blockIdx.y * SB;
  const int ns = min(SB, nsys - s0);
  const long long nf = (long long)t.fine.V * nd;
  for (int p = threadIdx.x; p < npos; p += blockDim.x) {
    const int x = agg_site(t, X, p);
    xs[p] = x;
    xpar[p] = site_parity(t.fine, x);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ns * npos * nd; e += blockDim.x) {
    const int sb = e / (npos * nd), rr = e - sb * (npos * nd);
    const int p = rr / nd, d = rr - p * nd;
    vx[e] = in[(size_t)(s0 + sb) * nf + (size_t)xs[p] * nd + d];
  }
  __syncthreads();
  const int kc = threadIdx.x % nch, g = threadIdx.x / nch;
  C acc0[SB][VPC], acc1[SB][VPC];
#pragma unroll
  for (int sb = 0; sb < SB; ++sb)
#pragma unroll
    for (int u = 0; u < VPC; ++u) { acc0[sb][u] = C{0, 0}; acc1[sb][u] = C{0, 0}; }
  if (g < groups) {
#pragma unroll 2
    for (int rr = g; rr < npos * nd; rr += groups) {
      const int p = rr / nd, d = rr - p * nd;
      const int chi = t.chi_mode == 0 ? xpar[p] : (d >= half ? 1 : 0);
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(P + ((size_t)xs[p] * nd + d) * nv) + kc);
      const SL* pe = reinterpret_cast<const SL*>(&raw);
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) {
        if (sb >= ns) break;
        const C v = vx[(size_t)sb * npos * nd + rr];
#pragma unroll
        for (int u = 0; u < VPC; ++u) {
          const C pv = ld<R>(pe, u);
          if (chi == 0) cfmac(acc0[sb][u], pv, v);
          else cfmac(acc1[sb][u], pv, v);
        }
      }
    }
  }
  const int N = 2 * nv;
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) {
    if (sb >= ns) break;
    if (g < groups) {
#pragma unroll
      for (int u = 0; u < VPC; ++u) {
        part[((size_t)g * 2 + 0) * nv + kc * VPC + u] = acc0[sb][u];
        part[((size_t)g * 2 + 1) * nv + kc * VPC + u] = acc1[sb][u];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kRed * N; e += blockDim.x) {
      const int j = e / N, i = e - j * N;
      C sum = C{0, 0};
      for (int gg = j; gg < groups; gg += kRed) sum = cadd(sum, part[(size_t)gg * N + i]);
      red[(size_t)j * N + i] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      C sum = C{0, 0};
      for (int j = 0; j < kRed; ++j) sum = cadd(sum, red[(size_t)j * N + i]);
      out[(size_t)(s0 + sb) * t.coarse.V * N + (size_t)X * N + i] = cscale(sum, pscale);
    }
    __syncthreads();
  }
}

// e(x, d) = sum_k P_k(x, d) ec(X(x), chi(x, d), k) for SB systems per thread
// (blockIdx.y picks the group): the prolongator row is read once for all.
template <typename R, typename SL, int SB>
__global__ void prolong_kernel(typename cplx<R>::T* __restrict__ out, const typename cplx<R>::T* __restrict__ in,
                               const SL* __restrict__ P, R pscale, TransferGeom t, int nsys, const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nf = (long long)t.fine.V * t.ndof;
  if (e >= nf) return;
  const int s0 = blockIdx.y * SB;
  const int ns = min(SB, nsys - s0);
  const int x = (int)(e / t.ndof), d = (int)(e % t.ndof);
  const int X = coarse_of(t, x);
  const int chi = chirality(t, x, d);
  const int N = 2 * t.nvec;
  const size_t cstride = (size_t)t.coarse.V * N;
  const C* vc = in + (size_t)s0 * cstride + (size_t)X * N + chi * t.nvec;
  const SL* Px = P + (size_t)e * t.nvec;
  C acc[SB];
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) acc[sb] = C{0, 0};
#pragma unroll 4
  for (int k = 0; k < t.nvec; ++k) {
    const C pk = ld<R>(Px, k);
#pragma unroll
    for (int sb = 0; sb < SB; ++sb)
      if (sb < ns) cfma(acc[sb], pk, vc[sb * cstride + k]);
  }
#pragma unroll
  for (int sb = 0; sb < SB; ++sb)
    if (sb < ns) out[(size_t)(s0 + sb) * nf + e] = cscale(acc[sb], pscale);
}

// Restriction with one CTA per aggregate and SB systems: thread (g, k) owns
// coarse vector k and every groups-th row of the aggregate, keeps both
// chirality sums for each system in registers (the row's chirality is the
// same for the whole warp), and reads each prolongator entry once for all SB
// systems; the row groups are added at the end in a fixed order.
template <typename R, typename SL, int SB>
__global__ void __launch_bounds__(256) restrict_agg_kernel(typename cplx<R>::T* __restrict__ out,
                                                           const typename cplx<R>::T* __restrict__ in,
                                                           const SL* __restrict__ P, R pscale, TransferGeom t,
                                                           int nsys, const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char ra_smem[];
  const int nv = t.nvec, nd = t.ndof, half = nd / 2;
  const int groups = blockDim.x / nv;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  C* part = reinterpret_cast<C*>(ra_smem);                        // [groups][SB][2][nv]
  int* xs = reinterpret_cast<int*>(part + (size_t)groups * SB * 2 * nv);
  int* xpar = xs + npos;
  const int X = blockIdx.x, s0 = blockIdx.y * SB;
  const int ns = min(SB, nsys - s0);
  const long long nf = (long long)t.fine.V * nd;
  for (int p = threadIdx.x; p < npos; p += blockDim.x) {
    const int x = agg_site(t, X, p);
    xs[p] = x;
    xpar[p] = site_parity(t.fine, x);
  }
  __syncthreads();
  const int k = threadIdx.x % nv, g = threadIdx.x / nv;
  C acc0[SB], acc1[SB];
#pragma unroll
  for (int sb = 0; sb < SB; ++sb) { acc0[sb] = C{0, 0}; acc1[sb] = C{0, 0}; }
  if (g < groups) {
#pragma unroll 4
    for (int rr = g; rr < npos * nd; rr += groups) {
      const int p = rr / nd, d = rr - p * nd;
      const int chi = t.chi_mode == 0 ? xpar[p] : (d >= half ? 1 : 0);
      const size_t row = (size_t)xs[p] * nd + d;
      const C pv = ld<R>(P, row * nv + k);
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) {
        if (sb >= ns) break;
        const C v = in[(size_t)(s0 + sb) * nf + row];
        if (chi == 0) cfmac(acc0[sb], pv, v);
        else cfmac(acc1[sb], pv, v);
      }
    }
#pragma unroll
    for (int sb = 0; sb < SB; ++sb) {
      part[(((size_t)g * SB + sb) * 2 + 0) * nv + k] = acc0[sb];
      part[(((size_t)g * SB + sb) * 2 + 1) * nv + k] = acc1[sb];
    }
  }
  __syncthreads();
  const int N = 2 * nv;
  for (int e = threadIdx.x; e < ns * N; e += blockDim.x) {
    const int sb = e / N, i = e - sb * N;                     // i = chi * nv + k
    C sum = C{0, 0};
    for (int gg = 0; gg < groups; ++gg) sum = cadd(sum, part[((size_t)gg * SB + sb) * N + i]);
    out[(size_t)(s0 + sb) * t.coarse.V * N + (size_t)X * N + i] = cscale(sum, pscale);
  }
}

// Prolongation with one CTA per aggregate and SB systems: the aggregate's
// coarse components of the SB systems are staged in shared memory, each
// thread takes rows of the aggregate and reads its prolongator row with
// 16-byte loads, once for all SB systems.
template <typename R, typename SL, int SB>
__global__ void __launch_bounds__(256) prolong_agg_kernel(typename cplx<R>::T* __restrict__ out,
                                                          const typename cplx<R>::T* __restrict__ in,
                                                          const SL* __restrict__ P, R pscale, TransferGeom t,
                                                          int nsys, const int* run) {
  using C = typename cplx<R>::T;
  constexpr int VPC = 16 / (int)sizeof(SL);
  if (run != nullptr && *run == 0) return;
  extern __shared__ __align__(16) unsigned char pa_smem[];
  const int nv = t.nvec, nd = t.ndof, half = nd / 2, N = 2 * nv;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  C* ec = reinterpret_cast<C*>(pa_smem);                          // [SB][2 nv]
  int* xs = reinterpret_cast<int*>(ec + (size_t)SB * N);
  int* xpar = xs + npos;
  const int X = blockIdx.x, s0 = blockIdx.y * SB;
  const int ns = min(SB, nsys - s0);
  const long long nf = (long long)t.fine.V * nd;
  for (int e = threadIdx.x; e < ns * N; e += blockDim.x) {
    const int sb = e / N, i = e - sb * N;
    ec[e] = in[(size_t)(s0 + sb) * t.coarse.V * N + (size_t)X * N + i];
  }
  for (int p = threadIdx.x; p < npos; p += blockDim.x) {
    const int x = agg_site(t, X, p);
    xs[p] = x;
    xpar[p] = site_parity(t.fine, x);
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < npos * nd; rr += blockDim.x) {
    const int p = rr / nd, d = rr - p * nd;
    const int chi = t.chi_mode == 0 ? xpar[p] : (d >= half ? 1 : 0);
    const size_t row = (size_t)xs[p] * nd + d;
    const uint4* Pr = reinterpret_cast<const uint4*>(P + row * nv);
    C acc[SB];
#pragma unroll
    for (int sb = 0; sb < SB; ++sb) acc[sb] = C{0, 0};
    for (int kc = 0; kc < nv / VPC; ++kc) {
      const uint4 raw = __ldg(Pr + kc);
      const SL* pe = reinterpret_cast<const SL*>(&raw);
#pragma unroll
      for (int u = 0; u < VPC; ++u) {
        const C pk = ld<R>(pe, u);
        const int kk = chi * nv + kc * VPC + u;
#pragma unroll
        for (int sb = 0; sb < SB; ++sb)
          if (sb < ns) cfma(acc[sb], pk, ec[(size_t)sb * N + kk]);
      }
    }
#pragma unroll
    for (int sb = 0; sb < SB; ++sb)
      if (sb < ns) out[(size_t)(s0 + sb) * nf + row] = cscale(acc[sb], pscale);
  }
}

// Raise a kernel's dynamic shared-memory limit once (not a stream operation,
// so it is never issued while a stream is being captured).
template <typename K>
void ensure_smem(K kernel, size_t bytes) {
  static std::vector<std::pair<const void*, size_t>> set;
  if (bytes <= 48 * 1024) return;
  for (auto& e : set)
    if (e.first == (const void*)kernel) {
      if (bytes <= e.second) return;
      SMG_CUDA_OK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      e.second = bytes;
      return;
    }
  SMG_CUDA_OK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  set.emplace_back((const void*)kernel, bytes);
}

}  // namespace

void block_orthonormalize(double2* raw, const TransferGeom& t, cudaStream_t st) {
  orthonormalize_kernel<<<dim3(t.coarse.V, 2), 256, 0, st>>>(raw, t);
  SMG_LAUNCH_OK();
}

void transfer_pack(Stored& dst, const double2* raw, const TransferGeom& t, cudaStream_t st) {
  const long long total = (long long)t.fine.V * t.nvec * t.ndof;
  unsigned grid = ceil_div(total, 256);
  if (grid > 8192) grid = 8192;
  dst.gscale = 1.0f;   // orthonormal columns: every entry has modulus <= 1
  if (dst.s == S64) transfer_pack_kernel<double2><<<grid, 256, 0, st>>>((double2*)dst.p, raw, t);
  else if (dst.s == S32) transfer_pack_kernel<float2><<<grid, 256, 0, st>>>((float2*)dst.p, raw, t);
  else transfer_pack_kernel<__half2><<<grid, 256, 0, st>>>((__half2*)dst.p, raw, t);
  SMG_LAUNCH_OK();
}

namespace {
// the restrict kernels for SB systems per CTA; false when the shared memory
// of the vectorised kernel does not fit (the caller then takes the plain one)
template <int SB>
bool launch_restrict_vec(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                         const int* run) {
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const size_t cb = prec_bytes(in.prec);
  const int vpc = (int)(16 / store_bytes(P.s));
  if (t.nvec % vpc != 0) return false;
  const int groups = 512 / (t.nvec / vpc);
  const size_t smem = cb * ((size_t)groups * 2 * t.nvec + 8 * 2 * t.nvec + (size_t)SB * npos * t.ndof) +
                      sizeof(int) * 2 * npos;
  if (smem > 200 * 1024) return false;
  dim3 grid(t.coarse.V, ceil_div(in.nsys, SB));
  if (in.prec == P64) {
    SMG_REQUIRE(P.s == S64, "restrict: FP64 vectors need FP64 prolongator");
    auto k = restrict_vec_kernel<double, double2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(512), smem, st, (double2*)out.p, (const double2*)in.p, (const double2*)P.p,
             (double)P.gscale, t, in.nsys, run);
  } else if (P.s == S32) {
    auto k = restrict_vec_kernel<float, float2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(512), smem, st, (float2*)out.p, (const float2*)in.p, (const float2*)P.p, P.gscale, t,
             in.nsys, run);
  } else {
    SMG_REQUIRE(P.s == S16, "restrict: unsupported storage");
    auto k = restrict_vec_kernel<float, __half2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(512), smem, st, (float2*)out.p, (const float2*)in.p, (const __half2*)P.p, P.gscale, t,
             in.nsys, run);
  }
  SMG_LAUNCH_OK();
  return true;
}

bool restrict_vec_sb(int sb, const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                     const int* run) {
  switch (sb) {
    case 1: return launch_restrict_vec<1>(out, in, t, P, st, run);
    case 2: return launch_restrict_vec<2>(out, in, t, P, st, run);
    case 4: return launch_restrict_vec<4>(out, in, t, P, st, run);
    default: return launch_restrict_vec<8>(out, in, t, P, st, run);
  }
}

template <int SB>
void launch_prolong(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                    const int* run) {
  dim3 grid(ceil_div(out.n, 256), ceil_div(in.nsys, SB));
  if (in.prec == P64) {
    SMG_REQUIRE(P.s == S64, "prolong: FP64 vectors need FP64 prolongator");
    launch_k(prolong_kernel<double, double2, SB>, grid, dim3(256), 0, st, (double2*)out.p, (const double2*)in.p,
             (const double2*)P.p, (double)P.gscale, t, in.nsys, run);
  } else if (P.s == S32) {
    launch_k(prolong_kernel<float, float2, SB>, grid, dim3(256), 0, st, (float2*)out.p, (const float2*)in.p,
             (const float2*)P.p, P.gscale, t, in.nsys, run);
  } else {
    SMG_REQUIRE(P.s == S16, "prolong: unsupported storage");
    launch_k(prolong_kernel<float, __half2, SB>, grid, dim3(256), 0, st, (float2*)out.p, (const float2*)in.p,
             (const __half2*)P.p, P.gscale, t, in.nsys, run);
  }
  SMG_LAUNCH_OK();
}

void prolong_sb(int sb, const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                const int* run) {
  switch (sb) {
    case 1: launch_prolong<1>(out, in, t, P, st, run); break;
    case 2: launch_prolong<2>(out, in, t, P, st, run); break;
    case 4: launch_prolong<4>(out, in, t, P, st, run); break;
    default: launch_prolong<8>(out, in, t, P, st, run); break;
  }
}

const char* sb_name(int sb) {
  return sb == 1 ? "1 system/CTA" : sb == 2 ? "2 systems/CTA" : sb == 4 ? "4 systems/CTA" : "8 systems/CTA";
}

// candidate ids of the aggregate kernels: 16 + systems per CTA
const char* agg_name(int sb) {
  return sb == 1 ? "aggregate CTA, 1 system" : sb == 2 ? "aggregate CTA, 2 systems"
                                            : sb == 4 ? "aggregate CTA, 4 systems" : "aggregate CTA, 8 systems";
}

template <int SB>
size_t restrict_agg_smem(const TransferGeom& t, size_t cb) {
  const int groups = 256 / t.nvec;
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  return cb * (size_t)groups * SB * 2 * t.nvec + sizeof(int) * 2 * npos;
}

template <int SB>
void launch_restrict_agg(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                         const int* run) {
  const size_t smem = restrict_agg_smem<SB>(t, prec_bytes(in.prec));
  dim3 grid(t.coarse.V, ceil_div(in.nsys, SB));
  if (in.prec == P64) {
    SMG_REQUIRE(P.s == S64, "restrict: FP64 vectors need FP64 prolongator");
    auto k = restrict_agg_kernel<double, double2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(256), smem, st, (double2*)out.p, (const double2*)in.p, (const double2*)P.p,
             (double)P.gscale, t, in.nsys, run);
  } else if (P.s == S32) {
    auto k = restrict_agg_kernel<float, float2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const float2*)P.p, P.gscale, t,
             in.nsys, run);
  } else {
    SMG_REQUIRE(P.s == S16, "restrict: unsupported storage");
    auto k = restrict_agg_kernel<float, __half2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const __half2*)P.p, P.gscale, t,
             in.nsys, run);
  }
  SMG_LAUNCH_OK();
}

void restrict_agg_sb(int sb, const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                     const int* run) {
  switch (sb) {
    case 1: launch_restrict_agg<1>(out, in, t, P, st, run); break;
    case 2: launch_restrict_agg<2>(out, in, t, P, st, run); break;
    case 4: launch_restrict_agg<4>(out, in, t, P, st, run); break;
    default: launch_restrict_agg<8>(out, in, t, P, st, run); break;
  }
}

template <int SB>
void launch_prolong_agg(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                        const int* run) {
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const size_t smem = prec_bytes(in.prec) * (size_t)SB * 2 * t.nvec + sizeof(int) * 2 * npos;
  dim3 grid(t.coarse.V, ceil_div(in.nsys, SB));
  if (in.prec == P64) {
    SMG_REQUIRE(P.s == S64, "prolong: FP64 vectors need FP64 prolongator");
    auto k = prolong_agg_kernel<double, double2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(256), smem, st, (double2*)out.p, (const double2*)in.p, (const double2*)P.p,
             (double)P.gscale, t, in.nsys, run);
  } else if (P.s == S32) {
    auto k = prolong_agg_kernel<float, float2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const float2*)P.p, P.gscale, t,
             in.nsys, run);
  } else {
    SMG_REQUIRE(P.s == S16, "prolong: unsupported storage");
    auto k = prolong_agg_kernel<float, __half2, SB>;
    ensure_smem(k, smem);
    launch_k(k, grid, dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const __half2*)P.p, P.gscale, t,
             in.nsys, run);
  }
  SMG_LAUNCH_OK();
}

void prolong_agg_sb(int sb, const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                    const int* run) {
  switch (sb) {
    case 1: launch_prolong_agg<1>(out, in, t, P, st, run); break;
    case 2: launch_prolong_agg<2>(out, in, t, P, st, run); break;
    case 4: launch_prolong_agg<4>(out, in, t, P, st, run); break;
    default: launch_prolong_agg<8>(out, in, t, P, st, run); break;
  }
}

// whether the aggregate kernels serve a transfer: whole nvec-wide thread rows
// in a CTA of 256, 16-byte prolongator rows
bool agg_kernels_ok(const TransferGeom& t, const Stored& P) {
  const int vpc = (int)(16 / store_bytes(P.s));
  return t.nvec >= 1 && t.nvec <= 256 && t.nvec % vpc == 0;
}

// the autotuner's choice of systems per CTA for one transfer launch
// candidate id of the tensor-core kernels
constexpr int kMmaId = 32;

template <class F>
int pick_sb(const char* family, const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P,
            cudaStream_t st, F&& launch, bool with_agg, bool with_mma) {
  std::vector<TuneCandidate> cands;
  for (int sb : {1, 2, 4, 8})
    if (sb == 1 || sb < 2 * in.nsys) cands.push_back({sb, sb_name(sb)});
  if (with_agg)
    for (int sb : {1, 2, 4, 8})
      if (sb == 1 || sb < 2 * in.nsys) cands.push_back({16 + sb, agg_name(sb)});
  if (with_mma) cands.push_back({kMmaId, "tensor cores, 16 systems/CTA"});
  if (cands.size() == 1) return cands[0].id;
  char key[192];
  std::snprintf(key, sizeof(key), "%s V=%d nvec=%d ndof=%d nsys=%d vec=%s store=%s", family, t.fine.V, t.nvec,
                t.ndof, in.nsys, in.prec == P64 ? "f64" : "f32",
                P.s == S16 ? "f16" : (P.s == S32 ? "f32" : "f64"));
  struct Scratch {
    void* p = nullptr;
    ~Scratch() { if (p) cudaFree(p); }
  } scratch;
  return tune_pick(key, cands, st, [&](int id) {
    if (scratch.p == nullptr) SMG_CUDA_OK(cudaMalloc(&scratch.p, out.bytes()));
    Vec o = out;
    o.p = scratch.p;
    launch(id, o);
  });
}
}  // namespace

void restrict_op(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                 const int* run) {
  SMG_REQUIRE(in.n == (long long)t.fine.V * t.ndof && out.n == (long long)t.coarse.V * 2 * t.nvec,
              "restrict: field sizes do not match the transfer");
  SMG_REQUIRE(in.nsys == out.nsys && in.prec == out.prec && t.nvec <= 128, "restrict: batch/precision mismatch");
  const int npos = t.agg[0] * t.agg[1] * t.agg[2] * t.agg[3];
  const size_t cb = prec_bytes(in.prec);
  const int vpc = (int)(16 / store_bytes(P.s));
  const bool mma = transfer_mma_ok(t, P, in.prec);
  if (t.nvec % vpc == 0 || mma) {
    // vectorised kernel: 512 threads, nvec / vpc threads per row; systems per
    // CTA by the autotuner among the group sizes whose shared memory fits
    const int groups = 512 / (t.nvec / vpc);
    auto fits = [&](int sb) {
      return cb * ((size_t)groups * 2 * t.nvec + 8 * 2 * t.nvec + (size_t)sb * npos * t.ndof) +
                 sizeof(int) * 2 * npos <= 200 * 1024;
    };
    if (fits(1) || mma) {
      const bool agg = agg_kernels_ok(t, P);
      const bool vec = t.nvec % vpc == 0 && fits(1);
      auto go = [&](int id, const Vec& o, const int* rr) {
        if (id == kMmaId) restrict_mma(o, in, t, P, st, rr);
        else if (id >= 16) restrict_agg_sb(id - 16, o, in, t, P, st, rr);
        else if (!vec) restrict_agg_sb(id, o, in, t, P, st, rr);
        else if (!fits(id) || !restrict_vec_sb(id, o, in, t, P, st, rr)) restrict_vec_sb(1, o, in, t, P, st, rr);
      };
      const int id = pick_sb("restrict", out, in, t, P, st, [&](int cid, const Vec& o) { go(cid, o, nullptr); }, agg,
                             mma);
      go(id, out, run);
      return;
    }
  }
  dim3 grid(t.coarse.V, in.nsys);
  const size_t smem = cb * (512 + (size_t)npos * t.ndof) + sizeof(int) * 2 * npos;
  SMG_REQUIRE(smem <= 200 * 1024, "restrict: aggregate too large for shared memory");
  if (in.prec == P64) {
    SMG_REQUIRE(P.s == S64, "restrict: FP64 vectors need FP64 prolongator");
    auto k = restrict_kernel<double, double2>;
    ensure_smem(k, smem);
    launch_k(k, dim3(grid), dim3(256), smem, st, (double2*)out.p, (const double2*)in.p, (const double2*)P.p, (double)P.gscale, t, run);
  } else if (P.s == S32) {
    auto k = restrict_kernel<float, float2>;
    ensure_smem(k, smem);
    launch_k(k, dim3(grid), dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const float2*)P.p, P.gscale, t, run);
  } else {
    SMG_REQUIRE(P.s == S16, "restrict: unsupported storage");
    auto k = restrict_kernel<float, __half2>;
    ensure_smem(k, smem);
    launch_k(k, dim3(grid), dim3(256), smem, st, (float2*)out.p, (const float2*)in.p, (const __half2*)P.p, P.gscale, t, run);
  }
  SMG_LAUNCH_OK();
}

void prolong_op(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                const int* run) {
  SMG_REQUIRE(out.n == (long long)t.fine.V * t.ndof && in.n == (long long)t.coarse.V * 2 * t.nvec,
              "prolong: field sizes do not match the transfer");
  SMG_REQUIRE(in.nsys == out.nsys && in.prec == out.prec, "prolong: batch/precision mismatch");
  const bool agg = agg_kernels_ok(t, P);
  const bool mma = transfer_mma_ok(t, P, in.prec);
  auto go = [&](int id, const Vec& o, const int* rr) {
    if (id == kMmaId) prolong_mma(o, in, t, P, st, rr);
    else if (id >= 16) prolong_agg_sb(id - 16, o, in, t, P, st, rr);
    else prolong_sb(id, o, in, t, P, st, rr);
  };
  const int id = pick_sb("prolong", out, in, t, P, st, [&](int cid, const Vec& o) { go(cid, o, nullptr); }, agg,
                         mma);
  go(id, out, run);
}

}  // namespace smg
