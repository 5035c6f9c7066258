// Multi-RHS coarse apply on the 5th-generation tensor cores (tcgen05 + TMA).
//
// Per coarse site the apply is the real GEMM D[128][32] = A[128][18N] B[18N][32]
// (N = 128 components per site): A is the FP16 stencil as stored (a site's
// 128 rows of 9N complex entries, (re, im) pairs along K), B the gathered
// neighbour vectors of up to 16 systems embedded as real 2x2 blocks (columns
// 2r, 2r+1 give Re, Im of system r), scaled per site and system by a power of
// two that puts the largest entry in [0.5, 1).
//
// One persistent CTA of four warps per SM slot walks the sites:
//   warp 0 lane 0  TMA producer: 128 x 64 FP16 stencil tiles (128-byte
//                  swizzle) into a 4-stage ring, completion on mbarriers;
//   warp 1 lane 0  MMA issuer: four tcgen05.mma (M=128, N=32, K=16, FP32
//                  accumulate in 32 TMEM columns) per stage, tcgen05.commit
//                  frees the stage;
//   warps 2..7     build the matching 32 x 64 FP16 B tile (same swizzle) of
//                  each stage from the FP32 vectors (float4 loads, the next
//                  chunk's loads issued before the current one is converted);
//   all warps      per-site scale before the K loop (the largest entry over
//                  the nine neighbours, from per-site maxima that a prepass
//                  kernel writes), and the epilogue:
//                  tcgen05.ld of the 128 x 32 accumulator (warp w owns TMEM
//                  lanes 32(w%4).. = rows and 16 of the 32 columns), row
//                  scale, 1/sigma.
// Every mbarrier wait is bounded (1 s of %globaltimer): on expiry the CTA
// sets the error word, lets its outstanding copies and MMAs drain (again
// bounded), frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>

#include "ops.cuh"

namespace smg {
namespace {

constexpr int UM = 128;          // GEMM rows = components per coarse site
constexpr int UN = 32;           // GEMM columns = 2 x 16 systems
constexpr int UKC = 64;          // FP16 K elements per stage (one 128-byte swizzle row)
constexpr int A_BYTES = UM * UKC * 2;   // 16 KiB
constexpr int B_BYTES = UN * UKC * 2;   // 4 KiB
constexpr int UTHREADS = 256;
constexpr int NBUILD = UTHREADS - 64;   // warps 2..7 build the B tiles
constexpr int kMaxRhsU = 16;

template <int STAGES>
struct UmmaSmem {
  uint8_t a[STAGES][A_BYTES];
  uint8_t b[STAGES][B_BYTES];
  unsigned long long full_a[STAGES], full_b[STAGES], empty[STAGES], done, drain;
  unsigned tmem_base;
  int err;
  int zero;                        // never written after init: a plain time limit for drain waits
  float sig[kMaxRhsU];
  unsigned vmax[kMaxRhsU];
  int nb[9];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, volatile int* err,
                                          unsigned long long limit_ns = 1000000000ull) {
  const unsigned a = smem_u32(b);
  const unsigned long long t0 = gtimer();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*err != 0 || gtimer() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// K-major operand, 128-byte swizzle, rows 128 bytes apart, 8-row groups 1024 bytes apart.
__device__ __forceinline__ unsigned long long umma_desc(const void* p) {
  const unsigned a = smem_u32(p);
  unsigned long long d = 0;
  d |= (unsigned long long)((a & 0x3FFFF) >> 4);
  d |= (unsigned long long)1 << 16;                  // leading byte offset (16 B; unused with swizzle)
  d |= (unsigned long long)(1024 >> 4) << 32;        // stride byte offset
  d |= (unsigned long long)1 << 46;                  // descriptor version
  d |= (unsigned long long)2 << 61;                  // 128-byte swizzle
  return d;
}
// kind::f16 instruction: FP32 accumulate, FP16 A and B, both K-major, M = 128, N = 32.
constexpr unsigned kIdesc = (1u << 4) | ((unsigned)(UN >> 3) << 17) | ((unsigned)(UM >> 4) << 24);

__device__ __forceinline__ void umma_f16(unsigned tmem, unsigned long long ad, unsigned long long bd, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ unsigned pack_h2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&h);
}

// smax[s][X] = max |Re|, |Im| of the N components of system s at site X:
// one warp per (site, system), 16-byte loads.
__global__ void __launch_bounds__(256) site_max_kernel(const float2* __restrict__ in, int nsys, int V, int N,
                                                       long long sys_stride, float* __restrict__ smax,
                                                       const int* run) {
  if (run != nullptr && *run == 0) return;
  const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= (long long)V * nsys) return;
  const int s = (int)(w / V), X = (int)(w - (long long)s * V);
  const float4* v = reinterpret_cast<const float4*>(in + (size_t)s * sys_stride + (size_t)X * N);
  float m = 0.f;
  for (int q = lane; q < N / 2; q += 32) {
    const float4 a = v[q];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) smax[(size_t)s * V + X] = m;
}

template <int STAGES>
__global__ void __launch_bounds__(UTHREADS, 1) coarse_umma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  float2* __restrict__ out,
                                                                  const float2* __restrict__ in,
                                                                  const float* __restrict__ rs, Geom g, int nsys,
                                                                  int s0, long long sys_stride,
                                                                  const float2* __restrict__ sub_from,
                                                                  const float* __restrict__ smax,
                                                                  int* __restrict__ gerr, const int* run) {
  if (run != nullptr && *run == 0) return;
  extern __shared__ unsigned char umma_raw[];
  UmmaSmem<STAGES>& sm = *reinterpret_cast<UmmaSmem<STAGES>*>(
      (unsigned char*)(((unsigned long long)umma_raw + 1023) & ~1023ull));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int N = UM;
  const int nrhs = min(kMaxRhsU, nsys - s0);
  const int nchunk = 9 * N * 2 / UKC;   // 36
  volatile int* err = &sm.err;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sm.full_a[s], 1);
      mbar_init(&sm.full_b[s], NBUILD);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.done, 1);
    mbar_init(&sm.drain, 1);
    sm.err = 0;
    sm.zero = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = sm.tmem_base;

  int site_iter = 0;
  long long it0 = 0;                  // stage uses issued so far (identical in every role)
  long long last_round[STAGES];       // producer: last round copied into each stage
#pragma unroll
  for (int s = 0; s < STAGES; ++s) last_round[s] = -1;
  for (int X = blockIdx.x; X < g.V && *err == 0; X += gridDim.x, ++site_iter, it0 += nchunk) {
    // ---- per-site scales and neighbours
    if (tid < 9) {
      int c[4];
      g.coords(X, c);
      sm.nb[tid] = tid == 0 ? X : g.shift(c, (tid - 1) >> 1, ((tid - 1) & 1) ? -1 : 1);
    }
    if (tid < kMaxRhsU) sm.vmax[tid] = 0u;
    __syncthreads();
    // the largest |Re|, |Im| over the nine neighbours, from the per-site
    // maxima of the prepass (one load per system and direction)
    for (int e = tid; e < nrhs * 9; e += UTHREADS) {
      const int r = e / 9, dir = e - 9 * r;
      atomicMax(&sm.vmax[r], __float_as_uint(smax[(size_t)(s0 + r) * g.V + sm.nb[dir]]));
    }
    __syncthreads();
    if (tid < kMaxRhsU) {
      const float m = tid < nrhs ? __uint_as_float(sm.vmax[tid]) : 0.f;
      int e2 = 0;
      if (m > 0.f) frexpf(m, &e2);
      sm.sig[tid] = ldexpf(1.f, -e2);
    }
    __syncthreads();
    // ---- pipelined K loop
    if (warp == 0) {
      if (lane == 0) {
        for (int c = 0; c < nchunk; ++c) {
          const long long i = it0 + c;
          const int s = (int)(i % STAGES);
          const long long round = i / STAGES;
          if (round > 0 && !mbar_wait(&sm.empty[s], (unsigned)((round - 1) & 1), err)) { atomicExch((int*)err, 1); break; }
          mbar_expect_tx(&sm.full_a[s], A_BYTES);
          tma_load_2d(sm.a[s], &tmap, c * UKC, X * UM, &sm.full_a[s]);
          last_round[s] = round;
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        for (int c = 0; c < nchunk; ++c) {
          const long long i = it0 + c;
          const int s = (int)(i % STAGES);
          const unsigned par = (unsigned)((i / STAGES) & 1);
          if (!mbar_wait(&sm.full_a[s], par, err) || !mbar_wait(&sm.full_b[s], par, err)) {
            atomicExch((int*)err, 1);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int kk = 0; kk < UKC / 16; ++kk)
            umma_f16(tmem, umma_desc(sm.a[s] + kk * 32), umma_desc(sm.b[s] + kk * 32), (c > 0 || kk > 0) ? 1u : 0u);
          umma_commit(&sm.empty[s]);
        }
        umma_commit(&sm.done);
      }
    } else {
      // B tile of chunk c: rows n = 2r + im (32), 64 FP16 along K = 32 complex
      // entries jj = 32c + 0..31; 16-byte granules (4 complex) at swizzled
      // slots.  Builder thread bt < 128 owns system r = bt / 8 and granule
      // column cc = bt % 8 of every chunk: one pair of 16-byte loads feeds both
      // rows (Re and Im) of its system, and the loads of chunk c + 1 are issued
      // before chunk c is converted, so two chunks' reads are in flight.
      const int bt = tid - 64;
      const bool owns = bt < kMaxRhsU * 8;
      const int r = bt >> 3, cc = bt & 7;
      const bool live = owns && r < nrhs;
      float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
      auto fetch = [&](int c) {
        if (!live) return;
        const int jj = 32 * c + 4 * cc;                     // 4 complex, never across a direction (N % 4 == 0)
        const int dir = jj / N, j = jj - dir * N;
        const float4* src =
            reinterpret_cast<const float4*>(in + (size_t)(s0 + r) * sys_stride + (size_t)sm.nb[dir] * N + j);
        q0 = src[0];
        q1 = src[1];
      };
      fetch(0);
      for (int c = 0; c < nchunk; ++c) {
        const long long i = it0 + c;
        const int s = (int)(i % STAGES);
        const long long round = i / STAGES;
        const float4 p0 = q0, p1 = q1;
        if (c + 1 < nchunk) fetch(c + 1);
        if (round > 0 && !mbar_wait(&sm.empty[s], (unsigned)((round - 1) & 1), err)) { atomicExch((int*)err, 1); break; }
        if (owns) {
          const float sg = live ? sm.sig[r] : 0.f;
          const float re[4] = {p0.x * sg, p0.z * sg, p1.x * sg, p1.z * sg};
          const float ii[4] = {p0.y * sg, p0.w * sg, p1.y * sg, p1.w * sg};
          unsigned wr[4], wi[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            wr[q] = pack_h2(re[q], -ii[q]);   // row 2r:     (Re, -Im)
            wi[q] = pack_h2(ii[q], re[q]);    // row 2r + 1: (Im,  Re)
          }
          const int n0 = 2 * r, n1 = 2 * r + 1;
          *reinterpret_cast<uint4*>(sm.b[s] + n0 * 128 + ((cc ^ (n0 & 7)) << 4)) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
          *reinterpret_cast<uint4*>(sm.b[s] + n1 * 128 + ((cc ^ (n1 & 7)) << 4)) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&sm.full_b[s]);
      }
    }
    // ---- epilogue: warp w reads TMEM lanes 32w..32w+31 (rows)
    bool ok = mbar_wait(&sm.done, (unsigned)(site_iter & 1), err);
    ok = __all_sync(0xffffffffu, ok && *err == 0);   // warp-uniform: tcgen05.ld is .sync.aligned
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      float d[16];
      const int quarter = warp & 3, half = warp >> 2;      // TMEM lanes 32*quarter.., columns 16*half..
      tmem_ld16(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(16 * half), d);
      const int row = quarter * 32 + lane;
      const float sc = rs[(size_t)X * N + row];
      for (int q = 0; q < 8; ++q) {
        const int r = 8 * half + q;
        if (r >= nrhs) break;
        const float f = sc / sm.sig[r];
        const size_t o = (size_t)(s0 + r) * sys_stride + (size_t)X * N + row;
        float2 v = make_float2(d[2 * q] * f, d[2 * q + 1] * f);
        if (sub_from != nullptr) v = csub(sub_from[o], v);
        out[o] = v;
      }
    } else {
      atomicExch((int*)err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // ---- teardown: on error let outstanding copies and MMAs finish (bounded), then free TMEM
  if (*err != 0) {
    volatile int* never = &sm.zero;
    if (tid == 32) {   // the MMA issuer: everything it issued has completed once `drain` fires
      umma_commit(&sm.drain);
      mbar_wait(&sm.drain, 0u, never);
    }
    if (tid == 0) {    // the producer: the last copy into each stage has landed
      for (int s = 0; s < STAGES; ++s)
        if (last_round[s] >= 0) mbar_wait(&sm.full_a[s], (unsigned)(last_round[s] & 1), never);
      atomicExch(gerr, 1);
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    SMG_CUDA_OK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    SMG_REQUIRE(q == cudaDriverEntryPointSuccess && p != nullptr, "cuTensorMapEncodeTiled unavailable");
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

bool coarse_umma_ok(const Vec& in, const CoarseParams& p, const Stored& S) {
  return in.prec == P32 && S.s == S16 && S.scale != nullptr && p.part < 0 && p.N == UM && in.nsys >= 2;
}

int* coarse_umma_err() {
  static int* err[64] = {};
  int dev = 0;
  SMG_CUDA_OK(cudaGetDevice(&dev));
  SMG_REQUIRE(dev >= 0 && dev < 64, "coarse_apply_umma: device ordinal out of range");
  if (err[dev] == nullptr) {
    SMG_CUDA_OK(cudaMalloc(&err[dev], sizeof(int)));
    SMG_CUDA_OK(cudaMemset(err[dev], 0, sizeof(int)));
    SMG_CUDA_OK(cudaDeviceSynchronize());
  }
  return err[dev];
}

bool coarse_umma_err_read_and_clear(cudaStream_t st) {
  int* e = coarse_umma_err();
  int h = 0;
  SMG_CUDA_OK(cudaMemcpyAsync(&h, e, sizeof(int), cudaMemcpyDeviceToHost, st));
  SMG_CUDA_OK(cudaStreamSynchronize(st));
  if (h != 0) {
    SMG_CUDA_OK(cudaMemsetAsync(e, 0, sizeof(int), st));
    SMG_CUDA_OK(cudaStreamSynchronize(st));
  }
  return h != 0;
}

namespace {
// Grow-only device buffer of per-site maxima (one per device; sized by the
// first, uncaptured call of a shape, so that a graph capture never allocates).
float* site_max_buffer(size_t n, cudaStream_t st) {
  static float* buf[64] = {};
  static size_t cap[64] = {};
  int dev = 0;
  SMG_CUDA_OK(cudaGetDevice(&dev));
  SMG_REQUIRE(dev >= 0 && dev < 64, "coarse_apply_umma: device ordinal out of range");
  if (cap[dev] < n) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SMG_CUDA_OK(cudaStreamIsCapturing(st, &cs));
    SMG_REQUIRE(cs == cudaStreamCaptureStatusNone,
                "coarse_apply_umma: a new batch shape met inside a graph capture (run it once uncaptured first)");
    if (buf[dev] != nullptr) {
      SMG_CUDA_OK(cudaDeviceSynchronize());
      SMG_CUDA_OK(cudaFree(buf[dev]));
      buf[dev] = nullptr;
    }
    SMG_CUDA_OK(cudaMalloc(&buf[dev], n * sizeof(float)));
    cap[dev] = n;
  }
  return buf[dev];
}

template <int STAGES>
void launch_umma(const CUtensorMap& map, const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S,
                 int* err, cudaStream_t st, const int* run, int grid) {
  const size_t smem = sizeof(UmmaSmem<STAGES>) + 1024;
  static bool attr = false;
  if (!attr) {
    SMG_CUDA_OK(cudaFuncSetAttribute(coarse_umma_kernel<STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    attr = true;
  }
  float* smax = site_max_buffer((size_t)in.nsys * p.g.V, st);
  const long long pairs = (long long)in.nsys * p.g.V;
  site_max_kernel<<<(unsigned)((pairs + 7) / 8), 256, 0, st>>>((const float2*)in.p, in.nsys, p.g.V, p.N, in.n, smax,
                                                              run);
  SMG_LAUNCH_OK();
  for (int s0 = 0; s0 < in.nsys; s0 += kMaxRhsU) {
    coarse_umma_kernel<STAGES><<<grid, UTHREADS, smem, st>>>(map, (float2*)out.p, (const float2*)in.p, S.scale, p.g,
                                                             in.nsys, s0, in.n, (const float2*)p.sub_from, smax, err,
                                                             run);
    SMG_LAUNCH_OK();
  }
}
}  // namespace

// err: device int, set to 1 if a CTA gave up on a wait (host reads it).
// ctas_per_sm: persistent CTAs per SM (1 or 2); stages: depth of the stencil
// ring (4 or 6; 6 stages leave room for one CTA per SM only).
void coarse_apply_umma(const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S, int* err,
                       cudaStream_t st, const int* run, int ctas_per_sm, int stages) {
  SMG_REQUIRE(coarse_umma_ok(in, p, S), "coarse_apply_umma: unsupported shape or precision");
  SMG_REQUIRE(((unsigned long long)S.p & 15ull) == 0, "coarse_apply_umma: stencil not 16-byte aligned");
  SMG_REQUIRE((ctas_per_sm == 1 || ctas_per_sm == 2) && (stages == 4 || stages == 6) &&
                  !(stages == 6 && ctas_per_sm == 2),
              "coarse_apply_umma: 1 or 2 CTAs per SM, 4 or 6 stages (6 with one CTA per SM)");
  // 2D view of the stencil: K = 18N FP16 per row (innermost), rows = Vc * N
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)18 * UM, (cuuint64_t)p.g.V * UM};
  const cuuint64_t gstride[1] = {(cuuint64_t)18 * UM * 2};
  const cuuint32_t box[2] = {UKC, UM};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, S.p, gdim, gstride, box, estride,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  SMG_REQUIRE(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed for the coarse stencil");
  int dev = 0, sms = 0;
  SMG_CUDA_OK(cudaGetDevice(&dev));
  SMG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::min(p.g.V, ctas_per_sm * sms);
  if (stages == 4) launch_umma<4>(map, out, in, p, S, err, st, run, grid);
  else launch_umma<6>(map, out, in, p, S, err, st, run, grid);
}

}  // namespace smg
