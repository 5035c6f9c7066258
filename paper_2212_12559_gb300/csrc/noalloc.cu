// Batched inner products that allocate nothing.
//
// The library's own reductions keep their per-CTA partial sums in device
// memory that the solver context allocates.  Some callers cannot afford any
// allocation on the call path: a framework whose caching allocator has
// reserved the whole device heap, or a latency-critical loop (an HMC
// trajectory, say) in which the implicit device-wide synchronisation of
// cudaMalloc/cudaFree is not acceptable.  This variant of the reduction keeps
// its scratch in a fixed file-scope device array instead.
//
// Scratch: kNoAllocPartials FP64 complex partial sums plus one arrival
// counter, 128 KiB + 256 B per device, held by every GPU that loads the
// library until the process exits.  A call needs nsys * nb partial sums,
// nb = number of CTAs per system, so nsys <= kNoAllocPartials.
//
// Host code cannot use the array's name as a device address (it is a host
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress, with that device current, and caches it.  That
// first call should therefore come before any stream capture.
//
// Every call shares the array: the arrival counter is cleared at the start of
// each call (cudaMemsetAsync on the call's stream), and calls that overlap
// on the GPU (different streams, no ordering between them) race on it.
#include <stdint.h>

#include <mutex>

#include "common.cuh"

namespace smg {

constexpr int kNoAllocPartials = 8192;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// partial sums [0, kNoAllocPartials), arrival counter at kNoAllocPartials
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocPartials + 16];

double2* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// out[s] = sum_i conj(x[s][i]) y[s][i]; the last CTA to arrive adds the
// partial sums in a fixed order.
__global__ void __launch_bounds__(kThreads) dot_noalloc_kernel(const double2* __restrict__ x,
                                                               const double2* __restrict__ y, long long n,
                                                               double2* __restrict__ scratch,
                                                               double2* __restrict__ out) {
  __shared__ double2 red[kThreads];
  __shared__ bool last;
  const int s = blockIdx.y, nb = gridDim.x, nsys = gridDim.y;
  const long long per = (n + nb - 1) / nb;
  const long long r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  double2 acc = make_double2(0, 0);
  for (long long i = r0 + threadIdx.x; i < r1; i += kThreads) cfmac(acc, x[s * n + i], y[s * n + i]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoAllocPartials);
  if (threadIdx.x == 0) {
    scratch[(size_t)s * nb + blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == (unsigned)(nb * nsys) - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int ss = threadIdx.x; ss < nsys; ss += kThreads) {
    double2 sum = make_double2(0, 0);
    for (int b = 0; b < nb; ++b) sum = cadd(sum, __ldcg(&scratch[(size_t)ss * nb + b]));
    out[ss] = sum;
  }
  if (threadIdx.x == 0) *counter = 0;
}

}  // namespace

// Runs the no-allocation reduction; returns an empty string on success or the
// reason it refused / failed.
std::string dot_noalloc(const void* x, const void* y, long long n, int nsys, void* out, cudaStream_t st) {
  if (x == nullptr || y == nullptr || out == nullptr) return "dot_noalloc: null pointer";
  if (n < 1) return "dot_noalloc: n must be >= 1";
  // the kernel reads and writes whole FP64 complex numbers (16 bytes)
  if ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)out)) & 15u)
    return "dot_noalloc: buffers must be 16-byte aligned";
  if (nsys < 1 || nsys > kNoAllocPartials)
    return "dot_noalloc: nsys must be 1.." + std::to_string(kNoAllocPartials) +
           " (the fixed scratch holds that many partial sums)";
  if (nsys > 65535) return "dot_noalloc: nsys must be <= 65535 (grid limit)";
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return std::string("cudaGetDevice: ") + cudaGetErrorString(e);
  if (dev < 0 || dev >= kMaxDevices) return "dot_noalloc: device ordinal out of range";
  double2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
      // set-up, once per device, with that device current
      e = cudaGetSymbolAddress((void**)&g_scratch_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      }
    }
    scratch = g_scratch_addr[dev];
  }
  long long nb = (n + 2 * kThreads - 1) / (2 * kThreads);
  const long long cap = kNoAllocPartials / nsys;
  if (nb > cap) nb = cap;
  if (nb > 304) nb = 304;
  if (nb < 1) nb = 1;
  e = cudaMemsetAsync(scratch + kNoAllocPartials, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
  dot_noalloc_kernel<<<dim3((unsigned)nb, (unsigned)nsys), kThreads, 0, st>>>(
      (const double2*)x, (const double2*)y, n, scratch, (double2*)out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return std::string("dot_noalloc launch: ") + cudaGetErrorString(e);
  ++g_launches;
  return std::string();
}

}  // namespace smg
