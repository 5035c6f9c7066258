// Shared device/host helpers of libsmg: complex arithmetic, storage types,
// batched field descriptors, launch helpers and error plumbing.
//
// Data conventions used by every kernel:
//  * a batched field holds nsys systems, each `n` complex numbers, stored
//    system-major: element (s, i) at offset s*n + i.  Fine fields are ordered
//    [site][colour], coarse fields [site][component].
//  * vector precision is FP64 (double2) or FP32 (float2); operator data
//    (links, KD block inverses, null vectors, coarse stencils) is stored as
//    double2, float2 or half2 (FP16 real/imag) with FP32 scale factors.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

namespace smg {

enum Prec { P64 = 0, P32 = 1 };
enum Store { S64 = 0, S32 = 1, S16 = 2 };

inline size_t prec_bytes(Prec p) { return p == P64 ? 16 : 8; }
inline size_t store_bytes(Store s) { return s == S64 ? 16 : (s == S32 ? 8 : 4); }

// ---------------------------------------------------------------- complex ops
template <typename R> struct cplx;
template <> struct cplx<double> { using T = double2; };
template <> struct cplx<float> { using T = float2; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { return C{a.x * s, a.y * s}; }
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __host__ __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// ------------------------------------------------------------ storage loads
template <typename R> __device__ __forceinline__ typename cplx<R>::T ld(const double2* p, size_t i) {
  double2 v = p[i]; return typename cplx<R>::T{(R)v.x, (R)v.y};
}
template <typename R> __device__ __forceinline__ typename cplx<R>::T ld(const float2* p, size_t i) {
  float2 v = p[i]; return typename cplx<R>::T{(R)v.x, (R)v.y};
}
template <typename R> __device__ __forceinline__ typename cplx<R>::T ld(const __half2* p, size_t i) {
  float2 v = __half22float2(p[i]); return typename cplx<R>::T{(R)v.x, (R)v.y};
}
__device__ __forceinline__ void st(double2* p, size_t i, double2 v) { p[i] = v; }
__device__ __forceinline__ void st(double2* p, size_t i, float2 v) { p[i] = make_double2(v.x, v.y); }
__device__ __forceinline__ void st(float2* p, size_t i, double2 v) { p[i] = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void st(float2* p, size_t i, float2 v) { p[i] = v; }

template <Store S> struct StoreT;
template <> struct StoreT<S64> { using T = double2; };
template <> struct StoreT<S32> { using T = float2; };
template <> struct StoreT<S16> { using T = __half2; };

// ------------------------------------------------------------ lattice helpers
struct Geom {
  int L[4];          // extents
  int V;             // volume
  __host__ __device__ __forceinline__ void coords(int i, int c[4]) const {
    c[0] = i % L[0]; i /= L[0];
    c[1] = i % L[1]; i /= L[1];
    c[2] = i % L[2]; c[3] = i / L[2];
  }
  __host__ __device__ __forceinline__ int index(const int c[4]) const {
    return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
  }
  // site index of c + k*mu_hat (periodic); one conditional wrap when
  // |k| <= L[mu] (every hop of the method), a modulo otherwise
  __host__ __device__ __forceinline__ int shift(const int c[4], int mu, int k) const {
    int d[4] = {c[0], c[1], c[2], c[3]};
    const int l = L[mu];
    int v = d[mu] + k;
    if (v >= l) v -= l;
    else if (v < 0) v += l;
    if (v < 0 || v >= l) { v %= l; if (v < 0) v += l; }
    d[mu] = v;
    return index(d);
  }
};

// ------------------------------------------------------------- error plumbing
struct Error {
  int code; std::string msg;
};

}  // namespace smg

#define SMG_CUDA_OK(expr)                                                       \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) {                                                    \
      throw smg::CudaError(_e, #expr, __FILE__, __LINE__);                      \
    }                                                                           \
  } while (0)

namespace smg {
// Number of kernels this library has launched (graph replays add their node count).
extern long long g_launches;
}
#define SMG_LAUNCH_OK()                  \
  do {                                   \
    ++smg::g_launches;                   \
    SMG_CUDA_OK(cudaGetLastError());     \
  } while (0)

namespace smg {
struct CudaError {
  cudaError_t err; std::string what;
  CudaError(cudaError_t e, const char* expr, const char* file, int line) : err(e) {
    what = std::string(cudaGetErrorString(e)) + " at " + file + ":" + std::to_string(line) + " (" + expr + ")";
  }
};
struct ArgError {
  std::string what;
  explicit ArgError(std::string w) : what(std::move(w)) {}
};
#define SMG_REQUIRE(cond, msg) do { if (!(cond)) throw smg::ArgError(msg); } while (0)

inline unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Kernel launch with explicit configuration (arguments converted to the
// kernel's parameter types).  Programmatic dependent launch was measured on
// the solver's kernel chain and made it slower (dependent CTAs waiting on
// SMs while the previous kernel drains), so launches are plain stream-ordered.
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  SMG_CUDA_OK(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}
}  // namespace smg
