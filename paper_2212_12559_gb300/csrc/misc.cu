// Lattice maps (exported for bit-exact checks) and the fermion-force
// outer-product kernel.
#include <algorithm>
#include <cstring>

#include "ops.cuh"

namespace smg {
namespace {

__global__ void site_maps_kernel(int* parity, int* kd_block, int* kd_pos, int* agg_idx, int* agg_pos, Geom g,
                                 int4 agg) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  g.coords(x, c);
  const int a[4] = {agg.x, agg.y, agg.z, agg.w};
  parity[x] = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int h[4] = {g.L[0] / 2, g.L[1] / 2, g.L[2] / 2, g.L[3] / 2};
  kd_block[x] = (c[0] >> 1) + h[0] * ((c[1] >> 1) + h[1] * ((c[2] >> 1) + h[2] * (c[3] >> 1)));
  kd_pos[x] = (c[0] & 1) + 2 * (c[1] & 1) + 4 * (c[2] & 1) + 8 * (c[3] & 1);
  const int cd[4] = {g.L[0] / a[0], g.L[1] / a[1], g.L[2] / a[2], g.L[3] / a[3]};
  agg_idx[x] = c[0] / a[0] + cd[0] * (c[1] / a[1] + cd[1] * (c[2] / a[2] + cd[2] * (c[3] / a[3])));
  agg_pos[x] = c[0] % a[0] + a[0] * (c[1] % a[1] + a[1] * (c[2] % a[2] + a[2] * (c[3] % a[3])));
}

// F_mu(x)[a][b] = -c eta_mu(x) ( Y_a(x) conj(X_b(x+k mu)) - X_a(x) conj(Y_b(x+k mu)) )
__global__ void force_kernel(double2* __restrict__ F, const double2* __restrict__ X, const double2* __restrict__ Y,
                             Geom g, int k, double coef, int bc_t) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= 4LL * g.V * 9) return;
  const int ab = (int)(e % 9);
  const long long q = e / 9;
  const int x = (int)(q % g.V), mu = (int)(q / g.V);
  const int a = ab / 3, b = ab % 3;
  int c[4];
  g.coords(x, c);
  int es = 0;
  for (int nu = 0; nu < mu; ++nu) es += c[nu];
  double eta = (es & 1) ? -1.0 : 1.0;
  if (mu == 3 && bc_t < 0 && c[3] + k >= g.L[3]) eta = -eta;   // the hop wraps around the time boundary
  const int xn = g.shift(c, mu, k);
  const double2 ya = Y[(size_t)x * 3 + a], xb = X[(size_t)xn * 3 + b];
  const double2 xa = X[(size_t)x * 3 + a], yb = Y[(size_t)xn * 3 + b];
  double2 t1 = cmul(ya, make_double2(xb.x, -xb.y));
  double2 t2 = cmul(xa, make_double2(yb.x, -yb.y));
  F[e] = make_double2(-coef * eta * (t1.x - t2.x), -coef * eta * (t1.y - t2.y));
}

// time links (mu = 3) of the sites with x_t + k >= L_t change sign
__global__ void boundary_flip_kernel(double2* __restrict__ links, Geom g, int k) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)g.V * 9) return;
  const int x = (int)(e / 9);
  int c[4];
  g.coords(x, c);
  if (c[3] + k < g.L[3]) return;
  double2* p = links + (size_t)3 * g.V * 9 + (size_t)e;
  *p = make_double2(-p->x, -p->y);
}

// largest |Re|, |Im| (float bits, non-negative, so the integer maximum is the float maximum)
__global__ void __launch_bounds__(256) absmax_kernel(const float2* __restrict__ v, long long n, unsigned* mx) {
  __shared__ float red[8];
  float m = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(v[e].x), fabsf(v[e].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(mx, __float_as_uint(m));
  }
}

__global__ void pack_h16_kernel(__half2* __restrict__ dst, const float2* __restrict__ src, long long n, float sc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = __floats2half2_rn(src[e].x / sc, src[e].y / sc);
}

__global__ void eps_mul_kernel(double2* out, const double2* in, Geom g) {   // may run in place
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.V * 3) return;
  int c[4];
  g.coords(e / 3, c);
  const double sg = ((c[0] + c[1] + c[2] + c[3]) & 1) ? -1.0 : 1.0;
  out[e] = make_double2(sg * in[e].x, sg * in[e].y);
}

}  // namespace

void eps_mul(double2* out, const double2* in, const Geom& g, cudaStream_t st) {
  eps_mul_kernel<<<ceil_div((long long)g.V * 3, 256), 256, 0, st>>>(out, in, g);
  SMG_LAUNCH_OK();
}

void site_maps(int* parity, int* kd_block, int* kd_pos, int* agg_idx, int* agg_pos, const Geom& g, const int agg[4],
               cudaStream_t st) {
  site_maps_kernel<<<ceil_div(g.V, 256), 256, 0, st>>>(parity, kd_block, kd_pos, agg_idx, agg_pos, g,
                                                       make_int4(agg[0], agg[1], agg[2], agg[3]));
  SMG_LAUNCH_OK();
}

void force_outer(double2* F, const double2* X, const double2* Y, const Geom& g, int k, double c, int bc_t,
                 cudaStream_t st) {
  force_kernel<<<ceil_div(4LL * g.V * 9, 256), 256, 0, st>>>(F, X, Y, g, k, c, bc_t);
  SMG_LAUNCH_OK();
}

float pack_fp16_global(__half2* dst, const float2* src, long long n, cudaStream_t st) {
  struct Word {
    unsigned* p = nullptr;
    ~Word() { if (p) cudaFree(p); }
  } mb;
  SMG_CUDA_OK(cudaMalloc(&mb.p, sizeof(unsigned)));
  SMG_CUDA_OK(cudaMemsetAsync(mb.p, 0, sizeof(unsigned), st));
  const unsigned grid = (unsigned)std::min<long long>(1216, std::max<long long>(1, (n + 255) / 256));
  absmax_kernel<<<grid, 256, 0, st>>>(src, n, mb.p);
  SMG_LAUNCH_OK();
  unsigned bits = 0;
  SMG_CUDA_OK(cudaMemcpyAsync(&bits, mb.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  SMG_CUDA_OK(cudaStreamSynchronize(st));
  float mx = 0.f;
  std::memcpy(&mx, &bits, sizeof(float));
  const float sc = mx > 0 ? mx : 1.f;
  pack_h16_kernel<<<grid, 256, 0, st>>>(dst, src, n, sc);
  SMG_LAUNCH_OK();
  return sc;
}

void boundary_flip_time(double2* links, const Geom& g, int k, cudaStream_t st) {
  boundary_flip_kernel<<<ceil_div((long long)g.V * 9, 256), 256, 0, st>>>(links, g, k);
  SMG_LAUNCH_OK();
}

}  // namespace smg
