// Fine staggered operator M = m + D (Sec. 2.2), naive or with Naik links.
//
//   (D psi)(x) = 1/2 sum_mu eta_mu(x) [ V_mu(x) psi(x+mu) - V_mu(x-mu)^dag psi(x-mu) ]
//              + c_N/2 sum_mu eta_mu(x) [ W_mu(x) psi(x+3mu) - W_mu(x-3mu)^dag psi(x-3mu) ]
//
// One thread per (site, colour row); blockIdx.y is the system of the batch.
// The three threads of a site read the three rows of each forward link and
// the three columns of each backward link, so a warp's link reads cover a
// contiguous run of 9-complex matrices; the neighbour spinor (3 complex) is
// shared by the three threads through L1.
//
// `part` restricts the operator to hops that stay inside an aggregate
// (part 0, plus the mass term) or that cross into the next / previous
// aggregate along one axis (part 1 + 2mu + dir); the Galerkin build probes the
// operator part by part.
#include "ops.cuh"

namespace smg {
namespace {

template <typename R, typename SL>
__device__ __forceinline__ void hop_accumulate(typename cplx<R>::T (&acc), const SL* __restrict__ links, R lscale,
                                               const typename cplx<R>::T* __restrict__ in, long long in_off,
                                               int V, int mu, int x, int xf, int xb, int a, R coef, bool use_f,
                                               bool use_b) {
  using C = typename cplx<R>::T;
  C t = C{0, 0};
  if (use_f) {
    const size_t lf = ((size_t)mu * V + x) * 9 + a * 3;
    const C* pf = in + in_off + (size_t)xf * 3;
#pragma unroll
    for (int b = 0; b < 3; ++b) cfma(t, ld<R>(links, lf + b), pf[b]);
  }
  if (use_b) {
    const size_t lb = ((size_t)mu * V + xb) * 9 + a;
    const C* pb = in + in_off + (size_t)xb * 3;
    C u = C{0, 0};
#pragma unroll
    for (int b = 0; b < 3; ++b) cfmac(u, ld<R>(links, lb + b * 3), pb[b]);
    t = csub(t, u);
  }
  acc.x = fma(coef * lscale, t.x, acc.x);
  acc.y = fma(coef * lscale, t.y, acc.y);
}

template <typename R, typename SL>
__global__ void __launch_bounds__(192) dslash_kernel(typename cplx<R>::T* __restrict__ out,
                                                     const typename cplx<R>::T* __restrict__ in,
                                                     const SL* __restrict__ fat, const SL* __restrict__ naik,
                                                     R fat_scale, R naik_scale, R half_c_naik,
                                                     const double* __restrict__ mass, double mass0, int dagger,
                                                     int part, int4 agg, Geom g,
                                                     const typename cplx<R>::T* __restrict__ sub_from,
                                                     const int* run) {
  using C = typename cplx<R>::T;
  if (run != nullptr && *run == 0) return;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * 3) return;
  const int s = blockIdx.y;
  const int x = tid / 3, a = tid - 3 * (tid / 3);
  const long long off = (long long)s * g.V * 3;
  int c[4];
  g.coords(x, c);
  const int ag[4] = {agg.x, agg.y, agg.z, agg.w};
  C acc = C{0, 0};
  int eta_sum = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const R eta = (eta_sum & 1) ? R(-1) : R(1);
    eta_sum += c[mu];
    const int r = c[mu] % ag[mu];
    // distance one
    {
      bool f = true, b = true;
      if (part >= 0) {
        const bool cf = r + 1 >= ag[mu], cb = r - 1 < 0;
        if (part == 0) { f = !cf; b = !cb; }
        else { f = (part == 1 + 2 * mu) && cf; b = (part == 2 + 2 * mu) && cb; }
      }
      if (f || b) {
        const int xf = g.shift(c, mu, 1), xb = g.shift(c, mu, -1);
        hop_accumulate<R, SL>(acc, fat, fat_scale, in, off, g.V, mu, x, xf, xb, a, R(0.5) * eta, f, b);
      }
    }
    if (naik != nullptr) {
      bool f = true, b = true;
      if (part >= 0) {
        const bool cf = r + 3 >= ag[mu], cb = r - 3 < 0;
        if (part == 0) { f = !cf; b = !cb; }
        else { f = (part == 1 + 2 * mu) && cf; b = (part == 2 + 2 * mu) && cb; }
      }
      if (f || b) {
        const int xf = g.shift(c, mu, 3), xb = g.shift(c, mu, -3);
        hop_accumulate<R, SL>(acc, naik, naik_scale, in, off, g.V, mu, x, xf, xb, a, half_c_naik * eta, f, b);
      }
    }
  }
  if (dagger) { acc.x = -acc.x; acc.y = -acc.y; }
  if (part <= 0) {
    const R m = (R)(mass != nullptr ? mass[s] : mass0);
    const C v = in[off + (size_t)x * 3 + a];
    acc.x = fma(m, v.x, acc.x);
    acc.y = fma(m, v.y, acc.y);
  }
  if (sub_from != nullptr) acc = csub(sub_from[off + (size_t)x * 3 + a], acc);
  out[off + (size_t)x * 3 + a] = acc;
}

template <typename R, typename SL>
void launch(const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run) {
  using C = typename cplx<R>::T;
  dim3 grid(ceil_div((long long)p.g.V * 3, 192), p.nsys);
  int4 agg = make_int4(p.agg[0], p.agg[1], p.agg[2], p.agg[3]);
  launch_k(dslash_kernel<R, SL>, dim3(grid), dim3(192), 0, st, (C*)out.p, (const C*)in.p, (const SL*)p.fat.p, (const SL*)p.naik.p,
                                             (R)p.fat.gscale, (R)p.naik.gscale, (R)(0.5 * p.c_naik), p.mass,
                                             p.mass0, p.dagger, p.part, agg, p.g, (const C*)p.sub_from, run);
  SMG_LAUNCH_OK();
}

}  // namespace

void dslash(const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run) {
  SMG_REQUIRE(in.n == (long long)p.g.V * 3 && out.n == in.n, "dslash: field size does not match the lattice");
  SMG_REQUIRE(in.nsys == p.nsys && out.nsys == p.nsys, "dslash: batch mismatch");
  SMG_REQUIRE(in.prec == out.prec, "dslash: precision mismatch");
  SMG_REQUIRE(p.naik.p == nullptr || p.naik.s == p.fat.s, "dslash: fat/naik storage mismatch");
  if (hop_dslash_ok(in, p)) {
    hop_dslash(out, in, p, st, run);
    return;
  }
  if (in.prec == P64) {
    SMG_REQUIRE(p.fat.s == S64, "dslash: FP64 vectors need FP64 links");
    launch<double, double2>(out, in, p, st, run);
  } else if (p.fat.s == S32) {
    launch<float, float2>(out, in, p, st, run);
  } else if (p.fat.s == S16) {
    launch<float, __half2>(out, in, p, st, run);
  } else {
    SMG_REQUIRE(false, "dslash: FP32 vectors with FP64 links are not supported");
  }
}

}  // namespace smg
