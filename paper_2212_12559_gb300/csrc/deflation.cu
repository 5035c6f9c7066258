// Host driver of the coarsest-level deflation setup (Table 1: SVD-deflated
// Chebyshev-basis CA-GCR): the Chebyshev-filtered subspace iteration that
// finds the lowest singular triplets of the coarsest operator, built from the
// block kernels of defl.cu and the coarse stencil apply.
#include <algorithm>
#include <cmath>
#include <vector>

#include "defl.cuh"
#include "solver.cuh"

namespace smg {

// The k lowest singular triplets of the coarsest operator A (Table 1's
// SVD-deflated coarsest solve) by Chebyshev-filtered subspace iteration on
// A^dag A in FP64: a block of kw = k + guard vectors is multiplied by the
// Chebyshev polynomial T_d((2 A^dag A - (a + b)) / (b - a)), which damps the
// spectrum on [a, b] (a = the block's largest Ritz value, b = 1.2 x a power
// iteration estimate of lambda_max) and grows the part below a; the degree is
// capped so that the growth over the block stays below 1e4 (the Gram matrix of
// the filtered block then keeps its rank in FP64).  Rayleigh-Ritz after each
// filter makes the block orthonormal with ascending Ritz values.  Converged
// when every wanted pair has |A^dag A v - lambda v| <= 1e-10 b.  Then
// sigma = sqrt(lambda), U = A V / sigma; the solve keeps V and U / sigma.
void build_deflation(Context& c, CoarseLevel& C, const void* start, int where) {
  const auto& P = c.params;
  const int k = P.coarsest_deflate;
  const int kw = k + defl_guard(k);
  const long long n = (long long)C.g.V * C.N;
  SMG_REQUIRE(kw <= kDeflMaxBlock, "coarsest_deflate: k + max(4, k/4) must be at most 64");
  SMG_REQUIRE(kw <= n, "coarsest_deflate: more vectors than coarsest unknowns");
  cudaStream_t st = c.stream;
  const size_t vb = (size_t)n * kw * sizeof(double2);
  DevBuf blk;
  blk.alloc(vb * 5);
  auto mk = [&](void* ptr, int ns) { Vec v; v.p = ptr; v.n = n; v.nsys = ns; v.prec = P64; return v; };
  void* buf[5];
  for (int i = 0; i < 5; ++i) buf[i] = (char*)blk.p + vb * i;
  Vec V = mk(buf[0], kw), W = mk(buf[1], kw), X = mk(buf[2], kw);
  void* tp[2] = {buf[3], buf[4]};     // two more Chebyshev iterates
  upload(V.p, start, vb, where, st);
  // A and A^dag of the level's operator (X^{-1} A_hat in block mode), FP64;
  // with the Schur form, S and S^dag on vectors that vanish on odd sites
  DevBuf sdag;
  sdag.alloc(C.S64.bytes);
  coarse_dagger(sdag.as<double2>(), C.S64.as<double2>(), C.g, C.N, st);
  const Stored SA{C.S64.p, nullptr, 1.0f, S64}, SD{sdag.p, nullptr, 1.0f, S64};
  CoarseParams cp;
  cp.g = C.g; cp.N = C.N; cp.allow_tc = 0;
  DevBuf sbuf;
  Vec t1, t2;
  if (C.schur) {
    SMG_REQUIRE(2 * kw <= n, "coarsest_deflate: more vectors than even-site unknowns");
    sbuf.alloc(vb * 2);
    t1 = mk(sbuf.p, kw);
    t2 = mk((char*)sbuf.p + vb, kw);
    parity_pick(V, &V, nullptr, C.g, C.N, st);
  }
  auto applyA = [&](const Vec& o, const Vec& i) {
    if (!C.schur) { coarse_apply(o, i, cp, SA, st); return; }
    Vec a = t1, b = t2;
    a.nsys = b.nsys = i.nsys;
    schur_apply(o, i, cp, SA, a, b, st, nullptr);
  };
  auto applyAd = [&](const Vec& o, const Vec& i) {
    if (!C.schur) { coarse_apply(o, i, cp, SD, st); return; }
    Vec a = t1, b = t2;
    a.nsys = b.nsys = i.nsys;
    schur_apply(o, i, cp, SD, a, b, st, nullptr);
  };
  const size_t kk = (size_t)kw * kw;
  DevBuf sm;
  sm.alloc(sizeof(double2) * (6 * kk + 4 * (size_t)kw + 8) + sizeof(double) * kw);
  double2* G = sm.as<double2>();
  double2* H = G + kk;
  double2* Y = H + kk;
  double2* rrs = Y + kk;               // 3 kk
  double2* coef = rrs + 3 * kk;        // [kw][3] recurrence / shift coefficients
  double2* dots = coef + 3 * kw;       // kw
  double2* small = dots + kw;          // 8
  double* lamd = (double*)(small + 8);
  std::vector<double> lam(kw);
  auto set_coef = [&](const std::vector<double2>& row) {
    std::vector<double2> h((size_t)kw * row.size());
    for (int s = 0; s < kw; ++s)
      for (size_t j = 0; j < row.size(); ++j) h[s * row.size() + j] = row[j];
    SMG_CUDA_OK(cudaMemcpyAsync(coef, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, st));
  };
  // lambda_max(A^dag A) by 30 power steps on the first start vector
  double rq = 0.0;
  {
    Vec x = mk(buf[3], 1), y = mk(buf[4], 1), z = mk(buf[2], 1);
    blas_copy(x, mk(V.p, 1), st);
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 0, 1};
    for (int it = 0; it < 30; ++it) {
      applyA(y, x);
      applyAd(z, y);
      Vec xz[2] = {x, z};
      blas_pair_dots(xz, 2, pi, pj, 3, small, 3, c.ws, st);
      double2 h[3];
      SMG_CUDA_OK(cudaMemcpyAsync(h, small, sizeof(h), cudaMemcpyDeviceToHost, st));
      SMG_CUDA_OK(cudaStreamSynchronize(st));
      SMG_REQUIRE(h[1].x > 0.0 && h[2].x > 0.0, "coarsest_deflate: zero power-iteration vector");
      rq = h[0].x / h[1].x;
      const double2 nz = make_double2(std::sqrt(h[2].x), 0.0);
      SMG_CUDA_OK(cudaMemcpyAsync(small + 4, &nz, sizeof(nz), cudaMemcpyHostToDevice, st));
      blas_copy(x, z, st);
      blas_scale(x, small + 4, true, st);
    }
  }
  double b = 1.2 * rq;
  auto ritz = [&]() {
    block_gram(V, V, G, c.ws, st);
    block_gram(W, W, H, c.ws, st);
    rayleigh_ritz(G, H, kw, Y, lamd, rrs, st);
    block_combine(X, V, Y, kw, st);
    std::swap(V.p, X.p);
    block_combine(X, W, Y, kw, st);
    std::swap(W.p, X.p);
    SMG_CUDA_OK(cudaMemcpyAsync(lam.data(), lamd, sizeof(double) * kw, cudaMemcpyDeviceToHost, st));
    SMG_CUDA_OK(cudaStreamSynchronize(st));
    SMG_REQUIRE(lam[0] < 1e299, "coarsest_deflate: the start block has no usable direction");
  };
  applyA(W, V);
  ritz();
  const int max_it = 200;
  int it = 0;
  double res = 0.0;
  for (; it < max_it; ++it) {
    // Chebyshev filter on [a, b]
    double a = lam[0];
    for (int j = 0; j < kw; ++j)
      if (lam[j] < 1e299) a = std::max(a, lam[j]);   // the largest Ritz value of the block
    b = std::max(b, 1.05 * a);
    if (!(a < b)) a = 0.5 * b;
    const double xmin = std::fabs((2.0 * lam[0] - a - b) / (b - a));
    int deg = 20;
    if (xmin > 1.0) deg = std::max(1, std::min(20, (int)(std::acosh(1e4) / std::acosh(xmin))));
    Vec T0 = V, T1 = mk(tp[0], kw), Tn = mk(tp[1], kw);
    applyA(W, T0);
    applyAd(X, W);
    set_coef({make_double2(2.0 / (b - a), 0.0), make_double2(-(a + b) / (b - a), 0.0)});
    Vec in2[2] = {X, T0};
    blas_maxpy(T1, in2, 2, coef, 2, 1.0, false, st);
    if (deg > 1) set_coef({make_double2(4.0 / (b - a), 0.0), make_double2(-2.0 * (a + b) / (b - a), 0.0),
                           make_double2(-1.0, 0.0)});
    for (int j = 1; j < deg; ++j) {
      applyA(W, T1);
      applyAd(X, W);
      Vec in3[3] = {X, T1, T0};
      blas_maxpy(Tn, in3, 3, coef, 3, 1.0, false, st);
      std::swap(T0.p, T1.p);    // T0 <- T1
      std::swap(T1.p, Tn.p);    // T1 <- Tn, Tn <- the old T0 (free)
    }
    // V <- T1; {T0, T1, Tn} is always a permutation of the three iterate
    // buffers, so T0 and Tn are the free pair
    V.p = T1.p;
    tp[0] = T0.p;
    tp[1] = Tn.p;
    applyA(W, V);
    ritz();
    // residuals of the k wanted pairs: A^dag W_j - lambda_j V_j
    applyAd(X, W);
    {
      std::vector<double2> h(kw);
      for (int s = 0; s < kw; ++s) h[s] = make_double2(lam[s] < 1e299 ? lam[s] : 0.0, 0.0);
      SMG_CUDA_OK(cudaMemcpyAsync(coef, h.data(), sizeof(double2) * kw, cudaMemcpyHostToDevice, st));
    }
    blas_maxpy(X, &V, 1, coef, 1, -1.0, true, st);
    const int p0[1] = {0};
    blas_pair_dots(&X, 1, p0, p0, 1, dots, 1, c.ws, st);
    std::vector<double2> d(kw);
    SMG_CUDA_OK(cudaMemcpyAsync(d.data(), dots, sizeof(double2) * kw, cudaMemcpyDeviceToHost, st));
    SMG_CUDA_OK(cudaStreamSynchronize(st));
    res = 0.0;
    for (int j = 0; j < k; ++j) res = std::max(res, std::sqrt(std::max(d[j].x, 0.0)) / b);
    if (res <= 1e-10) { ++it; break; }
  }
  SMG_REQUIRE(lam[k - 1] > 0.0 && lam[k - 1] < 1e299, "coarsest_deflate: fewer than k usable directions");
  C.defl_k = k;
  C.defl_iters = it;
  C.defl_res = res;
  C.sigma.resize(k);
  for (int j = 0; j < k; ++j) C.sigma[j] = std::sqrt(lam[j]);
  C.cheb_lmin = C.sigma[k - 1];
  C.cheb_lmax = std::sqrt(rq);
  // U / sigma = A V / sigma^2
  {
    std::vector<double2> h(k);
    for (int j = 0; j < k; ++j) h[j] = make_double2(lam[j], 0.0);
    SMG_CUDA_OK(cudaMemcpyAsync(coef, h.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, st));
    Vec Wk = mk(W.p, k);
    blas_scale(Wk, coef, true, st);
  }
  const size_t kb64 = (size_t)n * k * sizeof(double2);
  C.dV64.alloc(kb64);
  C.dU64.alloc(kb64);
  SMG_CUDA_OK(cudaMemcpyAsync(C.dV64.p, V.p, kb64, cudaMemcpyDeviceToDevice, st));
  SMG_CUDA_OK(cudaMemcpyAsync(C.dU64.p, W.p, kb64, cudaMemcpyDeviceToDevice, st));
  C.dV32.alloc((size_t)n * k * sizeof(float2));
  C.dU32.alloc((size_t)n * k * sizeof(float2));
  Vec v32 = mk(C.dV32.p, k);
  v32.prec = P32;
  Vec u32 = mk(C.dU32.p, k);
  u32.prec = P32;
  blas_copy(v32, mk(C.dV64.p, k), st);
  blas_copy(u32, mk(C.dU64.p, k), st);
  SMG_CUDA_OK(cudaStreamSynchronize(st));
}

// The deflation state of a saved setup: V and U diag(1/sigma) in FP64 as they
// were saved, their FP32 copies derived as build_deflation derives them.
void restore_deflation(Context& c, CoarseLevel& C, const DeflRestore& r) {
  const long long n = (long long)C.g.V * C.N;
  SMG_REQUIRE(r.k == c.params.coarsest_deflate && (int)r.sigma.size() == r.k && r.V && r.U,
              "load_setup: deflation block does not match the parameters");
  cudaStream_t st = c.stream;
  C.defl_k = r.k;
  C.defl_iters = r.iters;
  C.defl_res = r.res;
  C.sigma = r.sigma;
  C.cheb_lmin = r.lmin;
  C.cheb_lmax = r.lmax;
  const size_t kb64 = (size_t)n * r.k * sizeof(double2);
  C.dV64.alloc(kb64);
  C.dU64.alloc(kb64);
  upload(C.dV64.p, r.V, kb64, SMG_HOST, st);
  upload(C.dU64.p, r.U, kb64, SMG_HOST, st);
  C.dV32.alloc((size_t)n * r.k * sizeof(float2));
  C.dU32.alloc((size_t)n * r.k * sizeof(float2));
  auto mk = [&](void* p, Prec pr) { Vec v; v.p = p; v.n = n; v.nsys = r.k; v.prec = pr; return v; };
  blas_copy(mk(C.dV32.p, P32), mk(C.dV64.p, P64), st);
  blas_copy(mk(C.dU32.p, P32), mk(C.dU64.p, P64), st);
  SMG_CUDA_OK(cudaStreamSynchronize(st));
}

}  // namespace smg
