// The K-cycle multigrid preconditioner inside flexible GCR (Sec. 2.1, 2.3,
// Table 1), batched over systems, with every scalar of every Krylov method
// kept on the device.
//
// Levels:
//   0  M = m + D on the fine lattice: outer flexible GCR in FP64, restarted
//      every nkrylov directions with the residual recomputed in FP64; its
//      preconditioner K_0 runs in the preconditioner precision.
//   1  A = (B+m)^{-1} M on the fine lattice ("pseudo-fine", Sec. 2.3): GCR to
//      inner_tol or inner_maxiter iterations, preconditioned by K_1.
//   2, 3  Galerkin stencils R A P: GCR preconditioned by the next K-cycle, or
//      on the coarsest level an exact dense solve (dof <= dense_max) or plain
//      GCR to inner_tol / inner_maxiter.
// K_0(r):  e = GCR_1(A, (B+m)^{-1} r); e += CA-GCR_s(M, r - M e).
// K_l(r):  e = P_l solve_{l+1}(R_l r); e += CA-GCR_s(A_l, r - A_l e).
// No pre-smoothing (Table 1).  Inner loops launch a fixed kernel sequence;
// a device flag per loop makes the remaining launches return at once after
// convergence, so no host synchronisation happens inside K_0.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "defl.cuh"
#include "persist.cuh"
#include "solver.cuh"

namespace smg {

long long g_launches = 0;

// ------------------------------------------------------------- allocation
void DevBuf::alloc(size_t b) {
  release();
  if (b == 0) return;
  cudaError_t e = cudaMalloc(&p, b);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    throw OomError("cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
  }
  bytes = b;
  // fresh buffers start at zero so that no path ever reads uninitialised bits;
  // the memset runs on the legacy stream, so wait for it before any stream uses p
  SMG_CUDA_OK(cudaMemset(p, 0, b));
  SMG_CUDA_OK(cudaDeviceSynchronize());
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

void StoredBuf::alloc(Store s, size_t elems, size_t nscale) {
  v.alloc(elems * store_bytes(s));
  if (s == S16 && nscale > 0) sc.alloc(nscale * sizeof(float));
  else sc.release();
  st.p = v.p;
  st.scale = (s == S16) ? sc.as<float>() : nullptr;
  st.gscale = 1.0f;
  st.s = s;
}

void GcrWork::alloc(long long n, int ns, Prec p, int k) {
  K = k; nsys = ns;
  const size_t vb = (size_t)n * ns * prec_bytes(p);
  const int nv = 2 * K + 3;
  vbuf.alloc(vb * nv);
  z.resize(K); w.resize(K);
  auto mk = [&](int i) { Vec v; v.p = (char*)vbuf.p + vb * i; v.n = n; v.nsys = ns; v.prec = p; return v; };
  for (int i = 0; i < K; ++i) { z[i] = mk(i); w[i] = mk(K + i); }
  r = mk(2 * K); x = mk(2 * K + 1); b = mk(2 * K + 2);
  const int Kk = K > 0 ? K : 1;
  size_t nd2 = (size_t)ns * (Kk * 5 + 2 + Kk * Kk + 2 + 3);
  size_t bytes = nd2 * sizeof(double2) + (size_t)ns * 2 * sizeof(double) + ((size_t)ns * 2 + 1) * sizeof(int);
  sbuf.alloc(bytes);
  double2* d = sbuf.as<double2>();
  alpha = d; d += ns * Kk;
  gamma = d; d += ns * Kk;
  y = d; d += ns * Kk;
  tmp = d; d += ns * (Kk + 2);
  beta = d; d += ns * Kk * Kk;
  dd = d; d += ns * 2;
  na = d; d += ns;
  ginv = d; d += ns;
  r2 = d; d += ns;
  d += ns * Kk;   // spare
  double* dr = (double*)d;
  r02 = dr; dr += ns;
  thr2 = dr; dr += ns;
  int* ip = (int*)dr;
  active = ip; ip += ns;
  nk = ip; ip += ns;
  run = ip;
}

void SmoothWork::alloc(long long n, int ns, Prec p, int s_) {
  s = s_;
  const size_t vb = (size_t)n * ns * prec_bytes(p);
  vbuf.alloc(vb * (s + 1));
  V.resize(s + 1);
  for (int i = 0; i <= s; ++i) { V[i].p = (char*)vbuf.p + vb * i; V[i].n = n; V[i].nsys = ns; V[i].prec = p; }
  np = 0;
  for (int i = 0; i < s; ++i)
    for (int j = i; j < s; ++j) { pi[np] = i + 1; pj[np] = j + 1; ++np; }
  for (int i = 0; i < s; ++i) { pi[np] = i + 1; pj[np] = 0; ++np; }
  sbuf.alloc(sizeof(double2) * (size_t)ns * (kMaxPairs + s));
  gram = sbuf.as<double2>();
  coef = gram + (size_t)ns * kMaxPairs;
}

Context::~Context() {
  engine.reset();
  if (own_stream) cudaStreamDestroy(own_stream);
}

namespace {
__global__ void fill_consts(double2* ones, double2* mones, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { ones[i] = make_double2(1, 0); mones[i] = make_double2(-1, 0); }
}
}  // namespace

void Context::ensure_consts(int n) {
  if (n <= nconst) return;
  consts.alloc(sizeof(double2) * 2 * n);
  ones = consts.as<double2>();
  mones = ones + n;
  fill_consts<<<ceil_div(n, 128), 128, 0, stream>>>(ones, mones, n);
  SMG_LAUNCH_OK();
  nconst = n;
}

void upload(void* dst, const void* src, size_t bytes, int where, cudaStream_t st) {
  SMG_CUDA_OK(cudaMemcpyAsync(dst, src, bytes, where == SMG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              st));
}
void download(void* dst, const void* src, size_t bytes, int where, cudaStream_t st) {
  SMG_CUDA_OK(cudaMemcpyAsync(dst, src, bytes, where == SMG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                              st));
}

bool trace_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("SMG_TRACE");
    v = (e != nullptr && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

bool phase_profile_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("SMG_PHASES");
    v = (e != nullptr && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

// Opt-in (SMG_PHASES=1) device time per solver phase, from CUDA events
// recorded around each phase on the solver's stream; printed after each
// solve.  Only meaningful without the CUDA graph (use_graph = 0).
struct PhaseTimer {
  struct Rec { const char* name; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      SMG_CUDA_OK(cudaEventCreate(&e));
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(const char* name, cudaStream_t st) {
    Rec r{name, ev(), nullptr};
    SMG_CUDA_OK(cudaEventRecord(r.a, st));
    recs.push_back(r);
  }
  void end(cudaStream_t st) {
    for (auto it = recs.rbegin(); it != recs.rend(); ++it)
      if (it->b == nullptr) { it->b = ev(); SMG_CUDA_OK(cudaEventRecord(it->b, st)); return; }
  }
  // durations measured elsewhere (the persistent kernel's own trace)
  std::vector<std::pair<std::string, std::pair<double, int>>> ext;
  void add(const std::string& name, double ms) {
    for (auto& a : ext)
      if (a.first == name) { a.second.first += ms; a.second.second++; return; }
    ext.push_back({name, {ms, 1}});
  }
  void report(cudaStream_t st) {
    SMG_CUDA_OK(cudaStreamSynchronize(st));
    std::vector<std::pair<std::string, std::pair<double, int>>> acc;
    for (auto& r : recs) {
      float ms = 0;
      if (r.b) cudaEventElapsedTime(&ms, r.a, r.b);
      bool found = false;
      for (auto& a : acc)
        if (a.first == r.name) { a.second.first += ms; a.second.second++; found = true; }
      if (!found) acc.push_back({r.name, {ms, 1}});
    }
    for (auto& a : ext) acc.push_back(a);
    ext.clear();
    for (auto& a : acc)
      fprintf(stderr, "[smg phases] %-22s %10.3f ms  %6d calls\n", a.first.c_str(), a.second.first, a.second.second);
    recs.clear();
    used = 0;
  }
  ~PhaseTimer() { for (auto e : pool) cudaEventDestroy(e); }
};


// -------------------------------------------------------------------- engine
// Work areas and operator closures for one batch size and mass set.
struct Engine {
  Context& c;
  int nsys;
  int nlev;                         // number of coarse levels
  Prec vp;                          // preconditioner vector precision
  Store sp;                         // preconditioner storage
  DevBuf mass_dev, map_dev;
  const int* sys_map = nullptr;
  std::vector<double> masses;       // per shift
  std::vector<StoredBuf> kd_shift;  // per-shift block inverses (multi-mass)
  std::vector<Stored> kd_s;         // descriptors handed to kd_apply
  int nkd = 1;
  // level 0
  GcrWork outer;
  DevBuf target_buf;
  Vec r_s, tmpA, tmp_f, tmp64, zbuf;
  DevBuf fbuf;
  SmoothWork sm_f;
  // levels 1..nlev+1 (index = level)
  std::vector<GcrWork> lev;
  std::vector<SmoothWork> sm_c;     // smoother of coarse level l at index l
  std::vector<Vec> tmp_c;
  DevBuf cbuf;
  Workspace ws;                     // reduction partials, sized once so captured graphs stay valid
  DevBuf pbuf;                      // persistent coarse solver: partials, barrier words, error word
  PersistPlan pplan;                // its launch shape
  DevBuf trace_buf;                 // its phase trace (SMG_PHASES=1)
  PhaseTimer phases;
  bool prof = false;
  void pb(const char* n) { if (prof) phases.begin(n, st()); }
  void pe() { if (prof) phases.end(st()); }
  bool persistent = false;          // last GCR level solved by one cooperative launch
  // deflated coarsest level: Chebyshev basis Q_1..Q_{s-1} (Q_0 is the
  // residual), W_i = A Q_i, recurrence coefficients, Gram and flags
  struct ChebWork {
    int s = 0;
    std::vector<Vec> Q, W;
    DevBuf vbuf, sbuf;
    double2 *c1 = nullptr, *c2 = nullptr, *gram = nullptr, *coef = nullptr, *yd = nullptr, *rr = nullptr,
            *bb = nullptr;
    int *active = nullptr, *drun = nullptr;
    double2 *mgram = nullptr, *cscr = nullptr;   // per-system Gram sums, normal-equation scratch
    Vec t1, t2, t3, xe, rhs;          // Schur form: scratch, x_e and c_e - K_eo c_o
  } cw;
  // intermediate levels in Schur form: scratch t1..t3 and the saved right-hand side c, per level
  std::vector<std::vector<Vec>> sch;
  DevBuf schbuf;
  bool schur_lvl(int l) const { return l >= 2 && c.coarse[l - 2].schur_level; }
  // graph of K_0
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;
  long long graph_nodes = 0;

  int nrhs_ = 1;                    // systems per mass (consecutive)

  Engine(Context& ctx, int ns, const std::vector<double>& ms, int nrhs)
      : c(ctx), nsys(ns), masses(ms), nrhs_(nrhs) {
    const auto& P = c.params;
    nlev = P.n_coarse;
    vp = c.vprec();
    sp = c.sstore();
    const long long nf = (long long)c.g.V * 3;
    // per-system masses and block inverses
    std::vector<double> m(ns);
    std::vector<int> map(ns);
    for (int s = 0; s < ns; ++s) { map[s] = s / nrhs; m[s] = ms[map[s]]; }
    mass_dev.alloc(sizeof(double) * ns);
    SMG_CUDA_OK(cudaMemcpyAsync(mass_dev.p, m.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c.stream));
    nkd = (int)ms.size();
    if (nkd == 1 && ms[0] == c.mass) {
      kd_s.push_back(c.kd_of(sp));
    } else {
      SMG_REQUIRE(nkd <= 16, "multi_solve: at most 16 masses");
      map_dev.alloc(sizeof(int) * ns);
      SMG_CUDA_OK(cudaMemcpyAsync(map_dev.p, map.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, c.stream));
      sys_map = map_dev.as<int>();
      DevBuf row;
      row.alloc((size_t)(c.g.V / 16) * 48 * 48 * sizeof(double2));
      kd_shift.resize(nkd);
      for (int i = 0; i < nkd; ++i) {
        kd_build(row.as<double2>(), c.g, c.fat64.as<double2>(), ms[i], c.stream);
        kd_shift[i].alloc(sp, (size_t)(c.g.V / 16) * 48 * 48, (size_t)(c.g.V / 16) * 48);
        kd_pack(kd_shift[i].st, row.as<double2>(), c.g.V / 16, c.stream);
        kd_s.push_back(kd_shift[i].st);
      }
      SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    }
    outer.alloc(nf, ns, P64, P.nkrylov);
    target_buf.alloc(sizeof(double) * ns);
    const size_t fb = (size_t)nf * ns * prec_bytes(vp);
    fbuf.alloc(fb * 3 + (size_t)nf * ns * 16 * 2);
    auto mkv = [&](void* p, long long n, Prec pr) { Vec v; v.p = p; v.n = n; v.nsys = ns; v.prec = pr; return v; };
    r_s = mkv(fbuf.p, nf, vp);
    tmpA = mkv((char*)fbuf.p + fb, nf, vp);
    tmp_f = mkv((char*)fbuf.p + 2 * fb, nf, vp);
    tmp64 = mkv((char*)fbuf.p + 3 * fb, nf, P64);
    zbuf = mkv((char*)fbuf.p + 3 * fb + (size_t)nf * ns * 16, nf, P64);
    sm_f.alloc(nf, ns, vp, P.smoother_s);
    lev.resize(nlev + 2);
    sm_c.resize(nlev + 2);
    tmp_c.resize(nlev + 2);
    lev[1].alloc(nf, ns, vp, P.inner_maxiter);
    size_t cb = 0;
    for (int l = 2; l <= nlev + 1; ++l) cb += (size_t)c.coarse[l - 2].g.V * c.coarse[l - 2].N * ns * prec_bytes(vp);
    cbuf.alloc(cb > 0 ? cb : 16);
    size_t off = 0;
    for (int l = 2; l <= nlev + 1; ++l) {
      const CoarseLevel& C = c.coarse[l - 2];
      const long long n = (long long)C.g.V * C.N;
      const bool coarsest = (l == nlev + 1);
      lev[l].alloc(n, ns, vp, (coarsest && C.dense) ? 0 : c.inner_maxiter_of(l));
      if (!coarsest) sm_c[l].alloc(n, ns, vp, P.smoother_s);
      tmp_c[l] = mkv((char*)cbuf.p + off, n, vp);
      off += (size_t)n * ns * prec_bytes(vp);
    }
    c.ensure_consts(ns * 2 + 2);
    ws.get(sizeof(double2) * (size_t)(152 * 4) * kMaxPairs * ns);
    {
      sch.assign(nlev + 2, std::vector<Vec>());
      size_t sb = 0;
      for (int l = 2; l <= nlev; ++l)
        if (schur_lvl(l)) sb += (size_t)4 * c.coarse[l - 2].g.V * c.coarse[l - 2].N * ns * prec_bytes(vp);
      if (sb > 0) {
        schbuf.alloc(sb);
        size_t o = 0;
        for (int l = 2; l <= nlev; ++l) {
          if (!schur_lvl(l)) continue;
          const long long n = (long long)c.coarse[l - 2].g.V * c.coarse[l - 2].N;
          for (int i = 0; i < 4; ++i) {
            sch[l].push_back(mkv((char*)schbuf.p + o, n, vp));
            o += (size_t)n * ns * prec_bytes(vp);
          }
        }
      }
    }
    if (c.coarse.back().defl_k > 0) {
      SMG_REQUIRE(ns <= kDeflMaxBlock, "a deflated coarsest level solves at most 64 systems at once");
      const CoarseLevel& C = c.coarse.back();
      const long long n = (long long)C.g.V * C.N;
      const int s = P.coarsest_cheb_s;
      cw.s = s;
      const size_t vb = (size_t)n * ns * prec_bytes(vp);
      cw.vbuf.alloc(vb * (2 * s + (C.schur ? 5 : 0)));
      cw.Q.assign(s, Vec());
      cw.W.assign(s, Vec());
      for (int i = 0; i < s; ++i) {
        cw.W[i] = mkv((char*)cw.vbuf.p + vb * i, n, vp);
        if (i > 0) cw.Q[i] = mkv((char*)cw.vbuf.p + vb * (s + i), n, vp);
      }
      if (C.schur) {
        Vec* sv[5] = {&cw.t1, &cw.t2, &cw.t3, &cw.xe, &cw.rhs};
        for (int i = 0; i < 5; ++i) *sv[i] = mkv((char*)cw.vbuf.p + vb * (2 * s + i), n, vp);
      }
      const int npg = (s + 1) * (s + 2) / 2;       // Gram pairs of [r, W_0 .. W_{s-1}]
      const size_t nd = (size_t)ns * (2 + 3 + npg + s + 2 + 2 * s * s) + (size_t)C.defl_k * ns;
      cw.sbuf.alloc(sizeof(double2) * nd + sizeof(int) * (ns + 1));
      cw.c1 = cw.sbuf.as<double2>();
      cw.c2 = cw.c1 + 2 * ns;
      cw.mgram = cw.c2 + 3 * ns;
      cw.coef = cw.mgram + (size_t)npg * ns;
      cw.rr = cw.coef + (size_t)s * ns;
      cw.bb = cw.rr + ns;
      cw.cscr = cw.bb + ns;
      cw.yd = cw.cscr + (size_t)2 * s * s * ns;
      cw.active = (int*)(cw.yd + (size_t)C.defl_k * ns);
      cw.drun = cw.active + ns;
      // T = (A - c) / h maps [sigma_k, sigma_max] to [-1, 1]
      double cc = 0.5 * (C.cheb_lmax + C.cheb_lmin), h = 0.5 * (C.cheb_lmax - C.cheb_lmin);
      if (!(h > 0.0)) { h = C.cheb_lmax > 0.0 ? 0.5 * C.cheb_lmax : 1.0; cc = h; }
      std::vector<double2> hc((size_t)5 * ns);
      for (int q = 0; q < ns; ++q) {
        hc[2 * q] = make_double2(1.0 / h, 0.0);
        hc[2 * q + 1] = make_double2(-cc / h, 0.0);
        hc[2 * ns + 3 * q] = make_double2(2.0 / h, 0.0);
        hc[2 * ns + 3 * q + 1] = make_double2(-2.0 * cc / h, 0.0);
        hc[2 * ns + 3 * q + 2] = make_double2(-1.0, 0.0);
      }
      SMG_CUDA_OK(cudaMemcpyAsync(cw.c1, hc.data(), sizeof(double2) * hc.size(), cudaMemcpyHostToDevice, c.stream));
      ws.get(sizeof(double2) * (size_t)(2 * 152) * C.defl_k * ns);
      ws.get(sizeof(double2) * (size_t)(2 * 152 / ns + 1) * npg * ns);
      SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    }
    // one cooperative launch for the last GCR level when its coarser level is
    // the dense coarsest (or it is itself the coarsest without a dense solve)
    {
      const int l = c.coarse.back().dense ? nlev : nlev + 1;
      const bool deflated_target = (l == nlev + 1 && c.coarse.back().defl_k > 0);
      if (P.persistent && vp == P32 && l >= 2 && !deflated_target && !schur_lvl(l)) {
        const CoarseLevel& C = c.coarse[l - 2];
        const int nvec_next = l <= nlev ? c.coarse[l - 1].tg.nvec : 0;
        persistent = persist_supported(ns, c.inner_maxiter_of(l), P.smoother_s, C.N, (long long)C.g.V * C.N, sp);
        if (persistent) {
          pplan = persist_plan(C.g, C.N, ns, nvec_next, sp);
          pbuf.alloc(persist_buffer_bytes(pplan, nvec_next));
          if (trace_enabled() || phase_profile_enabled())
            fprintf(stderr, "[smg] persistent level %d: grid %d, %lld rows/CTA, %s, %d systems/stage, %zu B smem\n", l,
                    pplan.grid, pplan.per, pplan.resident ? "resident" : "streaming", pplan.sg, pplan.smem);
        }
      }
    }
  }

  ~Engine() {
    if (graph) cudaGraphExecDestroy(graph);
  }

  cudaStream_t st() const { return c.stream; }

  // debugging aid (SMG_TRACE=1, never inside a capture): prints ||v||^2 of system 0
  void dbg(const char* tag, const Vec& v) {
    if (!trace_enabled()) return;
    cudaStreamCaptureStatus cs;
    SMG_CUDA_OK(cudaStreamIsCapturing(st(), &cs));
    if (cs != cudaStreamCaptureStatusNone) return;
    const int p0[1] = {0};
    double2 h;
    blas_pair_dots(&v, 1, p0, p0, 1, outer.ginv, 1, ws, st());
    SMG_CUDA_OK(cudaMemcpyAsync(&h, outer.ginv, sizeof(double2), cudaMemcpyDeviceToHost, st()));
    SMG_CUDA_OK(cudaStreamSynchronize(st()));
    fprintf(stderr, "[smg]   %-12s |v|^2 = %.6e\n", tag, h.x);
  }

  // ---------------------------------------------------------------- operators
  DslashParams dparams(Store s, int dagger) const {
    DslashParams p;
    p.g = c.g;
    c.link_params(s, p);
    p.mass = mass_dev.as<double>();
    p.dagger = dagger;
    p.nsys = nsys;
    return p;
  }
  void M64(const Vec& out, const Vec& in, const int* run = nullptr, const Vec* sub = nullptr) {
    DslashParams p = dparams(S64, 0);
    p.sub_from = sub ? sub->p : nullptr;
    dslash(out, in, p, st(), run);
  }
  void Ms(const Vec& out, const Vec& in, const int* run, const Vec* sub = nullptr) {
    DslashParams p = dparams(sp, 0);
    p.sub_from = sub ? sub->p : nullptr;
    dslash(out, in, p, st(), run);
  }
  void Binv(const Vec& out, const Vec& in, const int* run, const Vec* sub = nullptr) {
    kd_apply(out, in, c.g, kd_s.data(), sys_map, nkd, 0, st(), run, sub ? sub->p : nullptr, nrhs_);
  }
  // A_1 = (B+m)^{-1} M_1; M_1 = M, or m + D_fat for the truncated operator
  void As(const Vec& out, const Vec& in, const int* run, const Vec* sub = nullptr) {
    DslashParams p = dparams(sp, 0);
    if (c.trunc1()) c.link_params(sp, p, true);
    dslash(tmpA, in, p, st(), run);
    Binv(out, tmpA, run, sub);
  }
  // out = A_l in, or out = sub - A_l in
  void op(int l, const Vec& out, const Vec& in, const int* run, const Vec* sub = nullptr) {
    if (l == 0) Ms(out, in, run, sub);
    else if (l == 1) As(out, in, run, sub);
    else {
      const CoarseLevel& C = c.coarse[l - 2];
      CoarseParams p;
      p.g = C.g; p.N = C.N;
      if (C.schur_level) {      // the Schur complement S of an intermediate level
        const std::vector<Vec>& T = sch[l];
        if (sub == nullptr) {
          schur_apply(out, in, p, C.Ss.st, T[0], T[1], st(), run);
        } else {
          schur_apply(T[2], in, p, C.Ss.st, T[0], T[1], st(), run);
          blas_sub(out, *sub, T[2], st(), run);
        }
        return;
      }
      p.sub_from = sub ? sub->p : nullptr;
      coarse_apply(out, in, p, C.Ss.st, st(), run);
    }
  }

  // CA-GCR(s) post-smoother: e += sum_i a_i A^i V0 with V0 = r - A e preset in
  // S.V[0]; one reduction for the whole Gram system (its Cholesky solve runs
  // in the reduction's last CTA).
  void smooth(int l, SmoothWork& S, const Vec& e, const int* run) {
    for (int i = 1; i <= S.s; ++i) op(l, S.V[i], S.V[i - 1], run);
    Epilogue ep;
    ep.kind = EPI_CA;
    ep.s = S.s;
    ep.d2a = S.coef;
    blas_pair_dots(S.V.data(), S.s + 1, S.pi, S.pj, S.np, S.gram, kMaxPairs, ws, st(), run, ep);
    blas_maxpy(e, S.V.data(), S.s, S.coef, S.s, 1.0, true, st(), run);
  }

  // Batched flexible GCR from G.b into G.x (Sec. 2.1), classical Gram-Schmidt
  // with one re-orthogonalisation pass.  Per iteration: preconditioner,
  // operator, two reductions (the second one's last CTA computes gamma_k,
  // alpha_k, the recursive |r|^2 and the convergence flags), one projection
  // and one fused normalise-and-update kernel.  `abs_target` (device, per
  // system) replaces tol^2 ||b||^2.  With `host`, r already holds the
  // residual and the host polls the run flag before each iteration.
  template <class Pre, class Op>
  int gcr(GcrWork& G, Op&& A, Pre&& precond, double tol, const double* abs_target, const int* run_outer,
          bool host, bool accumulate_x, int* iters_done = nullptr) {
    const int K = G.K;
    if (!accumulate_x) blas_zero(G.x, st(), run_outer);
    if (!host) blas_copy(G.r, G.b, st(), run_outer);
    {
      Epilogue ep;
      ep.kind = EPI_GCR_INIT;
      ep.tol2 = tol * tol;
      ep.abs_target = abs_target;
      ep.da = G.r02; ep.db = (double*)G.r2; ep.dc = G.thr2;
      ep.ia = G.active; ep.ib = G.nk; ep.run = G.run; ep.run_outer = run_outer;
      const int p0[1] = {0};
      blas_pair_dots(&G.r, 1, p0, p0, 1, G.dd, 1, ws, st(), run_outer, ep);
    }
    int done = 0;
    for (int k = 0; k < K; ++k) {
      if (host) {
        int runv = 0;
        SMG_CUDA_OK(cudaMemcpyAsync(&runv, G.run, sizeof(int), cudaMemcpyDeviceToHost, st()));
        SMG_CUDA_OK(cudaStreamSynchronize(st()));
        if (!runv) break;
      }
      precond(G.z[k], G.r, G.run);
      dbg("gcr.z", G.z[k]);
      const bool lvl1 = (&G == &lev[1]) || (&G == &outer);
      if (lvl1) pb(&G == &outer ? "outer.M64" : "L1.A");
      A(G.w[k], G.z[k], G.run);
      if (lvl1) { pe(); pb(&G == &outer ? "outer.gcr_ops" : "L1.gcr_ops"); }
      dbg("gcr.w", G.w[k]);
      int pi[kMaxPairs], pj[kMaxPairs];
      if (k > 0) {
        for (int j = 0; j < k; ++j) { pi[j] = j; pj[j] = k; }
        Epilogue ep;
        ep.kind = EPI_GCR_BETA1;
        ep.k = k; ep.K = K; ep.d2a = G.beta;
        blas_pair_dots(G.w.data(), k + 1, pi, pj, k, G.tmp, K + 2, ws, st(), G.run, ep);
        blas_maxpy(G.w[k], G.w.data(), k, G.tmp, K + 2, -1.0, true, st(), G.run);
      }
      // second pass: <w_j, w_k>, |w_k|^2, <w_k, r>, |r|^2 (the residual before
      // this step's update, summed afresh so that the convergence test never
      // rests on a running difference of squares)
      Vec vv[kMaxVecs + 1];
      for (int j = 0; j <= k; ++j) vv[j] = G.w[j];
      vv[k + 1] = G.r;
      for (int j = 0; j < k; ++j) { pi[j] = j; pj[j] = k; }
      pi[k] = k; pj[k] = k;
      pi[k + 1] = k; pj[k + 1] = k + 1;
      pi[k + 2] = k + 1; pj[k + 2] = k + 1;
      {
        Epilogue ep;
        ep.kind = EPI_GCR_STEP;
        ep.k = k; ep.K = K;
        ep.d2a = G.beta; ep.d2b = G.gamma; ep.d2c = G.alpha; ep.d2d = G.ginv; ep.d2e = G.na;
        ep.db = (double*)G.r2; ep.dc = G.thr2;
        ep.ia = G.active; ep.ib = G.nk; ep.run = G.run; ep.run_outer = run_outer;
        blas_pair_dots(vv, k + 2, pi, pj, k + 3, G.tmp, K + 2, ws, st(), G.run, ep);
      }
      blas_gcr_update(G.w.data(), k, G.tmp, K + 2, G.ginv, G.r, G.na, st(), G.run);
      if (lvl1) pe();
      if (host && trace_enabled()) {
        double h[1];
        SMG_CUDA_OK(cudaMemcpyAsync(h, G.r2, sizeof(double), cudaMemcpyDeviceToHost, st()));
        SMG_CUDA_OK(cudaStreamSynchronize(st()));
        fprintf(stderr, "[smg] outer k=%d |r|^2 (recursive) = %.3e\n", k, h[0]);
      }
      ++done;
    }
    blas_gcr_finish(G.x, G.z.data(), K, G.alpha, G.gamma, G.beta, G.nk, st(), run_outer);
    if (iters_done) *iters_done = done;
    return done;
  }

  // The level-l GCR (with its K-cycle down to the dense coarsest level) as
  // one cooperative launch.
  bool persistent_solve(int l, const int* run) {
    const bool coarsest = (l == nlev + 1);
    const int target = c.coarse.back().dense ? nlev : nlev + 1;
    if (!persistent || l != target) return false;
    const CoarseLevel& C = c.coarse[l - 2];
    GcrWork& G = lev[l];
    PersistArgs a{};
    a.g = C.g; a.N = C.N; a.S = C.Ss.st.p; a.Srs = C.Ss.st.s == S16 ? C.Ss.st.scale : nullptr;
    a.n = (long long)C.g.V * C.N;
    a.has_pre = coarsest ? 0 : 1;
    if (!coarsest) {
      const CoarseLevel& Cn = c.coarse[l - 1];
      a.tg = Cn.tg; a.P = Cn.Ps.st.p; a.D = Cn.D32.as<float2>(); a.nd = Cn.nd;
      a.rc = (float2*)lev[l + 1].b.p;
      a.ec = (float2*)lev[l + 1].x.p;
    }
    a.s = c.params.smoother_s;
    a.K = G.K;
    a.tol2 = c.inner_tol_of(l) * c.inner_tol_of(l);
    a.nsys = nsys;
    a.b = (float2*)G.b.p; a.x = (float2*)G.x.p; a.r = (float2*)G.r.p;
    for (int k = 0; k < G.K; ++k) { a.z[k] = (float2*)G.z[k].p; a.w[k] = (float2*)G.w[k].p; }
    if (!coarsest)
      for (int i = 0; i <= a.s; ++i) a.V[i] = (float2*)sm_c[l].V[i].p;
    const size_t part = ((size_t)pplan.grid * kPersistMaxSys * kPersistSums * sizeof(float2) + 15) & ~(size_t)15;
    a.partial = pbuf.as<float2>();
    a.rpart = (float2*)((char*)pbuf.p + part);
    a.plan = pplan;
    a.bar = (unsigned long long*)((char*)pbuf.p + pbuf.bytes - 64);
    a.exitc = (unsigned*)((char*)pbuf.p + pbuf.bytes - 64 + 8);
    a.err = (int*)((char*)pbuf.p + pbuf.bytes - 64 + 16);
    a.bar_limit_ns = c.dbg_bar_limit_ns;
    a.bar_extra = c.dbg_bar_extra;
    a.run = run;
    a.trace = nullptr;
    a.trace_cap = 0;
    if (prof) {
      // per-phase trace of this launch (CTA 0's barrier exits)
      const int cap = 4096;
      if (trace_buf.p == nullptr) trace_buf.alloc(sizeof(unsigned long long) * (1 + 2 * cap));
      SMG_CUDA_OK(cudaMemsetAsync(trace_buf.p, 0, sizeof(unsigned long long), st()));
      a.trace = trace_buf.as<unsigned long long>();
      a.trace_cap = cap;
    }
    persist_gcr(a, sp, st());
    if (prof) {
      std::vector<unsigned long long> h(1 + 2 * (size_t)a.trace_cap);
      SMG_CUDA_OK(cudaMemcpyAsync(h.data(), trace_buf.p, h.size() * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st()));
      SMG_CUDA_OK(cudaStreamSynchronize(st()));
      const size_t m = std::min<size_t>(h[0], (size_t)a.trace_cap);
      for (size_t i = 1; i < m; ++i)
        phases.add(persist_phase_name((int)h[1 + 2 * i], a.has_pre != 0),
                   1e-6 * (double)(h[2 + 2 * i] - h[2 + 2 * (i - 1)]));
    }
    return true;
  }

  // Bounded device waits that gave up since the last check: the tcgen05
  // coarse apply's error word, then the persistent solver's.
  void check_persistent_error() {
    if (coarse_umma_err_read_and_clear(st()))
      throw StateError("timeout: a bounded wait of the tcgen05 coarse apply gave up");
    if (!persistent) return;
    int err = 0;
    SMG_CUDA_OK(cudaMemcpyAsync(&err, (char*)pbuf.p + pbuf.bytes - 64 + 16, sizeof(int), cudaMemcpyDeviceToHost,
                                st()));
    SMG_CUDA_OK(cudaStreamSynchronize(st()));
    if (err) {
      // clear the barrier words so that a later solve starts from a clean state
      SMG_CUDA_OK(cudaMemsetAsync((char*)pbuf.p + pbuf.bytes - 64, 0, 64, st()));
      SMG_CUDA_OK(cudaStreamSynchronize(st()));
      throw StateError("timeout: a grid barrier of the persistent coarse solver gave up");
    }
  }

  // Table 1's coarsest solver: the deflated start x0 = V diag(1/sigma) U^dag b,
  // then up to inner_maxiter Chebyshev-basis CA-GCR(s) corrections, each one
  // only for the systems whose residual is still above 0.25 ||b||.  A(o, i,
  // run, sub) applies the operator (o = sub - A i when sub is given); r: residual scratch.
  template <class Op>
  void defl_cheb(const CoarseLevel& C, Op&& A, const Vec& b, const Vec& x, const Vec& r, const int* run) {
    const int s = cw.s;
    const long long n = (long long)C.g.V * C.N;
    Vec Ub;
    Ub.p = vp == P64 ? C.dU64.p : C.dU32.p;
    Ub.n = n; Ub.nsys = C.defl_k; Ub.prec = vp;
    Vec Vb = Ub;
    Vb.p = vp == P64 ? C.dV64.p : C.dV32.p;
    block_gram(Ub, b, cw.yd, ws, st(), run);
    block_combine(x, Vb, cw.yd, nsys, st(), run);
    const int p0[1] = {0};
    blas_pair_dots(&b, 1, p0, p0, 1, cw.bb, 1, ws, st(), run);
    const int lv = nlev + 1;    // the coarsest level
    const double tol2 = c.inner_tol_of(lv) * c.inner_tol_of(lv);
    for (int it = 0; it < c.inner_maxiter_of(lv); ++it) {
      const int* rn = it == 0 ? run : cw.drun;
      A(r, x, rn, &b);                                   // r = b - A x
      blas_pair_dots(&r, 1, p0, p0, 1, cw.rr, 1, ws, st(), rn);
      defl_active(cw.rr, cw.bb, tol2, cw.active, cw.drun, nsys, it == 0, st(), run);
      // Chebyshev: Q_0 = r, Q_1 = (A - c) Q_0 / h, Q_{i+1} = 2 (A - c) Q_i / h - Q_{i-1};
      // shifted power basis: Q_{i+1} = (A - c) Q_i / h;  W_i = A Q_i
      cw.Q[0] = r;
      const bool shifted = c.params.coarsest_basis == 1;
      for (int i = 0; i < s; ++i) {
        A(cw.W[i], cw.Q[i], cw.drun, nullptr);
        if (i + 1 == s) break;
        if (i == 0 || shifted) {
          Vec in2[2] = {cw.W[i], cw.Q[i]};
          blas_maxpy(cw.Q[i + 1], in2, 2, cw.c1, 2, 1.0, false, st(), cw.drun);
        } else {
          Vec in3[3] = {cw.W[i], cw.Q[i], cw.Q[i - 1]};
          blas_maxpy(cw.Q[i + 1], in3, 3, cw.c2, 3, 1.0, false, st(), cw.drun);
        }
      }
      // minimum residual over span(W): (W^dag W) a = W^dag r, x += sum_i a_i Q_i;
      // Gram eigenvalues below 1e-12 (FP64 vectors) or 1e-6 (FP32) of the
      // largest are rounding noise of the sums and are left out
      std::vector<Vec> L(s + 1);
      L[0] = r;
      for (int i = 0; i < s; ++i) L[i + 1] = cw.W[i];
      multi_gram(L.data(), s + 1, cw.mgram, ws, st(), cw.drun);
      cagcr_coef(cw.mgram, s, vp == P64 ? 1e-12 : 1e-6, cw.active, cw.coef, cw.cscr, nsys, st(), cw.drun);
      blas_maxpy(x, cw.Q.data(), s, cw.coef, s, 1.0, true, st(), cw.drun);
    }
  }

  // The deflated coarsest solve, on A or (Schur form) on S = 1 - K_eo K_oe of
  // A = 1 + K:  c_e - K_eo c_o = (c + R(c_o))_e with R(u) = u - A u = -K u,
  // S x_e = that, then x_o = c_o - K_oe x_e = (c + R(x_e))_o.
  void deflated_solve(int l, const int* run) {
    const CoarseLevel& C = c.coarse[l - 2];
    GcrWork& G = lev[l];
    CoarseParams cp;
    cp.g = C.g; cp.N = C.N;
    auto A = [&](const Vec& o, const Vec& i, const int* rr, const Vec* sub) {
      if (!C.schur) { op(l, o, i, rr, sub); return; }
      if (sub == nullptr) { schur_apply(o, i, cp, C.Ss.st, cw.t1, cw.t2, st(), rr); return; }
      schur_apply(cw.t3, i, cp, C.Ss.st, cw.t1, cw.t2, st(), rr);
      blas_sub(o, *sub, cw.t3, st(), rr);
    };
    if (!C.schur) {
      defl_cheb(C, A, G.b, G.x, G.r, run);
      return;
    }
    CoarseParams cr = cp;
    parity_pick(cw.t1, nullptr, &G.b, C.g, C.N, st(), run);      // c_o
    cr.sub_from = cw.t1.p;
    coarse_apply(cw.t2, cw.t1, cr, C.Ss.st, st(), run);           // R(c_o)
    Vec in2[2] = {G.b, cw.t2};
    blas_maxpy(cw.t1, in2, 2, c.ones, 2, 1.0, false, st(), run);  // c + R(c_o)
    parity_pick(cw.rhs, &cw.t1, nullptr, C.g, C.N, st(), run);
    defl_cheb(C, A, cw.rhs, cw.xe, G.r, run);
    cr.sub_from = cw.xe.p;
    coarse_apply(cw.t2, cw.xe, cr, C.Ss.st, st(), run);           // R(x_e)
    Vec in2b[2] = {G.b, cw.t2};
    blas_maxpy(cw.t1, in2b, 2, c.ones, 2, 1.0, false, st(), run);
    parity_pick(G.x, &cw.xe, &cw.t1, C.g, C.N, st(), run);
  }

  // solve on level l (>= 2): G = lev[l], input lev[l].b, output lev[l].x
  void coarse_solve(int l, const int* run) {
    const CoarseLevel& C = c.coarse[l - 2];
    GcrWork& G = lev[l];
    const bool coarsest = (l == nlev + 1);
    if (coarsest && C.defl_k > 0) {
      deflated_solve(l, run);
      return;
    }
    if (persistent_solve(l, run)) return;
    if (coarsest && C.dense) {
      if (vp == P64) dense_apply(G.x, G.b, C.D64.p, P64, C.nd, st(), run);
      else dense_apply(G.x, G.b, C.D32.p, P32, C.nd, st(), run);
      return;
    }
    auto A = [&](const Vec& o, const Vec& i, const int* r) { op(l, o, i, r); };
    if (coarsest) {
      auto pre = [&](const Vec& z, const Vec& r, const int* rr) { blas_copy(z, r, st(), rr); };
      gcr(G, A, pre, c.inner_tol_of(l), nullptr, run, false, false);
    } else if (C.schur_level) {
      // c_e - K_eo c_o = (c + R(c_o))_e, GCR on S, x_o = (c + R(x_e))_o
      const std::vector<Vec>& T = sch[l];
      CoarseParams cr;
      cr.g = C.g; cr.N = C.N;
      blas_copy(T[3], G.b, st(), run);
      parity_pick(T[0], nullptr, &T[3], C.g, C.N, st(), run);
      cr.sub_from = T[0].p;
      coarse_apply(T[1], T[0], cr, C.Ss.st, st(), run);
      Vec in2[2] = {T[3], T[1]};
      blas_maxpy(T[0], in2, 2, c.ones, 2, 1.0, false, st(), run);
      parity_pick(G.b, &T[0], nullptr, C.g, C.N, st(), run);
      auto pre = [&](const Vec& z, const Vec& r, const int* rr) { kcycle(l, z, r, rr); };
      gcr(G, A, pre, c.inner_tol_of(l), nullptr, run, false, false);
      cr.sub_from = G.x.p;
      coarse_apply(T[1], G.x, cr, C.Ss.st, st(), run);
      Vec in2b[2] = {T[3], T[1]};
      blas_maxpy(T[0], in2b, 2, c.ones, 2, 1.0, false, st(), run);
      parity_pick(G.x, &G.x, &T[0], C.g, C.N, st(), run);
    } else {
      auto pre = [&](const Vec& z, const Vec& r, const int* rr) { kcycle(l, z, r, rr); };
      gcr(G, A, pre, c.inner_tol_of(l), nullptr, run, false, false);
    }
  }

  // K_l for l >= 1: e = P solve(R r); e += CA-GCR(A_l, r - A_l e)
  void kcycle(int l, const Vec& e, const Vec& r, const int* run) {
    const CoarseLevel& C = c.coarse[l - 1];
    dbg("K.r", r);
    if (l == 1) pb("K1.restrict");
    restrict_op(lev[l + 1].b, r, C.tg, C.Ps.st, st(), run);
    // X^{-1} A_hat e = X^{-1} R r on a block-preconditioned level (Sec. 2.3)
    if (C.block && !C.dense)
      block_diag_apply(lev[l + 1].b, vp == P64 ? C.Xinv64.p : C.Xinv32.p, vp, C.N, st(), run);
    if (l == 1) { pe(); pb("K1.coarse_solve"); }
    dbg("K.rc", lev[l + 1].b);
    coarse_solve(l + 1, run);
    if (l == 1) { pe(); pb("K1.prolong"); }
    dbg("K.ec", lev[l + 1].x);
    prolong_op(e, lev[l + 1].x, C.tg, C.Ps.st, st(), run);
    // a Schur-form level keeps the even part of the full-system correction
    if (schur_lvl(l)) parity_pick(e, &e, nullptr, c.coarse[l - 2].g, c.coarse[l - 2].N, st(), run);
    if (l == 1) { pe(); pb("K1.smoother(A)"); }
    dbg("K.e", e);
    SmoothWork& S = (l == 1) ? sm_f : sm_c[l];
    op(l, S.V[0], e, run, &r);          // V0 = r - A_l e
    smooth(l, S, e, run);
    if (l == 1) pe();
    dbg("K.e+smooth", e);
  }

  // K_0: z (FP64) from r (FP64)
  void precond0_body(const Vec& z, const Vec& r) {
    blas_copy(r_s, r, st());
    dbg("K0.r_s", r_s);
    GcrWork& G = lev[1];
    Binv(G.b, r_s, nullptr);
    dbg("K0.b1", G.b);
    auto A = [&](const Vec& o, const Vec& i, const int* rr) { As(o, i, rr); };
    auto pre = [&](const Vec& zz, const Vec& rr, const int* run) { kcycle(1, zz, rr, run); };
    gcr(G, A, pre, c.inner_tol_of(1), nullptr, nullptr, false, false);
    dbg("K0.x1", G.x);
    pb("K0.smoother(M)");
    Ms(sm_f.V[0], G.x, nullptr, &r_s);   // V0 = r - M e
    smooth(0, sm_f, G.x, nullptr);
    pe();
    blas_copy(z, G.x, st());
  }

  void precond0(const Vec& z, const Vec& r) {
    if (!c.params.use_graph) { precond0_body(z, r); return; }
    if (!graph && !graph_tried) {
      graph_tried = true;
      // first call runs eagerly so that every scratch buffer exists before capture
      precond0_body(zbuf, r);
      SMG_CUDA_OK(cudaStreamSynchronize(st()));
      cudaGraph_t gr = nullptr;
      SMG_CUDA_OK(cudaStreamBeginCapture(st(), cudaStreamCaptureModeThreadLocal));
      const long long before = g_launches;
      precond0_body(zbuf, outer.r);
      graph_nodes = g_launches - before;
      g_launches = before;     // captured launches run when the graph is replayed
      SMG_CUDA_OK(cudaStreamEndCapture(st(), &gr));
      SMG_CUDA_OK(cudaGraphInstantiate(&graph, gr, 0));
      cudaGraphDestroy(gr);
      blas_copy(z, zbuf, st());
      return;
    }
    if (graph && r.p == outer.r.p) {
      SMG_CUDA_OK(cudaGraphLaunch(graph, st()));
      g_launches += graph_nodes;
      blas_copy(z, zbuf, st());
    } else {
      precond0_body(z, r);
    }
  }

  // Outer flexible GCR on M in FP64.  b, x: device FP64 [nsys][V][3].
  // Returns per-system true residuals through `res`.
  void solve(const Vec& b, const Vec& x, double tol, std::vector<double>& res, int& iters, int& restarts) {
    const auto& P = c.params;
    outer.x = x;
    blas_zero(x, st());
    blas_copy(outer.r, b, st());
    const int p0[1] = {0};
    blas_pair_dots(&b, 1, p0, p0, 1, outer.dd, 1, ws, st());
    std::vector<double2> hb(nsys);
    SMG_CUDA_OK(cudaMemcpyAsync(hb.data(), outer.dd, sizeof(double2) * nsys, cudaMemcpyDeviceToHost, st()));
    SMG_CUDA_OK(cudaStreamSynchronize(st()));
    std::vector<double> tgt(nsys), b2(nsys);
    for (int s = 0; s < nsys; ++s) { b2[s] = hb[s].x; tgt[s] = tol * tol * b2[s]; }
    SMG_CUDA_OK(cudaMemcpyAsync(target_buf.p, tgt.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st()));
    iters = 0;
    restarts = 0;
    res.assign(nsys, 0.0);
    prof = phase_profile_enabled() && !c.params.use_graph;
    std::vector<double2> hr(nsys);
    while (true) {
      auto A = [&](const Vec& o, const Vec& i, const int*) { M64(o, i); };
      auto pre = [&](const Vec& z, const Vec& r, const int*) { precond0(z, r); };
      const int left = P.max_outer - iters;
      if (left <= 0) break;
      const int Ksave = outer.K;
      if (left < outer.K) outer.K = left;
      int done = 0;
      gcr(outer, A, pre, 0.0, target_buf.as<double>(), nullptr, true, true, &done);
      outer.K = Ksave;
      iters += done;
      // true residual in FP64
      M64(outer.r, x, nullptr, &b);
      blas_pair_dots(&outer.r, 1, p0, p0, 1, outer.dd, 1, ws, st());
      SMG_CUDA_OK(cudaMemcpyAsync(hr.data(), outer.dd, sizeof(double2) * nsys, cudaMemcpyDeviceToHost, st()));
      SMG_CUDA_OK(cudaStreamSynchronize(st()));
      bool all = true, bad = false;
      for (int s = 0; s < nsys; ++s) {
        res[s] = b2[s] > 0 ? std::sqrt(hr[s].x / b2[s]) : 0.0;
        if (!std::isfinite(res[s])) bad = true;
        if (!(hr[s].x <= tgt[s])) all = false;
      }
      check_persistent_error();
      if (prof) phases.report(st());
      if (bad) throw StateError("breakdown: non-finite residual");
      if (all || done == 0) break;
      ++restarts;
    }
  }
};

void EngineDeleter::operator()(Engine* e) const { delete e; }

// ------------------------------------------------------------------ context
void Context::link_params(Store s, DslashParams& p, bool truncate) const {
  const bool naik = has_naik && !truncate;
  p.fat = fat_of(s);
  p.naik = naik ? naik_of(s) : Stored{};
  p.c_naik = naik ? c_naik : 0.0;
  if (s == S16 || s == S32) {
    if (has_naik && truncate) p.hop = s == S16 ? hop16f.st : hop32f.st;
    else p.hop = s == S16 ? hop16.st : hop32.st;
    p.hop_kinds = naik ? 2 : 1;
    p.hop_naik_scale = (s == S16 && naik) ? naik16.st.gscale : 1.0f;
  }
}

void ctx_set_gauge(Context& c, const void* fat, const void* naik, double c_naik, int where) {
  const size_t nl = (size_t)4 * c.g.V * 9;
  c.engine.reset();
  c.fat64.alloc(nl * sizeof(double2));
  upload(c.fat64.p, fat, nl * sizeof(double2), where, c.stream);
  c.has_naik = naik != nullptr;
  c.c_naik = c.has_naik ? c_naik : 0.0;
  if (c.has_naik) {
    c.naik64.alloc(nl * sizeof(double2));
    upload(c.naik64.p, naik, nl * sizeof(double2), where, c.stream);
  } else {
    c.naik64.release();
  }
  // antiperiodic time boundary: the hops that wrap around the time extent
  // carry -1, i.e. the wrapping time links change sign (fat: the last time
  // slice, Naik: the last three); every operator built from the links follows
  if (c.bc_t < 0) {
    boundary_flip_time(c.fat64.as<double2>(), c.g, 1, c.stream);
    if (c.has_naik) boundary_flip_time(c.naik64.as<double2>(), c.g, 3, c.stream);
  }
  c.fat64_st = Stored{c.fat64.p, nullptr, 1.0f, S64};
  c.naik64_st = Stored{c.naik64.p, nullptr, 1.0f, S64};
  // lower-precision copies; FP16 links carry one global scale (max |entry|)
  auto make_lp = [&](const DevBuf& s64, StoredBuf& d32, StoredBuf& d16) {
    d32.alloc(S32, nl, 0);
    Vec a; a.p = s64.p; a.n = (long long)nl; a.prec = P64;
    Vec b; b.p = d32.v.p; b.n = (long long)nl; b.prec = P32;
    blas_copy(b, a, c.stream);
    // FP16 from FP32 with global scale = max |entry| (device reduction and pack)
    d16.alloc(S16, nl, 0);
    d16.st.gscale = pack_fp16_global((__half2*)d16.v.p, (const float2*)d32.v.p, (long long)nl, c.stream);
  };
  make_lp(c.fat64, c.fat32, c.fat16);
  if (c.has_naik) make_lp(c.naik64, c.naik32, c.naik16);
  else { c.naik32 = StoredBuf(); c.naik16 = StoredBuf(); }
  {
    const double2* n64 = c.has_naik ? c.naik64.as<double2>() : nullptr;
    const float fs = c.fat16.st.gscale, ns = c.has_naik ? c.naik16.st.gscale : 1.0f;
    c.hop16.alloc(S16, hop_link_entries(c.g, c.has_naik, S16), 0);
    build_hop_links(c.hop16.v.p, S16, c.fat64.as<double2>(), n64, c.g, fs, ns, c.stream);
    c.hop16.st.gscale = fs;
    c.hop32.alloc(S32, hop_link_entries(c.g, c.has_naik, S32), 0);
    build_hop_links(c.hop32.v.p, S32, c.fat64.as<double2>(), n64, c.g, 1.0f, 1.0f, c.stream);
    c.hop32.st.gscale = 1.0f;
    if (c.has_naik) {   // fat-only records for the truncated level-1 operator
      c.hop16f.alloc(S16, hop_link_entries(c.g, false, S16), 0);
      build_hop_links(c.hop16f.v.p, S16, c.fat64.as<double2>(), nullptr, c.g, fs, 1.0f, c.stream);
      c.hop16f.st.gscale = fs;
      c.hop32f.alloc(S32, hop_link_entries(c.g, false, S32), 0);
      build_hop_links(c.hop32f.v.p, S32, c.fat64.as<double2>(), nullptr, c.g, 1.0f, 1.0f, c.stream);
      c.hop32f.st.gscale = 1.0f;
    } else {
      c.hop16f = StoredBuf();
      c.hop32f = StoredBuf();
    }
  }
  c.gauge_set = true;
  c.kd_valid = false;
  c.setup_done = false;
  c.coarse.clear();
  if (c.mass_set) ctx_build_kd(c);
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
}

void ctx_build_kd(Context& c) {
  SMG_REQUIRE(c.gauge_set, "set_gauge must come before the KD blocks are built");
  const long long nblk = c.g.V / 16;
  const size_t ne = (size_t)nblk * 48 * 48;
  c.kd_row64.alloc(ne * sizeof(double2));
  kd_build(c.kd_row64.as<double2>(), c.g, c.fat64.as<double2>(), c.mass, c.stream);
  c.kd64.alloc(S64, ne, 0);
  c.kd32.alloc(S32, ne, 0);
  c.kd16.alloc(S16, ne, (size_t)nblk * 48);
  kd_pack(c.kd64.st, c.kd_row64.as<double2>(), nblk, c.stream);
  kd_pack(c.kd32.st, c.kd_row64.as<double2>(), nblk, c.stream);
  kd_pack(c.kd16.st, c.kd_row64.as<double2>(), nblk, c.stream);
  c.kd_valid = true;
}

void ctx_set_mass(Context& c, double m) {
  SMG_REQUIRE(std::isfinite(m), "mass must be finite");
  c.mass = m;
  c.mass_set = true;
  c.engine.reset();
  if (c.gauge_set) ctx_build_kd(c);
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
}

namespace {

// Operator of level l (1 = A on the fine lattice, >= 2 coarse) in FP64 on a
// batch, restricted to one aggregate-crossing part (Galerkin probing).
void op_part64(Context& c, int l, const Vec& out, const Vec& in, Vec& tmp, int part, const int agg[4]) {
  if (l == 1) {
    DslashParams p;
    p.g = c.g;
    p.fat = c.fat64_st;
    if (c.has_naik && !c.trunc1()) {
      p.naik = c.naik64_st;
      p.c_naik = c.c_naik;
    }
    p.mass0 = c.mass;
    p.part = part;
    for (int mu = 0; mu < 4; ++mu) p.agg[mu] = agg[mu];
    p.nsys = in.nsys;
    dslash(tmp, in, p, c.stream);
    const Stored kd = c.kd64.st;
    kd_apply(out, tmp, c.g, &kd, nullptr, 1, 0, c.stream);
  } else {
    const CoarseLevel& C = c.coarse[l - 2];
    CoarseParams p;
    p.g = C.g; p.N = C.N; p.part = part;
    for (int mu = 0; mu < 4; ++mu) p.agg[mu] = agg[mu];
    Stored s{C.S64.p, nullptr, 1.0f, S64};
    coarse_apply(out, in, p, s, c.stream);
  }
}

// The same part of the level-l operator on FP32 vectors with the stored
// (preconditioner-precision) links, KD blocks or stencil: the operator side
// of the mixed-precision Galerkin product.
void op_part_s(Context& c, int l, const Vec& out, const Vec& in, Vec& tmp, int part, const int agg[4]) {
  const Store sp = c.sstore();
  if (l == 1) {
    DslashParams p;
    p.g = c.g;
    c.link_params(sp, p, c.trunc1());
    p.mass0 = c.mass;
    p.part = part;
    for (int mu = 0; mu < 4; ++mu) p.agg[mu] = agg[mu];
    p.nsys = in.nsys;
    dslash(tmp, in, p, c.stream);
    const Stored kd = c.kd_of(sp);
    kd_apply(out, tmp, c.g, &kd, nullptr, 1, 0, c.stream);
  } else {
    const CoarseLevel& C = c.coarse[l - 2];
    CoarseParams p;
    p.g = C.g; p.N = C.N; p.part = part;
    for (int mu = 0; mu < 4; ++mu) p.agg[mu] = agg[mu];
    coarse_apply(out, in, p, C.Ss.st, c.stream);
  }
}

// Level-l operator (and adjoint) in preconditioner precision for the setup CGNE.
struct SetupOp {
  Context& c;
  int l;
  Vec tmp;
  DevBuf tbuf;
  void apply(const Vec& out, const Vec& in, int dagger, const int* run) {
    const Store sp = c.sstore();
    if (l == 1) {
      DslashParams p;
      p.g = c.g;
      c.link_params(sp, p, c.trunc1());
      p.mass0 = c.mass;
      p.nsys = in.nsys;
      const Stored kd = c.kd_of(sp);
      if (!dagger) {
        p.dagger = 0;
        dslash(tmp, in, p, c.stream, run);
        kd_apply(out, tmp, c.g, &kd, nullptr, 1, 0, c.stream, run);
      } else {
        kd_apply(tmp, in, c.g, &kd, nullptr, 1, 1, c.stream, run);
        p.dagger = 1;
        dslash(out, tmp, p, c.stream, run);
      }
    } else {
      const CoarseLevel& C = c.coarse[l - 2];
      CoarseParams p;
      p.g = C.g; p.N = C.N;
      p.allow_tc = 0;   // near-null iterations keep FP32 inputs (CGNE's recursive residual would
                        // otherwise run below the FP16 input rounding)
      // the near-null CGNE runs on A_hat also when the level uses X^{-1} A_hat (Sec. 2.3)
      const Stored& S = dagger ? C.Sdags.st : (C.block ? C.Sraws.st : C.Ss.st);
      coarse_apply(out, in, p, S, c.stream, run);
    }
  }
};

}  // namespace


void ctx_mg_setup(Context& c, const smg_mg_params& P, const void* const* phi0, int where, const DeflRestore* restore) {
  SMG_REQUIRE(c.gauge_set && c.mass_set, "mg_setup needs set_gauge and set_mass first");
  SMG_REQUIRE(P.n_coarse >= 1 && P.n_coarse <= SMG_MAX_COARSE, "n_coarse must be 1..3");
  SMG_REQUIRE(P.inner_maxiter >= 1 && P.inner_maxiter <= 16, "inner_maxiter must be 1..16");
  SMG_REQUIRE(P.coarse_inner_maxiter >= 0 && P.coarse_inner_maxiter <= 16, "coarse_inner_maxiter must be 0..16");
  SMG_REQUIRE(P.coarse_inner_tol >= 0.0 && P.coarse_inner_tol < 1.0, "coarse_inner_tol must be in [0, 1)");
  SMG_REQUIRE(P.nkrylov >= 1 && P.nkrylov <= 16, "nkrylov must be 1..16");
  SMG_REQUIRE(P.smoother_s >= 1 && P.smoother_s <= 10, "smoother_s must be 1..10");
  SMG_REQUIRE(P.precision >= SMG_PREC_DOUBLE && P.precision <= SMG_PREC_HALF, "bad precision");
  SMG_REQUIRE(P.setup_maxiter >= 0 && P.max_outer >= 1, "bad iteration caps");
  SMG_REQUIRE(phi0 != nullptr, "phi0 must hold one start array per coarsening");
  SMG_REQUIRE(P.coarsest_deflate >= 0 && P.coarsest_deflate + defl_guard(P.coarsest_deflate) <= kDeflMaxBlock,
              "coarsest_deflate must be 0..51");
  SMG_REQUIRE(P.coarsest_deflate == 0 || (P.coarsest_cheb_s >= 1 && P.coarsest_cheb_s <= kCaBasisMax),
              "coarsest_cheb_s must be 1..16");
  SMG_REQUIRE(P.coarsest_basis == 0 || P.coarsest_basis == 1, "coarsest_basis must be 0 or 1");
  c.engine.reset();
  c.setup_done = false;
  c.params = P;
  c.coarse.clear();
  c.coarse.resize(P.n_coarse);
  if (!c.kd_valid) ctx_build_kd(c);
  c.setup_mass = c.mass;
  const Prec vp = c.vprec();
  const Store sp = c.sstore();
  cudaStream_t st = c.stream;
  Geom fg = c.g;
  int ndof = 3;
  for (int l = 0; l < P.n_coarse; ++l) {
    CoarseLevel& C = c.coarse[l];
    const int nvec = P.nvec[l];
    SMG_REQUIRE(nvec >= 1 && nvec <= 64, "nvec must be 1..64");
    Geom cg;
    for (int mu = 0; mu < 4; ++mu) {
      const int a = P.agg[l][mu];
      SMG_REQUIRE(a >= 1 && fg.L[mu] % a == 0, "aggregate extents must divide the level's lattice");
      if (l == 0) SMG_REQUIRE(a % 2 == 0 && a >= 4 - (c.has_naik ? 0 : 2),
                              "first aggregates must hold whole hypercubes (even, >= 4 with Naik links)");
      cg.L[mu] = fg.L[mu] / a;
    }
    cg.V = cg.L[0] * cg.L[1] * cg.L[2] * cg.L[3];
    C.g = cg;
    C.N = 2 * nvec;
    C.tg.fine = fg; C.tg.coarse = cg;
    for (int mu = 0; mu < 4; ++mu) C.tg.agg[mu] = P.agg[l][mu];
    C.tg.ndof = ndof; C.tg.nvec = nvec; C.tg.chi_mode = (l == 0) ? 0 : 1;
    if (l > 0) SMG_REQUIRE(ndof % 2 == 0, "coarse dof must be even");
    const long long n = (long long)fg.V * ndof;
    auto clock_phase = [&, t = std::chrono::steady_clock::now()](int ph) mutable {
      SMG_CUDA_OK(cudaStreamSynchronize(st));
      const auto now = std::chrono::steady_clock::now();
      C.setup_s[ph] += std::chrono::duration<double>(now - t).count();
      t = now;
    };
    // ---- near-null vectors: CGNE on A_l phi = 0 from phi0 (Table 1)
    DevBuf raw;
    raw.alloc((size_t)n * nvec * sizeof(double2));
    upload(raw.p, phi0[l], (size_t)n * nvec * sizeof(double2), where, st);
    C.setup_iters = 0;
    if (P.setup_maxiter > 0) {
      SetupOp A{c, l + 1, {}, {}};
      const size_t vb = (size_t)n * nvec * prec_bytes(vp);
      A.tbuf.alloc(vb);
      A.tmp.p = A.tbuf.p; A.tmp.n = n; A.tmp.nsys = nvec; A.tmp.prec = vp;
      DevBuf vbuf;
      vbuf.alloc(vb * 4);
      Vec x, r, p, q;
      Vec* vs[4] = {&x, &r, &p, &q};
      for (int i = 0; i < 4; ++i) { vs[i]->p = (char*)vbuf.p + vb * i; vs[i]->n = n; vs[i]->nsys = nvec; vs[i]->prec = vp; }
      Vec raw64; raw64.p = raw.p; raw64.n = n; raw64.nsys = nvec; raw64.prec = P64;
      blas_copy(x, raw64, st);
      DevBuf sb;
      sb.alloc(sizeof(double2) * nvec * 8 + sizeof(double) * nvec * 2 + sizeof(int) * (2 * nvec + 1));
      double2* rr = sb.as<double2>();
      double2* pp = rr + nvec;
      double2* alpha = pp + nvec;
      double2* nalpha = alpha + nvec;
      double2* bcoef = nalpha + nvec;    // [nvec][2]
      double* rr_prev = (double*)(bcoef + 2 * nvec + 2 * nvec);
      double* rr0 = rr_prev + nvec;
      int* active = (int*)(rr0 + nvec);
      int* iters = active + nvec;
      int* run = iters + nvec;
      c.ensure_consts(nvec);
      // r = -A x ; p = A^dag r
      A.apply(q, x, 0, nullptr);
      blas_maxpy(r, &q, 1, c.mones, 1, 1.0, false, st);
      A.apply(p, r, 1, nullptr);
      const int p0[1] = {0};
      Epilogue e0;
      e0.kind = EPI_CGNE_INIT;
      e0.da = rr_prev; e0.db = rr0; e0.ia = active; e0.ib = iters; e0.run = run;
      blas_pair_dots(&r, 1, p0, p0, 1, rr, 1, c.ws, st, nullptr, e0);
      const double tol2 = P.setup_tol * P.setup_tol;
      for (int it = 0; it < P.setup_maxiter; ++it) {
        if (it % 32 == 0) {
          int runv = 0;
          SMG_CUDA_OK(cudaMemcpyAsync(&runv, run, sizeof(int), cudaMemcpyDeviceToHost, st));
          SMG_CUDA_OK(cudaStreamSynchronize(st));
          if (!runv) break;
        }
        A.apply(q, p, 0, run);
        Epilogue ea;
        ea.kind = EPI_CGNE_ALPHA;
        ea.da = rr_prev; ea.ia = active; ea.d2a = alpha; ea.d2b = nalpha;
        blas_pair_dots(&p, 1, p0, p0, 1, pp, 1, c.ws, st, run, ea);
        blas_maxpy(x, &p, 1, alpha, 1, 1.0, true, st, run);
        blas_maxpy(r, &q, 1, nalpha, 1, 1.0, true, st, run);
        Epilogue eb;
        eb.kind = EPI_CGNE_BETA;
        eb.it = it; eb.tol2 = tol2;
        eb.da = rr_prev; eb.db = rr0; eb.ia = active; eb.ib = iters; eb.d2a = bcoef; eb.run = run;
        blas_pair_dots(&r, 1, p0, p0, 1, rr, 1, c.ws, st, run, eb);
        A.apply(q, r, 1, run);
        Vec pq[2] = {p, q};
        blas_maxpy(p, pq, 2, bcoef, 2, 1.0, false, st, run);
      }
      std::vector<int> hit(nvec);
      SMG_CUDA_OK(cudaMemcpyAsync(hit.data(), iters, sizeof(int) * nvec, cudaMemcpyDeviceToHost, st));
      blas_copy(raw64, x, st);
      SMG_CUDA_OK(cudaStreamSynchronize(st));
      for (int v : hit) C.setup_iters = std::max(C.setup_iters, v);
    }
    clock_phase(0);
    // ---- chiral doubling + block orthonormalisation (FP64); the vectors as
    // the setup produced them are kept for smg_save_setup
    C.pre64.alloc(raw.bytes);
    SMG_CUDA_OK(cudaMemcpyAsync(C.pre64.p, raw.p, raw.bytes, cudaMemcpyDeviceToDevice, st));
    block_orthonormalize(raw.as<double2>(), C.tg, st);
    C.raw64 = std::move(raw);
    C.P64.alloc(S64, (size_t)n * nvec, 0);
    transfer_pack(C.P64.st, C.raw64.as<double2>(), C.tg, st);
    if (sp != S64) {
      C.Ps.alloc(sp, (size_t)n * nvec, 0);
      transfer_pack(C.Ps.st, C.raw64.as<double2>(), C.tg, st);
    } else {
      C.Ps.st = C.P64.st;
    }
    clock_phase(1);
    // ---- Galerkin stencil by probing R A_part P e_j: column j of P on every
    // aggregate at once is P e_j; the part of A that stays in the aggregate or
    // crosses into one neighbour, restricted, gives that block column
    const int N = C.N;
    const long long nc = (long long)cg.V * N;
    C.S64.alloc((size_t)nc * 9 * N * sizeof(double2));
    SMG_CUDA_OK(cudaMemsetAsync(C.S64.p, 0, C.S64.bytes, st));
    if (P.galerkin_tc && sp == S16 && transfer_mma_ok(C.tg, C.Ps.st, P32)) {
      // mixed precision: FP16 prolongator (the K-cycle's), FP32 operator
      // parts, restriction P^dag (A P) on the tensor cores
      int chunk = N;
      const size_t per_col = (size_t)n * 8 * 3 + (size_t)nc * (8 * 2 + 16 * 2);
      while (chunk > 1 && per_col * chunk > ((size_t)16 << 30)) chunk = (chunk + 1) / 2;
      DevBuf pb;
      pb.alloc(per_col * chunk);
      for (int j0 = 0; j0 < N; j0 += chunk) {
        const int ncol = std::min(chunk, N - j0);
        char* base = (char*)pb.p;
        auto vec = [&](size_t off, long long len, Prec pr) {
          Vec v; v.p = base + off; v.n = len; v.nsys = ncol; v.prec = pr; return v;
        };
        const size_t c64 = (size_t)nc * 16 * chunk, c32 = (size_t)nc * 8 * chunk, f32 = (size_t)n * 8 * chunk;
        Vec E64 = vec(0, nc, P64), Cm64 = vec(c64, nc, P64);
        Vec E = vec(2 * c64, nc, P32), Cm = vec(2 * c64 + c32, nc, P32);
        Vec F = vec(2 * c64 + 2 * c32, n, P32), T = vec(2 * c64 + 2 * c32 + f32, n, P32);
        Vec T2 = vec(2 * c64 + 2 * c32 + 2 * f32, n, P32);
        unit_probes((double2*)E64.p, cg.V, N, j0, ncol, st);
        blas_copy(E, E64, st);
        prolong_op(F, E, C.tg, C.Ps.st, st);
        for (int dir = 0; dir < 9; ++dir) {
          op_part_s(c, l + 1, T, F, T2, dir, C.tg.agg);
          restrict_op(Cm, T, C.tg, C.Ps.st, st);
          blas_copy(Cm64, Cm, st);
          galerkin_scatter(C.S64.as<double2>(), (const double2*)Cm64.p, cg, N, dir, j0, ncol, st);
        }
      }
      SMG_CUDA_OK(cudaStreamSynchronize(st));
    } else {
      int chunk = N;
      const size_t per_col = (size_t)n * 16 * 3 + (size_t)nc * 16 * 2;
      while (chunk > 1 && per_col * chunk > ((size_t)8 << 30)) chunk = (chunk + 1) / 2;
      DevBuf pb;
      pb.alloc(per_col * chunk);
      for (int j0 = 0; j0 < N; j0 += chunk) {
        const int ncol = std::min(chunk, N - j0);
        Vec E, F, T, T2, Cm;
        char* base = (char*)pb.p;
        E.p = base; E.n = nc; E.nsys = ncol; E.prec = P64;
        Cm.p = base + (size_t)nc * 16 * chunk; Cm.n = nc; Cm.nsys = ncol; Cm.prec = P64;
        F.p = base + (size_t)nc * 16 * chunk * 2; F.n = n; F.nsys = ncol; F.prec = P64;
        T.p = (char*)F.p + (size_t)n * 16 * chunk; T.n = n; T.nsys = ncol; T.prec = P64;
        T2.p = (char*)T.p + (size_t)n * 16 * chunk; T2.n = n; T2.nsys = ncol; T2.prec = P64;
        unit_probes(E.p ? (double2*)E.p : nullptr, cg.V, N, j0, ncol, st);
        prolong_op(F, E, C.tg, C.P64.st, st);
        for (int dir = 0; dir < 9; ++dir) {
          op_part64(c, l + 1, T, F, T2, dir, C.tg.agg);
          restrict_op(Cm, T, C.tg, C.P64.st, st);
          galerkin_scatter(C.S64.as<double2>(), (const double2*)Cm.p, cg, N, dir, j0, ncol, st);
        }
      }
      SMG_CUDA_OK(cudaStreamSynchronize(st));
    }
    clock_phase(2);
    C.Sdag64.alloc(C.S64.bytes);
    coarse_dagger(C.Sdag64.as<double2>(), C.S64.as<double2>(), cg, N, st);
    // ---- block-preconditioned operator X^{-1} A_hat (Sec. 2.3): the level's GCR,
    // smoother and the next Galerkin product use it, the near-null CGNE keeps A_hat
    C.block = P.block_coarse != 0;
    if (C.block) {
      C.Sraw64.alloc(C.S64.bytes);
      SMG_CUDA_OK(cudaMemcpyAsync(C.Sraw64.p, C.S64.p, C.S64.bytes, cudaMemcpyDeviceToDevice, st));
      C.Xinv64.alloc((size_t)cg.V * N * N * sizeof(double2));
      DevBuf eb;
      eb.alloc(sizeof(int));
      SMG_CUDA_OK(cudaMemsetAsync(eb.p, 0, sizeof(int), st));
      block_precondition(C.S64.as<double2>(), C.Xinv64.as<double2>(), cg, N, eb.as<int>(), st);
      int sing = 0;
      SMG_CUDA_OK(cudaMemcpyAsync(&sing, eb.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      SMG_CUDA_OK(cudaStreamSynchronize(st));
      SMG_REQUIRE(!sing, "a coarse self block X is singular (block_coarse)");
      C.Xinv32.alloc((size_t)cg.V * N * N * sizeof(float2));
      Vec a; a.p = C.Xinv64.p; a.n = (long long)cg.V * N * N; a.prec = P64;
      Vec b; b.p = C.Xinv32.p; b.n = a.n; b.prec = P32;
      blas_copy(b, a, st);
    }
    if (sp != S64) {
      C.Ss.alloc(sp, (size_t)nc * 9 * N, (size_t)nc);
      coarse_pack(C.Ss.st, C.S64.as<double2>(), cg, N, st);
      C.Sdags.alloc(sp, (size_t)nc * 9 * N, (size_t)nc);
      coarse_pack(C.Sdags.st, C.Sdag64.as<double2>(), cg, N, st);
      if (C.block) {
        C.Sraws.alloc(sp, (size_t)nc * 9 * N, (size_t)nc);
        coarse_pack(C.Sraws.st, C.Sraw64.as<double2>(), cg, N, st);
      }
    } else {
      C.Ss.st = Stored{C.S64.p, nullptr, 1.0f, S64};
      C.Sdags.st = Stored{C.Sdag64.p, nullptr, 1.0f, S64};
      if (C.block) C.Sraws.st = Stored{C.Sraw64.p, nullptr, 1.0f, S64};
    }
    // ---- dense coarsest inverse; in block mode that of A_hat, since
    // (X^{-1} A_hat)^{-1} X^{-1} = A_hat^{-1} (the right-hand side then needs no X^{-1})
    C.dense = false;
    if (l == P.n_coarse - 1 && nc <= P.dense_max) {
      C.nd = (int)nc;
      C.D64.alloc((size_t)nc * nc * sizeof(double2));
      dense_from_stencil(C.D64.as<double2>(), (C.block ? C.Sraw64 : C.S64).as<double2>(), cg, N, st);
      DevBuf fac, perm;
      fac.alloc(sizeof(double2) * nc);
      perm.alloc(sizeof(int) * (nc + 1));
      dense_invert(C.D64.as<double2>(), (int)nc, fac.as<double2>(), perm.as<int>(), st);
      int sing = 0;
      SMG_CUDA_OK(cudaMemcpyAsync(&sing, perm.as<int>() + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
      SMG_CUDA_OK(cudaStreamSynchronize(st));
      SMG_REQUIRE(!sing, "coarsest operator is singular");
      C.D32.alloc((size_t)nc * nc * sizeof(float2));
      Vec a; a.p = C.D64.p; a.n = nc * nc; a.prec = P64;
      Vec b; b.p = C.D32.p; b.n = nc * nc; b.prec = P32;
      blas_copy(b, a, st);
      C.dense = true;
    }
    clock_phase(3);
    fg = cg;
    ndof = N;
  }
  if (P.schur_coarse)
    for (int l = 0; l + 1 < P.n_coarse; ++l) {
      CoarseLevel& C = c.coarse[l];
      SMG_REQUIRE(C.block, "schur_coarse needs block_coarse (identity self blocks)");
      for (int mu = 0; mu < 4; ++mu)
        SMG_REQUIRE(C.g.L[mu] % 2 == 0, "schur_coarse needs even coarse extents (every hop changes parity)");
      C.schur_level = true;
    }
  if (P.coarsest_deflate > 0 && !c.coarse.back().dense) {
    CoarseLevel& C = c.coarse.back();
    SMG_REQUIRE(restore != nullptr || phi0[P.n_coarse] != nullptr,
                "coarsest_deflate needs the start block phi0[n_coarse]");
    C.schur = P.coarsest_schur != 0;
    if (C.schur) {
      SMG_REQUIRE(C.block, "coarsest_schur needs block_coarse (identity self blocks)");
      for (int mu = 0; mu < 4; ++mu)
        SMG_REQUIRE(C.g.L[mu] % 2 == 0, "coarsest_schur needs even coarse extents (every hop changes parity)");
    }
    const auto t0 = std::chrono::steady_clock::now();
    if (restore != nullptr) restore_deflation(c, C, *restore);
    else build_deflation(c, C, phi0[P.n_coarse], where);
    SMG_CUDA_OK(cudaStreamSynchronize(st));
    C.setup_s[3] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  c.setup_done = true;
}

int ctx_solve(Context& c, int nrhs, const void* b, int nshift, const double* masses, void* x, double tol, int where,
              smg_solve_info* info) {
  SMG_REQUIRE(c.setup_done, "solve needs mg_setup first");
  SMG_REQUIRE(nrhs >= 1 && nshift >= 1 && nrhs * nshift <= 256, "1 <= nrhs*nshift <= 256");
  SMG_REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
  auto t0 = std::chrono::steady_clock::now();
  std::vector<double> ms;
  if (masses == nullptr) ms.push_back(c.mass);
  else for (int i = 0; i < nshift; ++i) { SMG_REQUIRE(std::isfinite(masses[i]), "masses must be finite"); ms.push_back(masses[i]); }
  const int ns = nrhs * nshift;
  bool reuse = c.engine && c.engine->nsys == ns && c.engine->masses == ms;
  if (!reuse) {
    c.engine.reset();
    c.engine.reset(new Engine(c, ns, ms, nrhs));
  }
  Engine& E = *c.engine;
  const long long nf = (long long)c.g.V * 3;
  const size_t vbytes = (size_t)nf * sizeof(double2);
  DevBuf bx;
  bx.alloc(vbytes * ns * 2);
  Vec bv; bv.p = bx.p; bv.n = nf; bv.nsys = ns; bv.prec = P64;
  Vec xv; xv.p = (char*)bx.p + vbytes * ns; xv.n = nf; xv.nsys = ns; xv.prec = P64;
  for (int sh = 0; sh < nshift; ++sh) upload(bv.sys(sh * nrhs), b, vbytes * nrhs, where, c.stream);
  std::vector<double> res;
  int iters = 0, restarts = 0;
  E.solve(bv, xv, tol, res, iters, restarts);
  download(x, xv.p, vbytes * ns, where, c.stream);
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool all = true;
  for (int s = 0; s < ns; ++s) {
    const bool conv = res[s] <= tol;
    all = all && conv;
    if (info) {
      info[s].converged = conv ? 1 : 0;
      info[s].iterations = iters;
      info[s].restarts = restarts;
      info[s].true_residual = res[s];
      info[s].seconds = secs;
    }
  }
  return all ? SMG_OK : SMG_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------- multi-shift CG
// M(m_i) x_i = b for several masses in one Krylov space (Sec. 4, the
// propagator workflow's multi-shift CG): CG on the base system
// M(m_0)^dag M(m_0) = m_0^2 + D^dag D with m_0 the lightest mass (one dslash
// pair per iteration), shift i = m_i^2 - m_0^2 carried by the scalar zeta_i
// of the three-term Lanczos recurrence (Jegerlehner 1996); then
// x_i = M(m_i)^dag y_i.  FP64 on the full operator.  The scalar recurrences run
// on the host from two device reductions per iteration; a shift stops moving
// once |zeta_i| ||r|| <= tol ||b|| / 2 (margin for the recomputed residual).
int ctx_multishift_cg(Context& c, const void* b, int nshift, const double* masses, void* x, double tol, int maxiter,
                      int where, smg_solve_info* info) {
  SMG_REQUIRE(c.gauge_set, "multishift_cg needs set_gauge first");
  SMG_REQUIRE(nshift >= 1 && nshift <= 64, "multishift_cg: 1 <= nshift <= 64");
  SMG_REQUIRE(tol > 0 && tol < 1 && maxiter >= 1, "multishift_cg: tol in (0, 1), maxiter >= 1");
  std::vector<double> ms(masses, masses + nshift);
  for (double m : ms) SMG_REQUIRE(std::isfinite(m) && m > 0, "multishift_cg: masses must be positive");
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = c.stream;
  const long long n = (long long)c.g.V * 3;
  const size_t vb = (size_t)n * sizeof(double2);
  DevBuf buf;
  buf.alloc(vb * (4 + 2 * (size_t)nshift));
  auto vec = [&](size_t slot, int nsys) {
    Vec v; v.p = (char*)buf.p + vb * slot; v.n = n; v.nsys = nsys; v.prec = P64;
    return v;
  };
  Vec bb = vec(0, 1), r = vec(1, 1), t = vec(2, 1), w = vec(3, 1);
  Vec X = vec(4, nshift), P = vec(4 + (size_t)nshift, nshift);
  // reduction outputs (nshift + 8 entries; entry 4 holds -alpha during the
  // iteration), then coef[3][nshift] and the masses
  const size_t nred = (size_t)nshift + 8;
  DevBuf sc;
  sc.alloc(sizeof(double2) * nred + sizeof(double) * 4 * (size_t)nshift);
  double2* red = sc.as<double2>();
  double* coef = (double*)((char*)sc.p + sizeof(double2) * nred);
  double* mdev = coef + 3 * (size_t)nshift;
  upload(bb.p, b, vb, where, st);
  SMG_CUDA_OK(cudaMemcpyAsync(r.p, bb.p, vb, cudaMemcpyDeviceToDevice, st));
  for (int i = 0; i < nshift; ++i) SMG_CUDA_OK(cudaMemcpyAsync(P.sys(i), bb.p, vb, cudaMemcpyDeviceToDevice, st));
  SMG_CUDA_OK(cudaMemsetAsync(X.p, 0, vb * nshift, st));
  const int p00[1] = {0};
  auto dot1 = [&](const Vec& a, const Vec& bv) {
    Vec vv[2] = {a, bv};
    const int pj[1] = {1};
    blas_pair_dots(vv, 2, p00, pj, 1, red, 1, c.ws, st);
    double2 h;
    SMG_CUDA_OK(cudaMemcpyAsync(&h, red, sizeof(double2), cudaMemcpyDeviceToHost, st));
    SMG_CUDA_OK(cudaStreamSynchronize(st));
    return h.x;
  };
  int base = 0;
  for (int i = 1; i < nshift; ++i) if (ms[i] < ms[base]) base = i;
  const double mb = ms[base];
  DslashParams dp;
  dp.g = c.g;
  c.link_params(S64, dp);
  dp.nsys = 1;
  dp.mass0 = mb;
  double rr = dot1(r, r);
  const double bn = std::sqrt(rr);
  std::vector<double> zeta(nshift, 1.0), zprev(nshift, 1.0), zn(nshift), hcoef(3 * (size_t)nshift);
  std::vector<char> active(nshift, bn > 0 ? 1 : 0);
  double a_prev = 1.0, b_prev = 0.0;
  int it = 0;
  auto any_active = [&]() { for (char a : active) if (a) return true; return false; };
  while (it < maxiter && any_active()) {
    Vec pb = P; pb.p = P.sys(base); pb.nsys = 1;
    dp.dagger = 0;
    dslash(t, pb, dp, st);
    dp.dagger = 1;
    dslash(w, t, dp, st);                        // w = (m_0^2 + D^dag D) p_0
    const double pw = dot1(pb, w);
    SMG_REQUIRE(pw > 0 && std::isfinite(pw), "multishift_cg: breakdown (p^dag A p <= 0)");
    const double a = rr / pw;
    for (int i = 0; i < nshift; ++i) {
      const double d = ms[i] * ms[i] - mb * mb;
      const double den = a * b_prev * (zprev[i] - zeta[i]) + zprev[i] * a_prev * (1.0 + d * a);
      zn[i] = den != 0.0 ? zeta[i] * zprev[i] * a_prev / den : 0.0;
      hcoef[i] = (active[i] && zeta[i] != 0.0) ? a * zn[i] / zeta[i] : 0.0;
    }
    const double2 na = make_double2(-a, 0.0);
    SMG_CUDA_OK(cudaMemcpyAsync(red + 4, &na, sizeof(double2), cudaMemcpyHostToDevice, st));
    blas_maxpy(r, &w, 1, red + 4, 1, 1.0, true, st);   // r -= a w
    const double rr_new = dot1(r, r);
    const double beta = rr_new / rr;
    for (int i = 0; i < nshift; ++i) {
      hcoef[nshift + i] = zn[i];
      hcoef[2 * nshift + i] = zeta[i] != 0.0 ? beta * (zn[i] / zeta[i]) * (zn[i] / zeta[i]) : 0.0;
    }
    SMG_CUDA_OK(cudaMemcpyAsync(coef, hcoef.data(), sizeof(double) * 3 * nshift, cudaMemcpyHostToDevice, st));
    blas_shift_update(X, P, r, coef, st);
    zprev = zeta;
    zeta = zn;
    a_prev = a;
    b_prev = beta;
    rr = rr_new;
    ++it;
    for (int i = 0; i < nshift; ++i)
      if (active[i] && !(std::fabs(zeta[i]) * std::sqrt(rr) > 0.5 * tol * bn)) active[i] = 0;
  }
  // x_i = M(m_i)^dag y_i into P, then b - M(m_i) x_i into X for the residuals
  SMG_CUDA_OK(cudaMemcpyAsync(mdev, ms.data(), sizeof(double) * nshift, cudaMemcpyHostToDevice, st));
  DslashParams q = dp;
  q.nsys = nshift;
  q.mass = mdev;
  q.dagger = 1;
  dslash(P, X, q, st);
  for (int i = 0; i < nshift; ++i) SMG_CUDA_OK(cudaMemcpyAsync(X.sys(i), bb.p, vb, cudaMemcpyDeviceToDevice, st));
  q.dagger = 0;
  q.sub_from = X.p;
  dslash(X, P, q, st);
  blas_pair_dots(&X, 1, p00, p00, 1, red, 1, c.ws, st);
  std::vector<double2> rn(nshift);
  SMG_CUDA_OK(cudaMemcpyAsync(rn.data(), red, sizeof(double2) * nshift, cudaMemcpyDeviceToHost, st));
  download(x, P.p, vb * nshift, where, st);
  SMG_CUDA_OK(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool all = true;
  for (int i = 0; i < nshift; ++i) {
    const double res = bn > 0 ? std::sqrt(std::fmax(rn[i].x, 0.0)) / bn : 0.0;
    const bool conv = res <= tol;
    all = all && conv;
    if (info) {
      info[i].converged = conv ? 1 : 0;
      info[i].iterations = it;
      info[i].restarts = 0;
      info[i].true_residual = res;
      info[i].seconds = secs;
    }
  }
  return all ? SMG_OK : SMG_ERR_NOT_CONVERGED;
}

// The propagator workflow's split (Sec. 4): the n_mg lightest masses by the
// MG solver of the current setup (coarse operators of the setup mass
// reused), the others by multi-shift CG.
int ctx_propagators(Context& c, const void* b, int nmass, const double* masses, int n_mg, void* x, double tol,
                    int cg_maxiter, int where, smg_solve_info* info) {
  SMG_REQUIRE(nmass >= 1 && nmass <= 64 && n_mg >= 0 && n_mg <= nmass, "propagators: 0 <= n_mg <= nmass <= 64");
  SMG_REQUIRE(n_mg == 0 || c.setup_done, "propagators: MG masses need mg_setup first");
  std::vector<int> order(nmass);
  for (int i = 0; i < nmass; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return masses[i] < masses[j]; });
  const long long n = (long long)c.g.V * 3;
  const size_t vb = (size_t)n * sizeof(double2);
  DevBuf bd, xd;
  bd.alloc(vb);
  xd.alloc(vb * (size_t)nmass);
  upload(bd.p, b, vb, where, c.stream);
  std::vector<smg_solve_info> inf(nmass);
  int rc_mg = SMG_OK, rc_cg = SMG_OK;
  if (n_mg > 0) {
    std::vector<double> ml(n_mg);
    for (int k = 0; k < n_mg; ++k) ml[k] = masses[order[k]];
    rc_mg = ctx_solve(c, 1, bd.p, n_mg, ml.data(), xd.p, tol, SMG_DEVICE, inf.data());
  }
  if (n_mg < nmass) {
    std::vector<double> mh(nmass - n_mg);
    for (int k = n_mg; k < nmass; ++k) mh[k - n_mg] = masses[order[k]];
    rc_cg = ctx_multishift_cg(c, bd.p, nmass - n_mg, mh.data(), (char*)xd.p + vb * n_mg, tol, cg_maxiter,
                              SMG_DEVICE, inf.data() + n_mg);
  }
  for (int k = 0; k < nmass; ++k) {
    download((char*)x + vb * order[k], (char*)xd.p + vb * k, vb, where, c.stream);
    if (info) info[order[k]] = inf[k];
  }
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
  return (rc_mg == SMG_OK && rc_cg == SMG_OK) ? SMG_OK : SMG_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------- test hooks
namespace {
struct Scratch {
  DevBuf a, b, t;
};
Vec conv_in(Context& c, DevBuf& buf, const void* in, long long n, int nsys, Prec p, int where) {
  DevBuf stage;
  stage.alloc((size_t)n * nsys * sizeof(double2));
  upload(stage.p, in, stage.bytes, where, c.stream);
  buf.alloc((size_t)n * nsys * prec_bytes(p));
  Vec s; s.p = stage.p; s.n = n; s.nsys = nsys; s.prec = P64;
  Vec d; d.p = buf.p; d.n = n; d.nsys = nsys; d.prec = p;
  blas_copy(d, s, c.stream);
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
  return d;
}
void conv_out(Context& c, void* out, const Vec& v, int where) {
  DevBuf stage;
  stage.alloc((size_t)v.n * v.nsys * sizeof(double2));
  Vec d; d.p = stage.p; d.n = v.n; d.nsys = v.nsys; d.prec = P64;
  blas_copy(d, v, c.stream);
  download(out, stage.p, stage.bytes, where, c.stream);
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
}
Store store_of(int prec) { return prec == SMG_PREC_DOUBLE ? S64 : (prec == SMG_PREC_SINGLE ? S32 : S16); }
Prec vprec_of(int prec) { return prec == SMG_PREC_DOUBLE ? P64 : P32; }
}  // namespace

void ctx_apply_fine(Context& c, int op, int prec, int nsys, const void* in, void* out, int where) {
  SMG_REQUIRE(c.gauge_set && c.mass_set, "set_gauge and set_mass first");
  SMG_REQUIRE(op >= SMG_OP_M && op <= SMG_OP_ADAG, "bad operator");
  SMG_REQUIRE(prec >= SMG_PREC_DOUBLE && prec <= SMG_PREC_HALF, "bad precision");
  SMG_REQUIRE(nsys >= 1 && nsys <= 65535, "bad nsys");
  if (!c.kd_valid) ctx_build_kd(c);
  const long long n = (long long)c.g.V * 3;
  const Prec vp = vprec_of(prec);
  const Store sp = store_of(prec);
  Scratch s;
  Vec vin = conv_in(c, s.a, in, n, nsys, vp, where);
  s.b.alloc(vin.bytes());
  s.t.alloc(vin.bytes());
  Vec vout = vin; vout.p = s.b.p;
  Vec tmp = vin; tmp.p = s.t.p;
  DslashParams p;
  p.g = c.g;
  c.link_params(sp, p);
  p.mass0 = c.mass;
  p.nsys = nsys;
  const Stored kd = c.kd_of(sp);
  switch (op) {
    case SMG_OP_M: p.dagger = 0; dslash(vout, vin, p, c.stream); break;
    case SMG_OP_MDAG: p.dagger = 1; dslash(vout, vin, p, c.stream); break;
    case SMG_OP_KD: kd_apply(vout, vin, c.g, &kd, nullptr, 1, 0, c.stream); break;
    case SMG_OP_KDDAG: kd_apply(vout, vin, c.g, &kd, nullptr, 1, 1, c.stream); break;
    case SMG_OP_A: dslash(tmp, vin, p, c.stream); kd_apply(vout, tmp, c.g, &kd, nullptr, 1, 0, c.stream); break;
    case SMG_OP_ADAG:
      kd_apply(tmp, vin, c.g, &kd, nullptr, 1, 1, c.stream);
      p.dagger = 1;
      dslash(vout, tmp, p, c.stream);
      break;
  }
  conv_out(c, out, vout, where);
}

// which: 0 restrict, 1 prolong, 2 coarse apply
void ctx_transfer(Context& c, int which, int l, int prec, int nsys, const void* in, void* out, int where) {
  SMG_REQUIRE(c.setup_done, "mg_setup first");
  SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "bad level");
  SMG_REQUIRE(prec >= SMG_PREC_DOUBLE && prec <= SMG_PREC_HALF, "bad precision");
  SMG_REQUIRE(nsys >= 1 && nsys <= 65535, "bad nsys");
  CoarseLevel& C = c.coarse[l];
  const Prec vp = vprec_of(prec);
  const Store sp = store_of(prec);
  const long long nfine = (long long)C.tg.fine.V * C.tg.ndof;
  const long long ncoarse = (long long)C.g.V * C.N;
  // the transfer and stencil are kept in FP64 and in the setup's preconditioner precision
  auto pick_P = [&]() -> Stored {
    if (sp == S64) return C.P64.st;
    SMG_REQUIRE(C.Ps.st.s == sp, "that precision was not built by mg_setup");
    return C.Ps.st;
  };
  Scratch s;
  if (which == 0) {
    Vec vin = conv_in(c, s.a, in, nfine, nsys, vp, where);
    s.b.alloc((size_t)ncoarse * nsys * prec_bytes(vp));
    Vec vout; vout.p = s.b.p; vout.n = ncoarse; vout.nsys = nsys; vout.prec = vp;
    restrict_op(vout, vin, C.tg, pick_P(), c.stream);
    conv_out(c, out, vout, where);
  } else if (which == 1) {
    Vec vin = conv_in(c, s.a, in, ncoarse, nsys, vp, where);
    s.b.alloc((size_t)nfine * nsys * prec_bytes(vp));
    Vec vout; vout.p = s.b.p; vout.n = nfine; vout.nsys = nsys; vout.prec = vp;
    prolong_op(vout, vin, C.tg, pick_P(), c.stream);
    conv_out(c, out, vout, where);
  } else {
    Vec vin = conv_in(c, s.a, in, ncoarse, nsys, vp, where);
    s.b.alloc((size_t)ncoarse * nsys * prec_bytes(vp));
    Vec vout = vin; vout.p = s.b.p;
    CoarseParams p;
    p.g = C.g; p.N = C.N;
    Stored S;
    if (sp == S64) S = Stored{C.S64.p, nullptr, 1.0f, S64};
    else { SMG_REQUIRE(C.Ss.st.s == sp, "that precision was not built by mg_setup"); S = C.Ss.st; }
    coarse_apply(vout, vin, p, S, c.stream);
    conv_out(c, out, vout, where);
  }
}

void ctx_coarse_solve(Context& c, int l, int nsys, const void* in, void* out, int where) {
  SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "coarse_solve: bad level");
  SMG_REQUIRE(nsys >= 1 && nsys <= 16, "coarse_solve: 1 <= nsys <= 16");
  const CoarseLevel& C = c.coarse[l];
  const long long n = (long long)C.g.V * C.N;
  // a new engine may grow the context's constant arrays, which a cached
  // engine's captured graph points into: drop the cached one first
  c.engine.reset();
  Engine E(c, nsys, std::vector<double>(1, c.mass), nsys);
  const int lv = l + 2;
  Scratch s;
  Vec vin = conv_in(c, s.a, in, n, nsys, E.vp, where);
  blas_copy(E.lev[lv].b, vin, c.stream);
  E.coarse_solve(lv, nullptr);
  E.check_persistent_error();
  conv_out(c, out, E.lev[lv].x, where);
}

// Fermion action S = phi^dag (M^dag M)^{-1} phi with its vectors:
// Z = M^{-1} (eps phi), Y = eps Z (= M^{-dag} phi since eps M eps = M^dag),
// X = M^{-1} Y, S = |Y|^2, dS/dm = -2 m |X|^2.  Two multigrid solves.
int ctx_fermion_action(Context& c, const void* phi, void* X, void* Y, double tol, int where, double* S,
                       double* dSdm, smg_solve_info* info) {
  SMG_REQUIRE(c.setup_done, "fermion_action needs mg_setup first");
  const size_t nb = (size_t)c.g.V * 3 * sizeof(double2);
  DevBuf buf;
  buf.alloc(nb * 4);
  char* b = (char*)buf.p;
  double2* dphi = (double2*)b;
  double2* dz = (double2*)(b + nb);
  double2* dy = (double2*)(b + 2 * nb);
  double2* dx = (double2*)(b + 3 * nb);
  upload(dphi, phi, nb, where, c.stream);
  eps_mul(dz, dphi, c.g, c.stream);                 // eps phi
  smg_solve_info i1{}, i2{};
  int rc1 = ctx_solve(c, 1, dz, 1, nullptr, dy, tol, SMG_DEVICE, &i1);   // Z
  eps_mul(dy, dy, c.g, c.stream);                   // Y = eps Z
  int rc2 = ctx_solve(c, 1, dy, 1, nullptr, dx, tol, SMG_DEVICE, &i2);   // X = M^{-1} Y
  Vec vy; vy.p = dy; vy.n = (long long)c.g.V * 3; vy.prec = P64;
  Vec vx = vy; vx.p = dx;
  Vec vv[2] = {vy, vx};
  const int pi[2] = {0, 1}, pj[2] = {0, 1};
  DevBuf ob;
  ob.alloc(sizeof(double2) * 2);
  blas_pair_dots(vv, 2, pi, pj, 2, ob.as<double2>(), 2, c.ws, c.stream);
  double2 h[2];
  SMG_CUDA_OK(cudaMemcpyAsync(h, ob.p, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
  if (X) download(X, dx, nb, where, c.stream);
  if (Y) download(Y, dy, nb, where, c.stream);
  SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
  *S = h[0].x;
  *dSdm = -2.0 * c.mass * h[1].x;
  if (info) {
    info[0] = i1;
    info[1] = i2;
  }
  return (rc1 == SMG_OK && rc2 == SMG_OK) ? SMG_OK : SMG_ERR_NOT_CONVERGED;
}

// The 9-point coarse apply (Sec. 3.1) on a caller's FP64 stencil
// [Vc][N][9][N], packed to the storage of `prec` as mg_setup packs its own,
// through kernel `path` (CPATH_*; 0 = the autotuner's choice).
void ctx_coarse_apply_stencil(Context& c, const int cdims[4], int N, int prec, int path, const void* stencil,
                              int nsys, const void* in, void* out, int where) {
  SMG_REQUIRE(N >= 1 && N <= 256 && nsys >= 1 && nsys <= 256, "coarse_apply_stencil: bad sizes");
  SMG_REQUIRE(prec >= SMG_PREC_DOUBLE && prec <= SMG_PREC_HALF, "coarse_apply_stencil: bad precision");
  SMG_REQUIRE(path >= CPATH_AUTO && path < CPATH_COUNT, "coarse_apply_stencil: bad path");
  Geom g;
  g.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    SMG_REQUIRE(cdims[mu] >= 1 && cdims[mu] <= 4096, "coarse_apply_stencil: bad extents");
    g.L[mu] = cdims[mu];
    g.V *= cdims[mu];
  }
  const Store sp = store_of(prec);
  const Prec vp = vprec_of(prec);
  SMG_REQUIRE(path == CPATH_AUTO || coarse_path_ok(path, N, nsys, vp, sp, true),
              "coarse_apply_stencil: that kernel does not serve this shape");
  const long long nc = (long long)g.V * N;
  DevBuf s64;
  s64.alloc((size_t)nc * 9 * N * sizeof(double2));
  upload(s64.p, stencil, s64.bytes, where, c.stream);
  StoredBuf S;
  if (sp != S64) {
    S.alloc(sp, (size_t)nc * 9 * N, (size_t)nc);
    coarse_pack(S.st, s64.as<double2>(), g, N, c.stream);
  } else {
    S.st = Stored{s64.p, nullptr, 1.0f, S64};
  }
  Scratch sc;
  Vec vin = conv_in(c, sc.a, in, nc, nsys, vp, where);
  sc.b.alloc(vin.bytes());
  Vec vout = vin;
  vout.p = sc.b.p;
  CoarseParams p;
  p.g = g;
  p.N = N;
  p.path = path;
  coarse_apply(vout, vin, p, S.st, c.stream);
  const bool tc_err = coarse_umma_err_read_and_clear(c.stream);
  if (tc_err) throw StateError("timeout: a bounded wait of the tcgen05 coarse apply gave up");
  conv_out(c, out, vout, where);
}

// Coarse 9-point apply on a synthetic stencil of a given shape (storage per
// `prec`, FP32 vectors or FP64 for SMG_PREC_DOUBLE), timed over nrep launches.
double ctx_bench_coarse(Context& c, const int cdims[4], int N, int nsys, int prec, int nrep) {
  SMG_REQUIRE(N >= 2 && N <= 256 && nsys >= 1 && nsys <= 64 && nrep >= 1, "bench_coarse: bad sizes");
  Geom g;
  g.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    SMG_REQUIRE(cdims[mu] >= 1, "bench_coarse: bad extents");
    g.L[mu] = cdims[mu];
    g.V *= cdims[mu];
  }
  const Store st = prec == SMG_PREC_DOUBLE ? S64 : (prec == SMG_PREC_SINGLE ? S32 : S16);
  const Prec vp = prec == SMG_PREC_DOUBLE ? P64 : P32;
  const long long ns = (long long)g.V * N * 9 * N;
  StoredBuf S;
  S.alloc(st, (size_t)ns, (size_t)g.V * N);
  synth_fill(S.v.p, st, ns, 12345u, c.stream);
  if (st == S16) synth_fill(S.sc.p, S32, (long long)g.V * N / 2, 777u, c.stream);   // scales: any finite values
  const long long n = (long long)g.V * N;
  DevBuf bi, bo;
  bi.alloc((size_t)n * nsys * prec_bytes(vp));
  bo.alloc((size_t)n * nsys * prec_bytes(vp));
  synth_fill(bi.p, vp == P64 ? S64 : S32, n * nsys, 99u, c.stream);
  Vec in; in.p = bi.p; in.n = n; in.nsys = nsys; in.prec = vp;
  Vec out = in; out.p = bo.p;
  CoarseParams p;
  p.g = g; p.N = N;
  coarse_apply(out, in, p, S.st, c.stream);
  cudaEvent_t e0, e1;
  SMG_CUDA_OK(cudaEventCreate(&e0));
  SMG_CUDA_OK(cudaEventCreate(&e1));
  SMG_CUDA_OK(cudaEventRecord(e0, c.stream));
  for (int i = 0; i < nrep; ++i) coarse_apply(out, in, p, S.st, c.stream);
  SMG_CUDA_OK(cudaEventRecord(e1, c.stream));
  SMG_CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0;
  SMG_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (double)ms / nrep;
}

// Average device time of one launch of a hot kernel on the context's
// stream, in the setup's preconditioner precision, timed with CUDA events
// over `nrep` back-to-back launches (after one warm-up launch).
double ctx_time_kernel(Context& c, int kernel, int l, int nsys, int nrep) {
  SMG_REQUIRE(nrep >= 1 && nsys >= 1 && nsys <= 256, "time_kernel: bad nrep/nsys");
  const Prec vp = c.setup_done ? c.vprec() : P64;
  const Store sp = c.setup_done ? c.sstore() : S64;
  SMG_REQUIRE(c.gauge_set && c.mass_set, "time_kernel needs set_gauge and set_mass");
  if (!c.kd_valid) ctx_build_kd(c);
  long long nin = (long long)c.g.V * 3, nout = nin;
  const CoarseLevel* C = nullptr;
  SMG_REQUIRE(kernel >= SMG_KERNEL_DSLASH && kernel <= SMG_KERNEL_COARSE_SOLVE, "time_kernel: unknown kernel");
  if (kernel == SMG_KERNEL_COARSE_SOLVE) {
    // a whole coarse-level solve through an engine of nsys systems; the
    // engine's work areas are set up before the timed launches
    SMG_REQUIRE(c.setup_done && l >= 0 && l < (int)c.coarse.size(), "time_kernel: bad level");
    SMG_REQUIRE(nsys <= 16, "time_kernel: at most 16 systems for a coarse solve");
    c.engine.reset();
    Engine E(c, nsys, std::vector<double>(1, c.mass), nsys);
    const int lv = l + 2;
    synth_fill(E.lev[lv].b.p, E.vp == P64 ? S64 : S32, E.lev[lv].b.n * nsys, 17u, c.stream);
    DevBuf keep;
    keep.alloc(E.lev[lv].b.bytes());
    SMG_CUDA_OK(cudaMemcpyAsync(keep.p, E.lev[lv].b.p, keep.bytes, cudaMemcpyDeviceToDevice, c.stream));
    auto solve_once = [&]() {
      // a Schur-form solve overwrites its right-hand side: restore it each time
      SMG_CUDA_OK(cudaMemcpyAsync(E.lev[lv].b.p, keep.p, keep.bytes, cudaMemcpyDeviceToDevice, c.stream));
      E.coarse_solve(lv, nullptr);
    };
    solve_once();
    cudaEvent_t e0, e1;
    SMG_CUDA_OK(cudaEventCreate(&e0));
    SMG_CUDA_OK(cudaEventCreate(&e1));
    SMG_CUDA_OK(cudaEventRecord(e0, c.stream));
    for (int i = 0; i < nrep; ++i) solve_once();
    SMG_CUDA_OK(cudaEventRecord(e1, c.stream));
    SMG_CUDA_OK(cudaEventSynchronize(e1));
    float ms = 0;
    SMG_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    E.check_persistent_error();
    return (double)ms / nrep;
  }
  if (kernel >= SMG_KERNEL_RESTRICT && kernel <= SMG_KERNEL_COARSE) {
    SMG_REQUIRE(c.setup_done && l >= 0 && l < (int)c.coarse.size(), "time_kernel: bad level");
    C = &c.coarse[l];
    const long long nf = (long long)C->tg.fine.V * C->tg.ndof, nc = (long long)C->g.V * C->N;
    if (kernel == SMG_KERNEL_RESTRICT) { nin = nf; nout = nc; }
    else if (kernel == SMG_KERNEL_PROLONG) { nin = nc; nout = nf; }
    else { nin = nc; nout = nc; }
  }
  DevBuf bi, bo, bt;
  bi.alloc((size_t)nin * nsys * prec_bytes(vp));
  bo.alloc((size_t)nout * nsys * prec_bytes(vp));
  bt.alloc((size_t)std::max(nin, nout) * nsys * prec_bytes(vp));
  Vec in; in.p = bi.p; in.n = nin; in.nsys = nsys; in.prec = vp;
  Vec out; out.p = bo.p; out.n = nout; out.nsys = nsys; out.prec = vp;
  Vec tmp; tmp.p = bt.p; tmp.n = nin; tmp.nsys = nsys; tmp.prec = vp;
  {
    Vec ones = in;
    c.ensure_consts(1);
    blas_zero(in, c.stream);
    Vec one1; one1.p = c.ones; one1.n = 1; one1.nsys = 1; one1.prec = P64;
    (void)one1; (void)ones;
  }
  DslashParams dp;
  dp.g = c.g;
  c.link_params(sp, dp);
  dp.mass0 = c.mass;
  dp.nsys = nsys;
  const Stored kd = c.kd_of(sp);
  auto launch = [&]() {
    switch (kernel) {
      case SMG_KERNEL_DSLASH: dslash(out, in, dp, c.stream); break;
      case SMG_KERNEL_KD: kd_apply(out, in, c.g, &kd, nullptr, 1, 0, c.stream); break;
      case SMG_KERNEL_RESTRICT: restrict_op(out, in, C->tg, C->Ps.st, c.stream); break;
      case SMG_KERNEL_PROLONG: prolong_op(out, in, C->tg, C->Ps.st, c.stream); break;
      case SMG_KERNEL_COARSE: {
        CoarseParams p; p.g = C->g; p.N = C->N;
        coarse_apply(out, in, p, C->Ss.st, c.stream);
        break;
      }
      case SMG_KERNEL_A:
        dslash(tmp, in, dp, c.stream);
        kd_apply(out, tmp, c.g, &kd, nullptr, 1, 0, c.stream);
        break;
      default: SMG_REQUIRE(false, "time_kernel: unknown kernel");
    }
  };
  launch();
  cudaEvent_t e0, e1;
  SMG_CUDA_OK(cudaEventCreate(&e0));
  SMG_CUDA_OK(cudaEventCreate(&e1));
  SMG_CUDA_OK(cudaEventRecord(e0, c.stream));
  for (int i = 0; i < nrep; ++i) launch();
  SMG_CUDA_OK(cudaEventRecord(e1, c.stream));
  SMG_CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0;
  SMG_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (double)ms / nrep;
}

}  // namespace smg
