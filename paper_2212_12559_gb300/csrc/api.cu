// The C ABI of libsmg (declared in include/smg.h): argument checks, error
// translation and host/device staging around the solver in solver.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "persist.cuh"
#include "solver.cuh"
#include "tune.cuh"

namespace smg {
std::string dot_noalloc(const void* x, const void* y, long long n, int nsys, void* out, cudaStream_t st);
}

struct smg_ctx {
  smg::Context c;
};

namespace {

template <class F>
int guarded(smg_ctx* ctx, F&& f) {
  if (ctx == nullptr) return SMG_ERR_ARG;
  try {
    ctx->c.err.clear();
    return f(ctx->c);
  } catch (const smg::ArgError& e) {
    ctx->c.err = e.what;
    return SMG_ERR_ARG;
  } catch (const smg::OomError& e) {
    ctx->c.err = e.what;
    return SMG_ERR_OOM;
  } catch (const smg::StateError& e) {
    ctx->c.err = e.what;
    if (e.what.rfind("breakdown", 0) == 0) return SMG_ERR_BREAKDOWN;
    if (e.what.rfind("timeout", 0) == 0) return SMG_ERR_TIMEOUT;
    return SMG_ERR_STATE;
  } catch (const smg::CudaError& e) {
    ctx->c.err = e.what;
    return SMG_ERR_CUDA;
  } catch (const std::exception& e) {
    ctx->c.err = e.what();
    return SMG_ERR_CUDA;
  }
}

bool valid_where(int w) { return w == SMG_HOST || w == SMG_DEVICE; }

}  // namespace

extern "C" {

int smg_persist_plan(int V, int N, int nsys, int nvec_next, int prec, int sms, long long smem_cap, long long out[10]) {
  if (out == nullptr || smem_cap <= 0 || (prec != SMG_PREC_SINGLE && prec != SMG_PREC_HALF)) return SMG_ERR_ARG;
  try {
    const smg::PersistPlan p = smg::persist_plan_for(V, N, nsys, nvec_next, prec == SMG_PREC_HALF ? smg::S16 : smg::S32,
                                                      sms, (size_t)smem_cap);
    out[0] = p.grid;
    out[1] = p.per;
    out[2] = p.nslot;
    out[3] = p.resident;
    out[4] = p.sg;
    out[5] = (long long)p.smem;
    out[6] = (long long)p.off_S;
    out[7] = (long long)p.off_sc;
    out[8] = (long long)p.off_P;
    out[9] = (long long)p.off_stg;
    return SMG_OK;
  } catch (...) {
    return SMG_ERR_ARG;
  }
}

void smg_default_params(smg_mg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_coarse = 1;
  for (int l = 0; l < SMG_MAX_COARSE; ++l) {
    for (int mu = 0; mu < 4; ++mu) p->agg[l][mu] = (l == 0) ? 4 : 2;
    p->nvec[l] = (l == 0) ? 24 : 32;
  }
  p->setup_tol = 1e-6;
  p->setup_maxiter = 2000;
  p->inner_tol = 0.25;
  p->inner_maxiter = 8;
  p->smoother_s = 8;
  p->dense_max = 4096;
  p->nkrylov = 16;
  p->max_outer = 500;
  p->precision = SMG_PREC_DOUBLE;
  p->use_graph = 0;
  p->persistent = 1;
  p->truncate_naik = 0;
  p->block_coarse = 0;
  p->coarsest_deflate = 0;
  p->coarsest_cheb_s = 8;
  p->coarsest_schur = 0;
  p->schur_coarse = 0;
  p->coarsest_basis = 0;
  p->coarse_inner_tol = 0.0;
  p->coarse_inner_maxiter = 0;
  p->galerkin_tc = 1;
}

int smg_create(const int dims[4], smg_ctx** out) {
  if (dims == nullptr || out == nullptr) return SMG_ERR_ARG;
  *out = nullptr;
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 4 || dims[mu] % 2 != 0) return SMG_ERR_ARG;
    V *= dims[mu];
  }
  if (V > (1LL << 30)) return SMG_ERR_ARG;
  smg_ctx* ctx = new (std::nothrow) smg_ctx();
  if (!ctx) return SMG_ERR_OOM;
  for (int mu = 0; mu < 4; ++mu) ctx->c.g.L[mu] = dims[mu];
  ctx->c.g.V = (int)V;
  if (cudaStreamCreateWithFlags(&ctx->c.own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return SMG_ERR_CUDA;
  }
  ctx->c.stream = ctx->c.own_stream;
  *out = ctx;
  return SMG_OK;
}

int smg_destroy(smg_ctx* ctx) {
  if (!ctx) return SMG_ERR_ARG;
  cudaStreamSynchronize(ctx->c.stream);
  delete ctx;
  return SMG_OK;
}

const char* smg_last_error(const smg_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->c.err.c_str();
}

int smg_set_stream(smg_ctx* ctx, void* stream) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    c.stream = stream ? (cudaStream_t)stream : c.own_stream;
    c.engine.reset();
    return SMG_OK;
  });
}

int smg_set_gauge(smg_ctx* ctx, const void* fat, const void* naik, double c_naik, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(fat != nullptr && valid_where(where), "set_gauge: null links or bad `where`");
    SMG_REQUIRE(std::isfinite(c_naik), "set_gauge: c_naik must be finite");
    smg::ctx_set_gauge(c, fat, naik, c_naik, where);
    return SMG_OK;
  });
}

int smg_set_boundary(smg_ctx* ctx, int flags) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(flags == 0 || flags == SMG_BC_T_ANTIPERIODIC, "set_boundary: unknown flags");
    c.bc_t = (flags & SMG_BC_T_ANTIPERIODIC) ? -1 : 1;
    c.engine.reset();
    c.gauge_set = false;
    c.kd_valid = false;
    c.setup_done = false;
    c.coarse.clear();
    return SMG_OK;
  });
}

int smg_set_mass(smg_ctx* ctx, double mass) {
  return guarded(ctx, [&](smg::Context& c) {
    smg::ctx_set_mass(c, mass);
    return SMG_OK;
  });
}

int smg_mg_setup(smg_ctx* ctx, const smg_mg_params* params, const void* const* phi0, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(params != nullptr && valid_where(where), "mg_setup: null params or bad `where`");
    if (!c.gauge_set || !c.mass_set) throw smg::StateError("mg_setup needs set_gauge and set_mass first");
    smg::ctx_mg_setup(c, *params, phi0, where);
    return SMG_OK;
  });
}

int smg_save_setup(smg_ctx* ctx, const char* path) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(path != nullptr, "save_setup: null path");
    if (!c.setup_done) throw smg::StateError("save_setup needs mg_setup first");
    smg::ctx_save_setup(c, path);
    return SMG_OK;
  });
}

int smg_load_setup(smg_ctx* ctx, const char* path, const smg_mg_params* params) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(path != nullptr, "load_setup: null path");
    if (!c.gauge_set || !c.mass_set) throw smg::StateError("load_setup needs set_gauge and set_mass first");
    smg::ctx_load_setup(c, path, params);
    return SMG_OK;
  });
}

int smg_solve(smg_ctx* ctx, const void* b, void* x, double tol, int where, smg_solve_info* info) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(b != nullptr && x != nullptr && valid_where(where), "solve: null buffer or bad `where`");
    if (!c.setup_done) throw smg::StateError("solve needs mg_setup first");
    return smg::ctx_solve(c, 1, b, 1, nullptr, x, tol, where, info);
  });
}

int smg_multi_solve(smg_ctx* ctx, int nrhs, const void* b, int nshift, const double* masses, void* x, double tol,
                    int where, smg_solve_info* info) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(b != nullptr && x != nullptr && masses != nullptr && valid_where(where),
                "multi_solve: null buffer or bad `where`");
    if (!c.setup_done) throw smg::StateError("multi_solve needs mg_setup first");
    return smg::ctx_solve(c, nrhs, b, nshift, masses, x, tol, where, info);
  });
}

int smg_multishift_cg(smg_ctx* ctx, const void* b, int nshift, const double* masses, void* x, double tol, int maxiter,
                      int where, smg_solve_info* info) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(b != nullptr && x != nullptr && masses != nullptr && valid_where(where),
                "multishift_cg: null buffer or bad `where`");
    if (!c.gauge_set) throw smg::StateError("multishift_cg needs set_gauge first");
    return smg::ctx_multishift_cg(c, b, nshift, masses, x, tol, maxiter, where, info);
  });
}

int smg_propagators(smg_ctx* ctx, const void* b, int nmass, const double* masses, int n_mg, void* x, double tol,
                    int cg_maxiter, int where, smg_solve_info* info) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(b != nullptr && x != nullptr && masses != nullptr && valid_where(where),
                "propagators: null buffer or bad `where`");
    if (!c.gauge_set) throw smg::StateError("propagators needs set_gauge first");
    if (n_mg > 0 && !c.setup_done) throw smg::StateError("propagators: MG masses need mg_setup first");
    return smg::ctx_propagators(c, b, nmass, masses, n_mg, x, tol, cg_maxiter, where, info);
  });
}

int smg_apply_fine(smg_ctx* ctx, int op, int prec, int nsys, const void* in, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(in != nullptr && out != nullptr && valid_where(where), "apply_fine: null buffer or bad `where`");
    if (!c.gauge_set || !c.mass_set) throw smg::StateError("apply_fine needs set_gauge and set_mass first");
    smg::ctx_apply_fine(c, op, prec, nsys, in, out, where);
    return SMG_OK;
  });
}

int smg_get_maps(smg_ctx* ctx, const int agg[4], int* parity, int* kd_block, int* kd_pos, int* agg_idx, int* agg_pos,
                 int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(agg && parity && kd_block && kd_pos && agg_idx && agg_pos && valid_where(where),
                "get_maps: null argument");
    for (int mu = 0; mu < 4; ++mu)
      SMG_REQUIRE(agg[mu] >= 1 && c.g.L[mu] % agg[mu] == 0, "get_maps: aggregate must divide the lattice");
    smg::DevBuf buf;
    const size_t V = c.g.V;
    buf.alloc(sizeof(int) * V * 5);
    int* d = buf.as<int>();
    smg::site_maps(d, d + V, d + 2 * V, d + 3 * V, d + 4 * V, c.g, agg, c.stream);
    int* outs[5] = {parity, kd_block, kd_pos, agg_idx, agg_pos};
    for (int i = 0; i < 5; ++i) smg::download(outs[i], d + i * V, sizeof(int) * V, where, c.stream);
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    return SMG_OK;
  });
}

int smg_get_kd_inverse(smg_ctx* ctx, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(out != nullptr && valid_where(where), "get_kd_inverse: null buffer");
    if (!c.gauge_set || !c.mass_set) throw smg::StateError("get_kd_inverse needs set_gauge and set_mass");
    if (!c.kd_valid) smg::ctx_build_kd(c);
    smg::download(out, c.kd_row64.p, c.kd_row64.bytes, where, c.stream);
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    return SMG_OK;
  });
}

int smg_get_null_vectors(smg_ctx* ctx, int l, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(out != nullptr && valid_where(where), "get_null_vectors: null buffer");
    if (!c.setup_done) throw smg::StateError("get_null_vectors needs mg_setup");
    SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "get_null_vectors: bad level");
    smg::download(out, c.coarse[l].raw64.p, c.coarse[l].raw64.bytes, where, c.stream);
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    return SMG_OK;
  });
}

int smg_get_coarse_op(smg_ctx* ctx, int l, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(out != nullptr && valid_where(where), "get_coarse_op: null buffer");
    if (!c.setup_done) throw smg::StateError("get_coarse_op needs mg_setup");
    SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "get_coarse_op: bad level");
    smg::download(out, c.coarse[l].S64.p, c.coarse[l].S64.bytes, where, c.stream);
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    return SMG_OK;
  });
}

int smg_get_coarse_xinv(smg_ctx* ctx, int l, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(out != nullptr && valid_where(where), "get_coarse_xinv: null buffer");
    if (!c.setup_done) throw smg::StateError("get_coarse_xinv needs mg_setup");
    SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "get_coarse_xinv: bad level");
    if (!c.coarse[l].block) throw smg::StateError("get_coarse_xinv needs a block_coarse setup");
    smg::download(out, c.coarse[l].Xinv64.p, c.coarse[l].Xinv64.bytes, where, c.stream);
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    return SMG_OK;
  });
}

int smg_get_deflation(smg_ctx* ctx, double* sigma, double* info) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(sigma != nullptr && info != nullptr, "get_deflation: null buffer");
    if (!c.setup_done || c.coarse.empty() || c.coarse.back().defl_k == 0)
      throw smg::StateError("get_deflation needs a setup with a deflated coarsest level");
    const smg::CoarseLevel& C = c.coarse.back();
    for (int i = 0; i < C.defl_k; ++i) sigma[i] = C.sigma[i];
    info[0] = C.cheb_lmin;
    info[1] = C.cheb_lmax;
    info[2] = C.defl_iters;
    info[3] = C.defl_res;
    return SMG_OK;
  });
}

int smg_coarse_solve(smg_ctx* ctx, int l, int nsys, const void* in, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(in && out && valid_where(where), "coarse_solve: null buffer");
    if (!c.setup_done) throw smg::StateError("coarse_solve needs mg_setup");
    smg::ctx_coarse_solve(c, l, nsys, in, out, where);
    return SMG_OK;
  });
}

int smg_restrict(smg_ctx* ctx, int l, int prec, int nsys, const void* in, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(in && out && valid_where(where), "restrict: null buffer");
    if (!c.setup_done) throw smg::StateError("restrict needs mg_setup");
    smg::ctx_transfer(c, 0, l, prec, nsys, in, out, where);
    return SMG_OK;
  });
}

int smg_prolong(smg_ctx* ctx, int l, int prec, int nsys, const void* in, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(in && out && valid_where(where), "prolong: null buffer");
    if (!c.setup_done) throw smg::StateError("prolong needs mg_setup");
    smg::ctx_transfer(c, 1, l, prec, nsys, in, out, where);
    return SMG_OK;
  });
}

int smg_coarse_apply(smg_ctx* ctx, int l, int prec, int nsys, const void* in, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(in && out && valid_where(where), "coarse_apply: null buffer");
    if (!c.setup_done) throw smg::StateError("coarse_apply needs mg_setup");
    smg::ctx_transfer(c, 2, l, prec, nsys, in, out, where);
    return SMG_OK;
  });
}

int smg_force(smg_ctx* ctx, const void* X, const void* Y, int which, void* F, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(X && Y && F && valid_where(where) && (which == 0 || which == 1), "force: bad argument");
    if (!c.gauge_set) throw smg::StateError("force needs set_gauge");
    SMG_REQUIRE(which == 0 || c.has_naik, "force: no Naik links were set");
    const size_t nv = (size_t)c.g.V * 3 * sizeof(double2);
    const size_t nf = (size_t)c.g.V * 36 * sizeof(double2);
    smg::DevBuf buf;
    buf.alloc(2 * nv + nf);
    char* b = (char*)buf.p;
    smg::upload(b, X, nv, where, c.stream);
    smg::upload(b + nv, Y, nv, where, c.stream);
    smg::force_outer((double2*)(b + 2 * nv), (const double2*)b, (const double2*)(b + nv), c.g, which ? 3 : 1,
                     which ? c.c_naik : 1.0, c.bc_t, c.stream);
    smg::download(F, b + 2 * nv, nf, where, c.stream);
    SMG_CUDA_OK(cudaStreamSynchronize(c.stream));
    return SMG_OK;
  });
}

int smg_setup_iterations(smg_ctx* ctx, int l, int* iters) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(iters != nullptr, "setup_iterations: null output");
    if (!c.setup_done) throw smg::StateError("setup_iterations needs mg_setup");
    SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "setup_iterations: bad level");
    *iters = c.coarse[l].setup_iters;
    return SMG_OK;
  });
}

int smg_setup_times(smg_ctx* ctx, int l, double secs[4]) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(secs != nullptr, "setup_times: null output");
    if (!c.setup_done) throw smg::StateError("setup_times needs mg_setup");
    SMG_REQUIRE(l >= 0 && l < (int)c.coarse.size(), "setup_times: bad level");
    for (int i = 0; i < 4; ++i) secs[i] = c.coarse[l].setup_s[i];
    return SMG_OK;
  });
}

int smg_fermion_action(smg_ctx* ctx, const void* phi, void* X, void* Y, double tol, int where, double* S,
                       double* dSdm, smg_solve_info* info) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(phi && S && dSdm && valid_where(where), "fermion_action: null argument");
    if (!c.setup_done) throw smg::StateError("fermion_action needs mg_setup first");
    SMG_REQUIRE(tol > 0 && tol < 1, "fermion_action: tol must be in (0, 1)");
    return smg::ctx_fermion_action(c, phi, X, Y, tol, where, S, dSdm, info);
  });
}

int smg_time_kernel(smg_ctx* ctx, int kernel, int l, int nsys, int nrep, double* ms_per_launch) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(ms_per_launch != nullptr, "time_kernel: null output");
    *ms_per_launch = smg::ctx_time_kernel(c, kernel, l, nsys, nrep);
    return SMG_OK;
  });
}

long long smg_kernel_launches(void) { return smg::g_launches; }

int smg_bench_coarse_apply(smg_ctx* ctx, const int cdims[4], int N, int nsys, int prec, int nrep,
                           double* ms_per_launch) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(cdims != nullptr && ms_per_launch != nullptr, "bench_coarse_apply: null argument");
    SMG_REQUIRE(prec >= SMG_PREC_DOUBLE && prec <= SMG_PREC_HALF, "bench_coarse_apply: bad precision");
    *ms_per_launch = smg::ctx_bench_coarse(c, cdims, N, nsys, prec, nrep);
    return SMG_OK;
  });
}

int smg_coarse_apply_stencil(smg_ctx* ctx, const int cdims[4], int N, int prec, int path, const void* stencil,
                             int nsys, const void* in, void* out, int where) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(cdims && stencil && in && out && valid_where(where), "coarse_apply_stencil: null argument");
    smg::ctx_coarse_apply_stencil(c, cdims, N, prec, path, stencil, nsys, in, out, where);
    return SMG_OK;
  });
}

int smg_coarse_paths(int N, int nsys, int prec, int* paths, int cap) {
  if (paths == nullptr || cap < 1 || N < 1 || nsys < 1 || prec < SMG_PREC_DOUBLE || prec > SMG_PREC_HALF)
    return SMG_ERR_ARG;
  const smg::Prec vp = prec == SMG_PREC_DOUBLE ? smg::P64 : smg::P32;
  const smg::Store sp = prec == SMG_PREC_DOUBLE ? smg::S64 : (prec == SMG_PREC_SINGLE ? smg::S32 : smg::S16);
  return smg::coarse_path_list(N, nsys, vp, sp, true, paths, cap);
}

int smg_debug_persist_barrier(smg_ctx* ctx, long long limit_ns, int extra_arrivals) {
  return guarded(ctx, [&](smg::Context& c) {
    SMG_REQUIRE(limit_ns >= 1000 && limit_ns <= 2000000000LL && (extra_arrivals == 0 || extra_arrivals == 1),
                "debug_persist_barrier: limit in [1 us, 2 s], extra arrivals 0 or 1");
    c.dbg_bar_limit_ns = (unsigned long long)limit_ns;
    c.dbg_bar_extra = extra_arrivals;
    return SMG_OK;
  });
}

int smg_tune_mode(int mode) {
  if (mode != 0 && mode != 1) return SMG_ERR_ARG;
  smg::tune_set_mode(mode);
  return SMG_OK;
}

long long smg_tune_table(char* buf, long long cap) {
  const std::string t = smg::tune_table_text();
  if (buf != nullptr && cap > 0) {
    const size_t m = std::min((size_t)(cap - 1), t.size());
    std::memcpy(buf, t.data(), m);
    buf[m] = '\0';
  }
  return (long long)t.size() + 1;
}

int smg_tune_load(const char* path) {
  if (path == nullptr) return SMG_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (f == nullptr) return SMG_ERR_ARG;
  std::string text;
  char buf[4096];
  size_t m;
  while ((m = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, m);
  std::fclose(f);
  return smg::tune_table_load(text) < 0 ? SMG_ERR_ARG : SMG_OK;
}

int smg_tune_save(const char* path) {
  if (path == nullptr) return SMG_ERR_ARG;
  FILE* f = std::fopen(path, "wb");
  if (f == nullptr) return SMG_ERR_ARG;
  const std::string t = smg::tune_table_text();
  const bool ok = std::fwrite(t.data(), 1, t.size(), f) == t.size();
  return (std::fclose(f) == 0 && ok) ? SMG_OK : SMG_ERR_ARG;
}

int smg_tune_clear(void) {
  smg::tune_table_clear();
  return SMG_OK;
}

int smg_dot_noalloc(smg_ctx* ctx, const void* x, const void* y, long long n, int nsys, void* out) {
  if (ctx == nullptr) return SMG_ERR_ARG;
  std::string err = smg::dot_noalloc(x, y, n, nsys, out, ctx->c.stream);
  if (err.empty()) return SMG_OK;
  const bool arg = err.rfind("dot_noalloc:", 0) == 0;
  ctx->c.err = std::move(err);
  return arg ? SMG_ERR_ARG : SMG_ERR_CUDA;
}

}  // extern "C"
