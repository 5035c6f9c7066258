// Host-side solver state: the context behind the C ABI, the multigrid
// hierarchy and the batched Krylov work areas.
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "ops.cuh"
#include "smg.h"

namespace smg {

struct OomError {
  std::string what;
  explicit OomError(std::string w) : what(std::move(w)) {}
};
struct StateError {
  std::string what;
  explicit StateError(std::string w) : what(std::move(w)) {}
};

// Owning device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t b);
  void release();
  template <class T> T* as() const { return (T*)p; }
};

// Operator data in one storage precision (values + optional FP16 scales).
struct StoredBuf {
  DevBuf v, sc;
  Stored st;
  void alloc(Store s, size_t elems, size_t nscale);
};

struct CoarseLevel {
  TransferGeom tg;          // fine side = the previous level
  StoredBuf P64, Ps;        // prolongator, FP64 and preconditioner precision
  DevBuf raw64;             // block-orthonormal vectors, FP64 [nvec][V][ndof]
  Geom g;                   // coarse lattice
  int N = 0;                // coarse dof per site
  DevBuf S64, Sdag64;       // FP64 stencil of the level's operator, adjoint of A_hat
  StoredBuf Ss, Sdags;      // preconditioner-precision copies
  bool block = false;       // the level's operator is X^{-1} A_hat (Sec. 2.3)
  DevBuf Sraw64, Xinv64, Xinv32;   // block mode: A_hat (near-null CGNE) and X^{-1} [Vc][N][N]
  StoredBuf Sraws;          // block mode: A_hat in preconditioner precision
  // deflated coarsest level (Table 1): V (right singular vectors) and
  // U diag(1/sigma) (left ones over sigma), [k][Vc][N], FP64 and FP32
  int defl_k = 0;
  bool schur = false;       // deflated solve on the even/odd Schur complement (vectors vanish on odd sites)
  bool schur_level = false; // intermediate level: GCR and smoother on the Schur complement
  DevBuf dV64, dU64, dV32, dU32;
  std::vector<double> sigma;
  double cheb_lmin = 0.0, cheb_lmax = 0.0, defl_res = 0.0;
  int defl_iters = 0;
  bool dense = false;       // exact coarsest solve
  DevBuf D64, D32;          // dense inverse
  int nd = 0;
  int setup_iters = 0;
  // wall-clock seconds of this coarsening's setup phases (stream synchronised
  // at each boundary): near-null CGNE, chiral doubling + block
  // orthonormalisation + packing, Galerkin stencil, the rest (dagger, block
  // preconditioning, packing, dense inverse or deflation)
  double setup_s[4] = {0, 0, 0, 0};
  DevBuf pre64;             // near-null vectors as the setup produced them (before chiral
                            // doubling and block orthonormalisation), FP64 [nvec][V][ndof]:
                            // what smg_save_setup writes
};

// Deflation state of the coarsest level read back from a saved setup.
struct DeflRestore {
  int k = 0, iters = 0;
  double lmin = 0.0, lmax = 0.0, res = 0.0;
  std::vector<double> sigma;
  const void* V = nullptr;   // host FP64 [k][Vc][N]
  const void* U = nullptr;   // host FP64 U diag(1/sigma), [k][Vc][N]
};

// Per-system scalars and vectors of one batched GCR.
struct GcrWork {
  int K = 0, nsys = 0;
  std::vector<Vec> z, w;
  Vec r, x, b;
  DevBuf vbuf, sbuf;
  double2 *alpha, *beta, *gamma, *y, *tmp, *dd, *na, *ginv, *r2;
  double *r02, *thr2;
  int *active, *nk, *run;
  void alloc(long long n, int nsys, Prec p, int K);
};

struct SmoothWork {
  int s = 0;
  std::vector<Vec> V;
  DevBuf vbuf, sbuf;
  double2 *gram, *coef;
  int pi[kMaxPairs], pj[kMaxPairs], np = 0;
  void alloc(long long n, int nsys, Prec p, int s);
};

struct Engine;
struct EngineDeleter {
  void operator()(Engine* e) const;
};

struct Context {
  Geom g{};
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  std::string err;
  // gauge field
  bool gauge_set = false, has_naik = false;
  double c_naik = 0.0;
  int bc_t = 1;               // time boundary: 1 periodic, -1 antiperiodic (smg_set_boundary)
  DevBuf fat64, naik64;
  StoredBuf fat32, naik32, fat16, naik16;
  StoredBuf hop32, hop16;     // phase-folded link copies (hop.cu)
  StoredBuf hop32f, hop16f;   // the same without the Naik links (truncated level-1 operator)
  // mass and KD blocks
  double mass = 0.0;
  bool mass_set = false, kd_valid = false;
  DevBuf kd_row64;            // [nblk][48][48] row-major FP64 (B+m)^{-1}
  StoredBuf kd64, kd32, kd16; // apply layout
  // multigrid
  bool setup_done = false;
  smg_mg_params params{};
  double setup_mass = 0.0;
  std::vector<CoarseLevel> coarse;
  Workspace ws;
  std::unique_ptr<Engine, EngineDeleter> engine;
  DevBuf consts;               // +1 / -1 coefficient arrays
  double2 *ones = nullptr, *mones = nullptr;
  int nconst = 0;
  // test hook (smg_debug_persist_barrier): grid-barrier wait limit and extra
  // expected arrivals of the persistent coarse solver
  unsigned long long dbg_bar_limit_ns = 2000000000ull;
  int dbg_bar_extra = 0;
  ~Context();

  Prec vprec() const { return params.precision == SMG_PREC_DOUBLE ? P64 : P32; }
  // inner GCR rule of level l >= 1 (levels >= 2 may have their own)
  double inner_tol_of(int l) const {
    return (l >= 2 && params.coarse_inner_tol > 0.0) ? params.coarse_inner_tol : params.inner_tol;
  }
  int inner_maxiter_of(int l) const {
    return (l >= 2 && params.coarse_inner_maxiter > 0) ? params.coarse_inner_maxiter : params.inner_maxiter;
  }
  Store sstore() const {
    return params.precision == SMG_PREC_DOUBLE ? S64 : (params.precision == SMG_PREC_SINGLE ? S32 : S16);
  }
  const Stored& fat_of(Store s) const { return s == S64 ? fat64_st : (s == S32 ? fat32.st : fat16.st); }
  const Stored& naik_of(Store s) const { return s == S64 ? naik64_st : (s == S32 ? naik32.st : naik16.st); }
  const Stored& kd_of(Store s) const { return s == S64 ? kd64.st : (s == S32 ? kd32.st : kd16.st); }
  // fat / Naik links (and their phase-folded copy) of storage s into a dslash
  // parameter block; `truncate` leaves the Naik hops out
  void link_params(Store s, DslashParams& p, bool truncate = false) const;
  // the level-1 (pseudo-fine) operator drops the Naik hops (Table 1, truncated operator)
  bool trunc1() const { return has_naik && params.truncate_naik != 0; }
  Stored fat64_st, naik64_st;
  void ensure_consts(int n);
};

// Host entry points used by the C ABI (api.cu).
void ctx_set_gauge(Context& c, const void* fat, const void* naik, double c_naik, int where);
void ctx_set_mass(Context& c, double m);
void ctx_mg_setup(Context& c, const smg_mg_params& p, const void* const* phi0, int where,
                  const DeflRestore* restore = nullptr);
// Checkpoint of the setup (Sec. 3.2: near-null and singular vectors generated
// once and reused): save writes it, load rebuilds the hierarchy from it for the
// context's gauge field and mass (setup_io.cu).
void ctx_save_setup(Context& c, const char* path);
void ctx_load_setup(Context& c, const char* path, const smg_mg_params* over = nullptr);
int ctx_multishift_cg(Context& c, const void* b, int nshift, const double* masses, void* x, double tol, int maxiter,
                      int where, smg_solve_info* info);
int ctx_propagators(Context& c, const void* b, int nmass, const double* masses, int n_mg, void* x, double tol,
                    int cg_maxiter, int where, smg_solve_info* info);
// The k = coarsest_deflate lowest singular triplets of the coarsest level C
// (or of its Schur complement when C.schur) from the start block `start`.
void build_deflation(Context& c, CoarseLevel& C, const void* start, int where);
// The same state from a saved setup (no subspace iteration).
void restore_deflation(Context& c, CoarseLevel& C, const DeflRestore& r);
void ctx_coarse_solve(Context& c, int l, int nsys, const void* in, void* out, int where);
int ctx_solve(Context& c, int nrhs, const void* b, int nshift, const double* masses, void* x, double tol, int where,
              smg_solve_info* info);
void ctx_apply_fine(Context& c, int op, int prec, int nsys, const void* in, void* out, int where);
void ctx_transfer(Context& c, int which, int l, int prec, int nsys, const void* in, void* out, int where);
void ctx_build_kd(Context& c);
double ctx_time_kernel(Context& c, int kernel, int l, int nsys, int nrep);
double ctx_bench_coarse(Context& c, const int cdims[4], int N, int nsys, int prec, int nrep);
void ctx_coarse_apply_stencil(Context& c, const int cdims[4], int N, int prec, int path, const void* stencil,
                              int nsys, const void* in, void* out, int where);
int ctx_fermion_action(Context& c, const void* phi, void* X, void* Y, double tol, int where, double* S,
                       double* dSdm, smg_solve_info* info);
void upload(void* dst, const void* src, size_t bytes, int where, cudaStream_t st);
void download(void* dst, const void* src, size_t bytes, int where, cudaStream_t st);

}  // namespace smg
