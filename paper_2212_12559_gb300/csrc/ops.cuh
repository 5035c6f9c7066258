// Launchers of the operator kernels: fine staggered dslash, Kahler-Dirac
// block inverse, restriction / prolongation, coarse 9-point stencil and the
// dense coarsest-level inverse.
#pragma once
#include "blas.cuh"

namespace smg {

// Stored operator data: values in one of three precisions plus optional
// FP32 scale factors (FP16 storage only).
struct Stored {
  void* p = nullptr;       // double2 / float2 / __half2
  float* scale = nullptr;  // per-row scales (layout depends on the operator)
  float gscale = 1.0f;     // one global scale (links, null vectors)
  Store s = S64;
};

// ------------------------------------------------------------------ dslash
// Section 2.2: M = m + D; fat links at distance 1 and Naik links at
// distance 3 (coefficient c_naik), staggered phases eta_mu(x).
struct DslashParams {
  Geom g;
  Stored fat, naik;          // [4][V][3][3]; naik.p == nullptr for the naive operator
  double c_naik = 0.0;
  const double* mass = nullptr;  // per system (device), or nullptr to use mass0
  double mass0 = 0.0;
  int dagger = 0;            // 1: m - D
  int part = -1;             // -1 full; 0 self + mass; 1 + 2*mu + (0 fwd | 1 bwd): crossing hops
  int agg[4] = {1, 1, 1, 1};
  int nsys = 1;
  const void* sub_from = nullptr;   // when set: out = sub_from - M in (residual form)
  // phase-folded copy of the links (FP16 / FP32, see hop.cu); used for FP32 vectors and part < 0
  Stored hop;                // gscale = fat scale (FP16)
  int hop_kinds = 0;         // 1 (naive) or 2 (with Naik links)
  float hop_naik_scale = 1.0f;
};
void dslash(const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run = nullptr);
// Phase-folded links: per (site, mu) eta_mu(x) V_mu(x) and eta_mu(x) W_mu(x), 16-byte padded.
size_t hop_link_entries(const Geom& g, bool naik, Store s);
void build_hop_links(void* H, Store s, const double2* fat, const double2* naik, const Geom& g, float fat_scale,
                     float naik_scale, cudaStream_t st);
bool hop_dslash_ok(const Vec& in, const DslashParams& p);
void hop_dslash(const Vec& out, const Vec& in, const DslashParams& p, cudaStream_t st, const int* run);

// -------------------------------------------------------- Kahler-Dirac blocks
// Site of position b = (x&1) + 2(y&1) + 4(z&1) + 8(t&1) in aligned hypercube blk
// (hypercubes ordered lexicographically on the half-extent lattice).
// Base (even) coordinates of aligned hypercube blk.
__device__ __forceinline__ void hypercube_coords(const Geom& g, int blk, int c[4]) {
  const int h0 = g.L[0] / 2, h1 = g.L[1] / 2, h2 = g.L[2] / 2;
  c[0] = blk % h0; blk /= h0;
  c[1] = blk % h1; blk /= h1;
  c[2] = blk % h2; c[3] = blk / h2;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) c[mu] *= 2;
}
__device__ __forceinline__ int hypercube_site(const Geom& g, int blk, int b) {
  int c[4];
  hypercube_coords(g, blk, c);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) c[mu] += (b >> mu) & 1;
  return g.index(c);
}
// Section 3.1: one dense 48x48 block (B+m)^{-1} per 2^4 hypercube, rows and
// columns ordered (position b in hypercube, colour a) -> 3b + a.
// Build: FP64 into `inv64` [nblk][48][48] row-major.
void kd_build(double2* inv64, const Geom& g, const double2* fat64, double mass, cudaStream_t st);
// Convert a row-major FP64 inverse to the apply layout (column-major per
// block, [nblk][48 col][48 row]) in storage `dst.s` (per-(block,row) scale for FP16).
void kd_pack(Stored& dst, const double2* inv64, long long nblk, cudaStream_t st);
// out[s] = K[sys_map[s]] in[s] (or K^dag).  kd[] holds one packed inverse per mass.
// With sub_from: out = sub_from - K in (residual form).  kd_run: with a
// sys_map, the number of consecutive systems that share one inverse (systems
// per mass), so that several systems per CTA can read each block once.
void kd_apply(const Vec& out, const Vec& in, const Geom& g, const Stored* kd, const int* sys_map, int nkd,
              int dagger, cudaStream_t st, const int* run = nullptr, const void* sub_from = nullptr,
              int kd_run = 1);

// ------------------------------------------------------- transfer operators
// A level's lattice with `ndof` components per site; aggregates of agg[]
// sites.  Chirality of component d at site x: parity(x) on the fine level
// (chi_mode 0), d >= ndof/2 on coarse levels (chi_mode 1).
struct TransferGeom {
  Geom fine;
  Geom coarse;
  int agg[4];
  int ndof;
  int nvec;
  int chi_mode;
};
// raw: FP64 [nvec][V][ndof]; orthonormalised in place per aggregate and chirality
// (modified Gram-Schmidt in vector order, twice).
void block_orthonormalize(double2* raw, const TransferGeom& t, cudaStream_t st);
// Pack orthonormal FP64 [nvec][V][ndof] into the transfer layout [V][ndof][nvec] (global scale 1 for FP16:
// orthonormal columns have entries of modulus <= 1).
void transfer_pack(Stored& dst, const double2* raw, const TransferGeom& t, cudaStream_t st);
// out (coarse, [Vc][2*nvec]) = R in ; R = P^dag
void restrict_op(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                 const int* run = nullptr);
// out (fine) = P in
void prolong_op(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                const int* run = nullptr);
// Tensor-core transfers (FP32 vectors, FP16 prolongator, nvec 32 or 64,
// 16 systems per CTA): whether a transfer has a supported shape, and the two
// launches (candidates of restrict_op / prolong_op's autotuner).
bool transfer_mma_ok(const TransferGeom& t, const Stored& P, Prec vp);
void restrict_mma(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                  const int* run);
void prolong_mma(const Vec& out, const Vec& in, const TransferGeom& t, const Stored& P, cudaStream_t st,
                 const int* run);

// ------------------------------------------------------- coarse 9-point op
// Stencil layout [Vc][N rows][9 dirs][N cols]; dir 0 = self, 1+2mu = hop to
// X+mu, 2+2mu = hop to X-mu.  FP16 storage carries one scale per (site, row).
struct CoarseParams {
  Geom g;
  int N;
  int part = -1;             // as DslashParams::part
  int agg[4] = {1, 1, 1, 1};
  const void* sub_from = nullptr;   // when set: out = sub_from - A_hat in
  int allow_tc = 1;          // 0: keep FP32 inputs (no FP16 rounding of the vectors), e.g. for the setup
  int path = 0;              // CPATH_*: 0 = the tuned (or default) choice for the shape
};
// Kernels of the coarse apply: CUDA cores (one CTA per site and system, a warp
// per row), mma.sync m16n8k16 (several systems, N % 16 == 0, N <= 128),
// tcgen05 + TMA (several systems, N = 128) with 1 or 2 CTAs per SM and a 4- or
// 6-stage stencil ring, and CUDA cores with the rows split evenly over a grid
// that fills the GPU once (a half warp per row; one system, or up to 8
// systems per CTA with FP32 vectors).
enum {
  CPATH_AUTO = 0, CPATH_CORES = 1, CPATH_MMA = 2, CPATH_UMMA_1x4 = 3, CPATH_UMMA_2x4 = 4, CPATH_UMMA_1x6 = 5,
  CPATH_ROWS = 6, CPATH_ROWS_MULTI = 7, CPATH_COUNT = 8
};
// Whether a path serves a shape (host logic only).
bool coarse_path_ok(int path, int N, int nsys, Prec vp, Store s, bool full_op);
// The paths that serve a shape in the autotuner's order (the untuned default
// first): writes up to cap of them, returns how many there are.
int coarse_path_list(int N, int nsys, Prec vp, Store s, bool full_op, int* out, int cap);
void coarse_apply(const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S, cudaStream_t st,
                  const int* run = nullptr);
// tcgen05 / TMA multi-RHS path (N = 128, FP16 stencil, FP32 vectors, >= 2 systems); err: device int
bool coarse_umma_ok(const Vec& in, const CoarseParams& p, const Stored& S);
void coarse_apply_umma(const Vec& out, const Vec& in, const CoarseParams& p, const Stored& S, int* err,
                       cudaStream_t st, const int* run = nullptr, int ctas_per_sm = 2, int stages = 4);
// Device error word of the tcgen05 coarse apply (set when a CTA gave up on a
// bounded wait); read_and_clear returns whether it was set.
int* coarse_umma_err();
bool coarse_umma_err_read_and_clear(cudaStream_t st);
// Hash-based synthetic values in [-1, 1) (benchmark inputs of a given shape)
void synth_fill(void* dst, Store s, long long n, unsigned seed, cudaStream_t st);
// S64 stencil -> stored copy in precision dst.s
void coarse_pack(Stored& dst, const double2* S64, const Geom& g, int N, cudaStream_t st);
// Adjoint stencil: X^dag, Y'_{+mu}(X) = Y_{-mu}(X+mu)^dag, Y'_{-mu}(X) = Y_{+mu}(X-mu)^dag
void coarse_dagger(double2* dst, const double2* src, const Geom& g, int N, cudaStream_t st);
// Scatter restricted probe columns into the stencil: C is [ncol systems][Vc][N],
// column j0 + s of direction `dir` at every coarse site.
void galerkin_scatter(double2* S64, const double2* C, const Geom& g, int N, int dir, int j0, int ncol,
                      cudaStream_t st);
// Unit coarse probes: E[s][X][i] = (i == j0 + s)
void unit_probes(double2* E, long long Vc, int N, int j0, int ncol, cudaStream_t st);

// Block-preconditioned stencil X^{-1} A_hat (Sec. 2.3), in place on the FP64
// stencil: self blocks become 1, hops X^{-1} Y_{+-mu}; X^{-1} goes to Xinv
// [Vc][N][N].  Sets *err (device int) when a self block is singular.
void block_precondition(double2* S64, double2* Xinv, const Geom& g, int N, int* err, cudaStream_t st);
// v[s](X) <- Xinv(X) v[s](X) on a coarse batch; Xinv in v's precision
void block_diag_apply(const Vec& v, const void* Xinv, Prec xprec, int N, cudaStream_t st, const int* run = nullptr);

// out = even sites of *even, odd sites of *odd (null: zero) on a coarse batch
void parity_pick(const Vec& out, const Vec* even, const Vec* odd, const Geom& g, int N, cudaStream_t st,
                 const int* run = nullptr);

// S v = mask_e(v - R(mask_o(R(v)))), R(u) = u - A u, for the Schur complement
// S = 1 - K_eo K_oe of a coarse operator A = 1 + K with identity self blocks,
// on fields that vanish on the odd sites (S^dag with the adjoint stencil);
// t1, t2: scratch shaped like v.
void schur_apply(const Vec& out, const Vec& in, const CoarseParams& cp, const Stored& S, const Vec& t1,
                 const Vec& t2, cudaStream_t st, const int* run = nullptr);

// ------------------------------------------------------- dense coarsest op
void dense_from_stencil(double2* Dn, const double2* S64, const Geom& g, int N, cudaStream_t st);
// In-place Gauss-Jordan inverse with partial pivoting (FP64); returns false if singular.
void dense_invert(double2* Dn, int n, double2* scratch, int* piv_dev, cudaStream_t st);
// out[s] = Dinv in[s] ; Dinv FP64 or FP32 [n][n] row-major
void dense_apply(const Vec& out, const Vec& in, const void* Dinv, Prec dprec, int n, cudaStream_t st,
                 const int* run = nullptr);

// ------------------------------------------------------- maps (test hooks)
// Per-site tables: parity, KD block, position in block, aggregate, position in aggregate.
void site_maps(int* parity, int* kd_block, int* kd_pos, int* agg_idx, int* agg_pos, const Geom& g,
               const int agg[4], cudaStream_t st);

// ------------------------------------------------------- fermion force
// F_mu(x) = -c eta_mu(x) b_mu(x) [ Y(x) X(x+k mu)^dag - X(x) Y(x+k mu)^dag ], with b_mu(x) = -1
// for the time links whose hop wraps around an antiperiodic time boundary (bc_t = -1), else 1
void force_outer(double2* F, const double2* X, const double2* Y, const Geom& g, int k, double c, int bc_t,
                 cudaStream_t st);
// Antiperiodic time boundary on FP64 links [4][V][3][3]: negates the time
// links of the sites whose hop of length k wraps around (x_t + k >= L_t).
void boundary_flip_time(double2* links, const Geom& g, int k, cudaStream_t st);
// FP16 copy of n FP32 complex numbers with one global scale: returns
// sc = max |Re|, |Im| (1 when all are zero) and writes dst = src / sc.
float pack_fp16_global(__half2* dst, const float2* src, long long n, cudaStream_t st);
// out = eps(x) in, eps(x) = (-1)^(x+y+z+t) (Sec. 2.2), one FP64 colour field
void eps_mul(double2* out, const double2* in, const Geom& g, cudaStream_t st);

}  // namespace smg
