// Checkpoint of the multigrid setup (Sec. 3.2: the near-null vectors and the
// coarsest level's singular vectors are generated once and reused for every
// later solve and mass).
//
// File layout (little-endian, as written by the host):
//   char     magic[8]          "SMGSETUP"
//   uint32   version           1
//   uint32   nblocks           n_coarse (+ 2 with a deflated coarsest level)
//   int32    dims[4]           fine lattice extents
//   double   setup_mass        mass the saved setup was built at
//   uint32   params_bytes      sizeof(smg_mg_params)
//   smg_mg_params params       as passed to smg_mg_setup
//   int32    setup_iters[SMG_MAX_COARSE]
//   deflation header (only with a deflated coarsest level):
//     int32 k, int32 iters, double lmin, lmax, res, double sigma[k]
//   nblocks x { uint64 count; count FP64 complex numbers }:
//     the near-null vectors of each coarsening as the setup produced them
//     (before chiral doubling and block orthonormalisation), then V and
//     U diag(1/sigma) of the deflation
//   uint64   FNV-1a 64 hash of every byte above
//
// Loading repeats the deterministic part of the setup (chiral doubling, block
// orthonormalisation, Galerkin products, storage copies) from the saved
// vectors for the context's current gauge field and mass; with the gauge field
// and mass of the save, every coarse stencil comes out bit for bit the same.
#include <cstdio>
#include <cstring>
#include <vector>

#include "solver.cuh"

namespace smg {
namespace {

constexpr char kMagic[8] = {'S', 'M', 'G', 'S', 'E', 'T', 'U', 'P'};
constexpr uint32_t kVersion = 1;

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  }
};

struct Writer {
  FILE* f = nullptr;
  Fnv fnv;
  std::string path;
  explicit Writer(const char* p) : path(p) {
    f = std::fopen(p, "wb");
    SMG_REQUIRE(f != nullptr, "save_setup: cannot open " + path + " for writing");
  }
  ~Writer() { if (f) std::fclose(f); }
  void put(const void* p, size_t n) {
    SMG_REQUIRE(std::fwrite(p, 1, n, f) == n, "save_setup: write to " + path + " failed");
    fnv.add(p, n);
  }
  template <class T> void val(const T& v) { put(&v, sizeof(T)); }
  void close() {
    const uint64_t h = fnv.h;
    SMG_REQUIRE(std::fwrite(&h, 1, sizeof(h), f) == sizeof(h), "save_setup: write to " + path + " failed");
    const int rc = std::fclose(f);
    f = nullptr;
    SMG_REQUIRE(rc == 0, "save_setup: closing " + path + " failed");
  }
};

struct Reader {
  FILE* f = nullptr;
  Fnv fnv;
  std::string path;
  explicit Reader(const char* p) : path(p) {
    f = std::fopen(p, "rb");
    SMG_REQUIRE(f != nullptr, "load_setup: cannot open " + path);
  }
  ~Reader() { if (f) std::fclose(f); }
  void get(void* p, size_t n) {
    SMG_REQUIRE(std::fread(p, 1, n, f) == n, "load_setup: " + path + " is truncated");
    fnv.add(p, n);
  }
  template <class T> T val() { T v; get(&v, sizeof(T)); return v; }
};

// Writes one FP64 complex device block, staged through host memory in chunks.
void put_block(Writer& w, const void* dev, size_t count, cudaStream_t st) {
  w.val<uint64_t>((uint64_t)count);
  const size_t chunk = (size_t)1 << 24;   // complex numbers per staging round (256 MiB)
  std::vector<double2> h(std::min(count, chunk));
  for (size_t off = 0; off < count; off += chunk) {
    const size_t m = std::min(chunk, count - off);
    SMG_CUDA_OK(cudaMemcpyAsync(h.data(), (const double2*)dev + off, m * sizeof(double2), cudaMemcpyDeviceToHost, st));
    SMG_CUDA_OK(cudaStreamSynchronize(st));
    w.put(h.data(), m * sizeof(double2));
  }
}

std::vector<double2> get_block(Reader& r, size_t want) {
  const uint64_t count = r.val<uint64_t>();
  SMG_REQUIRE(count == want, "load_setup: a vector block of " + r.path + " has the wrong size");
  std::vector<double2> h(count);
  r.get(h.data(), count * sizeof(double2));
  return h;
}

}  // namespace

void ctx_save_setup(Context& c, const char* path) {
  SMG_REQUIRE(path != nullptr, "save_setup: null path");
  SMG_REQUIRE(c.setup_done, "save_setup needs mg_setup first");
  const smg_mg_params& P = c.params;
  const CoarseLevel& last = c.coarse.back();
  const bool defl = last.defl_k > 0;
  Writer w(path);
  w.put(kMagic, sizeof(kMagic));
  w.val<uint32_t>(kVersion);
  w.val<uint32_t>((uint32_t)(P.n_coarse + (defl ? 2 : 0)));
  for (int mu = 0; mu < 4; ++mu) w.val<int32_t>(c.g.L[mu]);
  w.val<double>(c.setup_mass);
  w.val<uint32_t>((uint32_t)sizeof(smg_mg_params));
  w.put(&P, sizeof(P));
  for (int l = 0; l < SMG_MAX_COARSE; ++l) w.val<int32_t>(l < P.n_coarse ? c.coarse[l].setup_iters : 0);
  if (defl) {
    w.val<int32_t>(last.defl_k);
    w.val<int32_t>(last.defl_iters);
    w.val<double>(last.cheb_lmin);
    w.val<double>(last.cheb_lmax);
    w.val<double>(last.defl_res);
    w.put(last.sigma.data(), sizeof(double) * last.sigma.size());
  }
  for (int l = 0; l < P.n_coarse; ++l) put_block(w, c.coarse[l].pre64.p, c.coarse[l].pre64.bytes / sizeof(double2), c.stream);
  if (defl) {
    const size_t nk = (size_t)last.g.V * last.N * last.defl_k;
    put_block(w, last.dV64.p, nk, c.stream);
    put_block(w, last.dU64.p, nk, c.stream);
  }
  w.close();
}

void ctx_load_setup(Context& c, const char* path, const smg_mg_params* over) {
  SMG_REQUIRE(path != nullptr, "load_setup: null path");
  SMG_REQUIRE(c.gauge_set && c.mass_set, "load_setup needs set_gauge and set_mass first");
  Reader r(path);
  char magic[8];
  r.get(magic, sizeof(magic));
  SMG_REQUIRE(std::memcmp(magic, kMagic, sizeof(kMagic)) == 0, "load_setup: " + r.path + " is not a saved setup");
  SMG_REQUIRE(r.val<uint32_t>() == kVersion, "load_setup: unsupported file version");
  const uint32_t nblocks = r.val<uint32_t>();
  for (int mu = 0; mu < 4; ++mu)
    SMG_REQUIRE(r.val<int32_t>() == c.g.L[mu], "load_setup: the saved setup is for other lattice extents");
  (void)r.val<double>();   // the mass the setup was built at (the load uses the context's)
  SMG_REQUIRE(r.val<uint32_t>() == sizeof(smg_mg_params), "load_setup: parameter block size differs");
  smg_mg_params P;
  r.get(&P, sizeof(P));
  SMG_REQUIRE(P.n_coarse >= 1 && P.n_coarse <= SMG_MAX_COARSE, "load_setup: bad level count");
  int iters[SMG_MAX_COARSE];
  for (int l = 0; l < SMG_MAX_COARSE; ++l) iters[l] = r.val<int32_t>();
  // the level shapes the parameters imply
  std::vector<size_t> counts;
  Geom fg = c.g;
  int ndof = 3;
  for (int l = 0; l < P.n_coarse; ++l) {
    SMG_REQUIRE(P.nvec[l] >= 1 && P.nvec[l] <= 64, "load_setup: bad nvec");
    counts.push_back((size_t)fg.V * ndof * P.nvec[l]);
    Geom cg;
    cg.V = 1;
    for (int mu = 0; mu < 4; ++mu) {
      SMG_REQUIRE(P.agg[l][mu] >= 1 && fg.L[mu] % P.agg[l][mu] == 0, "load_setup: bad aggregates");
      cg.L[mu] = fg.L[mu] / P.agg[l][mu];
      cg.V *= cg.L[mu];
    }
    fg = cg;
    ndof = 2 * P.nvec[l];
  }
  const bool defl = nblocks == (uint32_t)P.n_coarse + 2;
  SMG_REQUIRE(defl || nblocks == (uint32_t)P.n_coarse, "load_setup: block count does not match the parameters");
  DeflRestore dr;
  if (defl) {
    dr.k = r.val<int32_t>();
    dr.iters = r.val<int32_t>();
    dr.lmin = r.val<double>();
    dr.lmax = r.val<double>();
    dr.res = r.val<double>();
    SMG_REQUIRE(dr.k == P.coarsest_deflate && dr.k >= 1 && dr.k <= 64, "load_setup: bad deflation block");
    dr.sigma.resize(dr.k);
    r.get(dr.sigma.data(), sizeof(double) * dr.k);
  }
  std::vector<std::vector<double2>> vecs;
  for (size_t cnt : counts) vecs.push_back(get_block(r, cnt));
  std::vector<double2> dV, dU;
  if (defl) {
    const size_t nk = (size_t)fg.V * ndof * dr.k;
    dV = get_block(r, nk);
    dU = get_block(r, nk);
    dr.V = dV.data();
    dr.U = dU.data();
  }
  const uint64_t want = r.fnv.h;
  uint64_t got = 0;
  SMG_REQUIRE(std::fread(&got, 1, sizeof(got), r.f) == sizeof(got), "load_setup: " + r.path + " is truncated");
  SMG_REQUIRE(got == want, "load_setup: checksum mismatch in " + r.path);
  // rebuild: the saved vectors are used as given (no CGNE), the deflation state
  // restored; other solver settings may replace the saved ones when the level
  // structure the vectors belong to is the same
  if (over != nullptr) {
    bool same = over->n_coarse == P.n_coarse && over->block_coarse == P.block_coarse &&
                over->coarsest_schur == P.coarsest_schur && over->coarsest_deflate == P.coarsest_deflate;
    for (int l = 0; l < P.n_coarse && same; ++l) {
      same = over->nvec[l] == P.nvec[l];
      for (int mu = 0; mu < 4; ++mu) same = same && over->agg[l][mu] == P.agg[l][mu];
    }
    SMG_REQUIRE(same, "load_setup: the parameters' level structure (n_coarse, agg, nvec, block_coarse, "
                      "coarsest_schur, coarsest_deflate) differs from the saved setup's");
    const int keep_iters = P.setup_maxiter;
    P = *over;
    P.setup_maxiter = keep_iters;
  }
  smg_mg_params Q = P;
  Q.setup_maxiter = 0;
  std::vector<const void*> phi0;
  for (auto& v : vecs) phi0.push_back(v.data());
  phi0.push_back(nullptr);
  ctx_mg_setup(c, Q, phi0.data(), SMG_HOST, defl ? &dr : nullptr);
  c.params = P;
  for (int l = 0; l < P.n_coarse; ++l) c.coarse[l].setup_iters = iters[l];
}

}  // namespace smg
