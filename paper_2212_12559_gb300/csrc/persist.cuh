// Persistent cooperative solver for one coarse level (see persist.cu).
#pragma once
#include "ops.cuh"

namespace smg {

constexpr int kPersistMaxSys = 16;
constexpr int kPersistMaxK = 8;
constexpr int kPersistSums = 72;      // reduction outputs per system (CA-GCR(10) Gram system: 65)
constexpr int kPersistMaxTouch = 8;   // lattice sites a CTA's rows may touch in the resident mode

// Launch plan, computed on the host from the level's shape and the device's
// shared-memory limit.
struct PersistPlan {
  int grid = 0;           // CTAs (one per SM, at most one per lattice site)
  long long per = 0;      // rows of every system owned by one CTA: [c*per, (c+1)*per)
  int nslot = 0;          // bound on the lattice sites one CTA's rows touch
  int resident = 0;       // 1: the CTA's stencil rows, row scales and prolongator rows live in shared memory
  int sg = 0;             // systems per input-staging round (resident mode)
  size_t smem = 0;        // dynamic shared memory per CTA
  size_t off_S = 0, off_sc = 0, off_P = 0, off_stg = 0;   // shared-memory offsets (resident mode)
};

struct PersistArgs {
  // the GCR level: coarse stencil, FP16 (row scales) or FP32
  Geom g;
  int N;
  const void* S;
  const float* Srs;
  long long n;               // unknowns per system on this level
  // preconditioner: restriction to the dense coarsest level and back
  int has_pre;
  TransferGeom tg;
  const void* P;             // prolongator of this level, storage as S, global scale 1
  const float2* D;           // dense coarsest inverse, FP32 [nd][nd]
  int nd;
  int s;                     // CA-GCR smoother length
  int K;                     // GCR iterations
  double tol2;
  int nsys;
  // FP32 work vectors [nsys][n] (rc, ec: [nsys][nd])
  float2 *b, *x, *r;
  float2* z[kPersistMaxK];
  float2* w[kPersistMaxK];
  float2* V[11];
  float2 *rc, *ec;
  float2* partial;           // [grid][kPersistMaxSys][kPersistSums]
  float2* rpart;             // [grid][nslot][kPersistMaxSys][2 nvec] per-CTA partial restrictions
  PersistPlan plan;
  unsigned long long* bar;   // barrier arrival counter, 0 between launches
  unsigned* exitc;           // CTAs that finished (the last one clears both counters)
  int* err;                  // set to 1 when a barrier wait times out
  unsigned long long bar_limit_ns = 2000000000ull;   // limit of one grid-barrier wait
  int bar_extra = 0;         // arrivals each barrier expects beyond the grid's: 0 in every
                             // solve; 1 (test hook) makes every barrier wait run out
  const int* run;            // skip the launch when *run == 0
  unsigned long long* trace; // optional phase trace (see persist.cu), or nullptr
  int trace_cap;
};
// names of the traced phase ids (index = id)
const char* persist_phase_name(int id, bool has_pre);

// n: unknowns per system on the level
bool persist_supported(int nsys, int K, int s, int N, long long n, Store st);
// nvec_next: null vectors of the next level (0 for the coarsest GCR level, no preconditioner)
PersistPlan persist_plan(const Geom& g, int N, int nsys, int nvec_next, Store st);
// The same for a device of `sms` SMs with `cap` bytes of shared memory per block (host only)
PersistPlan persist_plan_for(int V, int N, int nsys, int nvec_next, Store st, int sms, size_t cap);
// bytes of the device buffer behind partial, rpart and the barrier words
size_t persist_buffer_bytes(const PersistPlan& p, int nvec_next);
void persist_gcr(const PersistArgs& a, Store st, cudaStream_t stream);

}  // namespace smg
