// Persistent cooperative solver for one coarse level (see persist.cu).
#pragma once
#include "ops.cuh"

namespace smg {

constexpr int kPersistMaxSys = 16;
constexpr int kPersistMaxK = 8;

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
  double2* partial;          // [grid][kPersistMaxSys][64]
  unsigned* bar;             // barrier counter and generation
  int* err;                  // set to 1 when a barrier wait times out
  const int* run;            // skip the launch when *run == 0
};

bool persist_supported(int nsys, int K, int s, int N, Store st, int npos);
void persist_gcr(const PersistArgs& a, Store st, cudaStream_t stream);
int persist_grid_size();
size_t persist_smem_bytes();

}  // namespace smg
