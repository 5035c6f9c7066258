// One output row of the 9-point coarse stencil with 16-byte loads.
//
// The row's nine N-long blocks are one contiguous super-row of 9N entries
// ([site][row][dir][col] layout).  Each lane takes 16-byte chunks (4 FP16 or
// 2 FP32 complex entries) so a warp streams 512 contiguous bytes per load
// instruction; the matching input entries are fetched as float4 pairs.
// Requires N to be a multiple of 4 (a chunk never straddles two directions).
#pragma once
#include "common.cuh"

namespace smg {

template <typename SL> struct Chunk;
template <> struct Chunk<__half2> { static constexpr int C = 4; };
template <> struct Chunk<float2> { static constexpr int C = 2; };

// Neighbour site of direction dir among the nine held in nb[] (no dynamic
// register indexing: a select chain).
__device__ __forceinline__ int pick_site(const int nb[9], int dir) {
  int site = nb[0];
#pragma unroll
  for (int d = 1; d < 9; ++d) site = (dir == d) ? nb[d] : site;
  return site;
}

// sum_e S[e] * v(e) over the super-row; `vat(dir, j)` returns a pointer to
// the FP32 input entry j of the neighbour in direction dir (16-byte aligned
// for even j).
// LANES lanes share the row (lane in [0, LANES)).
template <int LANES, typename SL, typename VAt>
__device__ __forceinline__ float2 stencil_row_dot_lanes(const SL* __restrict__ sr, int N, int lane, VAt vat) {
  constexpr int C = Chunk<SL>::C;
  const int nchunk = 9 * N / C;
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int q = lane; q < nchunk; q += LANES) {
    const int e = q * C;
    const int dir = e / N, j = e - dir * N;
    const uint4 raw = __ldg(reinterpret_cast<const uint4*>(sr + e));
    const float4* v = reinterpret_cast<const float4*>(vat(dir, j));
    if constexpr (C == 4) {
      const __half2* h = reinterpret_cast<const __half2*>(&raw);
      const float4 v01 = v[0], v23 = v[1];
      cfma(a0, __half22float2(h[0]), make_float2(v01.x, v01.y));
      cfma(a1, __half22float2(h[1]), make_float2(v01.z, v01.w));
      cfma(a0, __half22float2(h[2]), make_float2(v23.x, v23.y));
      cfma(a1, __half22float2(h[3]), make_float2(v23.z, v23.w));
    } else {
      const float2* f = reinterpret_cast<const float2*>(&raw);
      const float4 v01 = v[0];
      cfma(a0, f[0], make_float2(v01.x, v01.y));
      cfma(a1, f[1], make_float2(v01.z, v01.w));
    }
  }
  return make_float2(a0.x + a1.x, a0.y + a1.y);
}

// A whole warp on the row.
template <typename SL, typename VAt>
__device__ __forceinline__ float2 stencil_row_dot(const SL* __restrict__ sr, int N, int lane, VAt vat) {
  return stencil_row_dot_lanes<32, SL>(sr, N, lane, vat);
}

}  // namespace smg
