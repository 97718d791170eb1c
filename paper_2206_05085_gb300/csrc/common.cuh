// Shared device/host helpers of the DVGOv2 GB300 library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dvgo.h"

namespace dvgo {

constexpr int kWarp = 32;
constexpr int kBrick = 8;           // brick side (voxels)
constexpr int kBrickVox = 512;      // voxels per brick
constexpr int kNumSMs = 152;        // GB300

#define DVGO_CHECK_ARG(cond)                 \
  do {                                       \
    if (!(cond)) return DVGO_ERR_INVALID_ARG; \
  } while (0)

inline int launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Grid-stride launch size: a multiple of the SM count, capped by the work.
inline int grid_for(int64_t work_items, int block, int per_sm = 8) {
  int64_t blocks = ceil_div(work_items, block);
  int64_t cap = (int64_t)kNumSMs * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// ------------------------------------------------------------- bricked layout
struct BrickGeom {
  int G[3];
  int nb[3];  // bricks per axis
  __host__ __device__ int64_t num_bricks() const { return (int64_t)nb[0] * nb[1] * nb[2]; }
};

inline BrickGeom make_geom(const int32_t G[3]) {
  BrickGeom g;
  for (int a = 0; a < 3; ++a) {
    g.G[a] = G[a];
    g.nb[a] = (G[a] + kBrick - 1) / kBrick;
  }
  return g;
}

// Morton order of a voxel inside its 8^3 brick: bit 3i+a holds bit i of axis a.
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}

// Voxel slot (in voxels, multiply by C for elements) of grid point (x, y, z).
__host__ __device__ __forceinline__ int64_t voxel_slot(const BrickGeom& g, int x, int y, int z) {
  int64_t b = ((int64_t)(z >> 3) * g.nb[1] + (y >> 3)) * g.nb[0] + (x >> 3);
  uint32_t local = spread3(x & 7) | (spread3(y & 7) << 1) | (spread3(z & 7) << 2);
  return b * kBrickVox + local;
}

__device__ __forceinline__ int64_t brick_of(const BrickGeom& g, int x, int y, int z) {
  return ((int64_t)(z >> 3) * g.nb[1] + (y >> 3)) * g.nb[0] + (x >> 3);
}

// ------------------------------------------------------------------- bf16
__device__ __forceinline__ float bf16_bits_to_f32(uint16_t h) {
  return __uint_as_float(((uint32_t)h) << 16);
}
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t*>(&b);
}

// ------------------------------------------------------------------- math
// softplus(x) = max(x, 0) + log1p(exp(-|x|))
__device__ __forceinline__ float softplus_f(float x) {
  return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x)));
}
__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// --------------------------------------------------------------- warp scans
__device__ __forceinline__ float warp_incl_sum(float v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// The exclusive prefix of lane k from an inclusive scan: lane k-1's inclusive
// sum (0 in lane 0), taken by a shuffle rather than incl - v, so that a large
// own term does not cancel against its prefix.
__device__ __forceinline__ float warp_excl_from_incl(float incl) {
  const float e = __shfl_up_sync(0xffffffffu, incl, 1);
  return (threadIdx.x & 31) ? e : 0.0f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Kahan-compensated running sum (carry between warp chunks).
struct Kahan {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
};

}  // namespace dvgo
