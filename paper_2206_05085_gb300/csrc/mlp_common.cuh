// Shared definitions of the colour MLP kernels (rgbnet, Tab. 1 "hybrid").
#pragma once

#include <algorithm>

#include "common.cuh"

namespace dvgo {

constexpr int kFeat = 12;        // feature-grid channels
constexpr int kIn = 39;          // 12 + 3 + 2*3*4 view-direction encoding
constexpr int kInP = 40;         // + constant 1 column carrying the layer-1 bias
constexpr int kHid = 128;
constexpr int kOut = 3;
constexpr int kTile = 128;       // samples per tile
constexpr int kNumFreq = 4;

// flat FP32 parameter layout: W1[128][39], b1, W2[128][128], b2, W3[3][128], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kNumParams = kOffB3 + kOut;  // 22019

__device__ __forceinline__ int64_t mlp_count(int64_t n_cap, const int64_t* n_dev) {
  if (!n_dev) return n_cap;
  int64_t n = *n_dev;
  return n < n_cap ? n : n_cap;
}

// Input row of sample j of the list: [k0 (12), d (3), sin(2^f d_a) (a major,
// f inner), cos(2^f d_a), 1].  Rows past the list end are zero (including
// the bias column), so they contribute nothing to any gradient.
// All 32 lanes of the warp call it together (rows j of the warp's lanes):
// the direction encoding is evaluated once per distinct ray among the
// warp's rows (up to 8 rays; 12 sine-cosine pairs per ray spread over the
// lanes, collected by shuffles), else per row.
__device__ __forceinline__ void encode_row(const float* __restrict__ k0,
                                           const float* __restrict__ rays_d,
                                           const int32_t* __restrict__ ray_id,
                                           const int32_t* __restrict__ idx, int64_t j, int64_t n,
                                           float row[kInP]) {
  const int lane = threadIdx.x & 31;
  const bool valid = j < n;
  int r = -1;
  float d[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < kInP; ++k) row[k] = 0.0f;
  if (valid) {
    const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
    const float4* kp = reinterpret_cast<const float4*>(k0 + s * kFeat);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float4 v = __ldg(kp + q);
      row[4 * q] = v.x;
      row[4 * q + 1] = v.y;
      row[4 * q + 2] = v.z;
      row[4 * q + 3] = v.w;
    }
    r = __ldg(ray_id + s);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __ldg(rays_d + 3 * (int64_t)r + a);
  }
  const unsigned peers = __match_any_sync(0xffffffffu, r);
  const int leader = __ffs(peers) - 1;
  const unsigned leaders = __ballot_sync(0xffffffffu, lane == leader);
  const int nd = __popc(leaders);
  if (nd <= 8) {   // warp-uniform
    const int rank = __popc(leaders & ((1u << leader) - 1u));
    const int ntask = kNumFreq * 3 * nd;   // 12 (axis, frequency) pairs per distinct ray
    for (int base = 0; base < ntask; base += 32) {
      const int t = min(base + lane, ntask - 1);
      const int ray = t / 12, pair = t % 12, a = pair >> 2, f = pair & 3;
      const int src = (int)__fns(leaders, 0, ray + 1);
      const float d0 = __shfl_sync(0xffffffffu, d[0], src);
      const float d1 = __shfl_sync(0xffffffffu, d[1], src);
      const float d2 = __shfl_sync(0xffffffffu, d[2], src);
      float sn, cs;
      sincosf((a == 0 ? d0 : (a == 1 ? d1 : d2)) * (float)(1 << f), &sn, &cs);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const int tq = rank * 12 + q - base;
        const float vs = __shfl_sync(0xffffffffu, sn, tq & 31);
        const float vc = __shfl_sync(0xffffffffu, cs, tq & 31);
        if (tq >= 0 && tq < 32) {
          row[kFeat + 3 + q] = vs;
          row[kFeat + 3 + 3 * kNumFreq + q] = vc;
        }
      }
    }
  } else if (valid) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int f = 0; f < kNumFreq; ++f) {
        float sn, cs;
        sincosf(d[a] * (float)(1 << f), &sn, &cs);
        row[kFeat + 3 + a * kNumFreq + f] = sn;
        row[kFeat + 3 + 3 * kNumFreq + a * kNumFreq + f] = cs;
      }
  }
  if (valid) {
#pragma unroll
    for (int a = 0; a < 3; ++a) row[kFeat + a] = d[a];
    row[kIn] = 1.0f;
  } else {
#pragma unroll
    for (int k = kFeat + 3; k < kIn; ++k) row[k] = 0.0f;
  }
}

// Upstream gradient of the colour of sample s: g_rgb[s] if given, else
// w[s] * g_color[ray_id[s]].
__device__ __forceinline__ void upstream_rgb_grad(const float* __restrict__ g_rgb,
                                                  const float* __restrict__ g_color,
                                                  const float* __restrict__ w,
                                                  const int32_t* __restrict__ ray_id, int64_t s,
                                                  float out[3]) {
  if (g_rgb) {
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = __ldg(g_rgb + 3 * s + c);
  } else {
    const float ws = __ldg(w + s);
    const int64_t r = __ldg(ray_id + s);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = ws * __ldg(g_color + 3 * r + c);
  }
}

// Butterfly reduce-scatter: lane l returns sum over the warp of v[l] (v is
// overwritten).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? v[j] : v[j + h];
      const float keep = up ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

}  // namespace dvgo
