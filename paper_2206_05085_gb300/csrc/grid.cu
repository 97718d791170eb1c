// Dense voxel grids (Tab. 1: explicit density grid, feature grid of the
// hybrid colour model): bricked storage, trilinear query and its adjoint,
// occupancy mask (Sec. 1), TV gradient (Sec. 2) and the fused sparse Adam
// step (Sec. 3 "Re-implement Adam optimizer").
#include <math.h>

#include "common.cuh"

namespace dvgo {

// Grid index of a position: u_a = (x_a - lo_a) (G_a - 1) / (hi_a - lo_a),
// written u = x S + C with S = (G - 1)/(hi - lo) and C = -lo S, each held as
// an unevaluated pair of floats (hi + lo parts, formed in double on the host).
struct TriArgs {
  BrickGeom g;
  float s_hi[3], s_lo[3];
  float c_hi[3], c_lo[3];
};

static bool make_tri(TriArgs& T, const dvgo_grid_desc* d) {
  for (int a = 0; a < 3; ++a) {
    if (d->G[a] < 2 || !(d->hi[a] > d->lo[a])) return false;
    const double S = (double)(d->G[a] - 1) / ((double)d->hi[a] - (double)d->lo[a]);
    const double C = -(double)d->lo[a] * S;
    T.s_hi[a] = (float)S;
    T.s_lo[a] = (float)(S - (double)T.s_hi[a]);
    T.c_hi[a] = (float)C;
    T.c_lo[a] = (float)(C - (double)T.c_hi[a]);
  }
  T.g = make_geom(d->G);
  return true;
}

struct Corners {
  int64_t slot[8];   // voxel slots of the 8 corners
  float w[8];
  int ix, iy, iz;    // lower corner
};

// Cell and fraction along one axis.  u = x S + C is carried as s + e: the
// product x S_hi split exactly by an FMA, the sum with C_hi split exactly by
// the two-sum, the small terms added into e.  The fraction f = (s - i) + e
// (s - i is exact) then has an absolute error of about one rounding of f
// itself, instead of one rounding of u (up to G 2^-24 grid units), which a
// steep field would multiply into the interpolated value.  Outside [0, G - 1]
// u is clamped to the border.
__device__ __forceinline__ void cell_1d(const TriArgs& T, int a, float x, int& i, float& f) {
  // explicit roundings (__f*_rn are never contracted into FMAs)
  const float p = __fmul_rn(x, T.s_hi[a]);
  const float pe = __fmaf_rn(x, T.s_hi[a], -p);            // x S_hi = p + pe
  const float s = __fadd_rn(p, T.c_hi[a]);
  const float bv = __fsub_rn(s, p);
  const float se = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bv)), __fsub_rn(T.c_hi[a], bv));   // p + C_hi = s + se
  const float e = __fadd_rn(se, __fadd_rn(__fmaf_rn(x, T.s_lo[a], pe), T.c_lo[a]));
  const float u = __fadd_rn(s, e);
  const int Gm = T.g.G[a] - 1;
  if (!(u > 0.0f)) {                                       // (also NaN)
    i = 0;
    f = 0.0f;
  } else if (u >= (float)Gm) {
    i = Gm - 1;
    f = 1.0f;
  } else {
    i = min((int)floorf(u), Gm - 1);
    f = __fadd_rn(__fsub_rn(s, (float)i), e);
    f = fminf(fmaxf(f, 0.0f), 1.0f);
  }
}

// Corners and weights of the position pos (already loaded).
__device__ __forceinline__ void corners_at(const TriArgs& T, const float pos[3], Corners& c) {
  int i0[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) cell_1d(T, a, pos[a], i0[a], f[a]);
  c.ix = i0[0];
  c.iy = i0[1];
  c.iz = i0[2];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    c.slot[k] = voxel_slot(T.g, i0[0] + dx, i0[1] + dy, i0[2] + dz);
    c.w[k] = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
  }
}

__device__ __forceinline__ void corners(const TriArgs& T, const float* __restrict__ xyz, int64_t s,
                                        Corners& c) {
  const float pos[3] = {__ldg(xyz + 3 * s), __ldg(xyz + 3 * s + 1), __ldg(xyz + 3 * s + 2)};
  corners_at(T, pos, c);
}

__device__ __forceinline__ int64_t live_n(int64_t n_cap, const int64_t* n_dev) {
  if (!n_dev) return n_cap;
  int64_t n = *n_dev;
  return n < n_cap ? n : n_cap;
}

// ---------------------------------------------------------------- gather
// One sample per thread and step of a grid-stride loop over a grid that
// stays resident; the next sample's position and the index after it are
// loaded before this sample's corners, so that the index -> position ->
// corners chain of one sample overlaps the corner loads of the previous one.
template <int C, bool kBF16>
__global__ void __launch_bounds__(256) gather_fwd_kernel(const void* __restrict__ grid, TriArgs T,
                                                         const float* __restrict__ xyz,
                                                         const int32_t* __restrict__ idx,
                                                         int64_t n_cap, const int64_t* n_dev,
                                                         float* __restrict__ out) {
  const int64_t n = live_n(n_cap, n_dev);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  auto sample_of = [&](int64_t k) -> int64_t { return idx ? (int64_t)__ldg(idx + k) : k; };
  int64_t s = sample_of(j);
  float pos[3] = {__ldg(xyz + 3 * s), __ldg(xyz + 3 * s + 1), __ldg(xyz + 3 * s + 2)};
  int64_t s_next = j + stride < n ? sample_of(j + stride) : -1;
  for (; j < n; j += stride) {
    float pos_next[3] = {0.0f, 0.0f, 0.0f};
    if (s_next >= 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) pos_next[a] = __ldg(xyz + 3 * s_next + a);
    }
    const int64_t s_after = j + 2 * stride < n ? sample_of(j + 2 * stride) : -1;
    Corners c;
    corners_at(T, pos, c);
    float acc[C];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) acc[ch] = 0.0f;
    if constexpr (!kBF16) {
      const float* g = reinterpret_cast<const float*>(grid);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float* p = g + c.slot[k] * C;
        if constexpr (C % 4 == 0) {
#pragma unroll
          for (int q = 0; q < C / 4; ++q) {
            float4 v = __ldg(reinterpret_cast<const float4*>(p) + q);
            acc[4 * q + 0] += c.w[k] * v.x;
            acc[4 * q + 1] += c.w[k] * v.y;
            acc[4 * q + 2] += c.w[k] * v.z;
            acc[4 * q + 3] += c.w[k] * v.w;
          }
        } else {
#pragma unroll
          for (int ch = 0; ch < C; ++ch) acc[ch] += c.w[k] * __ldg(p + ch);
        }
      }
    } else {
      const uint16_t* g = reinterpret_cast<const uint16_t*>(grid);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint16_t* p = g + c.slot[k] * C;
        if constexpr (C % 4 == 0) {
#pragma unroll
          for (int q = 0; q < C / 4; ++q) {
            uint2 v = __ldg(reinterpret_cast<const uint2*>(p) + q);
            acc[4 * q + 0] += c.w[k] * __uint_as_float(v.x << 16);
            acc[4 * q + 1] += c.w[k] * __uint_as_float(v.x & 0xffff0000u);
            acc[4 * q + 2] += c.w[k] * __uint_as_float(v.y << 16);
            acc[4 * q + 3] += c.w[k] * __uint_as_float(v.y & 0xffff0000u);
          }
        } else {
#pragma unroll
          for (int ch = 0; ch < C; ++ch) acc[ch] += c.w[k] * bf16_bits_to_f32(__ldg(p + ch));
        }
      }
    }
    float* o = out + s * C;
    if constexpr (C % 4 == 0) {
#pragma unroll
      for (int q = 0; q < C / 4; ++q)
        reinterpret_cast<float4*>(o)[q] =
            make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    } else {
#pragma unroll
      for (int ch = 0; ch < C; ++ch) o[ch] = acc[ch];
    }
    s = s_next;
#pragma unroll
    for (int a = 0; a < 3; ++a) pos[a] = pos_next[a];
    s_next = s_after;
  }
}

// Any channel count (scalar loads).
template <bool kBF16>
__global__ void gather_fwd_generic_kernel(const void* __restrict__ grid, TriArgs T, int C,
                                          const float* __restrict__ xyz,
                                          const int32_t* __restrict__ idx, int64_t n_cap,
                                          const int64_t* n_dev, float* __restrict__ out) {
  const int64_t n = live_n(n_cap, n_dev);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
    Corners c;
    corners(T, xyz, s, c);
    for (int ch = 0; ch < C; ++ch) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float v = kBF16 ? bf16_bits_to_f32(__ldg(reinterpret_cast<const uint16_t*>(grid) + c.slot[k] * C + ch))
                        : __ldg(reinterpret_cast<const float*>(grid) + c.slot[k] * C + ch);
        acc += c.w[k] * v;
      }
      out[s * C + ch] = acc;
    }
  }
}

// ---------------------------------------------------------------- scatter
__device__ __forceinline__ void mark_touched(uint8_t* touched, const TriArgs& T, const Corners& c) {
  if (!touched) return;
  // the cell spans at most two bricks per axis
  const int x1 = c.ix + 1, y1 = c.iy + 1, z1 = c.iz + 1;
  const bool sx = (c.ix >> 3) != (x1 >> 3), sy = (c.iy >> 3) != (y1 >> 3), sz = (c.iz >> 3) != (z1 >> 3);
  touched[brick_of(T.g, c.ix, c.iy, c.iz)] = 1;
  if (sx) touched[brick_of(T.g, x1, c.iy, c.iz)] = 1;
  if (sy) touched[brick_of(T.g, c.ix, y1, c.iz)] = 1;
  if (sz) touched[brick_of(T.g, c.ix, c.iy, z1)] = 1;
  if (sx && sy) touched[brick_of(T.g, x1, y1, c.iz)] = 1;
  if (sx && sz) touched[brick_of(T.g, x1, c.iy, z1)] = 1;
  if (sy && sz) touched[brick_of(T.g, c.ix, y1, z1)] = 1;
  if (sx && sy && sz) touched[brick_of(T.g, x1, y1, z1)] = 1;
}

template <int C>
__global__ void __launch_bounds__(256) scatter_bwd_kernel(const float* __restrict__ g_out, TriArgs T,
                                                          const float* __restrict__ xyz,
                                                          const int32_t* __restrict__ idx,
                                                          int64_t n_cap, const int64_t* n_dev,
                                                          float* __restrict__ g_grid,
                                                          uint8_t* __restrict__ touched) {
  const int64_t n = live_n(n_cap, n_dev);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
    Corners c;
    corners(T, xyz, s, c);
    float go[C];
    if constexpr (C % 4 == 0) {
#pragma unroll
      for (int q = 0; q < C / 4; ++q) {
        float4 v = __ldg(reinterpret_cast<const float4*>(g_out + s * C) + q);
        go[4 * q] = v.x;
        go[4 * q + 1] = v.y;
        go[4 * q + 2] = v.z;
        go[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int ch = 0; ch < C; ++ch) go[ch] = __ldg(g_out + s * C + ch);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float* p = g_grid + c.slot[k] * C;
      if constexpr (C % 4 == 0) {
#pragma unroll
        for (int q = 0; q < C / 4; ++q)
          atomicAdd(reinterpret_cast<float4*>(p) + q,
                    make_float4(c.w[k] * go[4 * q], c.w[k] * go[4 * q + 1], c.w[k] * go[4 * q + 2],
                                c.w[k] * go[4 * q + 3]));
      } else {
#pragma unroll
        for (int ch = 0; ch < C; ++ch) atomicAdd(p + ch, c.w[k] * go[ch]);
      }
    }
    mark_touched(touched, T, c);
  }
}

// Density (1 channel) and feature (12 channels) adjoints in one pass,
// warp-aggregated: a warp takes 32 consecutive list positions, and two
// neighbouring lanes whose samples lie in the same grid cell (consecutive
// samples of a ray often do) are merged - the first lane adds the second
// lane's weighted gradients to its own and issues one set of reductions for
// both.  Pairs are formed greedily along each run of equal cells.
__global__ void __launch_bounds__(256) scatter_bwd_1_12_kernel(
    const float* __restrict__ g_a, float* __restrict__ grid_a, uint8_t* __restrict__ touched_a,
    const float* __restrict__ g_b, float* __restrict__ grid_b, uint8_t* __restrict__ touched_b, TriArgs T,
    const float* __restrict__ xyz, const int32_t* __restrict__ idx, int64_t n_cap, const int64_t* n_dev) {
  const int64_t n = live_n(n_cap, n_dev);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j0 = warp0 * 32; j0 < n; j0 += nwarps * 32) {
    const int64_t j = j0 + lane;
    const bool valid = j < n;
    Corners c;
    float ga = 0.0f, gb[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) gb[i] = 0.0f;
    int64_t key = -1 - lane;   // distinct for invalid lanes
    if (valid) {
      const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
      corners(T, xyz, s, c);
      ga = __ldg(g_a + s);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(g_b + s * 12) + q);
        gb[4 * q] = v.x;
        gb[4 * q + 1] = v.y;
        gb[4 * q + 2] = v.z;
        gb[4 * q + 3] = v.w;
      }
      key = c.slot[0];
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c.w[k] = 0.0f;
        c.slot[k] = 0;
      }
    }
    // lanes continuing the previous lane's cell; greedy pairing along runs
    const int64_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned same = __ballot_sync(0xffffffffu, lane > 0 && prev == key);
    unsigned absorbed = 0u;
    for (int i = 1; i < 32; ++i)
      if (((same >> i) & 1u) && !((absorbed >> (i - 1)) & 1u)) absorbed |= 1u << i;
    // the next lane's weights and gradients (used when it is absorbed into this one)
    float wn[8], gan, gbn[12];
#pragma unroll
    for (int k = 0; k < 8; ++k) wn[k] = __shfl_down_sync(0xffffffffu, c.w[k], 1);
    gan = __shfl_down_sync(0xffffffffu, ga, 1);
#pragma unroll
    for (int i = 0; i < 12; ++i) gbn[i] = __shfl_down_sync(0xffffffffu, gb[i], 1);
    if (!valid || ((absorbed >> lane) & 1u)) continue;
    const bool pair = lane < 31 && ((absorbed >> (lane + 1)) & 1u);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w0 = c.w[k], w1 = pair ? wn[k] : 0.0f;
      atomicAdd(grid_a + c.slot[k], fmaf(w1, gan, w0 * ga));
      float4* p = reinterpret_cast<float4*>(grid_b + c.slot[k] * 12);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        atomicAdd(p + q, make_float4(fmaf(w1, gbn[4 * q], w0 * gb[4 * q]),
                                     fmaf(w1, gbn[4 * q + 1], w0 * gb[4 * q + 1]),
                                     fmaf(w1, gbn[4 * q + 2], w0 * gb[4 * q + 2]),
                                     fmaf(w1, gbn[4 * q + 3], w0 * gb[4 * q + 3])));
    }
    mark_touched(touched_a, T, c);
    mark_touched(touched_b, T, c);
  }
}

__global__ void scatter_bwd_generic_kernel(const float* __restrict__ g_out, TriArgs T, int C,
                                           const float* __restrict__ xyz,
                                           const int32_t* __restrict__ idx, int64_t n_cap,
                                           const int64_t* n_dev, float* __restrict__ g_grid,
                                           uint8_t* __restrict__ touched) {
  const int64_t n = live_n(n_cap, n_dev);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
    Corners c;
    corners(T, xyz, s, c);
    for (int ch = 0; ch < C; ++ch) {
      float go = __ldg(g_out + s * C + ch);
#pragma unroll
      for (int k = 0; k < 8; ++k) atomicAdd(g_grid + c.slot[k] * C + ch, c.w[k] * go);
    }
    mark_touched(touched, T, c);
  }
}

// ------------------------------------------------------------ pack/unpack
template <typename Tv>
__global__ void pack_kernel(const Tv* __restrict__ dense, Tv* __restrict__ bricked, BrickGeom g,
                            int C, bool to_bricked) {
  const int64_t nvox = (int64_t)g.G[0] * g.G[1] * g.G[2];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox;
       v += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(v % g.G[0]);
    int y = (int)((v / g.G[0]) % g.G[1]);
    int z = (int)(v / ((int64_t)g.G[0] * g.G[1]));
    int64_t slot = voxel_slot(g, x, y, z);
    for (int c = 0; c < C; ++c) {
      if (to_bricked) bricked[slot * C + c] = dense[v * C + c];
      else bricked[v * C + c] = dense[slot * C + c];  // here "dense" is the bricked input
    }
  }
}

// -------------------------------------------------------------- resample
// Progressive grid scaling (the grid-scaling schedule of the unbounded
// experiments, Sec. 5.4): a bricked FP32 grid of Gs points per axis resampled
// to Gd points per axis over the same box, by trilinear interpolation with
// corner-aligned grids.  Destination point x of axis a sits at source index
// u = x (Gs - 1) / (Gd - 1): the integer part and the remainder are exact
// integer arithmetic, the fraction r / (Gd - 1) one FP32 rounding.  One
// thread per destination voxel, all channels; dst is FP32 or (a renderer's
// BF16 copy) BF16, rounded to nearest.
__device__ __forceinline__ void resample_axis(int x, int gs, int gd, int& i, float& f) {
  if (gd == 1 || gs == 1) {
    i = 0;
    f = 0.0f;
    return;
  }
  const int64_t num = (int64_t)x * (gs - 1);
  i = (int)(num / (gd - 1));
  const int64_t r = num % (gd - 1);
  f = __fdiv_rn((float)r, (float)(gd - 1));
  if (i >= gs - 1) {   // the last point: the cell below it, fraction 1
    i = gs - 2;
    f = 1.0f;
  }
}

template <bool kBF16Out>
__global__ void __launch_bounds__(256) resample_kernel(const float* __restrict__ src, BrickGeom gs,
                                                       void* __restrict__ dst, BrickGeom gd, int C) {
  const int64_t nvox = (int64_t)gd.G[0] * gd.G[1] * gd.G[2];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % gd.G[0]), y = (int)((v / gd.G[0]) % gd.G[1]),
              z = (int)(v / ((int64_t)gd.G[0] * gd.G[1]));
    int i[3];
    float f[3];
    resample_axis(x, gs.G[0], gd.G[0], i[0], f[0]);
    resample_axis(y, gs.G[1], gd.G[1], i[1], f[1]);
    resample_axis(z, gs.G[2], gd.G[2], i[2], f[2]);
    int64_t sl[8];
    float w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const int cx = min(i[0] + dx, gs.G[0] - 1), cy = min(i[1] + dy, gs.G[1] - 1),
                cz = min(i[2] + dz, gs.G[2] - 1);
      sl[k] = voxel_slot(gs, cx, cy, cz);
      w[k] = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
    }
    const int64_t o = voxel_slot(gd, x, y, z) * C;
    for (int c = 0; c < C; ++c) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) acc = fmaf(w[k], __ldg(src + sl[k] * C + c), acc);
      if (kBF16Out)
        reinterpret_cast<uint16_t*>(dst)[o + c] = f32_to_bf16_bits(acc);
      else
        reinterpret_cast<float*>(dst)[o + c] = acc;
    }
  }
}

// ----------------------------------------------------------------- mask
__global__ void mask_kernel(const void* __restrict__ density, bool bf16, BrickGeom g, float thr,
                            uint8_t* __restrict__ mask) {
  const int64_t nvox = (int64_t)g.G[0] * g.G[1] * g.G[2];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox;
       v += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(v % g.G[0]);
    int y = (int)((v / g.G[0]) % g.G[1]);
    int z = (int)(v / ((int64_t)g.G[0] * g.G[1]));
    int64_t slot = voxel_slot(g, x, y, z);
    float raw = bf16 ? bf16_bits_to_f32(reinterpret_cast<const uint16_t*>(density)[slot])
                     : reinterpret_cast<const float*>(density)[slot];
    mask[v] = raw >= thr ? 1 : 0;
  }
}

// Progressive mask update: one block of 512 threads per listed brick, thread
// t on the brick's Morton slot t; padding voxels past the grid are skipped.
__global__ void __launch_bounds__(512) mask_update_kernel(const void* __restrict__ density, bool bf16,
                                                          BrickGeom g, float thr,
                                                          const int32_t* __restrict__ brick_list,
                                                          const int32_t* __restrict__ brick_count,
                                                          uint8_t* __restrict__ mask) {
  const int64_t nb = brick_list ? (int64_t)*brick_count : g.num_bricks();
  const uint32_t t = threadIdx.x;
  const int lx = (int)((t & 1u) | ((t >> 2) & 2u) | ((t >> 4) & 4u));
  const int ly = (int)(((t >> 1) & 1u) | ((t >> 3) & 2u) | ((t >> 5) & 4u));
  const int lz = (int)(((t >> 2) & 1u) | ((t >> 4) & 2u) | ((t >> 6) & 4u));
  for (int64_t i = blockIdx.x; i < nb; i += gridDim.x) {
    const int64_t b = brick_list ? (int64_t)__ldg(brick_list + i) : i;
    const int x = (int)(b % g.nb[0]) * 8 + lx, y = (int)((b / g.nb[0]) % g.nb[1]) * 8 + ly,
              z = (int)(b / ((int64_t)g.nb[0] * g.nb[1])) * 8 + lz;
    if (x >= g.G[0] || y >= g.G[1] || z >= g.G[2]) continue;
    const int64_t slot = b * kBrickVox + t;
    const float raw = bf16 ? bf16_bits_to_f32(reinterpret_cast<const uint16_t*>(density)[slot])
                           : reinterpret_cast<const float*>(density)[slot];
    mask[((int64_t)z * g.G[1] + y) * g.G[0] + x] = raw >= thr ? 1 : 0;
  }
}

// ------------------------------------------------------------------- TV
// One block per brick, 512 threads, thread t on the brick's Morton slot t, so a
// warp covers 32 consecutive voxels (contiguous memory) and the +-x/y/z
// neighbours of most voxels sit in the same or an adjacent warp's lines.
// Each thread handles all channels of its voxel with 128-bit loads when C % 4
// == 0.  Neighbours are summed in the order -x, +x, -y, +y, -z, +z.
__device__ __forceinline__ int compact3(uint32_t v) {
  return (int)((v & 1u) | ((v >> 2) & 2u) | ((v >> 4) & 4u));
}

template <bool kBF16>
__device__ __forceinline__ void load_vox4(const void* grid, int64_t slot, int C, int q, float v[4]) {
  if constexpr (kBF16) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(grid) + slot * C) + q);
    v[0] = __uint_as_float(u.x << 16);
    v[1] = __uint_as_float(u.x & 0xffff0000u);
    v[2] = __uint_as_float(u.y << 16);
    v[3] = __uint_as_float(u.y & 0xffff0000u);
  } else {
    float4 f = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(grid) + slot * C) + q);
    v[0] = f.x;
    v[1] = f.y;
    v[2] = f.z;
    v[3] = f.w;
  }
}

template <bool kBF16>
__device__ __forceinline__ float load_val(const void* grid, int64_t e) {
  return kBF16 ? bf16_bits_to_f32(__ldg(reinterpret_cast<const uint16_t*>(grid) + e))
               : __ldg(reinterpret_cast<const float*>(grid) + e);
}

// The six neighbour slots of voxel (x, y, z) = local Morton index t of brick
// b, in the order -x, +x, -y, +y, -z, +z, as offsets from the voxel's own
// slot (0 where the grid ends; has[d] says which exist; the host checks
// that a layer of nb[0] nb[1] bricks of 512 voxels fits an int32).  Inside the brick a step along axis a changes only a's
// interleaved bits (mask M): +1 is ((t | ~M) + 1) & M, -1 is ((t & M) - 1) & M,
// with t's other bits kept; at the brick face the neighbour is voxel 0 / 7 of
// the next / previous brick along a.
struct TvNbr {
  int32_t off[6];
  bool has[6];
};

__device__ __forceinline__ void tv_neighbours(const BrickGeom& g, int64_t b, int t, int x, int y, int z,
                                              TvNbr& q) {
  const int c[3] = {x, y, z};
  const int32_t bstride[3] = {kBrickVox, g.nb[0] * kBrickVox, g.nb[0] * g.nb[1] * kBrickVox};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int32_t M = 0x49 << a, u = t;
    q.has[2 * a] = c[a] > 0;
    q.has[2 * a + 1] = c[a] + 1 < g.G[a];
    // new local index minus the old, plus the brick step where the face is crossed
    const int32_t lo = (c[a] & 7) == 0 ? (u | M) - u - bstride[a] : ((((u & M) - 1) & M) | (u & ~M)) - u;
    const int32_t hi = (c[a] & 7) == 7 ? (u & ~M) - u + bstride[a] : ((((u | ~M) + 1) & M) | (u & ~M)) - u;
    q.off[2 * a] = q.has[2 * a] ? lo : 0;
    q.off[2 * a + 1] = q.has[2 * a + 1] ? hi : 0;
  }
}

// TV gradient of one voxel (thread t of brick b) of one grid.
template <bool kBF16>
__device__ __forceinline__ void tv_voxel(const void* __restrict__ grid, int C, float scale, float delta,
                                         int dense_mode, float* __restrict__ g_grid, int64_t b, int t,
                                         const TvNbr& q) {
  const int64_t self = b * kBrickVox + t;
  int64_t nbr[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nbr[d] = self + q.off[d];
  const bool* has = q.has;
  if (C % 4 == 0) {
    // sparse mode: a voxel whose data gradient is zero in every channel gets
    // no TV gradient, so its value and neighbours are not loaded at all
    if (!dense_mode) {
      bool any = false;
      for (int q = 0; q < C / 4; ++q) {
        const float4 gin = reinterpret_cast<const float4*>(g_grid + self * C)[q];
        any = any || gin.x != 0.0f || gin.y != 0.0f || gin.z != 0.0f || gin.w != 0.0f;
      }
      if (!any) return;
    }
    // per group of 4 channels: the gradient, the value and the six neighbours
    // are loaded together (no load waits on another)
    for (int q = 0; q < C / 4; ++q) {
      float4* gp = reinterpret_cast<float4*>(g_grid + self * C) + q;
      const float4 gin = *gp;
      float v[4], u[6][4];
      load_vox4<kBF16>(grid, self, C, q, v);
#pragma unroll
      for (int d = 0; d < 6; ++d) load_vox4<kBF16>(grid, nbr[d], C, q, u[d]);
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int d = 0; d < 6; ++d)
        if (has[d])
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] += fminf(fmaxf(v[i] - u[d][i], -delta), delta);
      // sparse mode adds the TV gradient only where the data gradient is non-zero
      const bool any = gin.x != 0.0f || gin.y != 0.0f || gin.z != 0.0f || gin.w != 0.0f;
      if (!dense_mode && !any) continue;
      float4 out = gin;
      if (dense_mode || gin.x != 0.0f) out.x = gin.x + scale * acc[0];
      if (dense_mode || gin.y != 0.0f) out.y = gin.y + scale * acc[1];
      if (dense_mode || gin.z != 0.0f) out.z = gin.z + scale * acc[2];
      if (dense_mode || gin.w != 0.0f) out.w = gin.w + scale * acc[3];
      *gp = out;
    }
  } else {
    for (int c = 0; c < C; ++c) {
      float* gp = g_grid + self * C + c;
      const float gin = *gp;
      if (!dense_mode && gin == 0.0f) continue;   // no TV gradient here: nothing to load
      const float v = load_val<kBF16>(grid, self * C + c);
      float u[6];
#pragma unroll
      for (int d = 0; d < 6; ++d) u[d] = load_val<kBF16>(grid, nbr[d] * C + c);
      float acc = 0.0f;
#pragma unroll
      for (int d = 0; d < 6; ++d)
        if (has[d]) acc += fminf(fmaxf(v - u[d], -delta), delta);
      *gp = gin + scale * acc;
    }
  }
}

constexpr int kMaxMulti = 4;

struct TvGridArgs {
  const void* grid;
  float* g_grid;
  uint8_t* touched;
  float scale;
  int C;
  int bf16;
};
struct TvMulti {
  TvGridArgs a[kMaxMulti];
  int count;
  const int32_t* list;    // flagged bricks (sparse mode) or NULL
  const int32_t* list_n;
};

// One block per brick of all grids (they share the geometry): every brick, or
// the bricks of the compacted list.
__global__ void __launch_bounds__(512, 2) tv_kernel(TvMulti M, BrickGeom g, float delta, int dense_mode) {
  const int64_t nb = M.list ? (int64_t)*M.list_n : g.num_bricks();
  const int t = threadIdx.x;
  const int lx = compact3(t), ly = compact3(t >> 1), lz = compact3(t >> 2);
  for (int64_t i = blockIdx.x; i < nb; i += gridDim.x) {
    const int64_t b = M.list ? (int64_t)M.list[i] : i;
    const int bx = (int)(b % g.nb[0]);
    const int by = (int)((b / g.nb[0]) % g.nb[1]);
    const int bz = (int)(b / ((int64_t)g.nb[0] * g.nb[1]));
    const int x = bx * 8 + lx, y = by * 8 + ly, z = bz * 8 + lz;
    const bool inside = x < g.G[0] && y < g.G[1] && z < g.G[2];
    TvNbr q;
    if (inside) tv_neighbours(g, b, t, x, y, z, q);   // shared by the grids
    for (int i = 0; i < M.count; ++i) {
      const TvGridArgs& A = M.a[i];
      if (!dense_mode && A.touched && A.touched[b] == 0) continue;
      if (dense_mode && A.touched && t == 0) A.touched[b] = 1;
      if (!inside) continue;
      if (A.bf16)
        tv_voxel<true>(A.grid, A.C, A.scale, delta, dense_mode, A.g_grid, b, t, q);
      else
        tv_voxel<false>(A.grid, A.C, A.scale, delta, dense_mode, A.g_grid, b, t, q);
    }
  }
}

// ------------------------------------------------------------------ Adam
struct AdamArgs {
  float lr, b1, b2, eps, inv_c1, inv_c2;
};

__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, const AdamArgs& a,
                                         bool& changed) {
  if (g == 0.0f) return;
  m = a.b1 * m + (1.0f - a.b1) * g;
  v = a.b2 * v + (1.0f - a.b2) * g * g;
  p = p - a.lr * (m * a.inv_c1) / (sqrtf(v * a.inv_c2) + a.eps);
  changed = true;
}

// One float4 group of Adam entries at i (p, m, v loaded by the caller when g
// is non-zero anywhere in the group).
__device__ __forceinline__ void adam_group(float* __restrict__ p, uint16_t* __restrict__ shadow,
                                           float* __restrict__ g, float* __restrict__ m,
                                           float* __restrict__ v, int64_t i, float4 gg, float4 pp,
                                           float4 mm, float4 vv, const AdamArgs& a, int zero_grad) {
  bool ch = false;
  adam_one(pp.x, gg.x, mm.x, vv.x, a, ch);
  adam_one(pp.y, gg.y, mm.y, vv.y, a, ch);
  adam_one(pp.z, gg.z, mm.z, vv.z, a, ch);
  adam_one(pp.w, gg.w, mm.w, vv.w, a, ch);
  *reinterpret_cast<float4*>(p + i) = pp;
  *reinterpret_cast<float4*>(m + i) = mm;
  *reinterpret_cast<float4*>(v + i) = vv;
  if (zero_grad) *reinterpret_cast<float4*>(g + i) = make_float4(0.f, 0.f, 0.f, 0.f);
  if (shadow) {
    uint2 sh;
    sh.x = (uint32_t)f32_to_bf16_bits(pp.x) | ((uint32_t)f32_to_bf16_bits(pp.y) << 16);
    sh.y = (uint32_t)f32_to_bf16_bits(pp.z) | ((uint32_t)f32_to_bf16_bits(pp.w) << 16);
    *reinterpret_cast<uint2*>(shadow + i) = sh;
  }
}

__device__ __forceinline__ bool nonzero4(float4 v) {
  return v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f;
}

// Adam over entries [base, end) of one array, float4 body (base a multiple of
// 4).  Two groups per thread and step, gradient and state loaded together
// (one memory round trip per step; the state of an all-zero group is read
// but neither updated nor written).
__device__ __forceinline__ void adam_range(float* __restrict__ p, uint16_t* __restrict__ shadow,
                                           float* __restrict__ g, float* __restrict__ m,
                                           float* __restrict__ v, int64_t base, int64_t end,
                                           const AdamArgs& a, int zero_grad) {
  const int64_t stride = 4 * (int64_t)blockDim.x;
  int64_t i = base + 4 * (int64_t)threadIdx.x;
  for (; i + stride + 4 <= end; i += 2 * stride) {
    const int64_t j = i + stride;
    const float4 g0 = *reinterpret_cast<const float4*>(g + i);
    const float4 g1 = *reinterpret_cast<const float4*>(g + j);
    const bool n0 = nonzero4(g0), n1 = nonzero4(g1);
    const float4 p0 = *reinterpret_cast<const float4*>(p + i);
    const float4 m0 = *reinterpret_cast<const float4*>(m + i);
    const float4 v0 = *reinterpret_cast<const float4*>(v + i);
    const float4 p1 = *reinterpret_cast<const float4*>(p + j);
    const float4 m1 = *reinterpret_cast<const float4*>(m + j);
    const float4 v1 = *reinterpret_cast<const float4*>(v + j);
    if (n0) adam_group(p, shadow, g, m, v, i, g0, p0, m0, v0, a, zero_grad);
    if (n1) adam_group(p, shadow, g, m, v, j, g1, p1, m1, v1, a, zero_grad);
  }
  for (; i < end; i += stride) {
    if (i + 4 <= end) {
      const float4 gg = *reinterpret_cast<const float4*>(g + i);
      if (!nonzero4(gg)) continue;
      adam_group(p, shadow, g, m, v, i, gg, *reinterpret_cast<const float4*>(p + i),
                 *reinterpret_cast<const float4*>(m + i), *reinterpret_cast<const float4*>(v + i), a,
                 zero_grad);
    } else {
      for (int64_t e = i; e < end; ++e) {
        bool ch = false;
        adam_one(p[e], g[e], m[e], v[e], a, ch);
        if (zero_grad) g[e] = 0.0f;
        if (shadow && ch) shadow[e] = f32_to_bf16_bits(p[e]);
      }
    }
  }
}

// One block per flagged block of entries (bricks of grids).
__global__ void __launch_bounds__(256) adam_blocks_kernel(float* __restrict__ p,
                                                          uint16_t* __restrict__ shadow,
                                                          float* __restrict__ g,
                                                          float* __restrict__ m,
                                                          float* __restrict__ v, int64_t n,
                                                          uint8_t* __restrict__ touched,
                                                          int64_t block_elems, AdamArgs a,
                                                          int zero_grad) {
  const int64_t nblk = (n + block_elems - 1) / block_elems;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    if (touched && touched[b] == 0) continue;
    // block_elems and the block starts are multiples of 4 (checked on the host)
    adam_range(p, shadow, g, m, v, b * block_elems, min((b + 1) * block_elems, n), a, zero_grad);
    if (touched && zero_grad) {
      __syncthreads();
      if (threadIdx.x == 0) touched[b] = 0;
    }
  }
}

struct AdamArray {
  float* p;
  uint16_t* shadow;
  float* g;
  float* m;
  float* v;
  int64_t n;
  uint8_t* touched;
  int64_t block_elems;
  const int32_t* list;     // flagged blocks (or NULL: every block)
  const int32_t* list_n;
  AdamArgs a;
};
struct AdamMulti {
  AdamArray x[kMaxMulti];
  int count;
  const int64_t* step;   // if set: t on the device, bias corrections formed in the kernel
};

// Blocks of all arrays in one index space: array i owns the next
// |list_i| (or ceil(n_i / block_elems_i)) indices.
__global__ void __launch_bounds__(256) adam_multi_kernel(AdamMulti M, int zero_grad) {
  // bias corrections of the device-side step count, formed once by step_increment_kernel
  float corr[2] = {0.0f, 0.0f};
  if (M.step) {
    const float* c = reinterpret_cast<const float*>(M.step + 1);
    corr[0] = c[0];
    corr[1] = c[1];
  }
  int64_t first[kMaxMulti + 1];
  first[0] = 0;
  for (int i = 0; i < M.count; ++i) {
    const AdamArray& A = M.x[i];
    first[i + 1] = first[i] + (A.list ? (int64_t)*A.list_n : (A.n + A.block_elems - 1) / A.block_elems);
  }
  for (int64_t b = blockIdx.x; b < first[M.count]; b += gridDim.x) {
    int i = 0;
    while (i + 1 < M.count && b >= first[i + 1]) ++i;
    const AdamArray& A = M.x[i];
    const int64_t lb = A.list ? (int64_t)A.list[b - first[i]] : b - first[i];
    if (A.touched && A.touched[lb] == 0) continue;
    AdamArgs a = A.a;
    if (M.step) {
      a.inv_c1 = corr[0];
      a.inv_c2 = corr[1];
    }
    adam_range(A.p, A.shadow, A.g, A.m, A.v, lb * A.block_elems, min((lb + 1) * A.block_elems, A.n), a,
               zero_grad);
    if (A.touched && zero_grad) {
      __syncthreads();
      if (threadIdx.x == 0) A.touched[lb] = 0;
    }
  }
}

// Flat parameter vectors of any length and alignment (scalar).
__global__ void adam_flat_kernel(float* __restrict__ p, uint16_t* __restrict__ shadow,
                                 float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, int64_t n, AdamArgs a, int zero_grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool ch = false;
    adam_one(p[i], g[i], m[i], v[i], a, ch);
    if (zero_grad) g[i] = 0.0f;
    if (shadow && ch) shadow[i] = f32_to_bf16_bits(p[i]);
  }
}

}  // namespace dvgo

using namespace dvgo;

extern "C" int64_t dvgo_grid_num_bricks(const int32_t G[3]) {
  if (!G || G[0] < 1 || G[1] < 1 || G[2] < 1) return -1;
  return make_geom(G).num_bricks();
}

extern "C" int64_t dvgo_grid_bricked_elems(const int32_t G[3], int32_t C) {
  int64_t nb = dvgo_grid_num_bricks(G);
  if (nb < 0 || C < 1) return -1;
  return nb * kBrickVox * C;
}

static int pack_impl(const void* src, void* dst, const int32_t G[3], int32_t C, int dtype,
                     void* stream, bool to_bricked) {
  DVGO_CHECK_ARG(src && dst && G && C >= 1 && (dtype == DVGO_F32 || dtype == DVGO_BF16));
  DVGO_CHECK_ARG(G[0] >= 1 && G[1] >= 1 && G[2] >= 1);
  BrickGeom g = make_geom(G);
  cudaStream_t st = as_stream(stream);
  size_t esz = dtype == DVGO_F32 ? 4 : 2;
  if (to_bricked) cudaMemsetAsync(dst, 0, (size_t)g.num_bricks() * kBrickVox * C * esz, st);
  int64_t nvox = (int64_t)G[0] * G[1] * G[2];
  int grid = grid_for(nvox, 256, 16);
  if (dtype == DVGO_F32) {
    if (to_bricked)
      pack_kernel<float><<<grid, 256, 0, st>>>((const float*)src, (float*)dst, g, C, true);
    else
      pack_kernel<float><<<grid, 256, 0, st>>>((const float*)src, (float*)dst, g, C, false);
  } else {
    pack_kernel<uint16_t><<<grid, 256, 0, st>>>((const uint16_t*)src, (uint16_t*)dst, g, C,
                                                to_bricked);
  }
  return launch_status();
}

extern "C" int dvgo_grid_pack(const void* dense, void* bricked, const int32_t G[3], int32_t C,
                              int dtype, void* stream) {
  return pack_impl(dense, bricked, G, C, dtype, stream, true);
}

extern "C" int dvgo_grid_resample(const float* src, const int32_t G_src[3], void* dst, int dst_dtype,
                                  const int32_t G_dst[3], int32_t C, void* stream) {
  DVGO_CHECK_ARG(src && dst && G_src && G_dst && C >= 1 && (dst_dtype == DVGO_F32 || dst_dtype == DVGO_BF16));
  for (int a = 0; a < 3; ++a) DVGO_CHECK_ARG(G_src[a] >= 2 && G_dst[a] >= 2);
  const BrickGeom gs = make_geom(G_src), gd = make_geom(G_dst);
  const int64_t nvox = (int64_t)G_dst[0] * G_dst[1] * G_dst[2];
  const int g = grid_for(nvox, 256, 16);
  cudaStream_t st = as_stream(stream);
  if (dst_dtype == DVGO_F32)
    resample_kernel<false><<<g, 256, 0, st>>>(src, gs, dst, gd, C);
  else
    resample_kernel<true><<<g, 256, 0, st>>>(src, gs, dst, gd, C);
  return launch_status();
}

extern "C" int dvgo_grid_unpack(const void* bricked, void* dense, const int32_t G[3], int32_t C,
                                int dtype, void* stream) {
  return pack_impl(bricked, dense, G, C, dtype, stream, false);
}

// alpha(raw) >= thr  <=>  raw >= log(expm1(-log1p(-thr)/interval)) - shift.
// The FP32 threshold is the smallest float not below the exact one, so the
// FP32 comparison decides exactly like the FP64 one.
static float mask_raw_threshold(float shift, float interval, float alpha_thres) {
  const double q = -log1p(-(double)alpha_thres) / (double)interval;
  const double thr64 = log(expm1(q)) - (double)shift;
  float thr = (float)thr64;
  if ((double)thr < thr64) thr = nextafterf(thr, INFINITY);
  return thr;
}

extern "C" int dvgo_update_mask(const void* density, int dtype, const dvgo_grid_desc* grid, float shift,
                                float interval, float alpha_thres, const int32_t* brick_list,
                                const int32_t* brick_count, uint8_t* mask, void* stream) {
  DVGO_CHECK_ARG(density && grid && mask && (dtype == DVGO_F32 || dtype == DVGO_BF16));
  DVGO_CHECK_ARG(interval > 0.0f && alpha_thres > 0.0f && alpha_thres < 1.0f);
  DVGO_CHECK_ARG(grid->G[0] >= 1 && grid->G[1] >= 1 && grid->G[2] >= 1);
  DVGO_CHECK_ARG((brick_list == nullptr) == (brick_count == nullptr));
  const float thr = mask_raw_threshold(shift, interval, alpha_thres);
  const BrickGeom g = make_geom(grid->G);
  const int blocks = (int)std::min<int64_t>(g.num_bricks(), (int64_t)kNumSMs * 4);
  mask_update_kernel<<<blocks, 512, 0, as_stream(stream)>>>(density, dtype == DVGO_BF16, g, thr, brick_list,
                                                             brick_count, mask);
  return launch_status();
}

extern "C" int dvgo_build_mask(const void* density, int dtype, const dvgo_grid_desc* grid,
                               float shift, float interval, float alpha_thres, uint8_t* mask,
                               void* stream) {
  DVGO_CHECK_ARG(density && grid && mask && (dtype == DVGO_F32 || dtype == DVGO_BF16));
  DVGO_CHECK_ARG(interval > 0.0f && alpha_thres > 0.0f && alpha_thres < 1.0f);
  DVGO_CHECK_ARG(grid->G[0] >= 1 && grid->G[1] >= 1 && grid->G[2] >= 1);
  const float thr = mask_raw_threshold(shift, interval, alpha_thres);
  BrickGeom g = make_geom(grid->G);
  int64_t nvox = (int64_t)grid->G[0] * grid->G[1] * grid->G[2];
  cudaStream_t st = as_stream(stream);
  mask_kernel<<<grid_for(nvox, 256, 16), 256, 0, st>>>(density, dtype == DVGO_BF16, g, thr, mask);
  return launch_status();
}

// ------------------------------------------------- density query + weights
// dvgo_sample_grid_fwd of the density (one channel) fused with the weights
// pass (dvgo_alpha_weights_fwd): one warp per ray, 32 samples at a time; each
// lane queries its sample's density, the warp scans log T, and the ray stops
// at the halt, so no sample past it is queried.  Same arithmetic as the two
// separate kernels.
template <bool kBF16>
__global__ void __launch_bounds__(256) density_alpha_kernel(
    const void* __restrict__ grid, TriArgs Tr, const float* __restrict__ xyz,
    const int64_t* __restrict__ ray_off, int64_t R, float shift, float interval,
    const float* __restrict__ delta, float T_stop,
    float* __restrict__ raw, float* __restrict__ w, float* __restrict__ T,
    int32_t* __restrict__ n_live, float* __restrict__ T_end) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp0; r < R; r += nwarps) {
    const int64_t b = ray_off[r];
    const int N = (int)(ray_off[r + 1] - b);
    Kahan carry;  // log T before the current chunk
    int stop = N;
    float t_end = 1.0f;
    int c0 = 0;
    for (; c0 < N; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < N;
      float rv = 0.0f;
      if (valid) {
        Corners c;
        corners(Tr, xyz, b + i, c);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if constexpr (kBF16)
            rv += c.w[k] * bf16_bits_to_f32(__ldg(reinterpret_cast<const uint16_t*>(grid) + c.slot[k]));
          else
            rv += c.w[k] * __ldg(reinterpret_cast<const float*>(grid) + c.slot[k]);
        }
        raw[b + i] = rv;
      }
      const float la = valid ? -(delta ? __ldg(delta + b + i) : interval) * softplus_f(rv + shift) : 0.0f;
      const float incl = warp_incl_sum(la);
      const float logT = __fadd_rn(carry.s, __fsub_rn(warp_excl_from_incl(incl), carry.c));
      const float Ti = expf(logT);
      const unsigned below = __ballot_sync(0xffffffffu, valid && Ti < T_stop);
      const int first = below ? __ffs(below) - 1 : 32;
      if (below) {
        stop = c0 + first;
        t_end = __shfl_sync(0xffffffffu, Ti, first);
      }
      if (valid) {
        if (lane < first) {
          w[b + i] = Ti * -expm1f(la);
          T[b + i] = Ti;
        } else {
          w[b + i] = 0.0f;
          T[b + i] = t_end;
        }
      }
      if (below) break;
      carry.add(__shfl_sync(0xffffffffu, incl, 31));
    }
    if (stop == N) t_end = expf(__fsub_rn(carry.s, carry.c));
    for (c0 += 32; c0 < N; c0 += 32) {
      const int i = c0 + lane;
      if (i < N) {
        raw[b + i] = 0.0f;   // past the halt: not queried
        w[b + i] = 0.0f;
        T[b + i] = t_end;
      }
    }
    if (lane == 0) {
      n_live[r] = stop;
      T_end[r] = t_end;
    }
  }
}

extern "C" int dvgo_density_alpha_fwd(const void* grid, int dtype, const dvgo_grid_desc* gd,
                                      const float* xyz, const int64_t* ray_off, int64_t R,
                                      float shift, float interval, const float* delta, float T_stop,
                                      float* raw, float* w, float* T, int32_t* n_live, float* T_end,
                                      void* stream) {
  DVGO_CHECK_ARG(gd && R >= 0 && interval > 0.0f && T_stop >= 0.0f);
  DVGO_CHECK_ARG(dtype == DVGO_F32 || dtype == DVGO_BF16);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(grid && xyz && ray_off && raw && w && T && n_live && T_end);
  TriArgs Tr;
  DVGO_CHECK_ARG(make_tri(Tr, gd));
  const int g = grid_for(R * 32, 256, 16);
  if (dtype == DVGO_F32)
    density_alpha_kernel<false><<<g, 256, 0, as_stream(stream)>>>(grid, Tr, xyz, ray_off, R, shift, interval,
                                                                   delta, T_stop, raw, w, T, n_live, T_end);
  else
    density_alpha_kernel<true><<<g, 256, 0, as_stream(stream)>>>(grid, Tr, xyz, ray_off, R, shift, interval,
                                                                  delta, T_stop, raw, w, T, n_live, T_end);
  return launch_status();
}

extern "C" int dvgo_sample_grid_fwd(const void* grid, int dtype, const dvgo_grid_desc* gd,
                                    int32_t C, const float* xyz, const int32_t* idx, int64_t n_cap,
                                    const int64_t* n_dev, float* out, void* stream) {
  DVGO_CHECK_ARG(gd && C >= 1 && n_cap >= 0 && (dtype == DVGO_F32 || dtype == DVGO_BF16));
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG(grid && xyz && out);
  TriArgs T;
  DVGO_CHECK_ARG(make_tri(T, gd));
  cudaStream_t st = as_stream(stream);
  const int block = 256;
  int g = grid_for(n_cap, block, 16);
  if (C == 1 || C == 12) {   // the specialised kernels loop: one resident wave of blocks
    static int per_sm[2][2] = {{0, 0}, {0, 0}};
    const int di = dtype == DVGO_F32 ? 0 : 1, ci = C == 1 ? 0 : 1;
    if (!per_sm[di][ci]) {
      const void* fn = di == 0 ? (ci == 0 ? (const void*)gather_fwd_kernel<1, false>
                                          : (const void*)gather_fwd_kernel<12, false>)
                               : (ci == 0 ? (const void*)gather_fwd_kernel<1, true>
                                          : (const void*)gather_fwd_kernel<12, true>);
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, block, 0) != cudaSuccess || b < 1) b = 1;
      per_sm[di][ci] = b;
    }
    g = (int)std::min<int64_t>(ceil_div(n_cap, block), (int64_t)kNumSMs * per_sm[di][ci]);
  }
  if (dtype == DVGO_F32) {
    if (C == 1) gather_fwd_kernel<1, false><<<g, block, 0, st>>>(grid, T, xyz, idx, n_cap, n_dev, out);
    else if (C == 12) gather_fwd_kernel<12, false><<<g, block, 0, st>>>(grid, T, xyz, idx, n_cap, n_dev, out);
    else gather_fwd_generic_kernel<false><<<g, block, 0, st>>>(grid, T, C, xyz, idx, n_cap, n_dev, out);
  } else {
    if (C == 1) gather_fwd_kernel<1, true><<<g, block, 0, st>>>(grid, T, xyz, idx, n_cap, n_dev, out);
    else if (C == 12) gather_fwd_kernel<12, true><<<g, block, 0, st>>>(grid, T, xyz, idx, n_cap, n_dev, out);
    else gather_fwd_generic_kernel<true><<<g, block, 0, st>>>(grid, T, C, xyz, idx, n_cap, n_dev, out);
  }
  return launch_status();
}

extern "C" int dvgo_sample_grid_bwd(const float* g_out, const dvgo_grid_desc* gd, int32_t C,
                                    const float* xyz, const int32_t* idx, int64_t n_cap,
                                    const int64_t* n_dev, float* g_grid, uint8_t* touched,
                                    void* stream) {
  DVGO_CHECK_ARG(gd && C >= 1 && n_cap >= 0);
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG(g_out && xyz && g_grid);
  TriArgs T;
  DVGO_CHECK_ARG(make_tri(T, gd));
  cudaStream_t st = as_stream(stream);
  const int block = 256;
  int g = grid_for(n_cap, block, 16);
  if (C == 1) scatter_bwd_kernel<1><<<g, block, 0, st>>>(g_out, T, xyz, idx, n_cap, n_dev, g_grid, touched);
  else if (C == 12) scatter_bwd_kernel<12><<<g, block, 0, st>>>(g_out, T, xyz, idx, n_cap, n_dev, g_grid, touched);
  else scatter_bwd_generic_kernel<<<g, block, 0, st>>>(g_out, T, C, xyz, idx, n_cap, n_dev, g_grid, touched);
  return launch_status();
}

extern "C" int dvgo_tv_add_grad(const void* grid, int dtype, const int32_t G[3], int32_t C,
                                float weight, float delta, int dense_mode, uint8_t* touched,
                                float* g_grid, void* stream) {
  dvgo_tv_grid one{grid, dtype, C, weight, touched, g_grid};
  return dvgo_tv_add_grad_multi(&one, 1, G, delta, dense_mode, nullptr, nullptr, stream);
}

extern "C" int dvgo_tv_add_grad_multi(const dvgo_tv_grid* grids, int32_t count, const int32_t G[3],
                                      float delta, int dense_mode, const int32_t* brick_list,
                                      const int32_t* brick_count, void* stream) {
  DVGO_CHECK_ARG(grids && count >= 1 && count <= kMaxMulti && G && delta > 0.0f);
  DVGO_CHECK_ARG(G[0] >= 1 && G[1] >= 1 && G[2] >= 1);
  BrickGeom g = make_geom(G);
  // neighbour offsets are int32: one layer of bricks must fit
  DVGO_CHECK_ARG((int64_t)g.nb[0] * g.nb[1] * kBrickVox <= (int64_t)INT32_MAX / 2);
  const double N = (double)G[0] * G[1] * G[2];
  TvMulti M{};
  M.count = count;
  for (int i = 0; i < count; ++i) {
    const dvgo_tv_grid& q = grids[i];
    DVGO_CHECK_ARG(q.grid && q.g_grid && q.C >= 1 && (q.dtype == DVGO_F32 || q.dtype == DVGO_BF16));
    M.a[i] = TvGridArgs{q.grid, q.g_grid, q.touched, (float)((double)q.weight * 2.0 / (N * q.C)), q.C,
                        q.dtype == DVGO_BF16 ? 1 : 0};
  }
  const bool use_list = !dense_mode && brick_list && brick_count;
  M.list = use_list ? brick_list : nullptr;
  M.list_n = use_list ? brick_count : nullptr;
  // with the list: persistent blocks over the flagged bricks; without: one
  // block per brick (blocks of unflagged bricks retire at once)
  const int nb = use_list ? (int)std::min<int64_t>(g.num_bricks(), (int64_t)kNumSMs * 2)
                          : (int)std::min<int64_t>(g.num_bricks(), (int64_t)1 << 30);
  tv_kernel<<<nb, 512, 0, as_stream(stream)>>>(M, g, delta, dense_mode);
  return launch_status();
}

extern "C" int dvgo_adam_step(float* p, uint16_t* p_shadow, float* g, float* m, float* v, int64_t n,
                              uint8_t* touched, int64_t block_elems, float lr, float beta1,
                              float beta2, float eps, int64_t step, int zero_grad, void* stream) {
  DVGO_CHECK_ARG(n >= 0 && step >= 1);
  if (n == 0) return DVGO_OK;
  DVGO_CHECK_ARG(p && g && m && v);
  AdamArgs a;
  a.lr = lr;
  a.b1 = beta1;
  a.b2 = beta2;
  a.eps = eps;
  a.inv_c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
  a.inv_c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
  cudaStream_t st = as_stream(stream);
  bool aligned = ((uintptr_t)p % 16 == 0) && ((uintptr_t)g % 16 == 0) && ((uintptr_t)m % 16 == 0) &&
                 ((uintptr_t)v % 16 == 0) && (!p_shadow || (uintptr_t)p_shadow % 8 == 0);
  if (touched) {
    DVGO_CHECK_ARG(block_elems > 0 && block_elems % 4 == 0 && aligned);
    int64_t nblk = (n + block_elems - 1) / block_elems;
    int grid = (int)std::min<int64_t>(nblk, (int64_t)kNumSMs * 8);
    adam_blocks_kernel<<<grid, 256, 0, st>>>(p, p_shadow, g, m, v, n, touched, block_elems, a,
                                             zero_grad);
  } else if (aligned && n % 4 == 0) {
    int64_t be = 4096;
    int64_t nblk = (n + be - 1) / be;
    int grid = (int)std::min<int64_t>(nblk, (int64_t)kNumSMs * 8);
    adam_blocks_kernel<<<grid, 256, 0, st>>>(p, p_shadow, g, m, v, n, nullptr, be, a, zero_grad);
  } else {
    adam_flat_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(p, p_shadow, g, m, v, n, a, zero_grad);
  }
  return launch_status();
}

extern "C" int dvgo_sample_grid_bwd2(const float* g_out_a, int32_t C_a, float* g_grid_a,
                                     uint8_t* touched_a, const float* g_out_b, int32_t C_b,
                                     float* g_grid_b, uint8_t* touched_b, const dvgo_grid_desc* gd,
                                     const float* xyz, const int32_t* idx, int64_t n_cap,
                                     const int64_t* n_dev, void* stream) {
  DVGO_CHECK_ARG(gd && C_a >= 1 && C_b >= 1 && n_cap >= 0);
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG(g_out_a && g_grid_a && g_out_b && g_grid_b && xyz);
  if (C_a == 1 && C_b == 12 && (uintptr_t)g_out_b % 16 == 0 && (uintptr_t)g_grid_b % 16 == 0) {
    TriArgs T;
    DVGO_CHECK_ARG(make_tri(T, gd));
    cudaStream_t st = as_stream(stream);
    scatter_bwd_1_12_kernel<<<grid_for(n_cap, 256, 16), 256, 0, st>>>(
        g_out_a, g_grid_a, touched_a, g_out_b, g_grid_b, touched_b, T, xyz, idx, n_cap, n_dev);
    return launch_status();
  }
  int r = dvgo_sample_grid_bwd(g_out_a, gd, C_a, xyz, idx, n_cap, n_dev, g_grid_a, touched_a, stream);
  if (r != DVGO_OK) return r;
  return dvgo_sample_grid_bwd(g_out_b, gd, C_b, xyz, idx, n_cap, n_dev, g_grid_b, touched_b, stream);
}

// beta^t in FP64 by binary exponentiation (about 2 log2 t products; this
// GPU's FP64 rate makes a general pow() cost several microseconds on one
// thread).
__device__ __forceinline__ double pow_int(double beta, int64_t t) {
  double r = 1.0;
  while (t > 0) {
    if (t & 1) r *= beta;
    beta *= beta;
    t >>= 1;
  }
  return r;
}

// step[0] += 1; step[1] holds the two FP32 bias corrections of the new t.
__global__ void step_increment_kernel(int64_t* step, float beta1, float beta2) {
  const int64_t t = step[0] + 1;
  step[0] = t;
  float* c = reinterpret_cast<float*>(step + 1);
  c[0] = (float)(1.0 / (1.0 - pow_int((double)beta1, t)));
  c[1] = (float)(1.0 / (1.0 - pow_int((double)beta2, t)));
}

static int adam_multi(const dvgo_adam_param* params, int32_t count, float beta1, float beta2, float eps,
                      int64_t step, int64_t* step_dev, int zero_grad, void* stream);

extern "C" int dvgo_adam_step_multi(const dvgo_adam_param* params, int32_t count, float beta1,
                                    float beta2, float eps, int64_t step, int zero_grad,
                                    void* stream) {
  DVGO_CHECK_ARG(step >= 1);
  return adam_multi(params, count, beta1, beta2, eps, step, nullptr, zero_grad, stream);
}

extern "C" int dvgo_adam_step_multi_dev(const dvgo_adam_param* params, int32_t count, float beta1,
                                        float beta2, float eps, int64_t* step, int zero_grad,
                                        void* stream) {
  DVGO_CHECK_ARG(step);
  step_increment_kernel<<<1, 1, 0, as_stream(stream)>>>(step, beta1, beta2);
  return adam_multi(params, count, beta1, beta2, eps, 1, step, zero_grad, stream);
}

static int adam_multi(const dvgo_adam_param* params, int32_t count, float beta1, float beta2, float eps,
                      int64_t step, int64_t* step_dev, int zero_grad, void* stream) {
  DVGO_CHECK_ARG(params && count >= 1 && count <= kMaxMulti);
  AdamMulti M{};
  M.count = 0;
  M.step = step_dev;
  int64_t total = 0;
  bool lists = false;
  const float inv_c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
  const float inv_c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
  for (int i = 0; i < count; ++i) {
    const dvgo_adam_param& q = params[i];
    DVGO_CHECK_ARG(q.n >= 0);
    if (q.n == 0) continue;
    DVGO_CHECK_ARG(q.p && q.g && q.m && q.v);
    DVGO_CHECK_ARG((uintptr_t)q.p % 16 == 0 && (uintptr_t)q.g % 16 == 0 && (uintptr_t)q.m % 16 == 0 &&
                   (uintptr_t)q.v % 16 == 0 && (!q.p_shadow || (uintptr_t)q.p_shadow % 8 == 0));
    const int64_t be = q.touched ? q.block_elems : 4096;
    DVGO_CHECK_ARG(be > 0 && be % 4 == 0);
    const bool use_list = q.touched && q.block_list && q.block_count;
    lists |= use_list;
    AdamArray& A = M.x[M.count++];
    A = AdamArray{q.p, q.p_shadow, q.g, q.m, q.v, q.n, q.touched, be,
                  use_list ? q.block_list : nullptr, use_list ? q.block_count : nullptr,
                  AdamArgs{q.lr, beta1, beta2, eps, inv_c1, inv_c2}};
    total += (q.n + be - 1) / be;
  }
  if (M.count == 0) return DVGO_OK;
  // with lists the block count is on the device: persistent blocks; else one
  // block per block of entries
  const int grid = lists ? (int)std::min<int64_t>(total, (int64_t)kNumSMs * 8)
                         : (int)std::min<int64_t>(total, (int64_t)1 << 30);
  adam_multi_kernel<<<grid, 256, 0, as_stream(stream)>>>(M, zero_grad);
  return launch_status();
}

__global__ void __launch_bounds__(256) touched_compact_kernel(const uint8_t* __restrict__ touched,
                                                              int64_t nb, int32_t* __restrict__ list,
                                                              int32_t* __restrict__ count) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const bool on = touched[b] != 0;
    // one counter update per warp
    const unsigned act = __activemask();
    const unsigned mask = __ballot_sync(act, on);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader && mask) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(act, base, leader);
    if (on) list[base + __popc(mask & ((1u << lane) - 1))] = (int32_t)b;
  }
}

extern "C" int dvgo_touched_compact(const uint8_t* touched, int64_t nb, int32_t* list, int32_t* count,
                                    void* stream) {
  DVGO_CHECK_ARG(nb >= 0 && count);
  cudaStream_t st = as_stream(stream);
  cudaMemsetAsync(count, 0, sizeof(int32_t), st);
  if (nb == 0) return launch_status();
  DVGO_CHECK_ARG(touched && list && nb < ((int64_t)1 << 31));
  touched_compact_kernel<<<grid_for(nb, 256, 4), 256, 0, st>>>(touched, nb, list, count);
  return launch_status();
}

extern "C" int dvgo_grid_adam_step(float* p, uint16_t* p_shadow, float* g, float* m, float* v,
                                   const int32_t G[3], int32_t C, uint8_t* touched, float lr, float beta1,
                                   float beta2, float eps, int64_t step, int zero_grad, void* stream) {
  DVGO_CHECK_ARG(G && C >= 1 && G[0] >= 1 && G[1] >= 1 && G[2] >= 1);
  const int64_t n = make_geom(G).num_bricks() * kBrickVox * C;
  return dvgo_adam_step(p, p_shadow, g, m, v, n, touched, (int64_t)kBrickVox * C, lr, beta1, beta2, eps,
                        step, zero_grad, stream);
}
