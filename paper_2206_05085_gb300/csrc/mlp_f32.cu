// Colour MLP (rgbnet, the shallow decoder of the hybrid representation of
// Tab. 1) in exact FP32 on the CUDA cores: 39 -> ReLU 128 -> ReLU 128 ->
// sigmoid 3.  Fused per tile of 128 samples.  The forward can store both
// hidden activations (list position j: act[j][0:128] = h1, act[j][128:256]
// = h2); the backward then reads them instead of recomputing the forward.
// Persistent CTAs keep their share of the weight gradients in registers
// across tiles and flush them once with atomics.
//
// 256 threads, ty = tid / 16, tx = tid % 16.  Shared-memory rows have
// pitches 44 (40-wide) and 132 (128-wide): multiples of 4 floats (128-bit
// loads) whose stride moves 16 threads onto 16 distinct bank quads.
//   NT products (k contiguous in both operands): thread rows ty + 16a,
//     columns tx + 16b, 128-bit loads along k.
//   TN products (reduction over the tile's samples): thread rows
//     {4ty..4ty+3, 64+4ty..}, columns {4tx..4tx+3, 64+4tx..}, 128-bit loads
//     along the row of each sample.
#include "common.cuh"
#include "mlp_common.cuh"

namespace dvgo {

constexpr int kP40 = 44;   // pitch of 40-wide rows
constexpr int kP128 = 132; // pitch of 128-wide rows
constexpr int kAct = 2 * kHid;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}
__device__ __forceinline__ float comp(float4 v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

// W1 (+ b1 as column 39) into [128][44]; W2 into [128][132].
__device__ __forceinline__ void load_w1(const float* __restrict__ params, float* W1S) {
  for (int e = threadIdx.x; e < kHid * kP40; e += blockDim.x) {
    const int o = e / kP40, k = e % kP40;
    W1S[e] = k < kIn ? params[kOffW1 + o * kIn + k] : (k == kIn ? params[kOffB1 + o] : 0.0f);
  }
}
__device__ __forceinline__ void load_w2(const float* __restrict__ params, float* W2S) {
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int o = e / kHid, i = e % kHid;
    W2S[o * kP128 + i] = params[kOffW2 + e];
  }
}

// acc[a][b] = sum_k A[(ty+16a)*lda + k] * B[(tx+16b)*ldb + k], K % 4 == 0
template <int K>
__device__ __forceinline__ void gemm_nt(const float* A, int lda, const float* B, int ldb, int ty,
                                        int tx, float acc[8][8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 2
  for (int k = 0; k < K; k += 4) {
    float4 av[8], bv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) av[a] = ld4(A + (ty + 16 * a) * lda + k);
#pragma unroll
    for (int b = 0; b < 8; ++b) bv[b] = ld4(B + (tx + 16 * b) * ldb + k);
    // outer-product order: 64 independent FMAs per k
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(comp(av[a], q), comp(bv[b], q), acc[a][b]);
  }
}

// Write the thread's 8x8 block (rows ty + 16a, columns tx + 16b) of a tile.
__device__ __forceinline__ void store_block(float* S, int ld, int ty, int tx, const float v[8][8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) S[(ty + 16 * a) * ld + tx + 16 * b] = v[a][b];
}

// Copy a [128][128] smem tile (pitch 132) to / from rows j0.. of a global
// [.][256] activation buffer at column offset col (rows past n skipped).
__device__ __forceinline__ void tile_to_global(const float* S, float* __restrict__ act, int64_t j0,
                                               int64_t n, int col) {
  for (int e = threadIdx.x; e < kTile * (kHid / 4); e += blockDim.x) {
    const int r = e >> 5, c4 = (e & 31) * 4;
    if (j0 + r < n) st4(act + (j0 + r) * kAct + col + c4, ld4(S + r * kP128 + c4));
  }
}
__device__ __forceinline__ void tile_from_global(float* S, const float* __restrict__ act, int64_t j0,
                                                 int64_t n, int col) {
  for (int e = threadIdx.x; e < kTile * (kHid / 4); e += blockDim.x) {
    const int r = e >> 5, c4 = (e & 31) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j0 + r < n) v = __ldg(reinterpret_cast<const float4*>(act + (j0 + r) * kAct + col + c4));
    st4(S + r * kP128 + c4, v);
  }
}

__device__ __forceinline__ void build_x_tile(float* XS, const float* __restrict__ k0,
                                             const float* __restrict__ rays_d,
                                             const int32_t* __restrict__ ray_id,
                                             const int32_t* __restrict__ idx, int64_t j0, int64_t n) {
  if (threadIdx.x < kTile) {
    float row[kInP];
    encode_row(k0, rays_d, ray_id, idx, j0 + threadIdx.x, n, row);
    float* dst = XS + threadIdx.x * kP40;
#pragma unroll
    for (int k = 0; k < kInP; k += 4) st4(dst + k, make_float4(row[k], row[k + 1], row[k + 2], row[k + 3]));
  }
}

__global__ void __launch_bounds__(256, 1) rgbnet_fwd_f32_kernel(
    const float* __restrict__ k0, const float* __restrict__ rays_d,
    const int32_t* __restrict__ ray_id, const int32_t* __restrict__ idx, int64_t n_cap,
    const int64_t* __restrict__ n_dev, const float* __restrict__ params, float* __restrict__ rgb,
    float* __restrict__ act) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* W1S = smem;                   // [128][44]
  float* W2S = W1S + kHid * kP40;      // [128][132]
  float* XS = W2S + kHid * kP128;      // [128][44]
  float* HS = XS + kTile * kP40;       // [128][132]  h1, then h2
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  load_w1(params, W1S);
  load_w2(params, W2S);
  float b2v[8], w3[3][8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    b2v[b] = __ldg(params + kOffB2 + tx + 16 * b);
#pragma unroll
    for (int c = 0; c < 3; ++c) w3[c][b] = __ldg(params + kOffW3 + c * kHid + tx + 16 * b);
  }
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t j0 = t * kTile;
    __syncthreads();
    build_x_tile(XS, k0, rays_d, ray_id, idx, j0, n);
    __syncthreads();
    float acc[8][8];
    gemm_nt<kInP>(XS, kP40, W1S, kP40, ty, tx, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaxf(acc[a][b], 0.0f);
    store_block(HS, kP128, ty, tx, acc);
    __syncthreads();
    if (act) tile_to_global(HS, act, j0, n, 0);
    gemm_nt<kHid>(HS, kP128, W2S, kP128, ty, tx, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaxf(acc[a][b] + b2v[b], 0.0f);
    if (act) {
      __syncthreads();  // h1 fully read
      store_block(HS, kP128, ty, tx, acc);
      __syncthreads();
      tile_to_global(HS, act, j0, n, kHid);
    }
    // layer 3: 8 rows x 3 outputs, reduced over the 16 threads sharing ty
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      float z[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int b = 0; b < 8; ++b) s = fmaf(w3[c][b], acc[a][b], s);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        z[c] = s + __ldg(params + kOffB3 + c);
      }
      const int64_t j = j0 + ty + 16 * a;
      if (tx == 0 && j < n) {
        const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
#pragma unroll
        for (int c = 0; c < 3; ++c) rgb[3 * s + c] = sigmoid_f(z[c]);
      }
    }
  }
}

// Backward.  Per tile: h1, h2 (stored, or recomputed when act is NULL), y =
// rgb -> g_z3 -> dW3/db3, g_z2 -> dW2/db2, g_h1 -> g_z1 -> dW1/db1, g_k0.
__global__ void __launch_bounds__(256, 1) rgbnet_bwd_f32_kernel(
    const float* __restrict__ g_rgb, const float* __restrict__ g_color, const float* __restrict__ w,
    const float* __restrict__ k0, const float* __restrict__ rays_d,
    const int32_t* __restrict__ ray_id, const int32_t* __restrict__ idx, int64_t n_cap,
    const int64_t* __restrict__ n_dev, const float* __restrict__ params,
    const float* __restrict__ act, const float* __restrict__ rgb_saved,
    float* __restrict__ g_params, float* __restrict__ g_k0) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* W2S = smem;                   // [128][132]
  float* H1S = W2S + kHid * kP128;     // [128][132]  h1, later g_z1
  float* GS = H1S + kTile * kP128;     // [128][132]  x (pitch 44), h2, g_z2, x again
  float* W1S = GS + kTile * kP128;     // [128][44]
  float* GZ3 = W1S + kHid * kP40;      // [128][4]    g_z3 per tile row
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  load_w1(params, W1S);
  load_w2(params, W2S);
  // persistent gradient partials
  float dW2[8][8], db2[8], dW1[8][3], db3[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    db2[a] = 0.0f;
#pragma unroll
    for (int b = 0; b < 8; ++b) dW2[a][b] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) dW1[a][c] = 0.0f;
  }
  const int o3 = tid & 127, half = tid >> 7;  // dW3: output column, sample half
  float w3o[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) w3o[c] = 0.0f;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t j0 = t * kTile;
    __syncthreads();
    if (act) {
      tile_from_global(H1S, act, j0, n, 0);
      tile_from_global(GS, act, j0, n, kHid);
    } else {
      build_x_tile(GS, k0, rays_d, ray_id, idx, j0, n);
      __syncthreads();
      float acc[8][8];
      gemm_nt<kInP>(GS, kP40, W1S, kP40, ty, tx, acc);
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaxf(acc[a][b], 0.0f);
      store_block(H1S, kP128, ty, tx, acc);
      __syncthreads();
      gemm_nt<kHid>(H1S, kP128, W2S, kP128, ty, tx, acc);
      __syncthreads();  // x no longer read
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
          acc[a][b] = fmaxf(acc[a][b] + __ldg(params + kOffB2 + tx + 16 * b), 0.0f);
      store_block(GS, kP128, ty, tx, acc);
    }
    __syncthreads();  // h1, h2 tiles complete
    // g_z3 = g_rgb * y (1 - y); y is the stored forward output (or recomputed)
    if (tid < kTile) {
      const int64_t j = j0 + tid;
      float g[3] = {0.f, 0.f, 0.f};
      if (j < n) {
        const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
        upstream_rgb_grad(g_rgb, g_color, w, ray_id, s, g);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float y;
          if (rgb_saved) {
            y = __ldg(rgb_saved + 3 * s + c);
          } else {
            float z = __ldg(params + kOffB3 + c);
            for (int o = 0; o < kHid; o += 4)
              z = dot4(ld4(GS + tid * kP128 + o), __ldg(reinterpret_cast<const float4*>(params + kOffW3 + c * kHid + o)), z);
            y = sigmoid_f(z);
          }
          g[c] *= y * (1.0f - y);
        }
      }
      st4(GZ3 + 4 * tid, make_float4(g[0], g[1], g[2], 0.0f));
    }
    __syncthreads();
    // dW3[c][o] += sum_s g_z3[s][c] h2[s][o]: thread = (o, half of the rows)
    {
      const float* h2 = GS + o3;
#pragma unroll 4
      for (int r = half * 64; r < half * 64 + 64; ++r) {
        const float4 g = ld4(GZ3 + 4 * r);
        const float hv = h2[r * kP128];
        w3o[0] = fmaf(g.x, hv, w3o[0]);
        w3o[1] = fmaf(g.y, hv, w3o[1]);
        w3o[2] = fmaf(g.z, hv, w3o[2]);
      }
      if (tid == 0)
        for (int r = 0; r < kTile; ++r) {
          const float4 g = ld4(GZ3 + 4 * r);
          db3[0] += g.x;
          db3[1] += g.y;
          db3[2] += g.z;
        }
    }
    __syncthreads();  // h2 read by everyone above
    // g_z2[s][o] = (h2 > 0) sum_c g_z3[s][c] W3[c][o], in place over h2
    for (int e = tid; e < kTile * kHid; e += blockDim.x) {
      const int r = e >> 7, o = e & 127;
      const float4 g = ld4(GZ3 + 4 * r);
      float* p = GS + r * kP128 + o;
      const float gs = g.x * __ldg(params + kOffW3 + o) + g.y * __ldg(params + kOffW3 + kHid + o) +
                       g.z * __ldg(params + kOffW3 + 2 * kHid + o);
      *p = *p > 0.0f ? gs : 0.0f;
    }
    __syncthreads();
    // dW2[o][i] += sum_s g_z2[s][o] h1[s][i]; db2[o] += sum_s g_z2[s][o]
    // this thread: o in {4ty.., 64+4ty..}, i in {4tx.., 64+4tx..}
#pragma unroll 2
    for (int r = 0; r < kTile; ++r) {
      const float4 g0 = ld4(GS + r * kP128 + 4 * ty), g1 = ld4(GS + r * kP128 + 64 + 4 * ty);
      const float4 h0 = ld4(H1S + r * kP128 + 4 * tx), h1 = ld4(H1S + r * kP128 + 64 + 4 * tx);
      const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
      const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        db2[a] += gv[a];
#pragma unroll
        for (int b = 0; b < 8; ++b) dW2[a][b] = fmaf(gv[a], hv[b], dW2[a][b]);
      }
    }
    // g_h1[s][i] = sum_o g_z2[s][o] W2[o][i]; rows ty + 16a, cols {4tx.., 64+4tx..}
    {
      float acc[8][8];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 1
      for (int o = 0; o < kHid; o += 4) {
        float4 av[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) av[a] = ld4(GS + (ty + 16 * a) * kP128 + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 b0 = ld4(W2S + (o + q) * kP128 + 4 * tx);
          const float4 b1 = ld4(W2S + (o + q) * kP128 + 64 + 4 * tx);
          const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            const float g = comp(av[a], q);
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(g, bv[b], acc[a][b]);
          }
        }
      }
      __syncthreads();  // dW2 finished reading h1
      // g_z1 = g_h1 * (h1 > 0), in place over h1
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float* row = H1S + (ty + 16 * a) * kP128;
        float4 h0 = ld4(row + 4 * tx), h1 = ld4(row + 64 + 4 * tx);
        h0 = make_float4(h0.x > 0.f ? acc[a][0] : 0.f, h0.y > 0.f ? acc[a][1] : 0.f,
                         h0.z > 0.f ? acc[a][2] : 0.f, h0.w > 0.f ? acc[a][3] : 0.f);
        h1 = make_float4(h1.x > 0.f ? acc[a][4] : 0.f, h1.y > 0.f ? acc[a][5] : 0.f,
                         h1.z > 0.f ? acc[a][6] : 0.f, h1.w > 0.f ? acc[a][7] : 0.f);
        st4(row + 4 * tx, h0);
        st4(row + 64 + 4 * tx, h1);
      }
    }
    __syncthreads();  // g_z2 no longer read
    build_x_tile(GS, k0, rays_d, ray_id, idx, j0, n);
    __syncthreads();
    // dW1[o][k] += sum_s g_z1[s][o] x[s][k]; o in {4ty.., 64+4ty..}, k in {tx, tx+16, tx+32}
#pragma unroll 2
    for (int r = 0; r < kTile; ++r) {
      const float4 g0 = ld4(H1S + r * kP128 + 4 * ty), g1 = ld4(H1S + r * kP128 + 64 + 4 * ty);
      const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
      float xv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) xv[c] = (tx + 16 * c < kInP) ? GS[r * kP40 + tx + 16 * c] : 0.0f;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) dW1[a][c] = fmaf(gv[a], xv[c], dW1[a][c]);
    }
    // g_k0[s][k] = sum_o g_z1[s][o] W1[o][k], k < 12: rows ty + 16a, k = tx
    if (tx < kFeat) {
      float gk[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) gk[a] = 0.0f;
#pragma unroll 2
      for (int o = 0; o < kHid; o += 4) {
        const float w0 = W1S[o * kP40 + tx], w1 = W1S[(o + 1) * kP40 + tx];
        const float w2 = W1S[(o + 2) * kP40 + tx], w3v = W1S[(o + 3) * kP40 + tx];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const float4 g = ld4(H1S + (ty + 16 * a) * kP128 + o);
          gk[a] = fmaf(g.x, w0, fmaf(g.y, w1, fmaf(g.z, w2, fmaf(g.w, w3v, gk[a]))));
        }
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t j = j0 + ty + 16 * a;
        if (j < n) {
          const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
          g_k0[s * kFeat + tx] = gk[a];
        }
      }
    }
  }
  // flush partials
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int o = (a < 4 ? 4 * ty + a : 64 + 4 * ty + (a - 4));
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = (b < 4 ? 4 * tx + b : 64 + 4 * tx + (b - 4));
      atomicAdd(g_params + kOffW2 + o * kHid + i, dW2[a][b]);
    }
    if (tx == 0) atomicAdd(g_params + kOffB2 + o, db2[a]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int k = tx + 16 * c;
      if (k < kIn) atomicAdd(g_params + kOffW1 + o * kIn + k, dW1[a][c]);
      else if (k == kIn) atomicAdd(g_params + kOffB1 + o, dW1[a][c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) atomicAdd(g_params + kOffW3 + c * kHid + o3, w3o[c]);
  if (tid == 0)
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(g_params + kOffB3 + c, db3[c]);
}

}  // namespace dvgo

using namespace dvgo;

int dvgo_rgbnet_fwd_f32(const float* k0, const float* rays_d, const int32_t* ray_id,
                        const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                        const float* params, float* rgb, float* act, cudaStream_t st) {
  const size_t smem = sizeof(float) * (2 * kHid * kP40 + 2 * kHid * kP128);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_fwd_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  rgbnet_fwd_f32_kernel<<<grid, 256, smem, st>>>(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb,
                                                 act);
  return launch_status();
}

int dvgo_rgbnet_bwd_f32(const float* g_rgb, const float* g_color, const float* w, const float* k0,
                        const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                        int64_t n_cap, const int64_t* n_dev, const float* params,
                        const float* act, const float* rgb, float* g_params, float* g_k0,
                        cudaStream_t st) {
  const size_t smem = sizeof(float) * (3 * kHid * kP128 + kHid * kP40 + 4 * kTile);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_bwd_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  rgbnet_bwd_f32_kernel<<<grid, 256, smem, st>>>(g_rgb, g_color, w, k0, rays_d, ray_id, idx, n_cap,
                                                 n_dev, params, act, rgb, g_params, g_k0);
  return launch_status();
}
