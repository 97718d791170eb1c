// Colour MLP (rgbnet, the shallow decoder of the hybrid representation of
// Tab. 1) in exact FP32 on the CUDA cores: 39 -> ReLU 128 -> ReLU 128 ->
// sigmoid 3.  Fused per tile of 128 samples: input encoding, both hidden
// layers, the output layer and (backward) every weight gradient.  Persistent
// CTAs keep their share of the weight gradients in registers across tiles and
// flush them once with atomics.
//
// Thread layout (256 threads): ty = tid / 16, tx = tid % 16; a thread owns
// rows ty + 16a and columns tx + 16b (a, b < 8) of every 128 x 128 tile, so
// row operands are warp broadcasts and column operands hit 16 distinct banks
// (row pitches are odd).
#include "common.cuh"
#include "mlp_common.cuh"

namespace dvgo {

constexpr int kP = 41;    // pitch of 40-wide rows
constexpr int kPH = 129;  // pitch of 128-wide rows

__device__ __forceinline__ void load_weights_f32(const float* __restrict__ params, float* W1S,
                                                 float* W2S) {
  for (int e = threadIdx.x; e < kHid * kInP; e += blockDim.x) {
    const int o = e / kInP, k = e % kInP;
    W1S[o * kP + k] = k < kIn ? params[kOffW1 + o * kIn + k] : params[kOffB1 + o];
  }
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int o = e / kHid, i = e % kHid;
    W2S[o * kPH + i] = params[kOffW2 + e];
  }
}

// acc[a][b] = sum_k A[(ty+16a)*lda + k] * B[(tx+16b)*ldb + k]
template <int K>
__device__ __forceinline__ void tile_gemm_nt(const float* A, int lda, const float* B, int ldb,
                                             int ty, int tx, float acc[8][8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float av[8], bv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) av[a] = A[(ty + 16 * a) * lda + k];
#pragma unroll
    for (int b = 0; b < 8; ++b) bv[b] = B[(tx + 16 * b) * ldb + k];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
  }
}

// Layer 3 for the 8 rows of this thread: z3[a][c] = b3[c] + sum_o W3[c][o] h2[a][o],
// reduced over the 16 threads that share ty.
__device__ __forceinline__ void layer3(const float h2[8][8], const float* __restrict__ params,
                                       int tx, float z3[8][3]) {
  float w3[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 8; ++b) w3[c][b] = __ldg(params + kOffW3 + c * kHid + tx + 16 * b);
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.0f;
#pragma unroll
      for (int b = 0; b < 8; ++b) s = fmaf(w3[c][b], h2[a][b], s);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      z3[a][c] = s + __ldg(params + kOffB3 + c);
    }
}

__global__ void __launch_bounds__(256, 1) rgbnet_fwd_f32_kernel(
    const float* __restrict__ k0, const float* __restrict__ rays_d,
    const int32_t* __restrict__ ray_id, const int32_t* __restrict__ idx, int64_t n_cap,
    const int64_t* __restrict__ n_dev, const float* __restrict__ params, float* __restrict__ rgb) {
  extern __shared__ float smem[];
  float* W1S = smem;                   // [128][41]
  float* W2S = W1S + kHid * kP;        // [128][129]
  float* XS = W2S + kHid * kPH;        // [128][41]
  float* H1S = XS + kTile * kP;        // [128][129]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  load_weights_f32(params, W1S, W2S);
  float b1v[8], b2v[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) b2v[b] = __ldg(params + kOffB2 + tx + 16 * b);
  (void)b1v;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (tid < kTile) {
      const int64_t j = t * kTile + tid;
      float row[kInP];
      encode_row(k0, rays_d, ray_id, idx, j, n, row);
#pragma unroll
      for (int k = 0; k < kInP; ++k) XS[tid * kP + k] = row[k];
    }
    __syncthreads();
    float acc[8][8];
    tile_gemm_nt<kInP>(XS, kP, W1S, kP, ty, tx, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) H1S[(ty + 16 * a) * kPH + tx + 16 * b] = fmaxf(acc[a][b], 0.0f);
    __syncthreads();
    tile_gemm_nt<kHid>(H1S, kPH, W2S, kPH, ty, tx, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaxf(acc[a][b] + b2v[b], 0.0f);
    float z3[8][3];
    layer3(acc, params, tx, z3);
    if (tx == 0) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t j = t * kTile + ty + 16 * a;
        if (j < n) {
          const int64_t s = idx ? (int64_t)idx[j] : j;
#pragma unroll
          for (int c = 0; c < 3; ++c) rgb[3 * s + c] = sigmoid_f(z3[a][c]);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256, 1) rgbnet_bwd_f32_kernel(
    const float* __restrict__ g_rgb, const float* __restrict__ g_color, const float* __restrict__ w,
    const float* __restrict__ k0,
    const float* __restrict__ rays_d, const int32_t* __restrict__ ray_id,
    const int32_t* __restrict__ idx, int64_t n_cap, const int64_t* __restrict__ n_dev,
    const float* __restrict__ params, float* __restrict__ g_params, float* __restrict__ g_k0) {
  extern __shared__ float smem[];
  float* W1S = smem;                   // [128][41]
  float* W2S = W1S + kHid * kP;        // [128][129]
  float* H1S = W2S + kHid * kPH;       // [128][129]  H1, later g_z1
  float* GS = H1S + kTile * kPH;       // [128][129]  X (pitch 41) then g_z2, then X again
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  load_weights_f32(params, W1S, W2S);
  float b2v[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) b2v[b] = __ldg(params + kOffB2 + tx + 16 * b);
  // persistent gradient partials
  float dW2[8][8], dW1[8][3], db2[8], dW3[3][8], db3[3];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
#pragma unroll
    for (int b = 0; b < 8; ++b) dW2[a][b] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) dW1[a][c] = 0.0f;
    db2[a] = 0.0f;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    db3[c] = 0.0f;
#pragma unroll
    for (int b = 0; b < 8; ++b) dW3[c][b] = 0.0f;
  }
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (tid < kTile) {
      float row[kInP];
      encode_row(k0, rays_d, ray_id, idx, t * kTile + tid, n, row);
#pragma unroll
      for (int k = 0; k < kInP; ++k) GS[tid * kP + k] = row[k];
    }
    __syncthreads();
    float acc[8][8];
    tile_gemm_nt<kInP>(GS, kP, W1S, kP, ty, tx, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) H1S[(ty + 16 * a) * kPH + tx + 16 * b] = fmaxf(acc[a][b], 0.0f);
    __syncthreads();
    tile_gemm_nt<kHid>(H1S, kPH, W2S, kPH, ty, tx, acc);  // z2 - b2
    float h2[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        acc[a][b] += b2v[b];
        h2[a][b] = fmaxf(acc[a][b], 0.0f);
      }
    float z3[8][3];
    layer3(h2, params, tx, z3);
    // g_z3 = w * g_color * y (1 - y)
    float gz3[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t j = t * kTile + ty + 16 * a;
      float gr[3] = {0.0f, 0.0f, 0.0f};
      if (j < n) upstream_rgb_grad(g_rgb, g_color, w, ray_id, idx ? (int64_t)__ldg(idx + j) : j, gr);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float y = sigmoid_f(z3[a][c]);
        gz3[a][c] = gr[c] * y * (1.0f - y);
      }
    }
    // g_z2, dW3, db2, db3
    float w3[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 8; ++b) w3[c][b] = __ldg(params + kOffW3 + c * kHid + tx + 16 * b);
    __syncthreads();  // GS (X) no longer read
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float g = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          g = fmaf(gz3[a][c], w3[c][b], g);
          dW3[c][b] = fmaf(gz3[a][c], h2[a][b], dW3[c][b]);
        }
        g = acc[a][b] > 0.0f ? g : 0.0f;
        db2[b] += g;
        GS[(ty + 16 * a) * kPH + tx + 16 * b] = g;
      }
    if (tx == 0)
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) db3[c] += gz3[a][c];
    __syncthreads();
    // dW2[o][i] += sum_s g_z2[s][o] h1[s][i]; this thread: o = ty + 16a, i = tx + 16b
#pragma unroll 2
    for (int s = 0; s < kTile; ++s) {
      float gv[8], hv[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) gv[a] = GS[s * kPH + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 8; ++b) hv[b] = H1S[s * kPH + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) dW2[a][b] = fmaf(gv[a], hv[b], dW2[a][b]);
    }
    __syncthreads();
    // g_h1[s][i] = sum_o g_z2[s][o] W2[o][i]; g_z1 = g_h1 * (h1 > 0), written over H1S
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 2
    for (int o = 0; o < kHid; ++o) {
      float gv[8], wv[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) gv[a] = GS[(ty + 16 * a) * kPH + o];
#pragma unroll
      for (int b = 0; b < 8; ++b) wv[b] = W2S[o * kPH + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(gv[a], wv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float* hp = H1S + (ty + 16 * a) * kPH + tx + 16 * b;
        *hp = *hp > 0.0f ? acc[a][b] : 0.0f;
      }
    __syncthreads();
    // rebuild X (pitch 41) in GS
    if (tid < kTile) {
      float row[kInP];
      encode_row(k0, rays_d, ray_id, idx, t * kTile + tid, n, row);
#pragma unroll
      for (int k = 0; k < kInP; ++k) GS[tid * kP + k] = row[k];
    }
    __syncthreads();
    // dW1[o][k] += sum_s g_z1[s][o] X[s][k]; o = ty + 16a, k = tx + 16c (k < 40)
#pragma unroll 2
    for (int s = 0; s < kTile; ++s) {
      float gv[8], xv[3];
#pragma unroll
      for (int a = 0; a < 8; ++a) gv[a] = H1S[s * kPH + ty + 16 * a];
#pragma unroll
      for (int c = 0; c < 3; ++c) xv[c] = (tx + 16 * c < kInP) ? GS[s * kP + tx + 16 * c] : 0.0f;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) dW1[a][c] = fmaf(gv[a], xv[c], dW1[a][c]);
    }
    // g_k0[s][k] = sum_o g_z1[s][o] W1[o][k], k < 12; s = ty + 16a, k = tx
    if (tx < kFeat) {
      float gk[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) gk[a] = 0.0f;
#pragma unroll 4
      for (int o = 0; o < kHid; ++o) {
        const float wv = W1S[o * kP + tx];
#pragma unroll
        for (int a = 0; a < 8; ++a) gk[a] = fmaf(H1S[(ty + 16 * a) * kPH + o], wv, gk[a]);
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t j = t * kTile + ty + 16 * a;
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
    const int o = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 8; ++b) atomicAdd(g_params + kOffW2 + o * kHid + tx + 16 * b, dW2[a][b]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int k = tx + 16 * c;
      if (k < kIn) atomicAdd(g_params + kOffW1 + o * kIn + k, dW1[a][c]);
      else if (k == kIn) atomicAdd(g_params + kOffB1 + o, dW1[a][c]);
    }
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int o = tx + 16 * b;
    atomicAdd(g_params + kOffB2 + o, db2[b]);
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(g_params + kOffW3 + c * kHid + o, dW3[c][b]);
  }
  if (tx == 0)
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(g_params + kOffB3 + c, db3[c]);
}

}  // namespace dvgo

using namespace dvgo;

int dvgo_rgbnet_fwd_f32(const float* k0, const float* rays_d, const int32_t* ray_id,
                        const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                        const float* params, float* rgb, cudaStream_t st) {
  const size_t smem = sizeof(float) * (2 * kHid * kP + 2 * kHid * kPH);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_fwd_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  rgbnet_fwd_f32_kernel<<<grid, 256, smem, st>>>(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb);
  return launch_status();
}

int dvgo_rgbnet_bwd_f32(const float* g_rgb, const float* g_color, const float* w, const float* k0,
                        const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                        int64_t n_cap, const int64_t* n_dev, const float* params,
                        float* g_params, float* g_k0, cudaStream_t st) {
  const size_t smem = sizeof(float) * (kHid * kP + 3 * kHid * kPH);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_bwd_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  rgbnet_bwd_f32_kernel<<<grid, 256, smem, st>>>(g_rgb, g_color, w, k0, rays_d, ray_id, idx, n_cap, n_dev,
                                                 params, g_params, g_k0);
  return launch_status();
}
