// Colour MLP (rgbnet) in BF16 on the 5th-generation tensor cores (tcgen05),
// FP32 accumulation in tensor memory.  One 128-sample tile per step of a
// persistent CTA of 128 threads (thread = tile row = TMEM lane).
//
// Forward, per tile:  X[128x48] (12 features, 27 view-encoding values, a 1
// carrying b1, zero pad) -> D1 = X W1^T (TMEM) -> H1 = relu(D1) (bf16, smem)
// -> D2 = H1 W2^T (TMEM) -> z2 = D2 + b2 -> layer 3 (3 outputs) on the CUDA
// cores in FP32 -> sigmoid.
// Backward, per tile (forward recomputed): g_z3 -> g_z2 (CUDA cores) ->
//   dW2 += g_z2^T [H1 | 1]      (TMEM, kept for the whole kernel; the ones
//                                column yields db2)
//   g_h1 = g_z2 W2, g_z1 = g_h1 * (H1 > 0)
//   dW1 += g_z1^T X             (TMEM, whole kernel; the X bias column
//                                yields db1)
//   g_X  = g_z1 W1[:, 0:16]     -> g_k0 (the 12 feature columns)
// dW3/db3 are reduced across each warp with a butterfly reduce-scatter.
// The same shared-memory bytes serve as K-major operand in one product and
// as MN-major operand in another (no transposed copies).
#include "common.cuh"
#include "mlp_common.cuh"
#include "tcgen05.cuh"

namespace dvgo {

__device__ int g_mlp_status;  // DVGO_ERR_TIMEOUT if a bounded wait gave up

namespace bf {

constexpr int kK1 = 48;                       // padded input width
constexpr uint32_t kSboX = (kK1 / 8) * 128;   // 768: 8-row group stride of 48-wide rows
constexpr uint32_t kSboH = (kHid / 8) * 128;  // 2048: of 128-wide rows
constexpr int kH1W = 144;                     // H1 width in the backward (+1 column, +pad)
constexpr uint32_t kSboH1b = (kH1W / 8) * 128;  // 2304

constexpr uint32_t kOffW1s = 0;
constexpr uint32_t kOffW2s = kOffW1s + kHid * kK1 * 2;      // 12288
constexpr uint32_t kOffXs = kOffW2s + kHid * kHid * 2;      // 45056
constexpr uint32_t kOffH1s = kOffXs + kTile * kK1 * 2;      // 57344
constexpr uint32_t kFwdOperandBytes = kOffH1s + kTile * kHid * 2;      // 90112
constexpr uint32_t kOffG2s = kOffH1s + kTile * kH1W * 2;    // 94208
constexpr uint32_t kBwdOperandBytes = kOffG2s + kTile * kHid * 2;      // 126976
// The backward reserves shared memory past its operands so that an MN-major
// descriptor read with its two strides exchanged (16 MN groups x 2048 B from
// the last K step of G2) would still stay inside the CTA's allocation.
constexpr uint32_t kBwdSmemBytes = 160 * 1024;

struct F32Side {  // epilogue constants (BF16-rounded values, kept in FP32)
  float W3[kOut * kHid];
  float b2[kHid];
  float b3[4];
  uint64_t bar;
  uint32_t tmem_slot;
};

constexpr uint32_t kSpin = 1u << 24;

__device__ __forceinline__ float bfr(float x) { return bf16_bits_to_f32(f32_to_bf16_bits(x)); }

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float x) {
  *reinterpret_cast<uint16_t*>(base + off) = f32_to_bf16_bits(x);
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  return (uint32_t)f32_to_bf16_bits(a) | ((uint32_t)f32_to_bf16_bits(b) << 16);
}

// Store 8 consecutive values (one 16-byte core-matrix row) of row `row`.
__device__ __forceinline__ void st_row8(uint8_t* base, int row, int k8, uint32_t sbo, const float* v) {
  uint4 q;
  q.x = pack2(v[0], v[1]);
  q.y = pack2(v[2], v[3]);
  q.z = pack2(v[4], v[5]);
  q.w = pack2(v[6], v[7]);
  *reinterpret_cast<uint4*>(base + tc::cm_off(row, k8, sbo)) = q;
}

__device__ __forceinline__ void ld_row8(const uint8_t* base, int row, int k8, uint32_t sbo, float* v) {
  uint4 q = *reinterpret_cast<const uint4*>(base + tc::cm_off(row, k8, sbo));
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// Weights into shared memory: W1 (+b1 column) and W2 as BF16 core matrices,
// W3/b2/b3 as BF16-rounded FP32.
__device__ void load_weights(const float* __restrict__ params, uint8_t* sm, F32Side* fs) {
  for (int e = threadIdx.x; e < kHid * kK1; e += blockDim.x) {
    const int o = e / kK1, k = e % kK1;
    float v = k < kIn ? params[kOffW1 + o * kIn + k] : (k == kIn ? params[kOffB1 + o] : 0.0f);
    st_bf16(sm + kOffW1s, tc::cm_off(o, k, kSboX), v);
  }
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int o = e / kHid, i = e % kHid;
    st_bf16(sm + kOffW2s, tc::cm_off(o, i, kSboH), params[kOffW2 + e]);
  }
  for (int e = threadIdx.x; e < kOut * kHid; e += blockDim.x) fs->W3[e] = bfr(params[kOffW3 + e]);
  for (int e = threadIdx.x; e < kHid; e += blockDim.x) fs->b2[e] = bfr(params[kOffB2 + e]);
  if (threadIdx.x < 4) fs->b3[threadIdx.x] = threadIdx.x < kOut ? bfr(params[kOffB3 + threadIdx.x]) : 0.0f;
}

__device__ __forceinline__ void write_x_row(uint8_t* sm, int row, const float x[kInP]) {
  float v[8];
#pragma unroll
  for (int kb = 0; kb < kK1 / 8; ++kb) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kb * 8 + i;
      v[i] = k < kInP ? x[k] : 0.0f;
    }
    st_row8(sm + kOffXs, row, kb * 8, kSboX, v);
  }
}

// Layer 1 / layer 2 MMAs (K-major A and B), issued by one thread.
__device__ __forceinline__ void issue_layer1(uint8_t* sm, uint32_t tmem_d) {
  const uint32_t xs = tc::smem_u32(sm + kOffXs), w1 = tc::smem_u32(sm + kOffW1s);
  const uint32_t id = tc::idesc_bf16(128, 128, 0, 0);
#pragma unroll
  for (int j = 0; j < kK1 / 16; ++j)
    tc::mma_bf16(tmem_d, tc::smem_desc(xs + 256 * j, 128, kSboX), tc::smem_desc(w1 + 256 * j, 128, kSboX),
                 id, j > 0);
}

__device__ __forceinline__ void issue_layer2(uint8_t* sm, uint32_t tmem_d, uint32_t sbo_h1) {
  const uint32_t h1 = tc::smem_u32(sm + kOffH1s), w2 = tc::smem_u32(sm + kOffW2s);
  const uint32_t id = tc::idesc_bf16(128, 128, 0, 0);
#pragma unroll
  for (int j = 0; j < kHid / 16; ++j)
    tc::mma_bf16(tmem_d, tc::smem_desc(h1 + 256 * j, 128, sbo_h1), tc::smem_desc(w2 + 256 * j, 128, kSboH),
                 id, j > 0);
}

// D1 (TMEM cols [0,128)) -> relu -> bf16 H1 row
__device__ __forceinline__ void epilogue_h1(uint8_t* sm, uint32_t taddr_row, int row, uint32_t sbo_h1) {
#pragma unroll 1
  for (int ch = 0; ch < 4; ++ch) {
    float v[32];
    tc::tmem_ld32(taddr_row + ch * 32, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) st_row8(sm + kOffH1s, row, ch * 32 + q * 8, sbo_h1, v + 8 * q);
  }
}

// z3 = b3 + W3 relu(D2 + b2)
__device__ __forceinline__ void layer3_z(const F32Side* fs, uint32_t taddr_d2, float z3[3]) {
  z3[0] = fs->b3[0];
  z3[1] = fs->b3[1];
  z3[2] = fs->b3[2];
#pragma unroll 1
  for (int ch = 0; ch < 4; ++ch) {
    float v[32];
    tc::tmem_ld32(taddr_d2 + ch * 32, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int o = ch * 32 + i;
      const float h = fmaxf(v[i] + fs->b2[o], 0.0f);
      z3[0] = fmaf(fs->W3[o], h, z3[0]);
      z3[1] = fmaf(fs->W3[kHid + o], h, z3[1]);
      z3[2] = fmaf(fs->W3[2 * kHid + o], h, z3[2]);
    }
  }
}

// Butterfly reduce-scatter: lane l returns sum over the warp of v[l].
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

}  // namespace bf

using namespace bf;

__global__ void __launch_bounds__(128, 1) rgbnet_fwd_bf16_kernel(
    const float* __restrict__ k0, const float* __restrict__ rays_d,
    const int32_t* __restrict__ ray_id, const int32_t* __restrict__ idx, int64_t n_cap,
    const int64_t* __restrict__ n_dev, const float* __restrict__ params, float* __restrict__ rgb) {
  extern __shared__ __align__(1024) uint8_t sm[];
  F32Side* fs = reinterpret_cast<F32Side*>(sm + kFwdOperandBytes);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (warp == 0) tc::tmem_alloc(&fs->tmem_slot, 256);
  if (tid == 0) tc::mbar_init(&fs->bar, 1);
  load_weights(params, sm, fs);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int64_t j = t * kTile + tid;
    {
      float x[kInP];
      encode_row(k0, rays_d, ray_id, idx, j, n, x);
      write_x_row(sm, tid, x);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_layer1(sm, tmem);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    epilogue_h1(sm, lane_base, tid, kSboH);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_layer2(sm, tmem + 128, kSboH);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    float z3[3];
    layer3_z(fs, lane_base + 128, z3);
    if (j < n) {
      const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
      rgb[3 * s] = sigmoid_f(z3[0]);
      rgb[3 * s + 1] = sigmoid_f(z3[1]);
      rgb[3 * s + 2] = sigmoid_f(z3[2]);
    }
    tc::fence_before_sync();
  }
  if (!ok && tid == 0) atomicExch(&g_mlp_status, (int)DVGO_ERR_TIMEOUT);
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

__global__ void __launch_bounds__(128, 1) rgbnet_bwd_bf16_kernel(
    const float* __restrict__ g_rgb, const float* __restrict__ g_color, const float* __restrict__ w,
    const float* __restrict__ k0,
    const float* __restrict__ rays_d, const int32_t* __restrict__ ray_id,
    const int32_t* __restrict__ idx, int64_t n_cap, const int64_t* __restrict__ n_dev,
    const float* __restrict__ params, float* __restrict__ g_params, float* __restrict__ g_k0) {
  extern __shared__ __align__(1024) uint8_t sm[];
  F32Side* fs = reinterpret_cast<F32Side*>(sm + kBwdOperandBytes);
  static_assert(kBwdOperandBytes + sizeof(F32Side) <= kBwdSmemBytes, "smem");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (warp == 0) tc::tmem_alloc(&fs->tmem_slot, 512);
  if (tid == 0) tc::mbar_init(&fs->bar, 1);
  load_weights(params, sm, fs);
  {  // constant columns of [H1 | 1 | 0...]: column 128 = 1
    float v[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    st_row8(sm + kOffH1s, tid, 128, kSboH1b, v);
    st_row8(sm + kOffH1s, tid, 136, kSboH1b, z);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  // TMEM columns: [0,128) D1 / g_h1, [128,256) D2 / g_X, [256,400) dW2|db2, [400,448) dW1|db1
  constexpr uint32_t cD1 = 0, cD2 = 128, cDW2 = 256, cDW1 = 400;
  const uint32_t sm_x = tc::smem_u32(sm + kOffXs), sm_w1 = tc::smem_u32(sm + kOffW1s);
  const uint32_t sm_w2 = tc::smem_u32(sm + kOffW2s), sm_h1 = tc::smem_u32(sm + kOffH1s);
  const uint32_t sm_g = tc::smem_u32(sm + kOffG2s);
  float dW3acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) dW3acc[i] = 0.0f;
  float db3acc[3] = {0.f, 0.f, 0.f};
  uint32_t phase = 0;
  bool ok = true;
  int it = 0;
  for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
    const int64_t j = t * kTile + tid;
    const bool valid = j < n;
    int64_t s = 0;
    float grgb[3] = {0.f, 0.f, 0.f};
    if (valid) {
      s = idx ? (int64_t)__ldg(idx + j) : j;
      upstream_rgb_grad(g_rgb, g_color, w, ray_id, s, grgb);
    }
    {
      float x[kInP];
      encode_row(k0, rays_d, ray_id, idx, j, n, x);
      write_x_row(sm, tid, x);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_layer1(sm, tmem + cD1);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    epilogue_h1(sm, lane_base + cD1, tid, kSboH1b);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_layer2(sm, tmem + cD2, kSboH1b);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    // ---- epilogue 2: g_z3, g_z2, dW3
    float z3[3];
    layer3_z(fs, lane_base + cD2, z3);
    float gz3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float y = sigmoid_f(z3[c]);
      gz3[c] = grgb[c] * y * (1.0f - y);
      db3acc[c] += gz3[c];
    }
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32], g[32];
      tc::tmem_ld32(lane_base + cD2 + ch * 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int o = ch * 32 + i;
        const float z2 = v[i] + fs->b2[o];
        const float gs = gz3[0] * fs->W3[o] + gz3[1] * fs->W3[kHid + o] + gz3[2] * fs->W3[2 * kHid + o];
        g[i] = z2 > 0.0f ? gs : 0.0f;
        v[i] = fmaxf(z2, 0.0f);  // h2
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) st_row8(sm + kOffG2s, tid, ch * 32 + q * 8, kSboH, g + 8 * q);
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        float p[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) p[i] = gz3[c] * v[i];
        dW3acc[c * 4 + ch] += reduce_scatter32(p, lane);
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      // dW2|db2 (+)= G2^T [H1 | 1]: M = o, N = 144, K = s; both operands MN-major
      const uint32_t id_dw2 = tc::idesc_bf16(128, kH1W, 1, 1);
#pragma unroll
      for (int k = 0; k < kTile / 16; ++k)
        tc::mma_bf16(tmem + cDW2, tc::smem_desc_mn(sm_g + k * 2 * kSboH, kSboH, 128),
                     tc::smem_desc_mn(sm_h1 + k * 2 * kSboH1b, kSboH1b, 128), id_dw2,
                     (it > 0 || k > 0) ? 1u : 0u);
      // g_h1 = G2 W2: M = s, N = i, K = o; A K-major, B (W2 stored [o][i]) MN-major
      const uint32_t id_gh = tc::idesc_bf16(128, 128, 0, 1);
#pragma unroll
      for (int k = 0; k < kHid / 16; ++k)
        tc::mma_bf16(tmem + cD1, tc::smem_desc(sm_g + k * 256, 128, kSboH),
                     tc::smem_desc_mn(sm_w2 + k * 2 * kSboH, kSboH, 128), id_gh, k > 0);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    // ---- epilogue 3: g_z1 = g_h1 * (H1 > 0), written over G2
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tc::tmem_ld32(lane_base + cD1 + ch * 32, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float h[8];
        ld_row8(sm + kOffH1s, tid, ch * 32 + q * 8, kSboH1b, h);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[8 * q + i] = h[i] > 0.0f ? v[8 * q + i] : 0.0f;
        st_row8(sm + kOffG2s, tid, ch * 32 + q * 8, kSboH, v + 8 * q);
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      // dW1|db1 (+)= G1^T X: M = o, N = 48, K = s; both MN-major
      const uint32_t id_dw1 = tc::idesc_bf16(128, kK1, 1, 1);
#pragma unroll
      for (int k = 0; k < kTile / 16; ++k)
        tc::mma_bf16(tmem + cDW1, tc::smem_desc_mn(sm_g + k * 2 * kSboH, kSboH, 128),
                     tc::smem_desc_mn(sm_x + k * 2 * kSboX, kSboX, 128), id_dw1,
                     (it > 0 || k > 0) ? 1u : 0u);
      // g_X[:, 0:16] = G1 W1: M = s, N = 16, K = o; A K-major, B (W1 stored [o][in]) MN-major
      const uint32_t id_gx = tc::idesc_bf16(128, 16, 0, 1);
#pragma unroll
      for (int k = 0; k < kHid / 16; ++k)
        tc::mma_bf16(tmem + cD2, tc::smem_desc(sm_g + k * 256, 128, kSboH),
                     tc::smem_desc_mn(sm_w1 + k * 2 * kSboX, kSboX, 128), id_gx, k > 0);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    {
      float gx[16];
      tc::tmem_ld16(lane_base + cD2, gx);
      if (valid) {
        float4* dst = reinterpret_cast<float4*>(g_k0 + s * kFeat);
        dst[0] = make_float4(gx[0], gx[1], gx[2], gx[3]);
        dst[1] = make_float4(gx[4], gx[5], gx[6], gx[7]);
        dst[2] = make_float4(gx[8], gx[9], gx[10], gx[11]);
      }
    }
    tc::fence_before_sync();
  }
  __syncthreads();
  tc::fence_after_sync();
  if (ok && it > 0) {
    // lane = output neuron o
    const int o = tid;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tc::tmem_ld32(lane_base + cDW2 + ch * 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) atomicAdd(g_params + kOffW2 + o * kHid + ch * 32 + i, v[i]);
    }
    {
      float v[16];
      tc::tmem_ld16(lane_base + cDW2 + 128, v);
      atomicAdd(g_params + kOffB2 + o, v[0]);
    }
    {
      float v[32], u[16];
      tc::tmem_ld32(lane_base + cDW1, v);
      tc::tmem_ld16(lane_base + cDW1 + 32, u);
#pragma unroll
      for (int k = 0; k < 32; ++k) atomicAdd(g_params + kOffW1 + o * kIn + k, v[k]);
#pragma unroll
      for (int k = 32; k < kIn; ++k) atomicAdd(g_params + kOffW1 + o * kIn + k, u[k - 32]);
      atomicAdd(g_params + kOffB1 + o, u[kIn - 32]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ch = 0; ch < 4; ++ch)
        atomicAdd(g_params + kOffW3 + c * kHid + ch * 32 + lane, dW3acc[c * 4 + ch]);
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(g_params + kOffB3 + c, db3acc[c]);
  }
  if (!ok && tid == 0) atomicExch(&g_mlp_status, (int)DVGO_ERR_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace dvgo

using namespace dvgo;

int dvgo_rgbnet_fwd_bf16(const float* k0, const float* rays_d, const int32_t* ray_id,
                         const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                         const float* params, float* rgb, cudaStream_t st) {
  const size_t smem = kFwdOperandBytes + sizeof(F32Side);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_fwd_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, 2 * kNumSMs);
  if (grid < 1) return DVGO_OK;
  rgbnet_fwd_bf16_kernel<<<grid, 128, smem, st>>>(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb);
  return launch_status();
}

int dvgo_rgbnet_bwd_bf16(const float* g_rgb, const float* g_color, const float* w, const float* k0,
                         const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                         int64_t n_cap, const int64_t* n_dev, const float* params,
                         float* g_params, float* g_k0, cudaStream_t st) {
  const size_t smem = kBwdSmemBytes;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_bwd_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  rgbnet_bwd_bf16_kernel<<<grid, 128, smem, st>>>(g_rgb, g_color, w, k0, rays_d, ray_id, idx, n_cap, n_dev,
                                                  params, g_params, g_k0);
  return launch_status();
}

int dvgo_mlp_status_read_and_clear(cudaStream_t st) {
  int v = 0, zero = 0;
  cudaMemcpyFromSymbolAsync(&v, g_mlp_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  cudaMemcpyToSymbolAsync(g_mlp_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return v;
}
