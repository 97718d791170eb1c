// Learned-proposal network (not part of the paper): position encoding
// [x, sin(2^f x_a), cos(2^f x_a)], f < 6 (39 values) -> ReLU 64 -> ReLU 64 ->
// 1 logit, on the 5th-generation tensor cores (tcgen05, FP32 accumulation in
// tensor memory).  One 128-sample tile per step of a persistent CTA
// (thread = tile row = TMEM lane).
//
// BF16 form.  The parameters are the stored BF16 values (W1, b1, W2 are one
// BF16 term each; W3, b2, b3 are BF16-rounded and used in FP32 on the CUDA
// cores).  Every other MMA operand -- the encoded inputs X, the hidden
// activations H1, the gradient rows G -- is kept as two BF16 terms, hi =
// bf16(v) and lo = bf16(v - hi) (16 significant bits between them), so no
// value is rounded to BF16 between layers: a product with a weight matrix is
// hi W + lo W (two MMAs), a weight gradient G^T A is Gh^T Ah + Gh^T Al +
// Gl^T Ah (three; the dropped lo*lo term is 2^-16 of the product).
//
// Forward, per tile:  X [128 x 48] (39 inputs, a 1 carrying b1, zero pad) ->
//   D1 = X W1^T -> H1 = relu(D1) -> D2 = H1 W2^T -> z = b3 + W3 relu(D2 + b2)
//   (output layer on the CUDA cores).
// Backward, per tile (the forward is recomputed): g_z -> G2 = (W3^T g_z) *
//   (z2 > 0) -> dW2|db2 += G2^T [H1 | 1] (the ones column yields db2), g_h1 =
//   G2 W2 -> G1 = g_h1 * (H1 > 0) -> dW1|db1 += G1^T X (X's ones column
//   yields db1).  The weight-gradient accumulators stay in tensor memory for
//   the whole kernel.  One warp issues the MMAs, four warps run the
//   epilogues.  Every wait on an mbarrier is bounded (DVGO_ERR_TIMEOUT).
#include "common.cuh"
#include "mlp_common.cuh"
#include "tcgen05.cuh"

namespace dvgo {

__device__ int g_mlp_status;  // DVGO_ERR_TIMEOUT if a bounded wait gave up

namespace prop {

constexpr int kH = 64;                        // hidden width
constexpr int kPropFreq = 6;
constexpr int oW1 = 0, oB1 = kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kK1 = 48;                       // padded input width
constexpr int kH1W = kH + 16;                 // [H1 | 1 | 0..] in the backward
constexpr int kGW = 128;                      // gradient-tile width (zero past kH): M = 128 products
constexpr uint32_t kSboX = (kK1 / 8) * 128;   // 768
constexpr uint32_t kSboW2 = (kH / 8) * 128;   // 1024
constexpr uint32_t kSboH1f = (kH / 8) * 128;  // forward H1 rows (64 wide)
constexpr uint32_t kSboH1 = (kH1W / 8) * 128; // 1280
constexpr uint32_t kSboG = (kGW / 8) * 128;   // 2048
constexpr uint32_t kXBytes = kTile * kK1 * 2;
constexpr uint32_t kSpin = 1u << 24;

// forward shared memory
constexpr uint32_t fW1 = 0, fW2 = fW1 + kH * kK1 * 2, fXh = fW2 + kH * kH * 2, fXl = fXh + kXBytes,
                   fH1h = fXl + kXBytes, fH1l = fH1h + kTile * kH * 2, fEnd = fH1l + kTile * kH * 2;
// backward shared memory
constexpr uint32_t bW1 = 0, bW2 = bW1 + kH * kK1 * 2, bXh = bW2 + kH * kH * 2, bXl = bXh + kXBytes,
                   bH1h = bXl + kXBytes, bH1l = bH1h + kTile * kH1W * 2, bGh = bH1l + kTile * kH1W * 2,
                   bGl = bGh + kTile * kGW * 2, bEnd = bGl + kTile * kGW * 2;
// backward tensor-memory columns: D (D1, D2, g_h1 in turn), dW2|db2, dW1|db1
constexpr uint32_t cD = 0, cDW2 = 128, cDW1 = 256;

struct Side {
  float W3[kH];
  float b2[kH];
  float b3;
  uint64_t ready;   // backward: the epilogue warps' operands of the next stage are written
  uint64_t done;    // MMAs of the stage finished
  uint64_t fin;     // backward: every MMA of the kernel finished
  uint32_t tmem_slot;
  int error;
};
static_assert(fEnd + sizeof(Side) <= 227 * 1024, "forward shared memory");
static_assert(bEnd + sizeof(Side) <= 227 * 1024, "backward shared memory");

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t u32_of(__nv_bfloat162 v) { return *reinterpret_cast<const uint32_t*>(&v); }

// Eight values of row `row` from column k8 as hi / lo BF16 core-matrix rows.
__device__ __forceinline__ void st_split8(uint8_t* hi, uint8_t* lo, int row, int k8, uint32_t sbo,
                                          const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h2);
    h[i] = u32_of(h2);
    l[i] = u32_of(__floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y));
  }
  const uint32_t off = tc::cm_off(row, k8, sbo);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// One stored BF16 parameter.
__device__ __forceinline__ void st_w(uint8_t* base, uint32_t off, float x) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(x);
}

// W1 | b1 (column 39) | 0 and W2 as BF16 core matrices; W3, b2, b3 BF16-rounded.
__device__ void load_weights(const float* __restrict__ params, uint8_t* w1, uint8_t* w2, Side* fs) {
  for (int e = threadIdx.x; e < kH * kK1; e += blockDim.x) {
    const int o = e / kK1, k = e % kK1;
    const float v = k < kIn ? params[oW1 + o * kIn + k] : (k == kIn ? params[oB1 + o] : 0.0f);
    st_w(w1, tc::cm_off(o, k, kSboX), v);
  }
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x)
    st_w(w2, tc::cm_off(e / kH, e % kH, kSboW2), params[oW2 + e]);
  for (int e = threadIdx.x; e < kH; e += blockDim.x) {
    fs->W3[e] = bfr(params[oW3 + e]);
    fs->b2[e] = bfr(params[oB2 + e]);
  }
  if (threadIdx.x == 0) fs->b3 = bfr(params[oB3]);
}

// Input row of list position j: [x (3), sin(2^f x_a) (a major, f inner),
// cos(2^f x_a), 1, 0 ...]; rows past the list end are zero.
__device__ __forceinline__ void encode(const float* __restrict__ xyz, const int32_t* __restrict__ idx,
                                       int64_t j, int64_t n, float row[kK1]) {
#pragma unroll
  for (int k = 0; k < kK1; ++k) row[k] = 0.0f;
  if (j >= n) return;
  const int64_t s = idx ? (int64_t)__ldg(idx + j) : j;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float x = __ldg(xyz + 3 * s + a);
    row[a] = x;
#pragma unroll
    for (int f = 0; f < kPropFreq; ++f) {
      float sn, cs;
      sincosf(x * (float)(1 << f), &sn, &cs);
      row[3 + a * kPropFreq + f] = sn;
      row[3 + 3 * kPropFreq + a * kPropFreq + f] = cs;
    }
  }
  row[kIn] = 1.0f;
}

__device__ __forceinline__ void write_x(uint8_t* xh, uint8_t* xl, int row, const float (&x)[kK1]) {
#pragma unroll
  for (int kb = 0; kb < kK1 / 8; ++kb) st_split8(xh, xl, row, kb * 8, kSboX, x + 8 * kb);
}

// D = A W^T with A split (hi, lo) and W one term: two MMAs per K step of 16.
__device__ __forceinline__ void mma_split_w(uint32_t d, uint32_t ah, uint32_t al, uint32_t a_sbo, uint32_t w,
                                            uint32_t w_sbo, int ksteps, uint32_t idesc) {
#pragma unroll 1
  for (int j = 0; j < ksteps; ++j) {
    const uint64_t dw = tc::smem_desc(w + 256 * j, 128, w_sbo);
    tc::mma_bf16(d, tc::smem_desc(ah + 256 * j, 128, a_sbo), dw, idesc, j > 0 ? 1u : 0u);
    tc::mma_bf16(d, tc::smem_desc(al + 256 * j, 128, a_sbo), dw, idesc, 1u);
  }
}

__device__ __forceinline__ void named_bar1() { tc::named_sync(1, 128); }

}  // namespace prop

using namespace prop;

// 128 threads.  Per tile: X -> layer 1 -> H1 -> layer 2 -> output layer.
__global__ void __launch_bounds__(128, 1) prop_fwd_kernel(const float* __restrict__ xyz,
                                                          const int32_t* __restrict__ idx, int64_t n_cap,
                                                          const int64_t* __restrict__ n_dev,
                                                          const float* __restrict__ params,
                                                          float* __restrict__ out) {
  extern __shared__ __align__(1024) uint8_t sm[];
  Side* fs = reinterpret_cast<Side*>(sm + fEnd);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (warp == 0) tc::tmem_alloc(&fs->tmem_slot, 128);
  if (tid == 0) tc::mbar_init(&fs->done, 1);
  load_weights(params, sm + fW1, sm + fW2, fs);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t sW1 = tc::smem_u32(sm + fW1), sW2 = tc::smem_u32(sm + fW2);
  const uint32_t sXh = tc::smem_u32(sm + fXh), sXl = tc::smem_u32(sm + fXl);
  const uint32_t sHh = tc::smem_u32(sm + fH1h), sHl = tc::smem_u32(sm + fH1l);
  const uint32_t id = tc::idesc_bf16(128, kH, 0, 0);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int64_t j = t * kTile + tid;
    {
      float x[kK1];
      encode(xyz, idx, j, n, x);
      write_x(sm + fXh, sm + fXl, tid, x);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      mma_split_w(tmem, sXh, sXl, kSboX, sW1, kSboX, kK1 / 16, id);
      tc::mma_commit(&fs->done);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->done, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
#pragma unroll 1
    for (int ch = 0; ch < kH / 32; ++ch) {          // H1 = relu(D1), split
      float v[32];
      tc::tmem_ld32(lane_base + ch * 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.0f);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        st_split8(sm + fH1h, sm + fH1l, tid, ch * 32 + q * 8, kSboH1f, v + 8 * q);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      mma_split_w(tmem + kH, sHh, sHl, kSboH1f, sW2, kSboW2, kH / 16, id);
      tc::mma_commit(&fs->done);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->done, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    float z = fs->b3;
#pragma unroll 1
    for (int ch = 0; ch < kH / 32; ++ch) {
      float v[32];
      tc::tmem_ld32(lane_base + kH + ch * 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) z = fmaf(fs->W3[ch * 32 + i], fmaxf(v[i] + fs->b2[ch * 32 + i], 0.0f), z);
    }
    if (j < n) out[idx ? (int64_t)__ldg(idx + j) : j] = z;
    tc::fence_before_sync();
  }
  if (!ok && tid == 0) atomicExch(&g_mlp_status, (int)DVGO_ERR_TIMEOUT);
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// Backward, 160 threads: warps 0-3 run the epilogues (thread = tile row),
// warp 4 issues the MMAs of each stage once the epilogue warps signal that
// its operands are in shared memory, and commits them to `done`.
//   stage 0: D = X W1^T
//   stage 1: D = H1 W2^T
//   stage 2: dW2|db2 += G2^T [H1 | 1];  D = G2 W2
//   stage 3: dW1|db1 += G1^T X
// g_params += the CTA's sums (atomics at the end of the kernel).
__global__ void __launch_bounds__(160, 1) prop_bwd_kernel(const float* __restrict__ g_out,
                                                          const float* __restrict__ xyz,
                                                          const int32_t* __restrict__ idx, int64_t n_cap,
                                                          const int64_t* __restrict__ n_dev,
                                                          const float* __restrict__ params,
                                                          float* __restrict__ g_params) {
  extern __shared__ __align__(1024) uint8_t sm[];
  Side* fs = reinterpret_cast<Side*>(sm + bEnd);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (warp == 4) tc::tmem_alloc(&fs->tmem_slot, 512);
  if (tid == 0) {
    tc::mbar_init(&fs->ready, 1);
    tc::mbar_init(&fs->done, 1);
    tc::mbar_init(&fs->fin, 1);
    fs->error = 0;
  }
  load_weights(params, sm + bW1, sm + bW2, fs);
  if (tid < kTile) {  // constant columns: [H1 | 1 | 0..] and G past the hidden width
    const float one[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    st_split8(sm + bH1h, sm + bH1l, tid, kH, kSboH1, one);
    st_split8(sm + bH1h, sm + bH1l, tid, kH + 8, kSboH1, z);
    for (int k = kH; k < kGW; k += 8) st_split8(sm + bGh, sm + bGl, tid, k, kSboG, z);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  float dW3acc[kH / 32] = {0.0f, 0.0f};
  float db3acc = 0.0f;
  if (warp == 4) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t sW1 = tc::smem_u32(sm + bW1), sW2 = tc::smem_u32(sm + bW2);
      const uint32_t sXh = tc::smem_u32(sm + bXh), sXl = tc::smem_u32(sm + bXl);
      const uint32_t sHh = tc::smem_u32(sm + bH1h), sHl = tc::smem_u32(sm + bH1l);
      const uint32_t sGh = tc::smem_u32(sm + bGh), sGl = tc::smem_u32(sm + bGl);
      const int64_t tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
      bool dw_started = false;   // the first accumulation initialises dW2 and dW1
      uint32_t ph = 0;
      for (int64_t st = 0; st < 4 * tiles; ++st) {
        if (!tc::mbar_wait(&fs->ready, ph, kSpin) || *(volatile int*)&fs->error) {
          atomicExch(&fs->error, 1);
          break;
        }
        ph ^= 1;
        tc::fence_after_sync();
        const int stage = (int)(st & 3);
        if (stage == 0) {
          mma_split_w(tmem + cD, sXh, sXl, kSboX, sW1, kSboX, kK1 / 16, tc::idesc_bf16(128, kH, 0, 0));
        } else if (stage == 1) {
          mma_split_w(tmem + cD, sHh, sHl, kSboH1, sW2, kSboW2, kH / 16, tc::idesc_bf16(128, kH, 0, 0));
        } else if (stage == 2) {
          // dW2|db2 += G2^T [H1 | 1]: Gh Hh + Gh Hl + Gl Hh (both MN-major; K = tile rows)
          const uint32_t id_dw2 = tc::idesc_bf16(128, kH1W, 1, 1);
#pragma unroll 1
          for (int k = 0; k < kTile / 16; ++k) {
            const uint64_t gh = tc::smem_desc_mn(sGh + k * 2 * kSboG, kSboG, 128);
            const uint64_t gl = tc::smem_desc_mn(sGl + k * 2 * kSboG, kSboG, 128);
            const uint64_t hh = tc::smem_desc_mn(sHh + k * 2 * kSboH1, kSboH1, 128);
            const uint64_t hl = tc::smem_desc_mn(sHl + k * 2 * kSboH1, kSboH1, 128);
            tc::mma_bf16(tmem + cDW2, gh, hh, id_dw2, (dw_started || k > 0) ? 1u : 0u);
            tc::mma_bf16(tmem + cDW2, gh, hl, id_dw2, 1u);
            tc::mma_bf16(tmem + cDW2, gl, hh, id_dw2, 1u);
          }
          // D = G2 W2: Gh W2 + Gl W2 (G K-major, W2 MN-major)
          const uint32_t id_gh = tc::idesc_bf16(128, kH, 0, 1);
#pragma unroll 1
          for (int k = 0; k < kH / 16; ++k) {
            const uint64_t w = tc::smem_desc_mn(sW2 + k * 2 * kSboW2, kSboW2, 128);
            tc::mma_bf16(tmem + cD, tc::smem_desc(sGh + k * 256, 128, kSboG), w, id_gh, k > 0 ? 1u : 0u);
            tc::mma_bf16(tmem + cD, tc::smem_desc(sGl + k * 256, 128, kSboG), w, id_gh, 1u);
          }
        } else {
          // dW1|db1 += G1^T X: Gh Xh + Gh Xl + Gl Xh
          const uint32_t id_dw1 = tc::idesc_bf16(128, kK1, 1, 1);
#pragma unroll 1
          for (int k = 0; k < kTile / 16; ++k) {
            const uint64_t gh = tc::smem_desc_mn(sGh + k * 2 * kSboG, kSboG, 128);
            const uint64_t gl = tc::smem_desc_mn(sGl + k * 2 * kSboG, kSboG, 128);
            const uint64_t xh = tc::smem_desc_mn(sXh + k * 2 * kSboX, kSboX, 128);
            const uint64_t xl = tc::smem_desc_mn(sXl + k * 2 * kSboX, kSboX, 128);
            tc::mma_bf16(tmem + cDW1, gh, xh, id_dw1, (dw_started || k > 0) ? 1u : 0u);
            tc::mma_bf16(tmem + cDW1, gh, xl, id_dw1, 1u);
            tc::mma_bf16(tmem + cDW1, gl, xh, id_dw1, 1u);
          }
          dw_started = true;
        }
        tc::mma_commit(&fs->done);
      }
      // every MMA issued has finished before tensor memory is read or released
      tc::mma_commit(&fs->fin);
      if (!tc::mbar_wait(&fs->fin, 0, kSpin)) atomicExch(&fs->error, 1);
    }
    __syncwarp();
  } else {
    // --------------------------------------------------- epilogue warps
    const int row = tid;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t ph = 0;
    auto signal = [&]() {
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      named_bar1();
      if (row == 0) tc::mbar_arrive(&fs->ready);
    };
    auto await = [&]() -> bool {
      const bool ok = tc::mbar_wait(&fs->done, ph, kSpin);
      ph ^= 1;
      if (!ok) atomicExch(&fs->error, 1);
      tc::fence_after_sync();
      return ok && !*(volatile int*)&fs->error;
    };
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t j = t * kTile + row;
      const bool valid = j < n;
      const float gup = valid ? __ldg(g_out + (idx ? (int64_t)__ldg(idx + j) : j)) : 0.0f;
      {
        float x[kK1];
        encode(xyz, idx, j, n, x);
        write_x(sm + bXh, sm + bXl, row, x);
      }
      signal();                                     // stage 0
      if (!await()) break;
#pragma unroll 1
      for (int ch = 0; ch < kH / 32; ++ch) {        // H1 = relu(D1), split
        float v[32];
        tc::tmem_ld32(lane_base + cD + ch * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q) st_split8(sm + bH1h, sm + bH1l, row, ch * 32 + q * 8, kSboH1, v + 8 * q);
      }
      signal();                                     // stage 1
      if (!await()) break;
      // output layer: g_z = the upstream logit gradient; G2 = (W3^T g_z) * (z2 > 0);
      // dW3 += g_z h2 (summed over the warp's rows by a reduce-scatter)
      db3acc += gup;
#pragma unroll 1
      for (int ch = 0; ch < kH / 32; ++ch) {
        float v[32], g[32];
        tc::tmem_ld32(lane_base + cD + ch * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int o = ch * 32 + i;
          const float z2 = v[i] + fs->b2[o];
          g[i] = z2 > 0.0f ? gup * fs->W3[o] : 0.0f;
          v[i] = gup * fmaxf(z2, 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) st_split8(sm + bGh, sm + bGl, row, ch * 32 + q * 8, kSboG, g + 8 * q);
        dW3acc[ch] += reduce_scatter32(v, lane);
      }
      signal();                                     // stage 2
      if (!await()) break;
#pragma unroll 1
      for (int ch = 0; ch < kH / 32; ++ch) {        // G1 = g_h1 * (H1 > 0), split
        float v[32];
        tc::tmem_ld32(lane_base + cD + ch * 32, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 hq = *reinterpret_cast<const uint4*>(sm + bH1h + tc::cm_off(row, ch * 32 + q * 8, kSboH1));
          const uint32_t hw[4] = {hq.x, hq.y, hq.z, hq.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {   // H1 > 0 <=> its hi term is positive
            if ((int16_t)(hw[i] & 0xffffu) <= 0) v[8 * q + 2 * i] = 0.0f;
            if ((int16_t)(hw[i] >> 16) <= 0) v[8 * q + 2 * i + 1] = 0.0f;
          }
          st_split8(sm + bGh, sm + bGl, row, ch * 32 + q * 8, kSboG, v + 8 * q);
        }
      }
      signal();                                     // stage 3
      if (!await()) break;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = fs->error == 0;
  if (ok && warp < 4 && (int64_t)blockIdx.x < ntiles) {
    // output layer: this warp's row sums (lane = hidden unit ch * 32 + lane)
#pragma unroll
    for (int ch = 0; ch < kH / 32; ++ch) atomicAdd(g_params + oW3 + ch * 32 + lane, dW3acc[ch]);
    float v = db3acc;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(g_params + oB3, v);
    // dW2|db2 and dW1|db1: TMEM lane = hidden unit o (lanes >= kH are padding)
    const int o = tid;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    if (warp < kH / 32) {
#pragma unroll 1
      for (int ch = 0; ch < kH / 32; ++ch) {
        float d[32];
        tc::tmem_ld32(lane_base + cDW2 + ch * 32, d);
#pragma unroll
        for (int i = 0; i < 32; ++i) atomicAdd(g_params + oW2 + o * kH + ch * 32 + i, d[i]);
      }
      float u[16];
      tc::tmem_ld16(lane_base + cDW2 + kH, u);
      atomicAdd(g_params + oB2 + o, u[0]);
      float d1[32], d2[16];
      tc::tmem_ld32(lane_base + cDW1, d1);
      tc::tmem_ld16(lane_base + cDW1 + 32, d2);
#pragma unroll
      for (int k = 0; k < 32; ++k) atomicAdd(g_params + oW1 + o * kIn + k, d1[k]);
#pragma unroll
      for (int k = 32; k < kIn; ++k) atomicAdd(g_params + oW1 + o * kIn + k, d2[k - 32]);
      atomicAdd(g_params + oB1 + o, d2[kIn - 32]);
    }
  }
  if (!ok && tid == 0) atomicExch(&g_mlp_status, (int)DVGO_ERR_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 4) tc::tmem_dealloc(tmem, 512);
}

}  // namespace dvgo

using namespace dvgo;

int dvgo_proposal_fwd_bf16(const float* xyz, const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                           const float* params, float* logits, cudaStream_t st) {
  const size_t smem = fEnd + sizeof(Side);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(prop_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, 2 * kNumSMs);
  if (grid < 1) return DVGO_OK;
  prop_fwd_kernel<<<grid, 128, smem, st>>>(xyz, idx, n_cap, n_dev, params, logits);
  return launch_status();
}

int dvgo_proposal_bwd_bf16(const float* g_logits, const float* xyz, const int32_t* idx, int64_t n_cap,
                           const int64_t* n_dev, const float* params, float* g_params, cudaStream_t st) {
  const size_t smem = bEnd + sizeof(Side);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(prop_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  prop_bwd_kernel<<<grid, 160, smem, st>>>(g_logits, xyz, idx, n_cap, n_dev, params, g_params);
  return launch_status();
}

int dvgo_mlp_status_read_and_clear(cudaStream_t st) {
  int v = 0, zero = 0;
  cudaMemcpyFromSymbolAsync(&v, g_mlp_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  cudaMemcpyToSymbolAsync(g_mlp_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return v;
}
