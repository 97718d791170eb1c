// Small MLPs in BF16 on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory: the colour MLP (rgbnet, 39 -> 128 -> 128 ->
// 3 sigmoid; the shallow decoder of the hybrid representation, Tab. 1) and the
// learned proposal network (position encoding 39 -> 64 -> 64 -> 1 logit).
// One 128-sample tile per step of a persistent CTA of 128 threads (thread =
// tile row = TMEM lane).
//
// Forward, per tile:  X[128x48] (39 inputs, a 1 carrying b1, zero pad) ->
// D1 = X W1^T (TMEM) -> H1 = relu(D1) (bf16, smem) -> D2 = H1 W2^T (TMEM) ->
// z2 = D2 + b2 -> output layer on the CUDA cores in FP32.
// Backward, per tile (forward recomputed): g_out -> g_z2 (CUDA cores) ->
//   dW2 += g_z2^T [H1 | 1]      (TMEM, kept for the whole kernel; the ones
//                                column yields db2)
//   g_h1 = g_z2 W2, g_z1 = g_h1 * (H1 > 0)
//   dW1 += g_z1^T X             (TMEM, whole kernel; the X bias column
//                                yields db1)
//   g_X  = g_z1 W1[:, 0:16]     (colour MLP only: -> g_k0, the 12 features)
// Output-layer gradients are reduced across each warp with a butterfly
// reduce-scatter.  The same shared-memory bytes serve as K-major operand in
// one product and as MN-major operand in another (no transposed copies).
// The gradient tile G is always 128 columns wide (zero past the hidden
// width), so every weight-gradient product is an M = 128 MMA.
#include "common.cuh"
#include "mlp_common.cuh"
#include "tcgen05.cuh"

namespace dvgo {

__device__ int g_mlp_status;  // DVGO_ERR_TIMEOUT if a bounded wait gave up

// All pointers a network may read or write (each uses a subset).
struct MlpIO {
  const float* k0;
  const float* rays_d;
  const int32_t* ray_id;
  const float* xyz;
  const int32_t* idx;
  int64_t n_cap;
  const int64_t* n_dev;
  const float* params;
  float* out;            // forward output rows at the sample index
  const float* g_out;    // per-sample upstream gradient (may be NULL for rgbnet)
  const float* g_color;  // rgbnet: upstream from compositing, w[s] * g_color[ray]
  const float* w;
  float* g_params;
  float* g_in;           // rgbnet: g_k0
  float* part;           // backward: per-CTA partial gradient rows of NP floats (NULL: atomics)
};

template <int H_, int OUT_>
struct NetShape {
  static constexpr int H = H_, OUT = OUT_;
  static constexpr int oW1 = 0, oB1 = H * kIn, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H,
                       oB3 = oW3 + OUT * H, NP = oB3 + OUT;
};

struct RgbNet : NetShape<kHid, kOut> {
  static constexpr bool kSigmoid = true, kInputGrad = true;
  static_assert(NP == kNumParams, "rgbnet layout");
  __device__ static void encode(const MlpIO& io, int64_t j, int64_t n, float row[kInP]) {
    encode_row(io.k0, io.rays_d, io.ray_id, io.idx, j, n, row);
  }
  __device__ static void upstream(const MlpIO& io, int64_t s, float g[3]) {
    upstream_rgb_grad(io.g_out, io.g_color, io.w, io.ray_id, s, g);
  }
};

constexpr int kPropFreq = 6;

struct PropNet : NetShape<64, 1> {
  static constexpr bool kSigmoid = false, kInputGrad = false;
  // [x (3), sin(2^f x_a) (a major, f inner), cos(2^f x_a), 1], f < 6
  __device__ static void encode(const MlpIO& io, int64_t j, int64_t n, float row[kInP]) {
    if (j >= n) {
#pragma unroll
      for (int k = 0; k < kInP; ++k) row[k] = 0.0f;
      return;
    }
    const int64_t s = io.idx ? (int64_t)__ldg(io.idx + j) : j;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float x = __ldg(io.xyz + 3 * s + a);
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
  __device__ static void upstream(const MlpIO& io, int64_t s, float g[1]) { g[0] = __ldg(io.g_out + s); }
};

namespace bf {

constexpr int kK1 = 48;                       // padded input width
constexpr uint32_t kSboX = (kK1 / 8) * 128;   // 768: 8-row group stride of 48-wide rows
constexpr int kGW = 128;                      // gradient-tile width (hidden width, zero padded)
constexpr uint32_t kSboG = (kGW / 8) * 128;   // 2048
constexpr uint32_t kSpin = 1u << 24;

template <class Net>
struct Layout {
  static constexpr int H = Net::H;
  static constexpr int H1W = H + 16;                    // [H1 | 1 | 0..]
  static constexpr uint32_t kSboW2 = (H / 8) * 128;
  static constexpr uint32_t kSboH1 = (H1W / 8) * 128;
  static constexpr uint32_t oW1 = 0;
  static constexpr uint32_t oW2 = oW1 + H * kK1 * 2;
  static constexpr uint32_t oX = oW2 + H * H * 2;
  static constexpr uint32_t oH1 = oX + kTile * kK1 * 2;
  static constexpr uint32_t oG = oH1 + kTile * H1W * 2;
  static constexpr uint32_t kFwdOperands = oG;
  static constexpr uint32_t kBwdOperands = oG + kTile * kGW * 2;
};

template <class Net>
struct F32Side {  // epilogue constants (BF16-rounded values, kept in FP32)
  float W3[Net::OUT * Net::H];
  float b2[Net::H];
  float b3[4];
  uint64_t bar;
  uint32_t tmem_slot;
};

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
template <class Net>
__device__ void load_weights(const float* __restrict__ params, uint8_t* sm, F32Side<Net>* fs) {
  using Lo = Layout<Net>;
  constexpr int H = Net::H;
  for (int e = threadIdx.x; e < H * kK1; e += blockDim.x) {
    const int o = e / kK1, k = e % kK1;
    float v = k < kIn ? params[Net::oW1 + o * kIn + k] : (k == kIn ? params[Net::oB1 + o] : 0.0f);
    st_bf16(sm + Lo::oW1, tc::cm_off(o, k, kSboX), v);
  }
  for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
    const int o = e / H, i = e % H;
    st_bf16(sm + Lo::oW2, tc::cm_off(o, i, Lo::kSboW2), params[Net::oW2 + e]);
  }
  for (int e = threadIdx.x; e < Net::OUT * H; e += blockDim.x) fs->W3[e] = bfr(params[Net::oW3 + e]);
  for (int e = threadIdx.x; e < H; e += blockDim.x) fs->b2[e] = bfr(params[Net::oB2 + e]);
  if (threadIdx.x < 4) fs->b3[threadIdx.x] = threadIdx.x < Net::OUT ? bfr(params[Net::oB3 + threadIdx.x]) : 0.0f;
}

template <class Net>
__device__ __forceinline__ void write_x_row(uint8_t* sm, int row, const float x[kInP]) {
  float v[8];
#pragma unroll
  for (int kb = 0; kb < kK1 / 8; ++kb) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kb * 8 + i;
      v[i] = k < kInP ? x[k] : 0.0f;
    }
    st_row8(sm + Layout<Net>::oX, row, kb * 8, kSboX, v);
  }
}

// Layer 1 / layer 2 MMAs (K-major A and B), issued by one thread.
template <class Net>
__device__ __forceinline__ void issue_layer1(uint8_t* sm, uint32_t tmem_d) {
  using Lo = Layout<Net>;
  const uint32_t xs = tc::smem_u32(sm + Lo::oX), w1 = tc::smem_u32(sm + Lo::oW1);
  const uint32_t id = tc::idesc_bf16(128, Net::H, 0, 0);
#pragma unroll
  for (int j = 0; j < kK1 / 16; ++j)
    tc::mma_bf16(tmem_d, tc::smem_desc(xs + 256 * j, 128, kSboX), tc::smem_desc(w1 + 256 * j, 128, kSboX),
                 id, j > 0);
}

template <class Net>
__device__ __forceinline__ void issue_layer2(uint8_t* sm, uint32_t tmem_d) {
  using Lo = Layout<Net>;
  const uint32_t h1 = tc::smem_u32(sm + Lo::oH1), w2 = tc::smem_u32(sm + Lo::oW2);
  const uint32_t id = tc::idesc_bf16(128, Net::H, 0, 0);
#pragma unroll
  for (int j = 0; j < Net::H / 16; ++j)
    tc::mma_bf16(tmem_d, tc::smem_desc(h1 + 256 * j, 128, Lo::kSboH1),
                 tc::smem_desc(w2 + 256 * j, 128, Lo::kSboW2), id, j > 0);
}

// D1 (TMEM) -> relu -> bf16 H1 row
template <class Net>
__device__ __forceinline__ void epilogue_h1(uint8_t* sm, uint32_t taddr_row, int row) {
  using Lo = Layout<Net>;
#pragma unroll 1
  for (int ch = 0; ch < Net::H / 32; ++ch) {
    float v[32];
    tc::tmem_ld32(taddr_row + ch * 32, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) st_row8(sm + Lo::oH1, row, ch * 32 + q * 8, Lo::kSboH1, v + 8 * q);
  }
}

// z3 = b3 + W3 relu(D2 + b2)
template <class Net>
__device__ __forceinline__ void layer3_z(const F32Side<Net>* fs, uint32_t taddr_d2, float (&z3)[Net::OUT]) {
#pragma unroll
  for (int c = 0; c < Net::OUT; ++c) z3[c] = fs->b3[c];
#pragma unroll 1
  for (int ch = 0; ch < Net::H / 32; ++ch) {
    float v[32];
    tc::tmem_ld32(taddr_d2 + ch * 32, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int o = ch * 32 + i;
      const float h = fmaxf(v[i] + fs->b2[o], 0.0f);
#pragma unroll
      for (int c = 0; c < Net::OUT; ++c) z3[c] = fmaf(fs->W3[c * Net::H + o], h, z3[c]);
    }
  }
}

}  // namespace bf

using namespace bf;

template <class Net>
__global__ void __launch_bounds__(128, 1) mlp_fwd_bf16_kernel(MlpIO io) {
  using Lo = Layout<Net>;
  extern __shared__ __align__(1024) uint8_t sm[];
  F32Side<Net>* fs = reinterpret_cast<F32Side<Net>*>(sm + Lo::kFwdOperands);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t n = mlp_count(io.n_cap, io.n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (warp == 0) tc::tmem_alloc(&fs->tmem_slot, 256);
  if (tid == 0) tc::mbar_init(&fs->bar, 1);
  load_weights<Net>(io.params, sm, fs);
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
      Net::encode(io, j, n, x);
      write_x_row<Net>(sm, tid, x);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_layer1<Net>(sm, tmem);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    epilogue_h1<Net>(sm, lane_base, tid);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_layer2<Net>(sm, tmem + 128);
      tc::mma_commit(&fs->bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&fs->bar, phase, kSpin));
    phase ^= 1;
    if (!ok) break;
    tc::fence_after_sync();
    float z3[Net::OUT];
    layer3_z<Net>(fs, lane_base + 128, z3);
    if (j < n) {
      const int64_t s = io.idx ? (int64_t)__ldg(io.idx + j) : j;
#pragma unroll
      for (int c = 0; c < Net::OUT; ++c)
        io.out[Net::OUT * s + c] = Net::kSigmoid ? sigmoid_f(z3[c]) : z3[c];
    }
    tc::fence_before_sync();
  }
  if (!ok && tid == 0) atomicExch(&g_mlp_status, (int)DVGO_ERR_TIMEOUT);
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Backward, warp specialised.  Two groups of four warps (WG0, WG1) take
// alternate tiles; each owns its shared-memory operand buffers (X, [H1 | 1],
// G) and a 128-column TMEM region that successively holds D1, D2, g_h1 and
// g_X of its tile.  A ninth warp issues every MMA: it waits until a group
// signals that the operands of the group's next stage are in shared memory,
// issues that stage and commits it to the group's "done" barrier, so the
// tensor core runs one group's products while the other group's epilogue
// runs on the CUDA cores.  The weight-gradient accumulators (dW2|db2,
// dW1|db1) sit in TMEM for the whole kernel and are only ever updated by
// the issuing thread.  Every wait is bounded.
namespace bf {

__device__ __forceinline__ void named_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(128) : "memory");
}

template <class Net>
struct WsLayout {
  static constexpr int H = Net::H;
  static constexpr int H1W = H + 16;
  static constexpr uint32_t kSboW2 = (H / 8) * 128;
  static constexpr uint32_t kSboH1 = (H1W / 8) * 128;
  static constexpr uint32_t oW1 = 0;
  static constexpr uint32_t oW2 = oW1 + H * kK1 * 2;
  static constexpr uint32_t oGroup = oW2 + H * H * 2;          // first group's buffers
  static constexpr uint32_t gX = 0;                             // offsets inside a group
  static constexpr uint32_t gH1 = gX + kTile * kK1 * 2;
  static constexpr uint32_t gG = gH1 + kTile * H1W * 2;
  static constexpr uint32_t kGroupBytes = gG + kTile * kGW * 2;
  static constexpr uint32_t kOperands = oGroup + 2 * kGroupBytes;
};

template <class Net>
struct WsSide {
  float W3[Net::OUT * Net::H];
  float b2[Net::H];
  float b3[4];
  uint64_t ready[2];
  uint64_t done[2];
  uint32_t tmem_slot;
  int error;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

}  // namespace bf

template <class Net>
__global__ void __launch_bounds__(288, 1) mlp_bwd_bf16_kernel(MlpIO io) {
  using Lo = WsLayout<Net>;
  constexpr int H = Net::H, OUT = Net::OUT, NCH = H / 32;
  constexpr uint32_t cDW2 = 256, cDW1 = 400;
  extern __shared__ __align__(1024) uint8_t sm[];
  WsSide<Net>* fs = reinterpret_cast<WsSide<Net>*>(sm + Lo::kOperands);
  static_assert(Lo::kOperands + sizeof(WsSide<Net>) <= 227 * 1024, "smem");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = mlp_count(io.n_cap, io.n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (warp == 8) tc::tmem_alloc(&fs->tmem_slot, 512);
  if (tid == 0) {
    tc::mbar_init(&fs->ready[0], 1);
    tc::mbar_init(&fs->ready[1], 1);
    tc::mbar_init(&fs->done[0], 1);
    tc::mbar_init(&fs->done[1], 1);
    fs->error = 0;
  }
  // weights (all 288 threads)
  for (int e = tid; e < H * kK1; e += blockDim.x) {
    const int o = e / kK1, k = e % kK1;
    float v = k < kIn ? io.params[Net::oW1 + o * kIn + k] : (k == kIn ? io.params[Net::oB1 + o] : 0.0f);
    st_bf16(sm + Lo::oW1, tc::cm_off(o, k, kSboX), v);
  }
  for (int e = tid; e < H * H; e += blockDim.x) {
    const int o = e / H, i = e % H;
    st_bf16(sm + Lo::oW2, tc::cm_off(o, i, Lo::kSboW2), io.params[Net::oW2 + e]);
  }
  for (int e = tid; e < OUT * H; e += blockDim.x) fs->W3[e] = bfr(io.params[Net::oW3 + e]);
  for (int e = tid; e < H; e += blockDim.x) fs->b2[e] = bfr(io.params[Net::oB2 + e]);
  if (tid < 4) fs->b3[tid] = tid < OUT ? bfr(io.params[Net::oB3 + tid]) : 0.0f;
  if (tid < 256) {  // constant columns of [H1 | 1 | 0..] and zero columns of G past H
    uint8_t* grp = sm + Lo::oGroup + (tid >> 7) * Lo::kGroupBytes;
    const int row = tid & 127;
    float one[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    st_row8(grp + Lo::gH1, row, H, Lo::kSboH1, one);
    st_row8(grp + Lo::gH1, row, H + 8, Lo::kSboH1, z);
    for (int k = H; k < kGW; k += 8) st_row8(grp + Lo::gG, row, k, kSboG, z);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  const uint32_t sm_w1 = tc::smem_u32(sm + Lo::oW1), sm_w2 = tc::smem_u32(sm + Lo::oW2);

  // output-layer gradient partials of the epilogue threads (zero in the issuer warp)
  float dW3acc[OUT * NCH];
#pragma unroll
  for (int i = 0; i < OUT * NCH; ++i) dW3acc[i] = 0.0f;
  float db3acc[OUT];
#pragma unroll
  for (int c = 0; c < OUT; ++c) db3acc[c] = 0.0f;
  if (warp == 8) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int64_t left[2];
      for (int w = 0; w < 2; ++w) {
        const int64_t first = blockIdx.x + (int64_t)w * gridDim.x;
        const int64_t tiles = first < ntiles ? (ntiles - 1 - first) / (2 * (int64_t)gridDim.x) + 1 : 0;
        left[w] = 4 * tiles;  // four MMA stages per tile
      }
      int stage[2] = {0, 0};
      uint32_t ph[2] = {0, 0};
      bool dw2_started = false, dw1_started = false;  // first accumulation initialises
      uint32_t spins = 0;
      while ((left[0] > 0 || left[1] > 0) && !*(volatile int*)&fs->error) {
        bool served = false;
        for (int w = 0; w < 2; ++w) {
          if (left[w] == 0 || !tc::mbar_try_wait(&fs->ready[w], ph[w])) continue;
          ph[w] ^= 1;
          served = true;
          tc::fence_after_sync();
          uint8_t* grp = sm + Lo::oGroup + w * Lo::kGroupBytes;
          const uint32_t sx = tc::smem_u32(grp + Lo::gX), sh1 = tc::smem_u32(grp + Lo::gH1);
          const uint32_t sg = tc::smem_u32(grp + Lo::gG);
          const uint32_t dcol = tmem + 128 * w;
          if (stage[w] == 0) {          // D = X W1^T
            const uint32_t id = tc::idesc_bf16(128, H, 0, 0);
#pragma unroll
            for (int j = 0; j < kK1 / 16; ++j)
              tc::mma_bf16(dcol, tc::smem_desc(sx + 256 * j, 128, kSboX),
                           tc::smem_desc(sm_w1 + 256 * j, 128, kSboX), id, j > 0);
          } else if (stage[w] == 1) {   // D = H1 W2^T
            const uint32_t id = tc::idesc_bf16(128, H, 0, 0);
#pragma unroll
            for (int j = 0; j < H / 16; ++j)
              tc::mma_bf16(dcol, tc::smem_desc(sh1 + 256 * j, 128, Lo::kSboH1),
                           tc::smem_desc(sm_w2 + 256 * j, 128, Lo::kSboW2), id, j > 0);
          } else if (stage[w] == 2) {   // dW2|db2 += G^T [H1 | 1];  D = G W2
            const uint32_t id_dw2 = tc::idesc_bf16(128, Lo::H1W, 1, 1);
#pragma unroll
            for (int k = 0; k < kTile / 16; ++k)
              tc::mma_bf16(tmem + cDW2, tc::smem_desc_mn(sg + k * 2 * kSboG, kSboG, 128),
                           tc::smem_desc_mn(sh1 + k * 2 * Lo::kSboH1, Lo::kSboH1, 128), id_dw2,
                           (dw2_started || k > 0) ? 1u : 0u);
            dw2_started = true;
            const uint32_t id_gh = tc::idesc_bf16(128, H, 0, 1);
#pragma unroll
            for (int k = 0; k < H / 16; ++k)
              tc::mma_bf16(dcol, tc::smem_desc(sg + k * 256, 128, kSboG),
                           tc::smem_desc_mn(sm_w2 + k * 2 * Lo::kSboW2, Lo::kSboW2, 128), id_gh, k > 0);
          } else {                      // dW1|db1 += G^T X;  D[:, 0:16] = G W1[:, 0:16]
            const uint32_t id_dw1 = tc::idesc_bf16(128, kK1, 1, 1);
#pragma unroll
            for (int k = 0; k < kTile / 16; ++k)
              tc::mma_bf16(tmem + cDW1, tc::smem_desc_mn(sg + k * 2 * kSboG, kSboG, 128),
                           tc::smem_desc_mn(sx + k * 2 * kSboX, kSboX, 128), id_dw1,
                           (dw1_started || k > 0) ? 1u : 0u);
            dw1_started = true;
            if (Net::kInputGrad) {
              const uint32_t id_gx = tc::idesc_bf16(128, 16, 0, 1);
#pragma unroll
              for (int k = 0; k < H / 16; ++k)
                tc::mma_bf16(dcol, tc::smem_desc(sg + k * 256, 128, kSboG),
                             tc::smem_desc_mn(sm_w1 + k * 2 * kSboX, kSboX, 128), id_gx, k > 0);
            }
          }
          tc::mma_commit(&fs->done[w]);
          stage[w] = (stage[w] + 1) & 3;
          --left[w];
        }
        if (served) spins = 0;
        else if (++spins > kSpin) atomicExch(&fs->error, 1);
      }
    }
    __syncwarp();
  } else {
    // --------------------------------------------------- epilogue groups
    const int w = warp >> 2;                 // group
    const int row = tid & 127;               // tile row = TMEM lane
    uint8_t* grp = sm + Lo::oGroup + w * Lo::kGroupBytes;
    const uint32_t lane_base = tmem + 128 * w + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t ph = 0;
    auto signal = [&]() {
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      named_bar(1 + w);
      if (row == 0) mbar_arrive(&fs->ready[w]);
    };
    auto await = [&]() -> bool {
      bool ok = tc::mbar_wait(&fs->done[w], ph, kSpin);
      ph ^= 1;
      if (!ok) atomicExch(&fs->error, 1);
      tc::fence_after_sync();
      return ok && !*(volatile int*)&fs->error;
    };
    for (int64_t t = blockIdx.x + (int64_t)w * gridDim.x; t < ntiles; t += 2 * (int64_t)gridDim.x) {
      const int64_t j = t * kTile + row;
      const bool valid = j < n;
      int64_t s = 0;
      float gup[OUT];
#pragma unroll
      for (int c = 0; c < OUT; ++c) gup[c] = 0.0f;
      if (valid) {
        s = io.idx ? (int64_t)__ldg(io.idx + j) : j;
        Net::upstream(io, s, gup);
      }
      {
        float x[kInP];
        Net::encode(io, j, n, x);
        float v[8];
#pragma unroll
        for (int kb = 0; kb < kK1 / 8; ++kb) {
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = kb * 8 + i < kInP ? x[kb * 8 + i] : 0.0f;
          st_row8(grp + Lo::gX, row, kb * 8, kSboX, v);
        }
      }
      signal();                                   // stage 0: D = X W1^T
      if (!await()) break;
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {          // epilogue 1: H1 = relu(D)
        float v[32];
        tc::tmem_ld32(lane_base + ch * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q) st_row8(grp + Lo::gH1, row, ch * 32 + q * 8, Lo::kSboH1, v + 8 * q);
      }
      signal();                                   // stage 1: D = H1 W2^T
      if (!await()) break;
      float z3[OUT];                              // epilogue 2
#pragma unroll
      for (int c = 0; c < OUT; ++c) z3[c] = fs->b3[c];
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {
        float v[32];
        tc::tmem_ld32(lane_base + ch * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int o = ch * 32 + i;
          const float h = fmaxf(v[i] + fs->b2[o], 0.0f);
#pragma unroll
          for (int c = 0; c < OUT; ++c) z3[c] = fmaf(fs->W3[c * H + o], h, z3[c]);
        }
      }
      float gz3[OUT];
#pragma unroll
      for (int c = 0; c < OUT; ++c) {
        if (Net::kSigmoid) {
          const float y = sigmoid_f(z3[c]);
          gz3[c] = gup[c] * y * (1.0f - y);
        } else {
          gz3[c] = gup[c];
        }
        db3acc[c] += gz3[c];
      }
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {
        float v[32], g[32];
        tc::tmem_ld32(lane_base + ch * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int o = ch * 32 + i;
          const float z2 = v[i] + fs->b2[o];
          float gs = 0.0f;
#pragma unroll
          for (int c = 0; c < OUT; ++c) gs = fmaf(gz3[c], fs->W3[c * H + o], gs);
          g[i] = z2 > 0.0f ? gs : 0.0f;
          v[i] = fmaxf(z2, 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) st_row8(grp + Lo::gG, row, ch * 32 + q * 8, kSboG, g + 8 * q);
#pragma unroll 1
        for (int c = 0; c < OUT; ++c) {
          float p[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) p[i] = gz3[c] * v[i];
          dW3acc[c * NCH + ch] += reduce_scatter32(p, lane);
        }
      }
      signal();                                   // stage 2: dW2 += G^T [H1|1]; D = G W2
      if (!await()) break;
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {          // epilogue 3: g_z1 over G
        float v[32];
        tc::tmem_ld32(lane_base + ch * 32, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float h[8];
          ld_row8(grp + Lo::gH1, row, ch * 32 + q * 8, Lo::kSboH1, h);
#pragma unroll
          for (int i = 0; i < 8; ++i) v[8 * q + i] = h[i] > 0.0f ? v[8 * q + i] : 0.0f;
          st_row8(grp + Lo::gG, row, ch * 32 + q * 8, kSboG, v + 8 * q);
        }
      }
      signal();                                   // stage 3: dW1 += G^T X; D = G W1
      if (!await()) break;
      if (Net::kInputGrad) {                      // epilogue 4
        float gx[16];
        tc::tmem_ld16(lane_base, gx);
        if (valid) {
          float4* dst = reinterpret_cast<float4*>(io.g_in + s * kFeat);
          dst[0] = make_float4(gx[0], gx[1], gx[2], gx[3]);
          dst[1] = make_float4(gx[4], gx[5], gx[6], gx[7]);
          dst[2] = make_float4(gx[8], gx[9], gx[10], gx[11]);
        }
      }
      tc::fence_before_sync();
      named_bar(1 + w);                           // TMEM region and X free for the next tile
    }
    if (!io.part) {
      // output-layer partials of this thread
#pragma unroll
      for (int c = 0; c < OUT; ++c)
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
          atomicAdd(io.g_params + Net::oW3 + c * H + ch * 32 + lane, dW3acc[c * NCH + ch]);
#pragma unroll
      for (int c = 0; c < OUT; ++c) atomicAdd(io.g_params + Net::oB3 + c, db3acc[c]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = fs->error == 0;
  if (io.part && warp < 8) {
    // output-layer partials of each epilogue warp into shared memory (every
    // group buffer is free once all warps have passed the barrier above)
    float* pr = reinterpret_cast<float*>(sm + Lo::oGroup);   // [8 warps][OUT][NCH][32]
    float* pr3 = pr + 8 * OUT * NCH * 32;                     // [8 warps][OUT]
#pragma unroll
    for (int c = 0; c < OUT; ++c)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) pr[((warp * OUT + c) * NCH + ch) * 32 + lane] = dW3acc[c * NCH + ch];
#pragma unroll
    for (int c = 0; c < OUT; ++c) {
      float v = db3acc[c];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) pr3[warp * OUT + c] = v;
    }
  }
  __syncthreads();
  if (io.part) {
    // This CTA's gradient into its own partial row (no atomics); a second
    // kernel sums the rows in CTA order.
    float* P = io.part + (size_t)blockIdx.x * Net::NP;
    const bool has = ntiles > blockIdx.x;
    const float* pr = reinterpret_cast<const float*>(sm + Lo::oGroup);
    const float* pr3 = pr + 8 * OUT * NCH * 32;
    for (int e = tid; has && e < OUT * H; e += blockDim.x) {
      const int c = e / H, o = e % H, ch = o >> 5, l = o & 31;
      float v = 0.0f;
      for (int w8 = 0; w8 < 8; ++w8) v += pr[((w8 * OUT + c) * NCH + ch) * 32 + l];
      P[Net::oW3 + e] = v;
    }
    if (has && tid < OUT) {
      float v = 0.0f;
      for (int w8 = 0; w8 < 8; ++w8) v += pr3[w8 * OUT + tid];
      P[Net::oB3 + tid] = v;
    }
    if (has && warp < 4 && warp * 32 < H) {
      // TMEM lane = output neuron o; rows through a 32 x 33 shared-memory
      // transpose so that each store covers 32 consecutive parameters
      float* tp = reinterpret_cast<float*>(sm + Lo::oGroup) + 8 * OUT * NCH * 32 + 64 + warp * 32 * 33;
      const int o0 = warp * 32;
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      const float keep = ok ? 1.0f : 0.0f;
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {
        float v[32];
        tc::tmem_ld32(lane_base + cDW2 + ch * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) tp[lane * 33 + i] = v[i] * keep;
        __syncwarp();
        for (int r = 0; r < 32; ++r) P[Net::oW2 + (o0 + r) * H + ch * 32 + lane] = tp[r * 33 + lane];
        __syncwarp();
      }
      {
        float v[16];
        tc::tmem_ld16(lane_base + cDW2 + H, v);
        P[Net::oB2 + o0 + lane] = v[0] * keep;
      }
      {
        float v[32], u[16];
        tc::tmem_ld32(lane_base + cDW1, v);
        tc::tmem_ld16(lane_base + cDW1 + 32, u);
#pragma unroll
        for (int i = 0; i < 32; ++i) tp[lane * 33 + i] = v[i] * keep;
        __syncwarp();
        for (int r = 0; r < 32; ++r) P[Net::oW1 + (o0 + r) * kIn + lane] = tp[r * 33 + lane];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i) tp[lane * 33 + i] = u[i] * keep;
        __syncwarp();
        for (int r = 0; r < 32; ++r) {
          if (lane < kIn - 32) P[Net::oW1 + (o0 + r) * kIn + 32 + lane] = tp[r * 33 + lane];
          else if (lane == kIn - 32) P[Net::oB1 + o0 + r] = tp[r * 33 + lane];
        }
      }
    }
  } else if (ok && warp < 4 && ntiles > blockIdx.x) {
    // TMEM lane = output neuron o (rows o >= H are padding)
    const int o = tid;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int ch = 0; ch < NCH; ++ch) {
      float v[32];
      tc::tmem_ld32(lane_base + cDW2 + ch * 32, v);
      if (o < H)
#pragma unroll
        for (int i = 0; i < 32; ++i) atomicAdd(io.g_params + Net::oW2 + o * H + ch * 32 + i, v[i]);
    }
    {
      float v[16];
      tc::tmem_ld16(lane_base + cDW2 + H, v);
      if (o < H) atomicAdd(io.g_params + Net::oB2 + o, v[0]);
    }
    {
      float v[32], u[16];
      tc::tmem_ld32(lane_base + cDW1, v);
      tc::tmem_ld16(lane_base + cDW1 + 32, u);
      if (o < H) {
#pragma unroll
        for (int k = 0; k < 32; ++k) atomicAdd(io.g_params + Net::oW1 + o * kIn + k, v[k]);
#pragma unroll
        for (int k = 32; k < kIn; ++k) atomicAdd(io.g_params + Net::oW1 + o * kIn + k, u[k - 32]);
        atomicAdd(io.g_params + Net::oB1 + o, u[kIn - 32]);
      }
    }
  }
  if (!ok && tid == 0) atomicExch(&g_mlp_status, (int)DVGO_ERR_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 8) tc::tmem_dealloc(tmem, 512);
}

// g_params += sum over the CTAs that had tiles of their partial rows, in CTA order.
__global__ void __launch_bounds__(256) bf16_partials_reduce_kernel(const float* __restrict__ part, int nrows,
                                                                   int np, int64_t n_cap,
                                                                   const int64_t* __restrict__ n_dev,
                                                                   float* __restrict__ g_params) {
  const int64_t n = mlp_count(n_cap, n_dev);
  const int rows = (int)std::min<int64_t>(nrows, (n + kTile - 1) / kTile);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int b = 0; b < rows; ++b) acc += part[(size_t)b * np + p];
    g_params[p] += acc;
  }
}

template <class Net>
static int launch_fwd(const MlpIO& io, cudaStream_t st) {
  const size_t smem = Layout<Net>::kFwdOperands + sizeof(F32Side<Net>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp_fwd_bf16_kernel<Net>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((io.n_cap + kTile - 1) / kTile, 2 * kNumSMs);
  if (grid < 1) return DVGO_OK;
  mlp_fwd_bf16_kernel<Net><<<grid, 128, smem, st>>>(io);
  return launch_status();
}

template <class Net>
static int launch_bwd(const MlpIO& io, cudaStream_t st) {
  const size_t smem = WsLayout<Net>::kOperands + sizeof(WsSide<Net>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp_bwd_bf16_kernel<Net>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int grid = (int)std::min<int64_t>((io.n_cap + kTile - 1) / kTile, kNumSMs);
  if (grid < 1) return DVGO_OK;
  mlp_bwd_bf16_kernel<Net><<<grid, 288, smem, st>>>(io);
  if (io.part)
    bf16_partials_reduce_kernel<<<(Net::NP + 255) / 256, 256, 0, st>>>(io.part, grid, Net::NP, io.n_cap,
                                                                      io.n_dev, io.g_params);
  return launch_status();
}

}  // namespace dvgo

using namespace dvgo;

int dvgo_rgbnet_fwd_bf16(const float* k0, const float* rays_d, const int32_t* ray_id,
                         const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                         const float* params, float* rgb, cudaStream_t st) {
  MlpIO io{};
  io.k0 = k0;
  io.rays_d = rays_d;
  io.ray_id = ray_id;
  io.idx = idx;
  io.n_cap = n_cap;
  io.n_dev = n_dev;
  io.params = params;
  io.out = rgb;
  return launch_fwd<RgbNet>(io, st);
}

int dvgo_rgbnet_bwd_bf16(const float* g_rgb, const float* g_color, const float* w, const float* k0,
                         const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                         int64_t n_cap, const int64_t* n_dev, const float* params,
                         float* g_params, float* g_k0, float* part, cudaStream_t st) {
  MlpIO io{};
  io.k0 = k0;
  io.rays_d = rays_d;
  io.ray_id = ray_id;
  io.idx = idx;
  io.n_cap = n_cap;
  io.n_dev = n_dev;
  io.params = params;
  io.g_out = g_rgb;
  io.g_color = g_color;
  io.w = w;
  io.g_params = g_params;
  io.g_in = g_k0;
  io.part = part;
  return launch_bwd<RgbNet>(io, st);
}

int dvgo_proposal_fwd_bf16(const float* xyz, const int32_t* idx, int64_t n_cap,
                           const int64_t* n_dev, const float* params, float* logits,
                           cudaStream_t st) {
  MlpIO io{};
  io.xyz = xyz;
  io.idx = idx;
  io.n_cap = n_cap;
  io.n_dev = n_dev;
  io.params = params;
  io.out = logits;
  return launch_fwd<PropNet>(io, st);
}

int dvgo_proposal_bwd_bf16(const float* g_logits, const float* xyz, const int32_t* idx,
                           int64_t n_cap, const int64_t* n_dev, const float* params,
                           float* g_params, cudaStream_t st) {
  MlpIO io{};
  io.xyz = xyz;
  io.idx = idx;
  io.n_cap = n_cap;
  io.n_dev = n_dev;
  io.params = params;
  io.g_out = g_logits;
  io.g_params = g_params;
  return launch_bwd<PropNet>(io, st);
}

int dvgo_mlp_status_read_and_clear(cudaStream_t st) {
  int v = 0, zero = 0;
  cudaMemcpyFromSymbolAsync(&v, g_mlp_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  cudaMemcpyToSymbolAsync(g_mlp_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return v;
}
