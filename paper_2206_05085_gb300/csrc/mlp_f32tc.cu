// Colour MLP (rgbnet, 39 -> ReLU 128 -> ReLU 128 -> sigmoid 3; the shallow
// decoder of the hybrid representation, Tab. 1) with FP32 accuracy on the
// 5th-generation tensor cores.
//
// Split operands.  A value v, first multiplied by an exact power of two s,
// is stored as two FP16 terms hi = fp16(s v) and lo = fp16(s v - hi); hi
// carries 11 significant bits and lo the next 11.  A product of two split
// matrices is accumulated in FP32 in tensor memory as hi*hi + hi*lo + lo*hi
// (three tcgen05.mma of kind::f16); the dropped lo*lo term is 2^-22 of the
// product, so each dot product carries an FP32-like relative error.  The
// scales keep the terms inside FP16's normal range: weights per matrix
// (largest |w| s in [2^13, 2^14)), layer inputs by 2^6, hidden activations
// by 2^4, and the backward's gradient rows G2 = g_z2 and G1 = g_z1 per sample
// from a bound on that sample's output-layer gradient, so that every sample's
// input gradient keeps FP32 relative accuracy however small it is.  The
// weight-gradient products (sums over samples) need one factor for all rows,
// S, the scale of the largest bound over the CTA's samples: dW2 reads H1 with
// row s multiplied by S / s_s, dW1 a second copy of G1's terms times S / s_s
// (a row far below the largest loses only terms below FP16's subnormal range,
// 2^-38 of the largest row).
// Every scale is an exact power of two, undone exactly in the epilogues.  A
// value whose scaled magnitude reaches 2^15 sets DVGO_ERR_RANGE.
//
// The same kernels also run the BF16 form (template parameter OpBF16): the
// parameters are the stored BF16 values, so each weight matrix is one BF16
// term (the products with its zero lo term are not issued) and the output
// layer reads BF16-rounded W3, b2, b3; every other operand (layer inputs,
// hidden activations, gradient rows) is split into two BF16 terms, hi with
// 8 significant bits and lo with the next 8, so that no rounding to BF16
// happens between layers.  BF16 has FP32's exponent range: the same
// power-of-two scales are applied (harmless) and no range limit applies.
//
// Forward, per 128-sample tile (thread = tile row = TMEM lane):
//   X (39 inputs, a 1 carrying b1, zero pad to 48) -> D1 = X W1^T -> H1 =
//   relu(D1) -> D2 = H1 W2^T -> z2 = D2 + b2 -> output layer and sigmoid on
//   the CUDA cores in FP32.  The split X and H1 of the tile (90112 bytes, the
//   shared-memory image) go to the act buffer with one bulk copy.
// Backward, per tile: bulk-load the tile's image; D2^T = W2 H1^T again (one
//   hidden unit per TMEM lane, so that sums over the tile's rows stay in a
//   thread's registers); on the CUDA cores g_z3 = g_rgb y (1 - y) from the
//   forward's output y, G2 = g_z2, dW3, db2 and db3; then dW2 += G2^T H1 and
//   g_h1 = G2 W2 (one shared-memory copy of G2 serves both); G1 = g_h1 *
//   (H1 > 0); dW1 (+db1 through X's ones column) += G1^T X and g_X =
//   G1 W1[:, 0:16] (-> g_k0).  dW2 and dW1 stay in tensor memory for the
//   whole kernel.
// Every wait on an mbarrier is bounded (DVGO_ERR_TIMEOUT).
#include <cuda_fp16.h>

#include "common.cuh"
#include "mlp_common.cuh"
#include "tcgen05.cuh"

namespace dvgo {

__device__ int g_mlp_tc_status;  // first error a kernel of this file met

namespace x3 {

constexpr int kK1 = 48;                           // padded input width
constexpr uint32_t kSboX = (kK1 / 8) * 128;       // 768: one term of an 8-row group, 48-wide rows
constexpr uint32_t kSboXs = 2 * kSboX;            // 1536: X's 8-row group, hi then lo terms
constexpr uint32_t kSboH = (kHid / 8) * 128;      // 2048: 128-wide rows
constexpr uint32_t kSboW1s = (32 / 8) * 128;      // 512: W1[:, 0:16] hi and lo side by side per 8 rows
constexpr uint32_t kXBytes = kTile * kK1 * 2;     // one term of X
constexpr uint32_t kHBytes = kTile * kHid * 2;    // one term of H1 or G
constexpr uint32_t kW1Bytes = kHid * kK1 * 2;
constexpr uint32_t kW1sBytes = kHid * 16 * 2;
constexpr uint32_t kW2Bytes = kHid * kHid * 2;
// Tile image [X | H1h | H1l]: X's hi and lo core matrices side by side in
// each 8-row group (so that [Xh | Xl] is one 96-wide operand of dW1).
constexpr uint32_t kImage = 2 * kXBytes + 2 * kHBytes;
constexpr uint32_t iX = 0, iHh = 2 * kXBytes, iHl = 2 * kXBytes + kHBytes;
constexpr uint32_t kActHeader = 256;
constexpr float kSX = 64.0f;     // input scale
constexpr float kSH = 16.0f;     // hidden-activation scale
constexpr float kRange = 32768.0f;   // FP16 terms: scaled magnitudes must stay below 2^15
constexpr uint32_t kSpin = 1u << 24;

__device__ __forceinline__ uint32_t u32_of(__half2 v) { return *reinterpret_cast<const uint32_t*>(&v); }
__device__ __forceinline__ uint32_t u32_of(__nv_bfloat162 v) { return *reinterpret_cast<const uint32_t*>(&v); }

// Operand term formats of the split products.
struct OpF16 {   // FP32 form: FP16 terms, every matrix split (weights too)
  static constexpr bool kBF = false;
  static constexpr bool kWeightLo = true;
  static constexpr float kMaxScaled = kRange;
  __host__ __device__ static constexpr uint32_t idesc(int M, int N, int a_mn, int b_mn) {
    return tc::idesc_f16(M, N, a_mn, b_mn);
  }
  // hi and lo terms of the pair (a, b), packed two per word
  __device__ static __forceinline__ uint32_t split2(float a, float b, uint32_t& lo) {
    const __half2 h2 = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h2);
    lo = u32_of(__floats2half2_rn(a - hf.x, b - hf.y));
    return u32_of(h2);
  }
  __device__ static __forceinline__ uint32_t weight2(float a, float b, uint32_t& lo) { return split2(a, b, lo); }
  // a pair of terms times a power of two r <= 1
  __device__ static __forceinline__ uint32_t mul2(uint32_t x, float r) {
    const __half2 y = __hmul2(*reinterpret_cast<const __half2*>(&x), __float2half2_rn(r));
    return u32_of(y);
  }
  __device__ static __forceinline__ float param(float x) { return x; }
};

struct OpBF16 {  // BF16 form: stored BF16 weights (one term), BF16 hi + lo terms elsewhere
  static constexpr bool kBF = true;
  static constexpr bool kWeightLo = false;
  static constexpr float kMaxScaled = 3.0e38f;   // only an overflow to infinity is reported
  __host__ __device__ static constexpr uint32_t idesc(int M, int N, int a_mn, int b_mn) {
    return tc::idesc_bf16(M, N, a_mn, b_mn);
  }
  __device__ static __forceinline__ uint32_t split2(float a, float b, uint32_t& lo) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h2);
    lo = u32_of(__floats2bfloat162_rn(a - hf.x, b - hf.y));
    return u32_of(h2);
  }
  __device__ static __forceinline__ uint32_t weight2(float a, float b, uint32_t& lo) {
    lo = 0u;
    return u32_of(__floats2bfloat162_rn(a, b));
  }
  __device__ static __forceinline__ uint32_t mul2(uint32_t x, float r) {
    const __nv_bfloat162 y =
        __hmul2(*reinterpret_cast<const __nv_bfloat162*>(&x), __float2bfloat162_rn(r));
    return u32_of(y);
  }
  __device__ static __forceinline__ float param(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
};

// backward shared memory
constexpr uint32_t bW2h = 0, bW2l = bW2h + kW2Bytes, bW1h = bW2l + kW2Bytes,
                   bImg = bW1h + 2 * kW1sBytes, bGh = bImg + kImage,
                   bGl = bGh + kHBytes, bEnd = bGl + kHBytes;
// tensor-memory columns of the backward
constexpr uint32_t cTmp = 0, cDW2 = 128, cDW1 = 256, cGX = 352, cGH = 384;

struct Side {
  float4 smp[kTile];  // per tile row: (g_z3[0..2], the row's gradient scale sG2)
  float red[32];      // block_max scratch: one entry per warp (17 warps)
  uint64_t bar_h;     // H1 terms of a tile image landed
  uint64_t bar_x;     // X terms landed
  uint64_t bar_d2;    // D2^T of a tile done
  uint64_t bar_gh;    // g_h1 done
  uint64_t bar_dw2;   // dW2 done (the tile's H1 terms are free)
  uint64_t bar_gx;    // g_X and dW1 done (G's shared memory and X are free)
  uint64_t bar_fin;   // every product done (before the accumulators are read)
  uint64_t g2_full;   // G2 of a tile in tensor and shared memory (16 warp arrivals)
  uint64_t g1_full;   // G1 of a tile in tensor and shared memory (16 warp arrivals)
  uint32_t tmem_slot;
  int abort;          // a wait gave up: later waits return at once
};
static_assert(bEnd + sizeof(Side) <= 227 * 1024, "backward shared memory");

// Largest value of v over the block (all threads call it).
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
  return r;
}

// 2^(13 - floor(log2 m)): maps the largest magnitude m into [2^13, 2^14).
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.0f) || !(m <= 3.0e38f)) return 1.0f;
  int e = ilogbf(m);
  e = max(-100, min(100, e));
  return ldexpf(1.0f, 13 - e);
}

// Split 8 (already scaled) values into the hi / lo core-matrix rows at (row,
// k8); vmax tracks the largest magnitude split (range check).  kWeight: the
// values are parameters (one term in the BF16 form).
template <class Op, bool kWeight>
__device__ __forceinline__ void st_split8(uint8_t* hi, uint8_t* lo, int row, int k8, uint32_t sbo,
                                          const float* v, float& vmax) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float a = v[2 * i], b = v[2 * i + 1];
    vmax = fmaxf(vmax, fmaxf(fabsf(a), fabsf(b)));
    h[i] = kWeight ? Op::weight2(a, b, l[i]) : Op::split2(a, b, l[i]);
  }
  const uint32_t off = tc::cm_off(row, k8, sbo);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// One scaled, split parameter (setup only).
template <class Op>
__device__ __forceinline__ void st_split1(uint8_t* hi, uint8_t* lo, uint32_t off, float v) {
  uint32_t l;
  const uint32_t h = Op::weight2(v, 0.0f, l);
  *reinterpret_cast<uint16_t*>(hi + off) = (uint16_t)(h & 0xffffu);
  *reinterpret_cast<uint16_t*>(lo + off) = (uint16_t)(l & 0xffffu);
}

// D (+)= A B^T over K = 16 * ksteps, split operands: three MMAs per K step
// (hi*hi, hi*lo, lo*hi; kALo / kBLo false: A's / B's lo term is zero and
// its product is not issued).  a_step / b_step: byte advance of the
// descriptors' start address per step (the start-address field holds
// address / 16, so a step adds step / 16).
template <bool kALo = true, bool kBLo = true>
__device__ __forceinline__ void mma3(uint32_t d, uint32_t ah, uint32_t al, uint32_t a_step, uint32_t a_lbo,
                                     uint32_t a_sbo, uint32_t bh, uint32_t bl, uint32_t b_step,
                                     uint32_t b_lbo, uint32_t b_sbo, int ksteps, uint32_t idesc,
                                     bool accumulate) {
  uint64_t dah = tc::smem_desc(ah, a_lbo, a_sbo), dal = tc::smem_desc(al, a_lbo, a_sbo);
  uint64_t dbh = tc::smem_desc(bh, b_lbo, b_sbo), dbl = tc::smem_desc(bl, b_lbo, b_sbo);
  const uint64_t ia = a_step >> 4, ib = b_step >> 4;
#pragma unroll 1
  for (int k = 0; k < ksteps; ++k) {
    tc::mma_bf16(d, dah, dbh, idesc, (accumulate || k > 0) ? 1u : 0u);
    if (kBLo) tc::mma_bf16(d, dah, dbl, idesc, 1u);
    if (kALo) tc::mma_bf16(d, dal, dbh, idesc, 1u);
    dah += ia;
    dal += ia;
    dbh += ib;
    dbl += ib;
  }
}

// D (+)= A B^T over K = 16 * ksteps with A (128 rows) in tensor memory as
// split terms: K-chunk q of 32 columns at a_tmem + 32 q, its hi terms packed
// two per column in the first 16 columns and its lo terms in the next 16.
template <bool kBLo = true>
__device__ __forceinline__ void mma3_ts(uint32_t d, uint32_t a_tmem, uint32_t bh, uint32_t bl, uint32_t b_step,
                                        uint32_t b_lbo, uint32_t b_sbo, int ksteps, uint32_t idesc,
                                        bool accumulate) {
  uint64_t dbh = tc::smem_desc(bh, b_lbo, b_sbo), dbl = tc::smem_desc(bl, b_lbo, b_sbo);
  const uint64_t ib = b_step >> 4;
#pragma unroll 1
  for (int j = 0; j < ksteps; ++j) {
    const uint32_t ah = a_tmem + 32u * (uint32_t)(j >> 1) + 8u * (uint32_t)(j & 1), al = ah + 16u;
    tc::mma_ts(d, ah, dbh, idesc, (accumulate || j > 0) ? 1u : 0u);
    if (kBLo) tc::mma_ts(d, ah, dbl, idesc, 1u);
    tc::mma_ts(d, al, dbh, idesc, 1u);
    dbh += ib;
    dbl += ib;
  }
}

// D (+)= A B^T over K = 16 * ksteps with A (128 rows) in tensor memory as
// split terms in 16-column chunks: K step j at a_tmem + 16 j, its hi terms
// packed two per column in the first 8 columns and its lo terms in the next 8.
template <bool kBLo = true>
__device__ __forceinline__ void mma3_ts16(uint32_t d, uint32_t a_tmem, uint32_t bh, uint32_t bl, uint32_t b_step,
                                          uint32_t b_lbo, uint32_t b_sbo, int ksteps, uint32_t idesc,
                                          bool accumulate) {
  uint64_t dbh = tc::smem_desc(bh, b_lbo, b_sbo), dbl = tc::smem_desc(bl, b_lbo, b_sbo);
  const uint64_t ib = b_step >> 4;
#pragma unroll 1
  for (int j = 0; j < ksteps; ++j) {
    const uint32_t ah = a_tmem + 16u * (uint32_t)j, al = ah + 8u;
    tc::mma_ts(d, ah, dbh, idesc, (accumulate || j > 0) ? 1u : 0u);
    if (kBLo) tc::mma_ts(d, ah, dbl, idesc, 1u);
    tc::mma_ts(d, al, dbh, idesc, 1u);
    dbh += ib;
    dbl += ib;
  }
}

// 16 values times s split into the 16-column chunk layout of mma3_ts16: hi
// terms of value pairs in words 0-7, lo terms in words 8-15.
template <class Op>
__device__ __forceinline__ void split16(const float (&v)[16], float s, uint32_t (&hl)[16], float& vmax) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float a = s * v[2 * c], b = s * v[2 * c + 1];
    vmax = fmaxf(vmax, fmaxf(fabsf(a), fabsf(b)));
    hl[c] = Op::split2(a, b, hl[8 + c]);
  }
}

// The split terms of split16 times r (a power of two <= 1) as the hi / lo
// core-matrix rows of columns k0 .. k0 + 15 of row `row` in shared memory.
template <class Op, bool kScale = true>
__device__ __forceinline__ void st_terms16(uint8_t* hi, uint8_t* lo, int row, int k0, const uint32_t (&hl)[16],
                                           float r) {
  auto m = [&](uint32_t x) { return kScale ? Op::mul2(x, r) : x; };
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint32_t off = tc::cm_off(row, k0 + 8 * q, kSboH);
    *reinterpret_cast<uint4*>(hi + off) =
        make_uint4(m(hl[4 * q]), m(hl[4 * q + 1]), m(hl[4 * q + 2]), m(hl[4 * q + 3]));
    *reinterpret_cast<uint4*>(lo + off) =
        make_uint4(m(hl[8 + 4 * q]), m(hl[9 + 4 * q]), m(hl[10 + 4 * q]), m(hl[11 + 4 * q]));
  }
}

// 32 values times s split into the tensor-memory chunk layout: hi terms of
// value pairs in words 0-15, lo terms in words 16-31 (one tcgen05.st).
template <class Op>
__device__ __forceinline__ void split32(const float (&v)[32], float s, uint32_t (&hl)[32],
                                        float& vmax) {
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const float a = s * v[2 * c], b = s * v[2 * c + 1];
    vmax = fmaxf(vmax, fmaxf(fabsf(a), fabsf(b)));
    hl[c] = Op::split2(a, b, hl[16 + c]);
  }
}

// The split terms of split32 times r (a power of two <= 1, exact in FP16
// down to its subnormal range, and in BF16) as the hi / lo core-matrix rows
// of columns k0 .. k0 + 31 of row `row` in shared memory.
template <class Op, bool kScale = true>
__device__ __forceinline__ void st_terms32(uint8_t* hi, uint8_t* lo, int row, int k0, const uint32_t (&hl)[32],
                                           float r) {
  auto m = [&](uint32_t x) { return kScale ? Op::mul2(x, r) : x; };
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t off = tc::cm_off(row, k0 + 8 * q, kSboH);
    *reinterpret_cast<uint4*>(hi + off) =
        make_uint4(m(hl[4 * q]), m(hl[4 * q + 1]), m(hl[4 * q + 2]), m(hl[4 * q + 3]));
    *reinterpret_cast<uint4*>(lo + off) =
        make_uint4(m(hl[16 + 4 * q]), m(hl[17 + 4 * q]), m(hl[18 + 4 * q]), m(hl[19 + 4 * q]));
  }
}

// Output-layer constants (FP32; the stored BF16 values in the BF16 form).
template <class Op, class SideT>
__device__ __forceinline__ void load_out_layer(const float* __restrict__ params, SideT* fs) {
  for (int o = threadIdx.x; o < kHid; o += blockDim.x)
    fs->ob[o] = make_float4(Op::param(params[kOffB2 + o]), Op::param(params[kOffW3 + o]),
                            Op::param(params[kOffW3 + kHid + o]), Op::param(params[kOffW3 + 2 * kHid + o]));
  if (threadIdx.x < 4) fs->b3[threadIdx.x] = threadIdx.x < kOut ? Op::param(params[kOffB3 + threadIdx.x]) : 0.0f;
}

// This thread's share of max |p[e]|, e < count (float4 loads, four in
// flight per thread, when p is 16-byte aligned and count a multiple of 4).
__device__ __forceinline__ float abs_max_part(const float* __restrict__ p, int count) {
  float m = 0.0f;
  if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (count & 3) == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const int n4 = count >> 2;
    for (int e0 = threadIdx.x; e0 < n4; e0 += 4 * blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = e < n4 ? __ldg(p4 + e) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
    }
  } else {
    for (int e = threadIdx.x; e < count; e += blockDim.x) m = fmaxf(m, fabsf(__ldg(p + e)));
  }
  return m;
}

// Rows o of W1 | b1 | 0 (width K = 8 kb, the bias in column kIn when K > kIn),
// scaled by s, as split K-major core matrices [o][k]; 8 columns per chunk.
template <class Op, int K>
__device__ __forceinline__ void load_w1(const float* __restrict__ params, uint8_t* hi, uint8_t* lo, uint32_t sbo,
                                        float s) {
  constexpr int kB = K / 8, kChunks = kHid * kB;
  float dummy = 0.0f;
  for (int c0 = threadIdx.x; c0 < kChunks; c0 += 2 * blockDim.x) {
    float v[2][8];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int c = c0 + u * blockDim.x, o = c / kB, k8 = (c % kB) * 8;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k8 + i;
        v[u][i] = c >= kChunks ? 0.0f
                               : (k < kIn ? __ldg(params + kOffW1 + o * kIn + k)
                                          : (k == kIn ? __ldg(params + kOffB1 + o) : 0.0f));
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int c = c0 + u * blockDim.x;
      if (c < kChunks) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[u][i] *= s;
        st_split8<Op, true>(hi, lo, c / kB, (c % kB) * 8, sbo, v[u], dummy);
      }
    }
  }
}

// W2 (scaled by s) as split K-major core matrices [o][i]; 8 columns per chunk.
template <class Op>
__device__ __forceinline__ void load_w2(const float* __restrict__ params, uint8_t* hi, uint8_t* lo, float s) {
  const float* w = params + kOffW2;
  float dummy = 0.0f;
  if ((reinterpret_cast<uintptr_t>(w) & 15u) != 0) {
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x)
      st_split1<Op>(hi, lo, tc::cm_off(e / kHid, e % kHid, kSboH), s * __ldg(w + e));
    return;
  }
  constexpr int kChunks = kHid * kHid / 8;
  for (int c0 = threadIdx.x; c0 < kChunks; c0 += 4 * blockDim.x) {
    float4 a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u * blockDim.x;
      if (c < kChunks) {
        a[u] = __ldg(reinterpret_cast<const float4*>(w + 8 * c));
        b[u] = __ldg(reinterpret_cast<const float4*>(w + 8 * c + 4));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u * blockDim.x;
      if (c < kChunks) {
        float v[8] = {s * a[u].x, s * a[u].y, s * a[u].z, s * a[u].w,
                      s * b[u].x, s * b[u].y, s * b[u].z, s * b[u].w};
        st_split8<Op, true>(hi, lo, c >> 4, (c & 15) * 8, kSboH, v, dummy);
      }
    }
  }
}

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_mlp_tc_status, 0, code); }

}  // namespace x3

using namespace x3;

// ------------------------------------------------------------------ forward
// Row inputs of the forward: the next tile's inputs are loaded in three
// dependent steps spread over the current tile (list index; feature row and
// ray id; direction), so their latency hides behind other work.
struct RowIn {
  int64_t s;       // sample index (-1 past the list end)
  int32_t r;       // ray id
  float k0[kFeat];
  float d[3];
};

__device__ __forceinline__ void row_in_l1(RowIn& in, const int32_t* __restrict__ idx, int64_t j, int64_t n) {
  in.s = j < n ? (idx ? (int64_t)__ldg(idx + j) : j) : -1;
}
__device__ __forceinline__ void row_in_l2(RowIn& in, const float* __restrict__ k0,
                                          const int32_t* __restrict__ ray_id, bool want_k0) {
  if (in.s < 0) return;
  if (want_k0) {
    const float4* kp = reinterpret_cast<const float4*>(k0 + in.s * kFeat);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 v = __ldg(kp + q);
      in.k0[4 * q] = v.x;
      in.k0[4 * q + 1] = v.y;
      in.k0[4 * q + 2] = v.z;
      in.k0[4 * q + 3] = v.w;
    }
  }
  in.r = __ldg(ray_id + in.s);
}
__device__ __forceinline__ void row_in_l3(RowIn& in, const float* __restrict__ rays_d) {
  if (in.s < 0) return;
#pragma unroll
  for (int a = 0; a < 3; ++a) in.d[a] = __ldg(rays_d + 3 * (int64_t)in.r + a);
}

// Input k-blocks (8 columns each) of warp quarter q: q0 blocks 0-1, q1 block
// 2, q2 block 3, q3 blocks 4-5 (the transcendental work is spread evenly).
__device__ __forceinline__ int x_first_block(int q) { return q == 0 ? 0 : (q == 3 ? 4 : q + 1); }
__device__ __forceinline__ int x_num_blocks(int q) { return (q == 0 || q == 3) ? 2 : 1; }

// Those columns of the input row [k0 (12), d (3), sin(2^f d_a) (a major, f
// inner; p = 4 a + f), cos(2^f d_a), 1, 0 ...] from loaded values; rows past
// the list end are zero.
__device__ __forceinline__ void quarter_x(const RowIn& in, int q, float v[16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = 0.0f;
  if (in.s < 0) return;
  auto arg = [&](int p) { return in.d[p >> 2] * (float)(1 << (p & 3)); };
  if (q == 0) {
#pragma unroll
    for (int k = 0; k < kFeat; ++k) v[k] = in.k0[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[kFeat + a] = in.d[a];
    v[15] = sinf(arg(0));
  } else if (q == 1) {
#pragma unroll
    for (int p = 1; p <= 8; ++p) v[p - 1] = sinf(arg(p));
  } else if (q == 2) {
#pragma unroll
    for (int p = 9; p <= 11; ++p) v[p - 9] = sinf(arg(p));
#pragma unroll
    for (int p = 0; p <= 4; ++p) v[3 + p] = cosf(arg(p));
  } else {
#pragma unroll
    for (int p = 5; p <= 11; ++p) v[p - 5] = cosf(arg(p));
    v[7] = 1.0f;
  }
}

// Column c (0..7) of quarter q (1..3) of the input row for a ray with
// direction d: q1 sin p = c + 1; q2 sin p = 9 + c (c < 3), cos p = c - 3;
// q3 cos p = 5 + c (c < 7), the constant 1 (c = 7); argument 2^f d_a, p = 4 a + f.
__device__ __forceinline__ float enc_col(int q, int c, float d0, float d1, float d2) {
  if (q == 3 && c == 7) return 1.0f;
  const bool is_cos = q == 3 || (q == 2 && c >= 3);
  const int p = q == 1 ? c + 1 : (q == 2 ? (c < 3 ? 9 + c : c - 3) : 5 + c);
  const float da = (p >> 2) == 0 ? d0 : ((p >> 2) == 1 ? d1 : d2);
  float sv, cv;
  sincosf(da * (float)(1 << (p & 3)), &sv, &cv);
  return is_cos ? cv : sv;
}

// quarter_x for q = 1..3, with the direction encoding evaluated once per
// distinct ray of the warp's 32 rows (consecutive samples mostly share a ray):
// for up to 8 distinct rays, lane 8 j' + c evaluates column c of the j-th
// ray (4 rays per round) and each row collects its 8 columns by shuffles.
__device__ __forceinline__ void quarter_x_shared(const RowIn& in, int q, int lane, float v[16]) {
  const int key = in.s >= 0 ? in.r : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(peers) - 1;
  const unsigned leaders = __ballot_sync(0xffffffffu, lane == leader);
  const int nd = __popc(leaders);
  if (nd > 8) {   // warp-uniform
    quarter_x(in, q, v);
    return;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = 0.0f;
  const int rank = __popc(leaders & ((1u << leader) - 1u));
  for (int r0 = 0; r0 < nd; r0 += 4) {
    const int j = min(r0 + (lane >> 3), nd - 1), c = lane & 7;
    const int src = (int)__fns(leaders, 0, j + 1);
    const float d0 = __shfl_sync(0xffffffffu, in.d[0], src);
    const float d1 = __shfl_sync(0xffffffffu, in.d[1], src);
    const float d2 = __shfl_sync(0xffffffffu, in.d[2], src);
    const float val = enc_col(q, c, d0, d1, d2);
    const bool mine = rank >= r0 && rank < r0 + 4;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const float t = __shfl_sync(0xffffffffu, val, ((rank - r0) & 3) * 8 + cc);
      if (mine) v[cc] = t;
    }
  }
  if (in.s < 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.0f;
  }
}

// Forward shared memory: split W1 and W2 (resident), two X buffers, and the
// staging copy of a tile's split H1 for the image.
constexpr uint32_t gW1h = 0, gW1l = gW1h + kW1Bytes, gW2h = gW1l + kW1Bytes, gW2l = gW2h + kW2Bytes,
                   gX0 = gW2l + kW2Bytes, gXBuf = 2 * kXBytes, gStage = gX0 + 2 * gXBuf,
                   gEnd = gStage + 2 * kHBytes;

struct FwdSide {
  float4 ob[kHid];   // per hidden unit o: (b2[o], W3[0][o], W3[1][o], W3[2][o])
  float b3[4];
  float red[32];         // block_max scratch: one entry per warp (17 warps)
  uint64_t x_full[2];    // X of the tile in buffer b written (16 warp arrivals)
  uint64_t l1_full[2];   // layer-1 MMAs of buffer b done (X buffer b free again)
  uint64_t h1_full[2];   // H1 of buffer b stored in tensor memory (16 warp arrivals)
  uint64_t l2_full[2];   // layer-2 MMAs of buffer b done
  uint64_t fin;          // every MMA of the kernel done
  uint32_t tmem_slot;
  int abort;             // a wait gave up: later waits return at once
};
static_assert(gEnd + sizeof(FwdSide) + 2 * 4 * kTile * kOut * sizeof(float) <= 227 * 1024,
              "forward shared memory");

// Bounded wait shared by all roles of the forward; after the first timeout
// every later wait returns false immediately, so that all threads still
// reach the same barriers and the kernel ends.
__device__ __forceinline__ bool fwd_wait(FwdSide* fs, uint64_t* bar, uint32_t parity) {
  if (*reinterpret_cast<volatile int*>(&fs->abort)) return false;
  if (tc::mbar_wait(bar, parity, kSpin)) return true;
  *reinterpret_cast<volatile int*>(&fs->abort) = 1;
  set_status(DVGO_ERR_TIMEOUT);
  return false;
}

// 544 threads.  Warps 0-15 compute (warp w: TMEM lane quarter w & 3 = tile
// rows 32 (w & 3) .. + 31, column quarter w / 4 = hidden columns 32 (w / 4)
// .. + 31 and a quarter of the input columns); warp 16 issues the MMAs, so
// that the tensor core runs while the compute warps work on other tiles.
// Two tiles are in flight, in tensor-memory buffers b = 0, 1 of 256 columns:
// columns 0-127 take D1 and then, in place, H1 split into FP16 hi / lo (the
// A operand of layer 2, read from tensor memory), columns 128-255 take D2.
// Column quarter q of H1 sits in columns 32 q .. 32 q + 31 of the buffer:
// hi terms of k = 32 q .. 32 q + 31 packed two per column in the first 16,
// lo terms in the next 16 (so each thread overwrites only the D1 columns it
// has read).  X (the layer-1 A operand) is double-buffered in shared memory.
// The tile image in the act buffer (the layout the backward loads) is written
// by bulk copies that the MMA warp issues: X from its buffer, H1 from a
// shared-memory staging copy that the compute warps fill beside the TMEM one.
// Before the layer-1 MMAs of tile k are committed the MMA thread waits until
// those copies have read their sources, so l1_full(k) also tells the compute
// warps that the staging area and X buffer k & 1 may be rewritten.
//
// Order per tile k of this CTA (b = k & 1):
//   compute: wait l1_full(k) -> H1(k) into TMEM and the image -> arrive
//            h1_full(k); write X(k + 1) -> arrive x_full(k + 1); wait
//            l2_full(k - 1) -> output layer and sigmoid of tile k - 1.
//   MMA:     wait h1_full(k - 1) -> layer 2 of k - 1 -> commit l2_full(k - 1);
//            wait x_full(k) (and l2_full(k - 2): buffer b's H1 read) -> layer 1
//            of k -> commit l1_full(k).
template <class Op>
__global__ void __launch_bounds__(544, 1) rgbnet_fwd_tc_kernel(
    const float* __restrict__ k0, const float* __restrict__ rays_d, const int32_t* __restrict__ ray_id,
    const int32_t* __restrict__ idx, int64_t n_cap, const int64_t* __restrict__ n_dev,
    const float* __restrict__ params, float* __restrict__ rgb, uint8_t* __restrict__ act) {
  extern __shared__ __align__(1024) uint8_t sm[];
  FwdSide* fs = reinterpret_cast<FwdSide*>(sm + gEnd);
  float* zx_all = reinterpret_cast<float*>(sm + gEnd + sizeof(FwdSide));  // [2][4][128][3]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lq = warp & 3, qw = warp >> 2, row = lq * 32 + lane;   // compute warps
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t nt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // the first tile's row inputs are fetched while the weights are prepared
  RowIn in;
  if (warp < 16 && nt > 0) row_in_l1(in, idx, (int64_t)blockIdx.x * kTile + row, n);
  if (warp == 0) tc::tmem_alloc(&fs->tmem_slot, 512);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&fs->x_full[b], 16);
      tc::mbar_init(&fs->l1_full[b], 1);
      tc::mbar_init(&fs->h1_full[b], 16);
      tc::mbar_init(&fs->l2_full[b], 1);
    }
    tc::mbar_init(&fs->fin, 1);
    fs->abort = 0;
  }
  // weights: W1 | b1 (column 39) and W2, split, each with its own scale
  const float m1 = abs_max_part(params + kOffW1, kHid * kIn + kHid);
  const float m2 = abs_max_part(params + kOffW2, kHid * kHid);
  const float sW1 = pow2_scale(block_max(m1, fs->red));
  const float sW2 = pow2_scale(block_max(m2, fs->red));
  if (warp < 16 && nt > 0) row_in_l2(in, k0, ray_id, qw == 0);
  load_w1<Op, kK1>(params, sm + gW1h, sm + gW1l, kSboX, sW1);
  load_w2<Op>(params, sm + gW2h, sm + gW2l, sW2);
  load_out_layer<Op>(params, fs);
  if (warp < 16 && nt > 0) row_in_l3(in, rays_d);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  uint8_t* act_img = act + kActHeader;
  float vmax = 0.0f;
  auto tile_of = [&](int64_t k) { return (int64_t)blockIdx.x + k * (int64_t)gridDim.x; };

  if (warp == 16) {
    // ------------------------------------------------------------ MMA warp
    const uint32_t id128 = Op::idesc(128, kHid, 0, 0);
    const uint32_t sW1h = tc::smem_u32(sm + gW1h), sW1l = tc::smem_u32(sm + gW1l);
    const uint32_t sW2h = tc::smem_u32(sm + gW2h), sW2l = tc::smem_u32(sm + gW2l);
    // lane 0 polls; the outcome is the warp's
    auto wait0 = [&](uint64_t* bar, uint32_t parity) -> bool {
      int r = 0;
      if (lane == 0) r = fwd_wait(fs, bar, parity) ? 1 : 0;
      return __shfl_sync(0xffffffffu, r, 0) != 0;
    };
    auto layer2 = [&](int64_t k) {
      const uint32_t b = (uint32_t)(k & 1), buf = tmem + 256u * b;
      if (!wait0(&fs->h1_full[b], (uint32_t)(k >> 1) & 1u)) return;
      tc::fence_after_sync();
      if (lane == 0) {
        tc::bulk_s2g(act_img + (size_t)tile_of(k) * kImage + iHh, sm + gStage, 2 * kHBytes);
        mma3_ts<Op::kWeightLo>(buf + 128u, buf, sW2h, sW2l, 256, 128, kSboH, kHid / 16, id128, false);
        tc::mma_commit(&fs->l2_full[b]);
      }
      __syncwarp();
    };
    auto layer1 = [&](int64_t k) {
      const uint32_t b = (uint32_t)(k & 1), buf = tmem + 256u * b;
      if (!wait0(&fs->x_full[b], (uint32_t)(k >> 1) & 1u)) return;
      // buffer b's H1 (tile k - 2) has been read by its layer-2 MMAs
      if (k >= 2 && !wait0(&fs->l2_full[b], (uint32_t)((k - 2) >> 1) & 1u)) return;
      tc::fence_after_sync();
      if (lane == 0) {
        uint8_t* xb = sm + gX0 + b * gXBuf;
        tc::bulk_wait_read();   // staging (H1 of k - 1) and X buffer b's older copy are read
        tc::bulk_s2g(act_img + (size_t)tile_of(k) * kImage + iX, xb, 2 * kXBytes);
        const uint32_t xs = tc::smem_u32(xb);
        mma3<true, Op::kWeightLo>(buf, xs, xs + kSboX, 256, 128, kSboXs, sW1h, sW1l, 256, 128, kSboX,
                                  kK1 / 16, id128, false);
        tc::mma_commit(&fs->l1_full[b]);
      }
      __syncwarp();
    };
    // issue order: L1(0), then per k: L2(k - 1) as soon as H1(k - 1) is in, L1(k)
    if (nt > 0) layer1(0);
    for (int64_t k = 1; k < nt; ++k) {
      layer2(k - 1);
      layer1(k);
    }
    if (nt > 0) layer2(nt - 1);
    // every MMA and copy this thread issued has finished before the memory is released
    if (lane == 0) {
      tc::mma_commit(&fs->fin);
      tc::mbar_wait(&fs->fin, 0, kSpin);
      tc::bulk_wait_all();
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------- compute warps
    const uint32_t lane_off = (uint32_t)(lq * 32) << 16;
    const float inv1 = kSH / (kSX * sW1), inv2 = 1.0f / (kSH * sW2);
    const int fb = x_first_block(qw), nb = x_num_blocks(qw);
    auto load_rows = [&](int64_t k) {
      row_in_l1(in, idx, tile_of(k) * kTile + row, n);
      row_in_l2(in, k0, ray_id, qw == 0);
      row_in_l3(in, rays_d);
    };
    // X of tile k (rows loaded in `in`) into buffer k & 1 and the image
    auto write_x = [&](int64_t k) {
      float x[16];
      if (qw == 0)
        quarter_x(in, 0, x);
      else
        quarter_x_shared(in, qw, lane, x);
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] *= kSX;
      uint8_t* xs = sm + gX0 + (k & 1) * gXBuf;
      st_split8<Op, false>(xs, xs + kSboX, row, fb * 8, kSboXs, x, vmax);
      if (nb == 2) st_split8<Op, false>(xs, xs + kSboX, row, fb * 8 + 8, kSboXs, x + 8, vmax);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&fs->x_full[k & 1]);
    };
    // H1 of tile k: relu(D1) scaled, split, into TMEM (in place) and the staging area
    auto layer1_out = [&](int64_t k) {
      const uint32_t b = (uint32_t)(k & 1);
      const uint32_t taddr = tmem + 256u * b + lane_off + 32u * qw;
      fwd_wait(fs, &fs->l1_full[b], (uint32_t)(k >> 1) & 1u);
      tc::fence_after_sync();
      uint32_t hl[32];
      {
        float v[32];
        tc::tmem_ld32(taddr, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float a = fmaxf(v[2 * c] * inv1, 0.0f), bb = fmaxf(v[2 * c + 1] * inv1, 0.0f);
          vmax = fmaxf(vmax, fmaxf(a, bb));
          hl[c] = Op::split2(a, bb, hl[16 + c]);
        }
      }
      tc::tmem_st32(taddr, hl);
      uint8_t* st = sm + gStage;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t off = tc::cm_off(row, 32 * qw + 8 * q, kSboH);
        *reinterpret_cast<uint4*>(st + off) = make_uint4(hl[4 * q], hl[4 * q + 1], hl[4 * q + 2], hl[4 * q + 3]);
        *reinterpret_cast<uint4*>(st + kHBytes + off) =
            make_uint4(hl[16 + 4 * q], hl[17 + 4 * q], hl[18 + 4 * q], hl[19 + 4 * q]);
      }
      tc::fence_proxy_async_smem();
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&fs->h1_full[b]);
    };
    // output layer and sigmoid of tile k (sample index s of this row)
    auto layer2_out = [&](int64_t k, int64_t s) {
      const uint32_t b = (uint32_t)(k & 1);
      fwd_wait(fs, &fs->l2_full[b], (uint32_t)(k >> 1) & 1u);
      tc::fence_after_sync();
      float z3[kOut] = {0.0f, 0.0f, 0.0f};
      {
        float v[32];
        tc::tmem_ld32(tmem + 256u * b + 128u + lane_off + 32u * qw, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float4 q = fs->ob[32 * qw + i];
          const float h = fmaxf(fmaf(v[i], inv2, q.x), 0.0f);
          z3[0] = fmaf(q.y, h, z3[0]);
          z3[1] = fmaf(q.z, h, z3[1]);
          z3[2] = fmaf(q.w, h, z3[2]);
        }
      }
      float* zx = zx_all + b * (4 * kTile * kOut);
#pragma unroll
      for (int c = 0; c < kOut; ++c) zx[(qw * kTile + row) * kOut + c] = z3[c];
      tc::named_sync(1 + lq, 128);
      if (qw < kOut && s >= 0) {   // quarter qw finishes output channel qw
        const float* zc = zx + row * kOut + qw;
        const float z = ((zc[0] + zc[kTile * kOut]) + zc[2 * kTile * kOut]) + zc[3 * kTile * kOut];
        rgb[3 * s + qw] = sigmoid_f(fs->b3[qw] + z);
      }
    };
    auto idx_of = [&](int64_t k) -> int64_t {
      const int64_t j = tile_of(k) * kTile + row;
      return j < n ? (idx ? (int64_t)__ldg(idx + j) : j) : -1;
    };
    // Per tile k: H1(k); X(k + 1); output layer of k - 1.  The three dependent
    // loads of a tile's rows (list index; feature row and ray id; direction)
    // are spread over the two iterations before its X is written.
    int64_t s_prev = -1, s_cur = -1, s_nn = -1;   // this row's sample in tiles k - 1, k, k + 2
    if (nt > 0) {
      write_x(0);
      s_cur = in.s;
      if (nt > 1) load_rows(1);
      if (nt > 2) s_nn = idx_of(2);
    }
    for (int64_t k = 0; k < nt; ++k) {
      layer1_out(k);
      int64_t s_next = -1;
      if (k + 1 < nt) {
        write_x(k + 1);
        s_next = in.s;
      }
      if (k + 2 < nt) {
        in.s = s_nn;
        row_in_l2(in, k0, ray_id, qw == 0);
      }
      if (k >= 1) layer2_out(k - 1, s_prev);
      if (k + 2 < nt) row_in_l3(in, rays_d);
      if (k + 3 < nt) s_nn = idx_of(k + 3);
      s_prev = s_cur;
      s_cur = s_next;
    }
    if (nt > 0) layer2_out(nt - 1, s_prev);
    __syncwarp();
  }
  if (vmax >= Op::kMaxScaled) set_status(DVGO_ERR_RANGE);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ----------------------------------------------------------------- backward
// 544 threads.  Warps 0-15 compute: warp w covers TMEM lane quarter w & 3
// and column quarter q = w / 4.  In the products with the tile rows on the
// TMEM lanes (g_h1, g_X) a thread holds row 32 (w & 3) + lane and hidden
// columns 32 q .. + 31; in the transposed layer 2 (D2^T) it holds hidden unit
// 32 (w & 3) + lane and tile rows 32 q .. + 31.  Warp 16 issues the MMAs and
// the X copies, so that the tensor core runs while the compute warps work:
// dW2 first (its completion frees H1's buffer for the next tile's copy),
// then g_h1, then the next tile's D2^T as soon as its H1 has landed, then
// this tile's g_X and dW1 once G1 is in.
//
// Order per tile t of this CTA (tn = the next one):
//   compute: wait h_full(t) -> row scales, relu mask (reads H1(t)); wait
//            d2(t) -> G2 epilogue; wait gx(t - 1) -> G2 into shared memory,
//            g_X(t - 1) -> g_k0; arrive g2_full(t).  Thread 0: wait dw2(t)
//            -> copy H1(tn) in.  Wait gh(t) -> G1 epilogue; arrive
//            g1_full(t).
//   MMA:     wait gx(t - 1) -> copy X(t) in; wait g2_full(t) -> dW2(t),
//            commit dw2; g_h1(t), commit gh; wait h_full(tn) -> D2^T(tn),
//            commit d2; wait g1_full(t) and X(t) -> g_X(t) and dW1(t),
//            commit gx.
// A tensor-memory column range or shared buffer is rewritten only after the
// barrier that follows its last reader.  The G2 and G1 split terms in tensor
// memory use 16-column chunks (mma3_ts16), so that each epilogue runs in two
// halves of 16 columns and rewrites only columns it has already read.  The
// upstream colour gradient of the next tile is loaded in three dependent
// steps over the current tile.
struct UpIn {
  int64_t s;       // sample index (-1 past the list end)
  int32_t r;
  float ws;
  float g[kOut];   // the upstream colour gradient, then (up_l3) g_z3
};

__device__ __forceinline__ void up_l1(UpIn& u, const int32_t* __restrict__ idx, int64_t j, int64_t n) {
  u.s = j < n ? (idx ? (int64_t)__ldg(idx + j) : j) : -1;
}
__device__ __forceinline__ void up_l2(UpIn& u, const float* __restrict__ g_rgb, const float* __restrict__ w,
                                      const int32_t* __restrict__ ray_id) {
  if (u.s < 0) return;
  if (g_rgb) {
#pragma unroll
    for (int c = 0; c < kOut; ++c) u.g[c] = __ldg(g_rgb + 3 * u.s + c);
  } else {
    u.ws = __ldg(w + u.s);
    u.r = __ldg(ray_id + u.s);
  }
}
// g_z3 = g_rgb * y (1 - y) with y = rgb[s], the forward's sigmoid output.
__device__ __forceinline__ void up_l3(UpIn& u, const float* __restrict__ g_rgb,
                                      const float* __restrict__ g_color, const float* __restrict__ rgb) {
  if (u.s < 0) return;
  float y[kOut];
#pragma unroll
  for (int c = 0; c < kOut; ++c) y[c] = __ldg(rgb + 3 * u.s + c);
  if (!g_rgb) {
#pragma unroll
    for (int c = 0; c < kOut; ++c) u.g[c] = u.ws * __ldg(g_color + 3 * (int64_t)u.r + c);
  }
#pragma unroll
  for (int c = 0; c < kOut; ++c) u.g[c] = u.g[c] * y[c] * (1.0f - y[c]);
}

// Bounded wait of the backward; after the first timeout every later wait
// returns false at once, so that both roles still reach the kernel's end.
__device__ __forceinline__ bool bwd_wait(Side* fs, uint64_t* bar, uint32_t parity) {
  if (*reinterpret_cast<volatile int*>(&fs->abort)) return false;
  if (tc::mbar_wait(bar, parity, kSpin)) return true;
  *reinterpret_cast<volatile int*>(&fs->abort) = 1;
  set_status(DVGO_ERR_TIMEOUT);
  return false;
}

template <class Op>
__global__ void __launch_bounds__(544, 1) rgbnet_bwd_tc_kernel(
    const float* __restrict__ g_rgb, const float* __restrict__ g_color, const float* __restrict__ w,
    const float* __restrict__ rgb, const int32_t* __restrict__ ray_id, const int32_t* __restrict__ idx,
    int64_t n_cap, const int64_t* __restrict__ n_dev, const float* __restrict__ params,
    const uint8_t* __restrict__ act, float* __restrict__ part, float* __restrict__ g_k0) {
  extern __shared__ __align__(1024) uint8_t sm[];
  Side* fs = reinterpret_cast<Side*>(sm + bEnd);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qw = (warp >> 2) & 3, row = (warp & 3) * 32 + lane;
  const bool compute = warp < 16;
  const int64_t n = mlp_count(n_cap, n_dev);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t nt = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto tile_of = [&](int64_t k) { return (int64_t)blockIdx.x + k * (int64_t)gridDim.x; };
  const uint8_t* img_g = act + kActHeader;
  uint8_t* img = sm + bImg;
  if (warp == 0) tc::tmem_alloc(&fs->tmem_slot, 512);
  if (tid == 0) {
    tc::mbar_init(&fs->bar_h, 1);
    tc::mbar_init(&fs->bar_x, 1);
    tc::mbar_init(&fs->bar_d2, 1);
    tc::mbar_init(&fs->bar_gh, 1);
    tc::mbar_init(&fs->bar_dw2, 1);
    tc::mbar_init(&fs->bar_gx, 1);
    tc::mbar_init(&fs->bar_fin, 1);
    tc::mbar_init(&fs->g2_full, 16);
    tc::mbar_init(&fs->g1_full, 16);
    fs->abort = 0;
    // the first image is fetched while the weights are prepared
    if (nt > 0) {
      tc::mbar_arrive_expect_tx(&fs->bar_h, 2 * kHBytes);
      tc::bulk_g2s(img + iHh, img_g + (size_t)tile_of(0) * kImage + iHh, 2 * kHBytes, &fs->bar_h);
      tc::mbar_arrive_expect_tx(&fs->bar_x, 2 * kXBytes);
      tc::bulk_g2s(img + iX, img_g + (size_t)tile_of(0) * kImage + iX, 2 * kXBytes, &fs->bar_x);
    }
  }
  UpIn cur, nxt;
  if (compute) up_l1(cur, idx, tile_of(0) * kTile + row, n);
  // scales: W2 and W1[:, 0:16] per matrix; G2 from the upstream bound, G1 from G2's
  float m1 = 0.0f, m3 = 0.0f;
#pragma unroll 4
  for (int e = tid; e < kHid * 16; e += blockDim.x)
    m1 = fmaxf(m1, fabsf(__ldg(params + kOffW1 + (e >> 4) * kIn + (e & 15))));
  const float m2 = abs_max_part(params + kOffW2, kHid * kHid);
  for (int o = tid; o < kHid; o += blockDim.x) {
    float a = 0.0f;
#pragma unroll
    for (int c = 0; c < kOut; ++c) a += fabsf(params[kOffW3 + c * kHid + o]);
    m3 = fmaxf(m3, a);
  }
  const float mw1 = block_max(m1, fs->red);
  const float mw2 = block_max(m2, fs->red);
  const float mw3 = block_max(m3, fs->red);
  const float sW1 = pow2_scale(mw1), sW2 = pow2_scale(mw2);
  // Largest upstream colour gradient over this CTA's own tiles.  S2 and S1
  // need only be uniform within the CTA: its partial gradient row carries
  // its own scale.
  float gm = 0.0f;
  {
    const int64_t cnt = nt * kTile;
    for (int64_t e0 = tid; e0 < cnt; e0 += 4 * (int64_t)blockDim.x) {
      int64_t sv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t e = e0 + u * (int64_t)blockDim.x;
        const int64_t j = tile_of(e / kTile) * kTile + e % kTile;
        sv[u] = (e < cnt && j < n) ? (idx ? (int64_t)__ldg(idx + j) : j) : -1;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (sv[u] < 0) continue;
        float g[kOut];
        upstream_rgb_grad(g_rgb, g_color, w, ray_id, sv[u], g);
        gm = fmaxf(gm, fmaxf(fabsf(g[0]), fmaxf(fabsf(g[1]), fabsf(g[2]))));
      }
    }
  }
  const float gmax = block_max(gm, fs->red);
  // |g_z2[s]| <= max_o sum_c |W3[c][o]| * max_c |g_z3[s][c]| and g_z3 <= g_rgb / 4;
  // |g_h1[s]| <= 128 max|W2| max|g_z2[s]|.  S2 / S1: the scales of the largest bounds.
  const float w21 = mw2 * (float)kHid;
  const float S2 = pow2_scale(0.25f * gmax * mw3);
  const float S1 = pow2_scale(0.25f * gmax * mw3 * w21);
  if (compute) up_l2(cur, g_rgb, w, ray_id);
  // W1[:, 0:16] split, hi and lo core matrices side by side in each 8-row
  // group, so that [hi | lo] is one 32-wide B operand of g_X = G1 W1[:, 0:16]
  load_w1<Op, 16>(params, sm + bW1h, sm + bW1h + 256, kSboW1s, sW1);
  load_w2<Op>(params, sm + bW2h, sm + bW2l, sW2);
  if (compute) up_l3(cur, g_rgb, g_color, rgb);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = fs->tmem_slot;
  const uint32_t sW1h = tc::smem_u32(sm + bW1h);
  const uint32_t sW2h = tc::smem_u32(sm + bW2h), sW2l = tc::smem_u32(sm + bW2l);
  const uint32_t sX = tc::smem_u32(img + iX);
  const uint32_t sHh = tc::smem_u32(img + iHh), sHl = tc::smem_u32(img + iHl);
  const uint32_t sGh = tc::smem_u32(sm + bGh), sGl = tc::smem_u32(sm + bGl);
  float vmax = 0.0f;   // largest magnitude split (range check)
  // per-thread partial sums of dW3, db2 (hidden unit oh) and db3 (tile row)
  float dW3acc[kOut] = {0.0f, 0.0f, 0.0f}, db2acc = 0.0f, db3acc[kOut] = {0.0f, 0.0f, 0.0f};
  if (warp == 16) {
    // ------------------------------------------------------------ MMA warp
    // lane 0 polls and issues; the outcome of a wait is the warp's
    auto wait0 = [&](uint64_t* bar, uint32_t parity) -> bool {
      int r = 0;
      if (lane == 0) r = bwd_wait(fs, bar, parity) ? 1 : 0;
      return __shfl_sync(0xffffffffu, r, 0) != 0;
    };
    bool inflight_x = nt > 0;   // lane 0: an X copy not yet seen landed
    uint32_t ph_h = 0, ph_x = 0, ph_gx = 0, ph_g2 = 0, ph_g1 = 0;
    auto load_x = [&](int64_t k) {
      tc::mbar_arrive_expect_tx(&fs->bar_x, 2 * kXBytes);
      tc::bulk_g2s(img + iX, img_g + (size_t)tile_of(k) * kImage + iX, 2 * kXBytes, &fs->bar_x);
      inflight_x = true;
    };
    // D2^T = W2 H1^T of the tile whose H1 terms have landed (TMEM lane =
    // hidden unit, column = tile row); after a failed wait only the commit
    auto d2 = [&](bool h_ok) {
      if (h_ok) {
        mma3<Op::kWeightLo, true>(tmem + cTmp, sW2h, sW2l, 256, 128, kSboH, sHh, sHl, 256, 128, kSboH,
                                  kHid / 16, Op::idesc(128, kTile, 0, 0), false);
      }
      tc::mma_commit(&fs->bar_d2);
    };
    if (nt > 0) {
      const bool h_ok = wait0(&fs->bar_h, ph_h);
      ph_h ^= 1;
      tc::fence_after_sync();
      if (lane == 0) d2(h_ok);
      __syncwarp();
    }
    for (int64_t k = 0; k < nt; ++k) {
      const bool has_next = k + 1 < nt;
      // X(k): the buffer is free once g_X and dW1 of tile k - 1 are done
      if (k > 0) {
        if (wait0(&fs->bar_gx, ph_gx) && lane == 0) load_x(k);
        ph_gx ^= 1;
      }
      // dW2 += G2^T H1 (A from tensor memory), then g_h1 = G2 W2 (A MN-major)
      const bool g2 = wait0(&fs->g2_full, ph_g2);
      ph_g2 ^= 1;
      tc::fence_after_sync();
      if (lane == 0) {
        if (g2)
          mma3_ts16(tmem + cDW2, tmem + cTmp, sHh, sHl, 2 * kSboH, kSboH, 128, kTile / 16,
                    Op::idesc(128, kHid, 0, 1), k > 0);
        tc::mma_commit(&fs->bar_dw2);
        if (g2)
          mma3<true, Op::kWeightLo>(tmem + cGH, sGh, sGl, 2 * kSboH, kSboH, 128, sW2h, sW2l, 2 * kSboH,
                                    kSboH, 128, kHid / 16, Op::idesc(128, kHid, 1, 1), false);
        tc::mma_commit(&fs->bar_gh);
      }
      __syncwarp();
      // the next tile's D2^T once its H1 has landed (compute thread 0 copies
      // it in when dW2 has read this one's); it needs no G1 of this tile
      if (has_next) {
        const bool h_ok = wait0(&fs->bar_h, ph_h);
        ph_h ^= 1;
        tc::fence_after_sync();
        if (lane == 0) d2(h_ok);
        __syncwarp();
      }
      // once G1 and X are in: g_X = G1 W1[:, 0:16] (A from tensor memory) and
      // dW1|db1 += G1^T X
      const bool g1 = wait0(&fs->g1_full, ph_g1);
      ph_g1 ^= 1;
      tc::fence_after_sync();
      if (lane == 0) {
        const bool x_ok = g1 && bwd_wait(fs, &fs->bar_x, ph_x);
        ph_x ^= 1;
        if (x_ok) {
          inflight_x = false;
          {   // per K step: G1h [W1h | W1l] (N = 32: hi*hi in columns 0-15, hi*lo in 16-31), G1l W1h
            const uint32_t id32 = Op::idesc(128, 32, 0, 1), id16 = Op::idesc(128, 16, 0, 1);
            uint64_t db = tc::smem_desc(sW1h, kSboW1s, 128);
#pragma unroll 1
            for (uint32_t j = 0; j < kHid / 16; ++j) {
              const uint32_t ah = tmem + cGH + 16u * j, al = ah + 8u;
              tc::mma_ts(tmem + cGX, ah, db, id32, j > 0 ? 1u : 0u);
              tc::mma_ts(tmem + cGX, al, db, id16, 1u);
              db += (2 * kSboW1s) >> 4;
            }
          }
          {   // per K step: G1h [Xh | Xl] (N = 96: hi*hi in columns 0-47, hi*lo in 48-95), G1l Xh
            const uint32_t id96 = Op::idesc(128, 2 * kK1, 1, 1), id48 = Op::idesc(128, kK1, 1, 1);
            uint64_t dah = tc::smem_desc(sGh, kSboH, 128), dal = tc::smem_desc(sGl, kSboH, 128);
            uint64_t dbx = tc::smem_desc(sX, kSboXs, 128);
#pragma unroll 1
            for (int kk = 0; kk < kTile / 16; ++kk) {
              tc::mma_bf16(tmem + cDW1, dah, dbx, id96, (k > 0 || kk > 0) ? 1u : 0u);
              tc::mma_bf16(tmem + cDW1, dal, dbx, id48, 1u);
              dah += (2 * kSboH) >> 4;
              dal += (2 * kSboH) >> 4;
              dbx += (2 * kSboXs) >> 4;
            }
          }
        }
        tc::mma_commit(&fs->bar_gx);
      }
      __syncwarp();
    }
    // every product has finished before the accumulators are read and the
    // tensor memory is released; a copy issued but never seen landed (only
    // after a failed wait) lands before exit
    if (lane == 0) {
      tc::mma_commit(&fs->bar_fin);
      if (!tc::mbar_wait(&fs->bar_fin, 0, kSpin)) {
        *reinterpret_cast<volatile int*>(&fs->abort) = 1;
        set_status(DVGO_ERR_TIMEOUT);
      }
      if (inflight_x) tc::mbar_wait(&fs->bar_x, ph_x, kSpin);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------- compute warps
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const float inv2 = 1.0f / (kSH * sW2);           // D2 -> z2 - b2
    // this thread's hidden unit in the transposed layer-2 products (TMEM lane)
    const int oh = (warp & 3) * 32 + lane;
    const float b2o = Op::param(__ldg(params + kOffB2 + oh)), w3o0 = Op::param(__ldg(params + kOffW3 + oh)),
                w3o1 = Op::param(__ldg(params + kOffW3 + kHid + oh)),
                w3o2 = Op::param(__ldg(params + kOffW3 + 2 * kHid + oh));
    uint32_t ph_h = 0, ph_d2 = 0, ph_gh = 0, ph_gx = 0, ph_dw2 = 0;
    bool inflight_h = tid == 0 && nt > 0;   // thread 0: an H1 copy not yet seen landed
    int64_t prev_s = -1;       // the previous tile's row: its g_X is stored one tile later
    float prev_invX = 0.0f;
    // g_X = G1 W1[:, 0:16] of the previous tile (lane quarter qw == 0) -> g_k0
    auto store_gx = [&]() {
      float ga[16], gb[16];
      tc::tmem_ld16(lane_base + cGX, ga);
      tc::tmem_ld16(lane_base + cGX + 16, gb);
      if (prev_s >= 0) {
        float4* dst = reinterpret_cast<float4*>(g_k0 + prev_s * kFeat);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          dst[q] = make_float4((ga[4 * q] + gb[4 * q]) * prev_invX, (ga[4 * q + 1] + gb[4 * q + 1]) * prev_invX,
                               (ga[4 * q + 2] + gb[4 * q + 2]) * prev_invX,
                               (ga[4 * q + 3] + gb[4 * q + 3]) * prev_invX);
      }
    };
    for (int64_t k = 0; k < nt; ++k) {
      const bool valid = cur.s >= 0;
      const int64_t s = cur.s;
      up_l1(nxt, idx, tile_of(k + 1) * kTile + row, n);
      // this tile's H1 terms (for the relu mask)
      if (bwd_wait(fs, &fs->bar_h, ph_h)) inflight_h = false;
      ph_h ^= 1;
      // g_z3 of this row's sample and its gradient scales (for g_h1 and g_X);
      // the weight-gradient products take the CTA-wide S2, S1 instead
      float fG1, invX, r1;
      {
        float gz3[kOut] = {0.0f, 0.0f, 0.0f};
        if (valid) {
#pragma unroll
          for (int c = 0; c < kOut; ++c) gz3[c] = cur.g[c];
        }
        const float b2s = mw3 * fmaxf(fabsf(gz3[0]), fmaxf(fabsf(gz3[1]), fabsf(gz3[2])));
        const float sG2 = b2s > 0.0f ? fmaxf(pow2_scale(b2s), S2) : S2;
        const float sG1 = b2s > 0.0f ? fmaxf(pow2_scale(b2s * w21), S1) : S1;
        fG1 = sG1 / (sG2 * sW2);             // (sG2 G2)(sW2 W2) -> sG1 g_h1
        invX = 1.0f / (sG1 * sW1);           // g_X
        r1 = S1 / sG1;                       // G1 terms -> the dW1 copy
        if (qw == 0) {
          fs->smp[row] = make_float4(gz3[0], gz3[1], gz3[2], sG2);
#pragma unroll
          for (int c = 0; c < kOut; ++c) db3acc[c] += gz3[c];
        }
      }
      // relu mask of layer 1 on this quarter's columns (H1 > 0 <=> hi > 0)
      uint32_t m1b = 0u;
#pragma unroll
      for (int k8 = 0; k8 < 32; k8 += 8) {
        const uint4 q = *reinterpret_cast<const uint4*>(img + iHh + tc::cm_off(row, 32 * qw + k8, kSboH));
        const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int kq = k8 + 2 * i;
          if ((int16_t)(wd[i] & 0xffffu) > 0) m1b |= 1u << kq;
          if ((int16_t)(wd[i] >> 16) > 0) m1b |= 1u << (kq + 1);
        }
      }
      up_l2(nxt, g_rgb, w, ray_id);
      tc::named_sync(1, 512);   // every row's g_z3 and scale are in fs->smp
      bwd_wait(fs, &fs->bar_d2, ph_d2);
      ph_d2 ^= 1;
      tc::fence_after_sync();
      // Hidden unit oh over the tile rows 32 qw .. 32 qw + 31 (two halves of
      // 16): G2 = (W3^T g_z3) * (z2 > 0), and the sums over rows dW3 +=
      // g_z3 h2^T, db2 += G2 in registers.  G2 goes out twice: at the
      // CTA-wide scale S2 into tensor memory over the half's own D2 columns
      // (lane = unit, K = row: the A operand of dW2), and at each row's own
      // scale sG2 into shared memory as [unit][row] core matrices (the
      // MN-major A operand of g_h1).
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int r0 = 32 * qw + 16 * h;
        float v[16];
        tc::tmem_ld16(lane_base + cTmp + r0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float4 q = fs->smp[r0 + i];
          const float z2 = fmaf(v[i], inv2, b2o);
          const float gs = fmaf(w3o2, q.z, fmaf(w3o1, q.y, w3o0 * q.x));
          const float g = z2 > 0.0f ? gs : 0.0f;
          const float hh = fmaxf(z2, 0.0f);
          db2acc += g;
          dW3acc[0] = fmaf(q.x, hh, dW3acc[0]);
          dW3acc[1] = fmaf(q.y, hh, dW3acc[1]);
          dW3acc[2] = fmaf(q.z, hh, dW3acc[2]);
          v[i] = g;
        }
        uint32_t hl[16];
        split16<Op>(v, S2, hl, vmax);
        tc::tmem_st16(lane_base + cTmp + r0, hl);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] *= fs->smp[r0 + i].w;
        split16<Op>(v, 1.0f, hl, vmax);
        // the previous tile's g_X and dW1 (readers of G's shared memory, X and
        // the g_X columns) are done
        if (h == 0 && k > 0) {
          bwd_wait(fs, &fs->bar_gx, ph_gx);
          ph_gx ^= 1;
          tc::fence_after_sync();
        }
        st_terms16<Op, false>(sm + bGh, sm + bGl, oh, r0, hl, 1.0f);
      }
      if (k > 0 && qw == 0) store_gx();
      tc::tmem_wait_st();
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&fs->g2_full);
      up_l3(nxt, g_rgb, g_color, rgb);
      // the next tile's H1 terms, once dW2 has read this tile's
      if (tid == 0 && k + 1 < nt) {
        if (bwd_wait(fs, &fs->bar_dw2, ph_dw2)) {
          tc::mbar_arrive_expect_tx(&fs->bar_h, 2 * kHBytes);
          tc::bulk_g2s(img + iHh, img_g + (size_t)tile_of(k + 1) * kImage + iHh, 2 * kHBytes, &fs->bar_h);
          inflight_h = true;
        }
        ph_dw2 ^= 1;
      }
      bwd_wait(fs, &fs->bar_gh, ph_gh);
      ph_gh ^= 1;
      tc::fence_after_sync();
      // G1 = g_h1 * (H1 > 0): at S1 in shared memory (dW1), at sG1 in tensor
      // memory (g_X), in two halves of 16 hidden units
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int c0 = 32 * qw + 16 * h;
        float v[16];
        tc::tmem_ld16(lane_base + cGH + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = ((m1b >> (16 * h + i)) & 1u) ? v[i] : 0.0f;
        uint32_t hl[16];
        split16<Op>(v, fG1, hl, vmax);
        tc::tmem_st16(lane_base + cGH + c0, hl);
        st_terms16<Op>(sm + bGh, sm + bGl, row, c0, hl, r1);
      }
      tc::tmem_wait_st();
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&fs->g1_full);
      prev_s = valid ? s : -1;
      prev_invX = invX;
      cur = nxt;
    }
    // the last tile's g_X
    if (nt > 0) {
      bwd_wait(fs, &fs->bar_gx, ph_gx);
      tc::fence_after_sync();
      if (qw == 0) store_gx();
    }
    // a copy issued but never seen landed (only after a failed wait) lands before exit
    if (inflight_h) tc::mbar_wait(&fs->bar_h, ph_h, kSpin);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = !*reinterpret_cast<volatile int*>(&fs->abort);
  if (vmax >= Op::kMaxScaled) set_status(DVGO_ERR_RANGE);
  // This CTA's gradient goes to its own row of the partials array (every
  // parameter written, no atomics); a second kernel sums the rows in a fixed
  // order.  Output-layer and b2 sums of the four lane quarters meet in shared
  // memory first (the G and image buffers are free now).
  float* pr = reinterpret_cast<float*>(sm + bGh);            // [16 warps][4][32]
  float* pr3 = pr + 16 * 4 * 32;                             // [4 lane quarters][3]
  if (compute) {
#pragma unroll
    for (int c = 0; c < kOut; ++c) pr[(warp * 4 + c) * 32 + lane] = dW3acc[c];
    pr[(warp * 4 + 3) * 32 + lane] = db2acc;
  }
  if (compute && qw == 0) {
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
      float v = db3acc[c];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) pr3[(warp & 3) * kOut + c] = v;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  float* P = part + (size_t)blockIdx.x * kNumParams;
  const bool has_tiles = (int64_t)blockIdx.x < ntiles;
  if (has_tiles && compute && qw == 0) {   // warp l: W3[:, 32 l + lane] and b2[32 l + lane] over the 4 row quarters
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float v = ((pr[((warp + 0) * 4 + c) * 32 + lane] + pr[((warp + 4) * 4 + c) * 32 + lane]) +
                       pr[((warp + 8) * 4 + c) * 32 + lane]) + pr[((warp + 12) * 4 + c) * 32 + lane];
      P[(c < kOut ? kOffW3 + c * kHid : kOffB2) + 32 * warp + lane] = v;
    }
  }
  if (has_tiles && tid < kOut) P[kOffB3 + tid] = ((pr3[tid] + pr3[kOut + tid]) + pr3[2 * kOut + tid]) + pr3[3 * kOut + tid];
  if (has_tiles && compute) {
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    // dW2 / dW1 rows (TMEM lane = output neuron) through a per-warp 32 x 33
    // shared-memory transpose, so that each store covers 32 consecutive
    // parameters of one row
    float* tp = reinterpret_cast<float*>(sm + bImg) + warp * 32 * 33;
    const float u2 = ok ? 1.0f / (S2 * kSH) : 0.0f, u1 = ok ? 1.0f / (S1 * kSX) : 0.0f;
    const int o0 = (warp & 3) * 32;
    // columns col (plus columns col2, when given) of this warp's 32 lanes
    auto flush32 = [&](uint32_t col, float scale, int base, int stride, uint32_t col2 = 0) {
      float v[32];
      tc::tmem_ld32(lane_base + col, v);
      if (col2) {
        float v2[32];
        tc::tmem_ld32(lane_base + col2, v2);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += v2[i];
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) tp[lane * 33 + i] = v[i] * scale;
      __syncwarp();
      for (int r = 0; r < 32; ++r) P[base + (o0 + r) * stride + lane] = tp[r * 33 + lane];
      __syncwarp();
    };
    flush32(cDW2 + 32 * qw, u2, kOffW2 + 32 * qw, kHid);
    // dW1 | db1: the sum of the hi*hi + lo*hi columns and the hi*lo columns
    if (qw == 0) {
      flush32(cDW1, u1, kOffW1, kIn, cDW1 + kK1);              // W1[:, 0:32]
    } else if (qw == 1) {
      float v[16], v2[16];
      tc::tmem_ld16(lane_base + cDW1 + 32, v);                  // W1[:, 32:39] and b1 (column 39)
      tc::tmem_ld16(lane_base + cDW1 + kK1 + 32, v2);
#pragma unroll
      for (int i = 0; i < 8; ++i) tp[lane * 33 + i] = (v[i] + v2[i]) * u1;
      __syncwarp();
      for (int r = 0; r < 32; ++r) {
        if (lane < kIn - 32) P[kOffW1 + (o0 + r) * kIn + 32 + lane] = tp[r * 33 + lane];
        else if (lane == kIn - 32) P[kOffB1 + o0 + r] = tp[r * 33 + lane];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// g_params += sum of the partial rows of the CTAs that had tiles: block =
// 32 parameters x 8 row groups; each group sums its rows in order, then the
// eight group sums are added in order (a fixed association: deterministic).
__global__ void __launch_bounds__(256) partials_reduce_kernel(const float* __restrict__ part, int nrows,
                                                              int64_t n_cap, const int64_t* __restrict__ n_dev,
                                                              float* __restrict__ g_params) {
  __shared__ float acc[8][33];
  const int64_t n = mlp_count(n_cap, n_dev);
  const int rows = (int)std::min<int64_t>(nrows, (n + kTile - 1) / kTile);
  const int j = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + j;
  const int per = (rows + 7) / 8, b0 = grp * per, b1 = std::min(rows, b0 + per);
  float a = 0.0f;
  if (p < kNumParams) {
#pragma unroll 8
    for (int b = b0; b < b1; ++b) a += __ldg(part + (size_t)b * kNumParams + p);
  }
  acc[grp][j] = a;
  __syncthreads();
  if (grp == 0 && p < kNumParams) {
    float t = acc[0][j];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += acc[q][j];
    g_params[p] += t;
  }
}

}  // namespace dvgo

using namespace dvgo;

// act layout: [256 reserved bytes | one 90112-byte image per 128-position tile |
// kNumSMs partial gradient rows of kNumParams floats]
static int64_t act_images_end(int64_t n_cap) {
  return (int64_t)kActHeader + (n_cap + kTile - 1) / kTile * (int64_t)kImage;
}

int64_t rgbnet_act_bytes_tc(int64_t n_cap) {
  return act_images_end(n_cap) + (int64_t)kNumSMs * kNumParams * (int64_t)sizeof(float);
}

template <class Op>
static int rgbnet_fwd_tc(const float* k0, const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                         int64_t n_cap, const int64_t* n_dev, const float* params, float* rgb, float* act,
                         cudaStream_t st) {
  const size_t smem = gEnd + sizeof(FwdSide) + 2 * 4 * kTile * kOut * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_fwd_tc_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  rgbnet_fwd_tc_kernel<Op><<<grid, 544, smem, st>>>(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb,
                                                    reinterpret_cast<uint8_t*>(act));
  return launch_status();
}

template <class Op>
static int rgbnet_bwd_tc(const float* g_rgb, const float* g_color, const float* w, const float* rgb,
                         const int32_t* ray_id, const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                         const float* params, float* act, float* g_params, float* g_k0, cudaStream_t st) {
  const size_t smem = bEnd + sizeof(Side);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rgbnet_bwd_tc_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int grid = (int)std::min<int64_t>((n_cap + kTile - 1) / kTile, kNumSMs);
  float* part = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(act) + act_images_end(n_cap));
  rgbnet_bwd_tc_kernel<Op><<<grid, 544, smem, st>>>(g_rgb, g_color, w, rgb, ray_id, idx, n_cap, n_dev,
                                                    params, reinterpret_cast<const uint8_t*>(act), part,
                                                    g_k0);
  partials_reduce_kernel<<<(kNumParams + 31) / 32, 256, 0, st>>>(part, grid, n_cap, n_dev, g_params);
  return launch_status();
}

// bf16_form: the BF16 form (stored BF16 parameters, BF16 operand terms);
// otherwise the FP32 form (FP16 operand terms).
int dvgo_rgbnet_fwd_tc(const float* k0, const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                       int64_t n_cap, const int64_t* n_dev, const float* params, float* rgb, float* act,
                       bool bf16_form, cudaStream_t st) {
  return bf16_form ? rgbnet_fwd_tc<OpBF16>(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb, act, st)
                   : rgbnet_fwd_tc<OpF16>(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb, act, st);
}

int dvgo_rgbnet_bwd_tc(const float* g_rgb, const float* g_color, const float* w, const float* rgb,
                       const int32_t* ray_id, const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                       const float* params, float* act, float* g_params, float* g_k0, bool bf16_form,
                       cudaStream_t st) {
  return bf16_form ? rgbnet_bwd_tc<OpBF16>(g_rgb, g_color, w, rgb, ray_id, idx, n_cap, n_dev, params, act,
                                           g_params, g_k0, st)
                   : rgbnet_bwd_tc<OpF16>(g_rgb, g_color, w, rgb, ray_id, idx, n_cap, n_dev, params, act,
                                          g_params, g_k0, st);
}

int dvgo_mlp_tc_status_read_and_clear(cudaStream_t st) {
  int v = 0, zero = 0;
  cudaMemcpyFromSymbolAsync(&v, g_mlp_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  cudaMemcpyToSymbolAsync(g_mlp_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return v;
}
