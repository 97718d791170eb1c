// Volume rendering over ragged per-ray sample lists: raw->alpha with
// log-space transmittance and early stop (Sec. 3 "Re-implement rendering
// utils"), colour accumulation and its adjoint, the O(N) distortion loss and
// its gradient (Sec. 2), and the photometric loss.  One warp per ray; the
// samples of a ray are processed in chunks of 32 with warp scans and a
// carried running value between chunks.
#include "common.cuh"

namespace dvgo {

__device__ __forceinline__ void ray_range(const int64_t* __restrict__ ray_off,
                                          const int32_t* __restrict__ seg_len, int64_t r,
                                          int64_t& b, int& n, int& N) {
  b = ray_off[r];
  N = (int)(ray_off[r + 1] - b);
  n = N;
  if (seg_len) n = min(n, (int)seg_len[r]);
}

#define DVGO_WARP_LOOP(R)                                                   \
  const int lane = threadIdx.x & 31;                                        \
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; \
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;            \
  for (int64_t r = warp0; r < (R); r += nwarps)

// The alpha interval of sample s: delta[s] when a per-sample interval is
// given (a proposal pick standing for the gap to the next pick), else the
// common interval.
__device__ __forceinline__ float interval_of(const float* __restrict__ delta, float interval, int64_t s) {
  return delta ? __ldg(delta + s) : interval;
}

// ------------------------------------------------------------- weights fwd
__global__ void __launch_bounds__(256) alpha_weights_kernel(
    const float* __restrict__ raw, const int64_t* __restrict__ ray_off, int64_t R, float shift,
    float interval, const float* __restrict__ delta, float T_stop, float* __restrict__ w, float* __restrict__ T,
    int32_t* __restrict__ n_live, float* __restrict__ T_end) {
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, nullptr, r, b, n, N);
    Kahan carry;  // log T before the current chunk
    int stop = N;
    float t_end = 1.0f;
    int c0 = 0;
    for (; c0 < N; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < N;
      const float la =
          valid ? -interval_of(delta, interval, b + i) * softplus_f(__ldg(raw + b + i) + shift) : 0.0f;
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

// --------------------------------------------------------- colour forward
__global__ void __launch_bounds__(256) composite_rgb_kernel(
    const float* __restrict__ w, const float* __restrict__ rgb, const int64_t* __restrict__ ray_off,
    const int32_t* __restrict__ n_live, const float* __restrict__ T_end, int64_t R, float bg0,
    float bg1, float bg2, float* __restrict__ color) {
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, n_live, r, b, n, N);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float wi = __ldg(w + b + i);
      a0 += wi * __ldg(rgb + 3 * (b + i));
      a1 += wi * __ldg(rgb + 3 * (b + i) + 1);
      a2 += wi * __ldg(rgb + 3 * (b + i) + 2);
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
      const float te = T_end[r];
      color[3 * r] = a0 + te * bg0;
      color[3 * r + 1] = a1 + te * bg1;
      color[3 * r + 2] = a2 + te * bg2;
    }
  }
}

// -------------------------------------------------------- composite bwd
// The adjoint reverse recurrence R_k = g_{k+1} alpha_{k+1} + (1 -
// alpha_{k+1}) R_{k+1}, R_{n-1} = g_T, enters the gradient only as
// T_{k+1} R_k, which unrolls to the suffix sum
//   S_k = T_{k+1} R_k = sum_{j > k} g_j w_j + g_T T_end,
// so g_raw_k = interval sigmoid(raw_k + shift) (T_{k+1} g_k - S_k).  S_k is
// formed as a sum (per 32-sample chunk by shuffles, across chunks with a
// compensated carry): no product of (1 - alpha) factors along the ray, so the
// rounding error does not grow with the ray's length.
__global__ void __launch_bounds__(256) composite_bwd_kernel(
    const float* __restrict__ g_color, const float* __restrict__ g_w, const float* __restrict__ raw,
    const float* __restrict__ T, const float* __restrict__ rgb, const int64_t* __restrict__ ray_off,
    const int32_t* __restrict__ n_live, int64_t R, float shift, float interval,
    const float* __restrict__ delta, float bg0, float bg1, float bg2, float* __restrict__ g_raw,
    float* __restrict__ g_rgb) {
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, n_live, r, b, n, N);
    const float gc0 = __ldg(g_color + 3 * r), gc1 = __ldg(g_color + 3 * r + 1),
                gc2 = __ldg(g_color + 3 * r + 2);
    const float gT = bg0 * gc0 + bg1 * gc1 + bg2 * gc2;
    Kahan suf;   // sum of g_j w_j over the chunks after the current one, + g_T T_end
    const int last_chunk = n > 0 ? ((n - 1) & ~31) : -32;
    for (int c0 = last_chunk; c0 >= 0; c0 -= 32) {
      const int k = c0 + lane;
      const bool valid = k < n;
      float gk = 0.0f, la = 0.0f, rk = 0.0f, Tk = 0.0f, al = 0.0f, dk = 0.0f;
      if (valid) {
        const int64_t s = b + k;
        rk = __ldg(raw + s);
        dk = interval_of(delta, interval, s);
        la = -dk * softplus_f(rk + shift);
        al = -expm1f(la);
        if (rgb) gk = __ldg(rgb + 3 * s) * gc0 + __ldg(rgb + 3 * s + 1) * gc1 + __ldg(rgb + 3 * s + 2) * gc2;
        if (g_w) gk += __ldg(g_w + s);
        Tk = __ldg(T + s);
      }
      const float Tk1 = Tk * expf(la);
      if (c0 == last_chunk) suf.add(gT * __shfl_sync(0xffffffffu, Tk1, (n - 1) & 31));   // T_end
      const float wk = Tk * al;
      const float v = valid ? gk * wk : 0.0f;
      float sv = v;   // inclusive suffix sum within the chunk (lane .. 31)
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float a = __shfl_down_sync(0xffffffffu, sv, o);
        if (lane + o < 32) sv += a;
      }
      float ex = __shfl_down_sync(0xffffffffu, sv, 1);
      if (lane == 31) ex = 0.0f;
      const float Sk = __fadd_rn(suf.s, __fsub_rn(ex, suf.c));
      if (valid) {
        g_raw[b + k] = dk * sigmoid_f(rk + shift) * (Tk1 * gk - Sk);
        if (g_rgb) {
          g_rgb[3 * (b + k)] = wk * gc0;
          g_rgb[3 * (b + k) + 1] = wk * gc1;
          g_rgb[3 * (b + k) + 2] = wk * gc2;
        }
      }
      suf.add(__shfl_sync(0xffffffffu, sv, 0));
    }
    for (int k = n + lane; k < N; k += 32) {
      g_raw[b + k] = 0.0f;
      if (g_rgb) {
        g_rgb[3 * (b + k)] = 0.0f;
        g_rgb[3 * (b + k) + 1] = 0.0f;
        g_rgb[3 * (b + k) + 2] = 0.0f;
      }
    }
  }
}

// ------------------------------------------------------------ distortion
// Midpoints are measured from the segment's first midpoint (the loss and its
// gradient only depend on differences of m), which keeps the prefix-sum
// difference m_i W_{<i} - WM_{<i} free of cancellation against large m.
__global__ void __launch_bounds__(256) distortion_fwd_kernel(
    const float* __restrict__ w, const float* __restrict__ m, const float* __restrict__ ds,
    const int64_t* __restrict__ ray_off, const int32_t* __restrict__ seg_len, int64_t R,
    float* __restrict__ L_r) {
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, seg_len, r, b, n, N);
    const float m0 = n > 0 ? __ldg(m + b) : 0.0f;
    Kahan cW, cWM;
    float acc = 0.0f;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < n;
      const float wi = valid ? __ldg(w + b + i) : 0.0f;
      const float mi = valid ? __ldg(m + b + i) - m0 : 0.0f;
      const float di = valid ? __ldg(ds + b + i) : 0.0f;
      const float iw = warp_incl_sum(wi);
      const float iwm = warp_incl_sum(wi * mi);
      const float Wlt = __fadd_rn(cW.s, __fsub_rn(iw - wi, cW.c));
      const float WMlt = __fadd_rn(cWM.s, __fsub_rn(iwm - wi * mi, cWM.c));
      acc += 2.0f * wi * (mi * Wlt - WMlt) + wi * wi * di * (1.0f / 3.0f);
      cW.add(__shfl_sync(0xffffffffu, iw, 31));
      cWM.add(__shfl_sync(0xffffffffu, iwm, 31));
    }
    acc = warp_sum(acc);
    if (lane == 0) L_r[r] = acc;
  }
}

__global__ void __launch_bounds__(256) distortion_bwd_kernel(
    const float* __restrict__ g_L, float g_L_scalar, const float* __restrict__ w,
    const float* __restrict__ m, const float* __restrict__ ds, const int64_t* __restrict__ ray_off,
    const int32_t* __restrict__ seg_len, int64_t R, float* __restrict__ g_w) {
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, seg_len, r, b, n, N);
    const float gl = g_L ? __ldg(g_L + r) : g_L_scalar;
    const float m0 = n > 0 ? __ldg(m + b) : 0.0f;
    // totals
    Kahan tW, tWM;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const float wi = i < n ? __ldg(w + b + i) : 0.0f;
      const float mi = i < n ? __ldg(m + b + i) - m0 : 0.0f;
      tW.add(warp_sum(wi));
      tWM.add(warp_sum(wi * mi));
    }
    const float Wt = __fsub_rn(tW.s, tW.c), WMt = __fsub_rn(tWM.s, tWM.c);
    Kahan cW, cWM;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < n;
      const float wi = valid ? __ldg(w + b + i) : 0.0f;
      const float mi = valid ? __ldg(m + b + i) - m0 : 0.0f;
      const float di = valid ? __ldg(ds + b + i) : 0.0f;
      const float iw = warp_incl_sum(wi);
      const float iwm = warp_incl_sum(wi * mi);
      const float Wlt = __fadd_rn(cW.s, __fsub_rn(iw - wi, cW.c));
      const float WMlt = __fadd_rn(cWM.s, __fsub_rn(iwm - wi * mi, cWM.c));
      const float Wgt = Wt - Wlt - wi;
      const float WMgt = WMt - WMlt - wi * mi;
      if (valid)
        g_w[b + i] = gl * (2.0f * (mi * (Wlt - Wgt) - WMlt + WMgt) + (2.0f / 3.0f) * wi * di);
      cW.add(__shfl_sync(0xffffffffu, iw, 31));
      cWM.add(__shfl_sync(0xffffffffu, iwm, 31));
    }
    for (int k = n + lane; k < N; k += 32) g_w[b + k] = 0.0f;
  }
}

// Compositing adjoint with the distortion gradient formed in place, for ray
// r (samples b .. b + N, the first n live) given its totals W and WM of w and
// w m (Kahan): chunks from the last to the first, Kahan-compensated suffix
// sums W_{>i}, WM_{>i} give g_w_i (W_{<i} = W - W_{>i} - w_i), which enters
// the colour adjoint's suffix sum S_k = sum_{j>k} g_j w_j + g_T T_end (see
// composite_bwd_kernel) directly (g_w is never stored).  One warp; every
// lane calls it.
__device__ __forceinline__ void composite_distortion_bwd_ray(
    int lane, int64_t b, int n, int N, float gc0, float gc1, float gc2, float Wt, float WMt, float g_L,
    const float* __restrict__ w, const float* __restrict__ raw, const float* __restrict__ T,
    const float* __restrict__ rgb, const float* __restrict__ m, const float* __restrict__ ds,
    float shift, float interval, const float* __restrict__ delta, float bg0, float bg1, float bg2,
    float* __restrict__ g_raw) {
  const float m0 = n > 0 ? __ldg(m + b) : 0.0f;
  Kahan sW, sWM;                                     // sums over the chunks after the current one
  Kahan suf;                                         // sum_{j in later chunks} g_j w_j + g_T T_end
  const float gT = bg0 * gc0 + bg1 * gc1 + bg2 * gc2;
  const int last_chunk = n > 0 ? ((n - 1) & ~31) : -32;
  for (int c0 = last_chunk; c0 >= 0; c0 -= 32) {
    const int k = c0 + lane;
    const bool valid = k < n;
    float wi = 0.0f, mi = 0.0f, di = 0.0f, rk = 0.0f, Tk = 0.0f, la = 0.0f, dk = 0.0f;
    float c_rgb = 0.0f;
    if (valid) {
      const int64_t s = b + k;
      wi = __ldg(w + s);
      mi = __ldg(m + s) - m0;
      di = __ldg(ds + s);
      rk = __ldg(raw + s);
      Tk = __ldg(T + s);
      c_rgb = __ldg(rgb + 3 * s) * gc0 + __ldg(rgb + 3 * s + 1) * gc1 + __ldg(rgb + 3 * s + 2) * gc2;
      dk = interval_of(delta, interval, s);
      la = -dk * softplus_f(rk + shift);
    }
    const float Tk1 = Tk * expf(la);
    if (c0 == last_chunk) suf.add(gT * __shfl_sync(0xffffffffu, Tk1, (n - 1) & 31));   // T_end
    // inclusive suffix sums within the chunk (lane .. 31)
    float sw = wi, swm = wi * mi;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float a = __shfl_down_sync(0xffffffffu, sw, o);
      const float c = __shfl_down_sync(0xffffffffu, swm, o);
      if (lane + o < 32) {
        sw += a;
        swm += c;
      }
    }
    const float Wgt = __fadd_rn(sW.s, __fsub_rn(sw - wi, sW.c));
    const float WMgt = __fadd_rn(sWM.s, __fsub_rn(swm - wi * mi, sWM.c));
    const float Wlt = Wt - Wgt - wi;
    const float WMlt = WMt - WMgt - wi * mi;
    const float gw = g_L * (2.0f * (mi * (Wlt - Wgt) - WMlt + WMgt) + (2.0f / 3.0f) * wi * di);
    const float gk = valid ? c_rgb + gw : 0.0f;
    const float v = gk * wi;
    float sv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float a = __shfl_down_sync(0xffffffffu, sv, o);
      if (lane + o < 32) sv += a;
    }
    float ex = __shfl_down_sync(0xffffffffu, sv, 1);
    if (lane == 31) ex = 0.0f;
    const float Sk = __fadd_rn(suf.s, __fsub_rn(ex, suf.c));
    if (valid) g_raw[b + k] = dk * sigmoid_f(rk + shift) * (Tk1 * gk - Sk);
    suf.add(__shfl_sync(0xffffffffu, sv, 0));
    sW.add(__shfl_sync(0xffffffffu, sw, 0));
    sWM.add(__shfl_sync(0xffffffffu, swm, 0));
  }
  for (int k = n + lane; k < N; k += 32) g_raw[b + k] = 0.0f;
}

// ------------------------------------------------ fused per-ray tails
// Colour accumulation and the distortion loss of the live samples in one pass
// over each ray (both read w; same arithmetic as the two kernels above).
// With kLoss the photometric loss of dvgo_rgb_loss is formed too: each ray's
// squared error and g_color beside its colour, per-block partial sums, and
// the last block to finish (a ticket counter it resets) adds the partials in
// block order (deterministic).
// With kBwd (and kLoss) the compositing adjoint of each ray follows its
// forward pass in the same warp (composite_distortion_bwd_ray with the g_color
// just formed): one pass of the per-ray tail for the whole step.
struct BwdTail {
  float g_L;
  const float* raw;
  const float* T;
  float shift, interval;
  const float* delta;   // per-sample intervals (may be NULL)
  float* g_raw;
};

struct LossTail {
  const float* target;
  float lambda_dist;
  float* g_color;
  float* loss_out;
  unsigned int* ticket;
  float* part;       // [gridDim.x][2]
};

template <bool kLoss, bool kBwd = false>
__global__ void __launch_bounds__(256) composite_distortion_fwd_kernel(
    const float* __restrict__ w, const float* __restrict__ rgb, const float* __restrict__ m,
    const float* __restrict__ ds, const int64_t* __restrict__ ray_off, const int32_t* __restrict__ n_live,
    const float* __restrict__ T_end, int64_t R, float bg0, float bg1, float bg2,
    float* __restrict__ color, float* __restrict__ L_r, LossTail lt, BwdTail bt = BwdTail{}) {
  static_assert(kLoss || !kBwd, "the adjoint needs the loss gradient");
  float sq = 0.0f, dsum = 0.0f;   // lane 0: this warp's rays
  const float gscale = 2.0f / (3.0f * (float)R);
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, n_live, r, b, n, N);
    const float m0 = n > 0 ? __ldg(m + b) : 0.0f;
    // lane 0's per-ray inputs, loaded before the chunk loop that they follow
    float te = 0.0f, tg0 = 0.0f, tg1 = 0.0f, tg2 = 0.0f;
    if (lane == 0) {
      te = __ldg(T_end + r);
      if constexpr (kLoss) {
        tg0 = __ldg(lt.target + 3 * r);
        tg1 = __ldg(lt.target + 3 * r + 1);
        tg2 = __ldg(lt.target + 3 * r + 2);
      }
    }
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, acc = 0.0f;
    Kahan cW, cWM, tW, tWM;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < n;
      float wi = 0.0f, mi = 0.0f, di = 0.0f;
      if (valid) {
        const int64_t s = b + i;
        wi = __ldg(w + s);
        mi = __ldg(m + s) - m0;
        di = __ldg(ds + s);
        a0 += wi * __ldg(rgb + 3 * s);
        a1 += wi * __ldg(rgb + 3 * s + 1);
        a2 += wi * __ldg(rgb + 3 * s + 2);
      }
      const float iw = warp_incl_sum(wi);
      const float iwm = warp_incl_sum(wi * mi);
      const float Wlt = __fadd_rn(cW.s, __fsub_rn(iw - wi, cW.c));
      const float WMlt = __fadd_rn(cWM.s, __fsub_rn(iwm - wi * mi, cWM.c));
      acc += 2.0f * wi * (mi * Wlt - WMlt) + wi * wi * di * (1.0f / 3.0f);
      cW.add(__shfl_sync(0xffffffffu, iw, 31));
      cWM.add(__shfl_sync(0xffffffffu, iwm, 31));
      if constexpr (kBwd) {   // the adjoint's totals, summed as its own kernel sums them
        tW.add(warp_sum(wi));
        tWM.add(warp_sum(wi * mi));
      }
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    acc = warp_sum(acc);
    float gc0 = 0.0f, gc1 = 0.0f, gc2 = 0.0f;
    if (lane == 0) {
      const float c0 = a0 + te * bg0, c1 = a1 + te * bg1, c2 = a2 + te * bg2;
      color[3 * r] = c0;
      color[3 * r + 1] = c1;
      color[3 * r + 2] = c2;
      L_r[r] = acc;
      if constexpr (kLoss) {
        const float e0 = c0 - tg0, e1 = c1 - tg1, e2 = c2 - tg2;
        gc0 = gscale * e0;
        gc1 = gscale * e1;
        gc2 = gscale * e2;
        lt.g_color[3 * r] = gc0;
        lt.g_color[3 * r + 1] = gc1;
        lt.g_color[3 * r + 2] = gc2;
        sq += (e0 * e0 + e1 * e1) + e2 * e2;
        dsum += acc;
      }
    }
    if constexpr (kBwd) {
      gc0 = __shfl_sync(0xffffffffu, gc0, 0);
      gc1 = __shfl_sync(0xffffffffu, gc1, 0);
      gc2 = __shfl_sync(0xffffffffu, gc2, 0);
      composite_distortion_bwd_ray(lane, b, n, N, gc0, gc1, gc2, __fsub_rn(tW.s, tW.c),
                                   __fsub_rn(tWM.s, tWM.c), bt.g_L, w, bt.raw, bt.T, rgb, m, ds,
                                   bt.shift, bt.interval, bt.delta, bg0, bg1, bg2, bt.g_raw);
    }
  }
  if constexpr (kLoss) {
    __shared__ float s1[8], s2[8];
    __shared__ bool last;
    const int wid = threadIdx.x >> 5;
    if (lane == 0) {
      s1[wid] = sq;
      s2[wid] = dsum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = 0.0f, d = 0.0f;
      for (int i = 0; i < 8; ++i) {
        a += s1[i];
        d += s2[i];
      }
      lt.part[2 * blockIdx.x] = a;
      lt.part[2 * blockIdx.x + 1] = d;
      __threadfence();
      last = atomicAdd(lt.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      // thread t adds blocks t, t + 256, ... in order; the warp and block
      // steps below always pair the same partners
      float a = 0.0f, d = 0.0f;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        a += __ldcg(lt.part + 2 * b);
        d += __ldcg(lt.part + 2 * b + 1);
      }
      a = warp_sum(a);
      d = warp_sum(d);
      __syncthreads();
      if (lane == 0) {
        s1[wid] = a;
        s2[wid] = d;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        a = 0.0f;
        d = 0.0f;
        for (int i = 0; i < 8; ++i) {
          a += s1[i];
          d += s2[i];
        }
        const float lr = a / (3.0f * (float)R);
        const float ld = d / (float)R;
        lt.loss_out[0] = lr;
        lt.loss_out[1] = ld;
        lt.loss_out[2] = lr + lt.lambda_dist * ld;
        *lt.ticket = 0u;   // ready for the next call
      }
    }
  }
}

// The adjoint for each ray: one forward pass for the totals W and WM, then
// composite_distortion_bwd_ray.
__global__ void __launch_bounds__(256) composite_distortion_bwd_kernel(
    const float* __restrict__ g_color, float g_L, const float* __restrict__ w,
    const float* __restrict__ raw, const float* __restrict__ T, const float* __restrict__ rgb,
    const float* __restrict__ m, const float* __restrict__ ds, const int64_t* __restrict__ ray_off,
    const int32_t* __restrict__ n_live, int64_t R, float shift, float interval,
    const float* __restrict__ delta, float bg0, float bg1, float bg2, float* __restrict__ g_raw) {
  DVGO_WARP_LOOP(R) {
    int64_t b;
    int n, N;
    ray_range(ray_off, n_live, r, b, n, N);
    const float gc0 = __ldg(g_color + 3 * r), gc1 = __ldg(g_color + 3 * r + 1),
                gc2 = __ldg(g_color + 3 * r + 2);
    const float m0 = n > 0 ? __ldg(m + b) : 0.0f;
    Kahan tW, tWM;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const float wi = i < n ? __ldg(w + b + i) : 0.0f;
      const float mi = i < n ? __ldg(m + b + i) - m0 : 0.0f;
      tW.add(warp_sum(wi));
      tWM.add(warp_sum(wi * mi));
    }
    composite_distortion_bwd_ray(lane, b, n, N, gc0, gc1, gc2, __fsub_rn(tW.s, tW.c),
                                 __fsub_rn(tWM.s, tWM.c), g_L, w, raw, T, rgb, m, ds, shift, interval,
                                 delta, bg0, bg1, bg2, g_raw);
  }
}

// ------------------------------------------------------------------ loss
__global__ void __launch_bounds__(1024) rgb_loss_kernel(const float* __restrict__ color,
                                                        const float* __restrict__ target,
                                                        const float* __restrict__ L_r, int64_t R,
                                                        float lambda_dist,
                                                        float* __restrict__ loss_out,
                                                        float* __restrict__ g_color) {
  __shared__ float s1[32], s2[32];
  float a = 0.0f, d = 0.0f;
  const float gscale = 2.0f / (3.0f * (float)R);
  // eight independent loads in flight per thread and step
  constexpr int U = 8;
  for (int64_t i0 = threadIdx.x; i0 < 3 * R; i0 += U * (int64_t)blockDim.x) {
    float c[U], t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * (int64_t)blockDim.x;
      c[u] = i < 3 * R ? __ldg(color + i) : 0.0f;
      t[u] = i < 3 * R ? __ldg(target + i) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * (int64_t)blockDim.x;
      const float e = c[u] - t[u];
      a += e * e;
      if (i < 3 * R) g_color[i] = gscale * e;
    }
  }
  if (L_r)
    for (int64_t i0 = threadIdx.x; i0 < R; i0 += U * (int64_t)blockDim.x) {
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + u * (int64_t)blockDim.x;
        v[u] = i < R ? __ldg(L_r + i) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) d += v[u];
    }
  a = warp_sum(a);
  d = warp_sum(d);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s1[wid] = a;
    s2[wid] = d;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? s1[lane] : 0.0f;
    d = lane < nw ? s2[lane] : 0.0f;
    a = warp_sum(a);
    d = warp_sum(d);
    if (lane == 0) {
      const float lr = a / (3.0f * (float)R);
      const float ld = d / (float)R;
      loss_out[0] = lr;
      loss_out[1] = ld;
      loss_out[2] = lr + lambda_dist * ld;
    }
  }
}

}  // namespace dvgo

using namespace dvgo;

static int warp_grid(int64_t R) { return grid_for(R * 32, 256, 16); }

extern "C" int dvgo_alpha_weights_fwd(const float* raw, const int64_t* ray_off, int64_t R,
                                      float shift, float interval, const float* delta, float T_stop,
                                      float* w, float* T, int32_t* n_live, float* T_end, void* stream) {
  DVGO_CHECK_ARG(R >= 0 && interval > 0.0f && T_stop >= 0.0f);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(raw && ray_off && w && T && n_live && T_end);
  alpha_weights_kernel<<<warp_grid(R), 256, 0, as_stream(stream)>>>(raw, ray_off, R, shift,
                                                                    interval, delta, T_stop, w, T, n_live,
                                                                    T_end);
  return launch_status();
}

extern "C" int dvgo_composite_rgb_fwd(const float* w, const float* rgb, const int64_t* ray_off,
                                      const int32_t* n_live, const float* T_end, int64_t R,
                                      const float bg[3], float* color, void* stream) {
  DVGO_CHECK_ARG(R >= 0);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(w && rgb && ray_off && T_end && bg && color);
  composite_rgb_kernel<<<warp_grid(R), 256, 0, as_stream(stream)>>>(w, rgb, ray_off, n_live, T_end,
                                                                    R, bg[0], bg[1], bg[2], color);
  return launch_status();
}

extern "C" int dvgo_composite_bwd(const float* g_color, const float* g_w, const float* raw,
                                  const float* T, const float* rgb, const int64_t* ray_off,
                                  const int32_t* n_live, int64_t R, float shift, float interval,
                                  const float* delta, const float bg[3], float* g_raw, float* g_rgb,
                                  void* stream) {
  DVGO_CHECK_ARG(R >= 0 && interval > 0.0f);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(g_color && raw && T && ray_off && n_live && bg && g_raw);
  composite_bwd_kernel<<<warp_grid(R), 256, 0, as_stream(stream)>>>(
      g_color, g_w, raw, T, rgb, ray_off, n_live, R, shift, interval, delta, bg[0], bg[1], bg[2], g_raw,
      g_rgb);
  return launch_status();
}

extern "C" int dvgo_distortion_fwd(const float* w, const float* m, const float* ds,
                                   const int64_t* ray_off, const int32_t* seg_len, int64_t R,
                                   float* L_r, void* stream) {
  DVGO_CHECK_ARG(R >= 0);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(w && m && ds && ray_off && L_r);
  distortion_fwd_kernel<<<warp_grid(R), 256, 0, as_stream(stream)>>>(w, m, ds, ray_off, seg_len, R,
                                                                     L_r);
  return launch_status();
}

extern "C" int dvgo_distortion_bwd(const float* g_L, float g_L_scalar, const float* w,
                                   const float* m, const float* ds, const int64_t* ray_off,
                                   const int32_t* seg_len, int64_t R, float* g_w, void* stream) {
  DVGO_CHECK_ARG(R >= 0);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(w && m && ds && ray_off && g_w);
  distortion_bwd_kernel<<<warp_grid(R), 256, 0, as_stream(stream)>>>(g_L, g_L_scalar, w, m, ds,
                                                                     ray_off, seg_len, R, g_w);
  return launch_status();
}

extern "C" int dvgo_rgb_loss(const float* color, const float* target, const float* L_r, int64_t R,
                             float lambda_dist, float* loss_out, float* g_color, void* stream) {
  DVGO_CHECK_ARG(R > 0 && color && target && loss_out && g_color);
  rgb_loss_kernel<<<1, 1024, 0, as_stream(stream)>>>(color, target, L_r, R, lambda_dist, loss_out,
                                                     g_color);
  return launch_status();
}

extern "C" int dvgo_composite_distortion_fwd(const float* w, const float* rgb, const float* m,
                                             const float* ds, const int64_t* ray_off,
                                             const int32_t* n_live, const float* T_end, int64_t R,
                                             const float bg[3], float* color, float* L_r,
                                             void* stream) {
  DVGO_CHECK_ARG(R >= 0);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(w && rgb && m && ds && ray_off && T_end && bg && color && L_r);
  composite_distortion_fwd_kernel<false><<<warp_grid(R), 256, 0, as_stream(stream)>>>(
      w, rgb, m, ds, ray_off, n_live, T_end, R, bg[0], bg[1], bg[2], color, L_r, LossTail{});
  return launch_status();
}

// workspace: a ticket counter (16 bytes) and two partial sums per block
extern "C" size_t dvgo_composite_loss_workspace_size(int64_t R) {
  return 16 + (size_t)2 * sizeof(float) * (size_t)warp_grid(R < 1 ? 1 : R);
}

extern "C" int dvgo_composite_distortion_loss_fwd(const float* w, const float* rgb, const float* m,
                                                  const float* ds, const int64_t* ray_off,
                                                  const int32_t* n_live, const float* T_end, int64_t R,
                                                  const float bg[3], const float* target,
                                                  float lambda_dist, float* color, float* L_r,
                                                  float* g_color, float* loss_out, void* ws,
                                                  void* stream) {
  DVGO_CHECK_ARG(R > 0);
  DVGO_CHECK_ARG(w && rgb && m && ds && ray_off && T_end && bg && color && L_r && target && g_color &&
                 loss_out && ws);
  DVGO_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 15u) == 0);
  LossTail lt{target, lambda_dist, g_color, loss_out, reinterpret_cast<unsigned int*>(ws),
              reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(ws) + 16)};
  composite_distortion_fwd_kernel<true><<<warp_grid(R), 256, 0, as_stream(stream)>>>(
      w, rgb, m, ds, ray_off, n_live, T_end, R, bg[0], bg[1], bg[2], color, L_r, lt);
  return launch_status();
}

extern "C" int dvgo_composite_distortion_loss_fwd_bwd(
    const float* w, const float* rgb, const float* m, const float* ds, const int64_t* ray_off,
    const int32_t* n_live, const float* T_end, int64_t R, const float bg[3], const float* target,
    float lambda_dist, float g_L, const float* raw, const float* T, float shift, float interval,
    const float* delta, float* color, float* L_r, float* g_color, float* loss_out, float* g_raw, void* ws,
    void* stream) {
  DVGO_CHECK_ARG(R > 0);
  DVGO_CHECK_ARG(w && rgb && m && ds && ray_off && T_end && bg && color && L_r && target && g_color &&
                 loss_out && ws && raw && T && g_raw);
  DVGO_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 15u) == 0);
  LossTail lt{target, lambda_dist, g_color, loss_out, reinterpret_cast<unsigned int*>(ws),
              reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(ws) + 16)};
  BwdTail bt{g_L, raw, T, shift, interval, delta, g_raw};
  composite_distortion_fwd_kernel<true, true><<<warp_grid(R), 256, 0, as_stream(stream)>>>(
      w, rgb, m, ds, ray_off, n_live, T_end, R, bg[0], bg[1], bg[2], color, L_r, lt, bt);
  return launch_status();
}

extern "C" int dvgo_composite_distortion_bwd(const float* g_color, float g_L, const float* w,
                                             const float* raw, const float* T, const float* rgb,
                                             const float* m, const float* ds,
                                             const int64_t* ray_off, const int32_t* n_live,
                                             int64_t R, float shift, float interval,
                                             const float* delta, const float bg[3], float* g_raw,
                                             void* stream) {
  DVGO_CHECK_ARG(R >= 0 && interval > 0.0f);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(g_color && w && raw && T && rgb && m && ds && ray_off && n_live && bg && g_raw);
  composite_distortion_bwd_kernel<<<warp_grid(R), 256, 0, as_stream(stream)>>>(
      g_color, g_L, w, raw, T, rgb, m, ds, ray_off, n_live, R, shift, interval, delta, bg[0], bg[1], bg[2],
      g_raw);
  return launch_status();
}

extern "C" int dvgo_composite_fwd(const float* raw, const float* rgb, const int64_t* ray_off, int64_t R,
                                  float shift, float interval, const float* delta, float T_stop,
                                  const float bg[3], float* color, float* w, float* T, int32_t* n_live,
                                  float* T_end, void* stream) {
  const int r = dvgo_alpha_weights_fwd(raw, ray_off, R, shift, interval, delta, T_stop, w, T, n_live, T_end,
                                       stream);
  if (r != DVGO_OK) return r;
  return dvgo_composite_rgb_fwd(w, rgb, ray_off, n_live, T_end, R, bg, color, stream);
}
