// Learned proposal (sample reduction; not part of the paper): per-ray
// softmax cross-entropy against the plain renderer's compositing weights,
// inverse-CDF selection of the samples to keep, and compaction of the kept
// samples into a new ragged list.  The proposal network itself runs in
// mlp_prop.cu.
#include "common.cuh"

int dvgo_proposal_fwd_bf16(const float*, const int32_t*, int64_t, const int64_t*, const float*,
                           float*, cudaStream_t);
int dvgo_proposal_bwd_bf16(const float*, const float*, const int32_t*, int64_t, const int64_t*,
                           const float*, float*, cudaStream_t);

namespace dvgo {

// Warp per ray.  q = softmax of the ray's logits; with a target, p_j =
// (w_j / W + eps) / (1 + N eps) (uniform when W = sum w = 0), loss_r =
// -sum p_j log q_j and g_logit_j = g_scale (q_j - p_j).
__global__ void __launch_bounds__(256) proposal_xent_kernel(
    const float* __restrict__ logits, const float* __restrict__ w, const int64_t* __restrict__ ray_off,
    int64_t R, float eps_u, float g_scale, float* __restrict__ loss_r, float* __restrict__ g_logits,
    float* __restrict__ q) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp0; r < R; r += nwarps) {
    const int64_t b = ray_off[r];
    const int N = (int)(ray_off[r + 1] - b);
    float mx = -INFINITY, W = 0.0f;
    for (int i = lane; i < N; i += 32) {
      mx = fmaxf(mx, __ldg(logits + b + i));
      if (w) W += __ldg(w + b + i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    W = warp_sum(W);
    float se = 0.0f;
    for (int i = lane; i < N; i += 32) se += expf(__ldg(logits + b + i) - mx);
    se = warp_sum(se);
    const float lse = mx + logf(se);
    const float norm = 1.0f / (1.0f + (float)N * eps_u);
    float loss = 0.0f;
    for (int i = lane; i < N; i += 32) {
      const float z = __ldg(logits + b + i);
      const float qi = expf(z - lse);
      if (q) q[b + i] = qi;
      if (w) {
        const float p = W > 0.0f ? (__ldg(w + b + i) / W + eps_u) * norm : 1.0f / (float)N;
        loss -= p * (z - lse);
        if (g_logits) g_logits[b + i] = g_scale * (qi - p);
      }
    }
    loss = warp_sum(loss);
    if (lane == 0 && loss_r) loss_r[r] = N > 0 ? loss : 0.0f;
  }
}

// One thread per ray: inverse CDF of q at u_k = (k + 0.5)/n_draw, the CDF
// summed sequentially in FP32 in candidate order; repeated picks collapse.
__global__ void proposal_select_kernel(const float* __restrict__ q, const int64_t* __restrict__ ray_off,
                                       int64_t R, int n_draw, int32_t* __restrict__ sel,
                                       int32_t* __restrict__ n_sel) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = ray_off[r];
    const int N = (int)(ray_off[r + 1] - b);
    int32_t* out = sel + r * n_draw;
    int cnt = 0;
    if (N > 0) {
      int j = 0;
      float cdf = q[b];
      const float nd = (float)n_draw;
      for (int k = 0; k < n_draw; ++k) {
        const float u = __fdiv_rn(__fadd_rn((float)k, 0.5f), nd);
        while (j < N - 1 && !(u < cdf)) {
          ++j;
          cdf = __fadd_rn(cdf, q[b + j]);
        }
        if (cnt == 0 || out[cnt - 1] != j) out[cnt++] = j;
      }
    }
    n_sel[r] = cnt;
    for (int k = cnt; k < n_draw; ++k) out[k] = -1;
  }
}

__global__ void scan_i32_kernel(const int32_t* __restrict__ counts, int64_t n,
                                int64_t* __restrict__ off) {
  // one block: exclusive scan into off[0..n]
  __shared__ int64_t wt[32];
  const int t = threadIdx.x, nt = blockDim.x;
  int64_t chunk = (n + nt - 1) / nt;
  int64_t b = min((int64_t)t * chunk, n), e = min(b + chunk, n);
  int64_t local = 0;
  for (int64_t i = b; i < e; ++i) local += counts[i];
  const int lane = t & 31, wid = t >> 5;
  int64_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wt[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t v = lane < (nt >> 5) ? wt[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < (nt >> 5)) wt[lane] = v;
  }
  __syncthreads();
  int64_t run = (wid > 0 ? wt[wid - 1] : 0) + incl - local;
  for (int64_t i = b; i < e; ++i) {
    off[i] = run;
    run += counts[i];
  }
  if (t == nt - 1) off[n] = run;
}

__global__ void compact_kernel(const int32_t* __restrict__ sel, const int32_t* __restrict__ n_sel,
                               int n_draw, const int64_t* __restrict__ ray_off, int64_t R,
                               const float* __restrict__ xyz, const int32_t* __restrict__ ray_id,
                               const int32_t* __restrict__ step_k, const float* __restrict__ s_mid,
                               const float* __restrict__ s_len, const int64_t* __restrict__ out_off,
                               float* __restrict__ o_xyz, int32_t* __restrict__ o_ray_id,
                               int32_t* __restrict__ o_step_k, float* __restrict__ o_s_mid,
                               float* __restrict__ o_s_len, int32_t* __restrict__ o_src,
                               float interval, float* __restrict__ o_delta) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp0; r < R; r += nwarps) {
    const int n = n_sel[r];
    const int64_t dst0 = out_off[r], src0 = ray_off[r];
    const int n_cand = (int)(ray_off[r + 1] - src0);
    for (int i = lane; i < n; i += 32) {
      const int j = sel[r * n_draw + i];
      const int64_t src = src0 + j;
      const int64_t dst = dst0 + i;
      o_xyz[3 * dst] = xyz[3 * src];
      o_xyz[3 * dst + 1] = xyz[3 * src + 1];
      o_xyz[3 * dst + 2] = xyz[3 * src + 2];
      o_ray_id[dst] = ray_id[src];
      o_step_k[dst] = step_k[src];
      if (o_delta) {
        // the pick stands for every candidate up to the next pick (the last
        // one up to the end of the ray's candidates)
        const int j_next = i + 1 < n ? sel[r * n_draw + i + 1] : n_cand;
        const float start = __fsub_rn(s_mid[src], __fmul_rn(0.5f, s_len[src]));
        const int64_t e = src0 + (j_next < n_cand ? j_next : n_cand - 1);
        const float end = j_next < n_cand ? __fsub_rn(s_mid[e], __fmul_rn(0.5f, s_len[e]))
                                          : __fadd_rn(s_mid[e], __fmul_rn(0.5f, s_len[e]));
        o_s_mid[dst] = __fmul_rn(0.5f, __fadd_rn(start, end));
        o_s_len[dst] = __fsub_rn(end, start);
        o_delta[dst] = __fmul_rn(interval, (float)(j_next - j));
      } else {
        o_s_mid[dst] = s_mid[src];
        o_s_len[dst] = s_len[src];
      }
      if (o_src) o_src[dst] = (int32_t)src;
    }
  }
}

}  // namespace dvgo

using namespace dvgo;

extern "C" int dvgo_proposal_fwd(const float* xyz, const int32_t* idx, int64_t n_cap,
                                 const int64_t* n_dev, const float* params, float* logits,
                                 void* stream) {
  DVGO_CHECK_ARG(n_cap >= 0);
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG(xyz && params && logits);
  return dvgo_proposal_fwd_bf16(xyz, idx, n_cap, n_dev, params, logits, as_stream(stream));
}

extern "C" int dvgo_proposal_bwd(const float* g_logits, const float* xyz, const int32_t* idx,
                                 int64_t n_cap, const int64_t* n_dev, const float* params,
                                 float* g_params, void* stream) {
  DVGO_CHECK_ARG(n_cap >= 0);
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG(g_logits && xyz && params && g_params);
  return dvgo_proposal_bwd_bf16(g_logits, xyz, idx, n_cap, n_dev, params, g_params, as_stream(stream));
}

extern "C" int dvgo_proposal_xent(const float* logits, const float* w_target, const int64_t* ray_off,
                                  int64_t R, float eps_u, float g_scale, float* loss_r,
                                  float* g_logits, float* q, void* stream) {
  DVGO_CHECK_ARG(R >= 0 && eps_u >= 0.0f);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(logits && ray_off && (q || w_target));
  proposal_xent_kernel<<<grid_for(R * 32, 256, 16), 256, 0, as_stream(stream)>>>(
      logits, w_target, ray_off, R, eps_u, g_scale, loss_r, g_logits, q);
  return launch_status();
}

extern "C" int dvgo_proposal_select(const float* q, const int64_t* ray_off, int64_t R, int32_t n_draw,
                                    int32_t* sel, int32_t* n_sel, void* stream) {
  DVGO_CHECK_ARG(R >= 0 && n_draw >= 1);
  if (R == 0) return DVGO_OK;
  DVGO_CHECK_ARG(q && ray_off && sel && n_sel);
  proposal_select_kernel<<<(int)ceil_div(R, 128), 128, 0, as_stream(stream)>>>(q, ray_off, R, n_draw,
                                                                              sel, n_sel);
  return launch_status();
}

extern "C" int dvgo_compact_samples(const int32_t* sel, const int32_t* n_sel, int32_t n_draw,
                                    const int64_t* ray_off, int64_t R, const float* xyz,
                                    const int32_t* ray_id, const int32_t* step_k, const float* s_mid,
                                    const float* s_len, int64_t* out_ray_off, float* out_xyz,
                                    int32_t* out_ray_id, int32_t* out_step_k, float* out_s_mid,
                                    float* out_s_len, int32_t* out_src, float interval,
                                    float* out_delta, void* stream) {
  DVGO_CHECK_ARG(R >= 0 && n_draw >= 1);
  DVGO_CHECK_ARG(!out_delta || interval > 0.0f);
  DVGO_CHECK_ARG(out_ray_off);
  cudaStream_t st = as_stream(stream);
  if (R == 0) {
    cudaMemsetAsync(out_ray_off, 0, sizeof(int64_t), st);
    return launch_status();
  }
  DVGO_CHECK_ARG(sel && n_sel && ray_off && xyz && ray_id && step_k && s_mid && s_len);
  DVGO_CHECK_ARG(out_xyz && out_ray_id && out_step_k && out_s_mid && out_s_len);
  scan_i32_kernel<<<1, 1024, 0, st>>>(n_sel, R, out_ray_off);
  compact_kernel<<<grid_for(R * 32, 256, 16), 256, 0, st>>>(
      sel, n_sel, n_draw, ray_off, R, xyz, ray_id, step_k, s_mid, s_len, out_ray_off, out_xyz,
      out_ray_id, out_step_k, out_s_mid, out_s_len, out_src, interval, out_delta);
  return launch_status();
}
