/*
 * dvgo.h — C ABI of the GB300 (sm_103a) DVGOv2 training-step library.
 *
 * Sun, Sun, Chen, "Improved Direct Voxel Grid Optimization for Radiance
 * Fields Reconstruction" (arXiv 2206.05085).  The library computes one
 * training iteration of the differentiable volume renderer: ray sampling
 * inside the scene bbox with occupancy culling, trilinear grid queries,
 * softplus-shifted raw->alpha, front-to-back compositing with early stop,
 * the colour MLP, the O(N) distortion loss, the TV gradient and the sparse
 * Adam grid step, each with its backward.
 *
 * Conventions (apply to every call unless stated):
 *  - Return value: DVGO_OK (0) or a negative dvgo_status.  Arguments are
 *    validated on the host before any launch; invalid arguments launch
 *    nothing.  DVGO_ERR_CUDA reports a launch error (cudaGetLastError).
 *  - No call allocates or frees memory, and no call synchronises except
 *    dvgo_device_status (a host read of the device status word, which must
 *    wait for the stream).  Every buffer is caller-owned device memory unless
 *    marked "host".  Scratch is passed as (ws, ws_bytes); the required size
 *    comes from the matching *_workspace_size call.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Ragged sample lists are CSR: ray_off[R+1] int64, non-decreasing,
 *    ray_off[0] = 0; the samples of ray r are [ray_off[r], ray_off[r+1]).
 *    Where a call takes seg_len[R] (int32, may be NULL), ray r is limited to
 *    its first seg_len[r] samples (the live samples before early stop).
 *  - Sample counts: calls over samples take a capacity n_cap (host) and an
 *    optional device count n_dev (int64, may be NULL).  With n_dev set only
 *    the first *n_dev (<= n_cap) samples are processed, so a whole
 *    iteration can run without reading counts back to the host.
 *  - Grids are corner aligned: grid point i along axis a sits at
 *    lo_a + i (hi_a - lo_a)/(G_a - 1).  Library-side grid storage is
 *    "bricked": 8x8x8 bricks in raster order (x fastest), Morton (z-order)
 *    order of the 512 voxels inside a brick, channels innermost.
 *    dvgo_grid_pack/unpack convert from/to the dense layout
 *    g[((z*Gy + y)*Gx + x)*C + c].
 *
 * Which calls are the operations of the method, and which are fusions:
 *  - The operations (one call each, each the plain form of one step):
 *    dvgo_sample_rays, dvgo_sample_grid_fwd / _bwd, dvgo_alpha_weights_fwd,
 *    dvgo_composite_fwd / _bwd, dvgo_composite_rgb_fwd,
 *    dvgo_distortion_fwd / _bwd, dvgo_rgb_loss, dvgo_rgbnet_fwd / _bwd,
 *    dvgo_tv_add_grad, dvgo_adam_step, dvgo_grid_adam_step, dvgo_build_mask,
 *    dvgo_update_mask, dvgo_grid_resample, dvgo_live_samples, and the
 *    learned proposal (dvgo_proposal_*, dvgo_compact_samples).
 *  - Fusions the training step uses, each equal to a sequence of the calls
 *    above (stated at each): dvgo_density_alpha_fwd, dvgo_sample_grid_bwd2,
 *    dvgo_composite_distortion_fwd / _bwd,
 *    dvgo_composite_distortion_loss_fwd / _fwd_bwd, dvgo_tv_add_grad_multi,
 *    dvgo_adam_step_multi / _multi_dev, dvgo_touched_compact.
 *  - Variants: dvgo_live_samples_cull (low-weight colour-query cull),
 *    dvgo_sample_rays_noalloc (no workspace).
 *  - Helpers: grid geometry, workspace sizes, dvgo_device_status, and one
 *    measurement aid that is no step of the method (dvgo_read_probe, last).
 */
#ifndef DVGO_H_
#define DVGO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DVGO_OK = 0,
  DVGO_ERR_INVALID_ARG = -1, /* null pointer, bad enum or parameter */
  DVGO_ERR_SHAPE = -2,       /* inconsistent sizes / capacity too small */
  DVGO_ERR_CUDA = -3,        /* a CUDA runtime error was reported */
  DVGO_ERR_BOUNDS = -4,      /* device-side bounds check failed (checked builds) */
  DVGO_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  DVGO_ERR_UNSUPPORTED = -6, /* valid but not implemented combination */
  DVGO_ERR_WORKSPACE = -7,   /* ws_bytes smaller than the required size */
  DVGO_ERR_RANGE = -8        /* a value left the range a split-FP16 operand holds */
} dvgo_status;

/* Arithmetic forms.  DVGO_F32_TC is a colour-MLP precision only: FP32
 * accuracy on the tensor cores (see dvgo_rgbnet_fwd). */
typedef enum { DVGO_F32 = 0, DVGO_BF16 = 1, DVGO_F32_TC = 2 } dvgo_dtype;

/* Scene grid: box [lo, hi] and grid points per axis (corner aligned). */
typedef struct {
  float lo[3];
  float hi[3];
  int32_t G[3];
} dvgo_grid_desc;

/* Ray sampler (Sec. 3 "Re-implement rendering utils", Sec. 5.3, Sec. 5.4).
 * mode 0 (bbox): t_k = t_lo + (k + step_offset) step, k < n, where
 *   [t_lo, t_hi] = [near, far], clipped to the ray/bbox slab when use_slab,
 *   n = min(max_steps, ceil((t_hi - t_lo)/step - step_offset)); a sample
 *   exists iff its point lies in the box and, with a mask, the mask is on at
 *   its nearest grid point.  All these decisions are IEEE FP32 with the
 *   operation order written in the sampler source, so they are reproducible
 *   bit for bit.  s_mid/s_len (the distortion loss's normalised interval)
 *   are (k + step_offset) step/(t_hi - t_lo) and step/(t_hi - t_lo).
 * mode 1 (contracted, Eq. ub): march x_{k+1} = x_k + h_k d from
 *   x_0 = o + near d with h_k = step_c / |J(x_k) d| (J the Jacobian of the
 *   contraction with parameter b, p = inf when p_inf else 2); emits the
 *   contracted points for k < max_steps while their contracted p-norm
 *   radius stays below (1 + b) - step_c; s_mid = (k + 0.5)/max_steps,
 *   s_len = 1/max_steps.
 * mode 2 (forward-facing, Sec. 5.3 "Points parameterization and sampling"):
 *   each world ray (d_z < 0, the camera looking down -z) is moved to the
 *   plane z = -ndc_near and warped to normalized device coordinates, o' =
 *   (-fx o_x/o_z, -fy o_y/o_z, 1 + 2 ndc_near/o_z), d' = (-fx (d_x/d_z -
 *   o_x/o_z), -fy (d_y/d_z - o_y/o_z), -2 ndc_near/o_z) with fx = ndc_fx, fy =
 *   ndc_fy (focal / half the image width / height); the grid is a stack of
 *   G_z depth layers over the box's z extent (multiplane images), and the
 *   samples are the ray's crossings of the layer planes z_k = lo_z + k step
 *   (hi_z - lo_z)/(G_z - 1), k < K = min(max_steps, floor((G_z - 1)/step) + 1)
 *   (step in layers); a crossing exists iff it lies in the box and, with a
 *   mask, the mask is on at its nearest grid point.  All in IEEE FP32 with
 *   the operation order of the sampler source.  s_mid = (k + 0.5)/K, s_len =
 *   1/K. */
typedef struct {
  int32_t mode;
  float near;
  float far;
  float step;
  float step_offset;
  int32_t use_slab;
  int32_t max_steps;
  float contract_b;
  int32_t p_inf;
  float step_c;
  float ndc_fx;
  float ndc_fy;
  float ndc_near;
} dvgo_sampler_desc;

int dvgo_version(void);
const char* dvgo_status_string(int status);

/* ------------------------------------------------------------------ grid */
/* Number of elements (voxels x C, including brick padding) of a bricked
 * grid with G points per axis and C channels. */
int64_t dvgo_grid_bricked_elems(const int32_t G[3], int32_t C);
int64_t dvgo_grid_num_bricks(const int32_t G[3]);

/* dense -> bricked (pack) and bricked -> dense (unpack).  dtype applies to
 * both buffers; padding voxels of the bricked grid are set to zero by pack. */
int dvgo_grid_pack(const void* dense, void* bricked, const int32_t G[3], int32_t C, int dtype,
                   void* stream);
int dvgo_grid_unpack(const void* bricked, void* dense, const int32_t G[3], int32_t C, int dtype,
                     void* stream);

/* Progressive grid scaling (Sec. 5.4, the grid-scaling schedule): the
 * bricked FP32 grid src (G_src points per axis, C channels) trilinearly
 * resampled to G_dst points per axis over the same box (corner-aligned
 * grids: destination point x of axis a sits at source index x (G_src - 1) /
 * (G_dst - 1)).  dst is bricked, dtype F32 or BF16 (rounded to nearest; the
 * renderer's copy of a BF16-stored grid).  Any G >= 2 on both sides
 * (down-sampling too).  Applied by the caller to each grid and to its Adam
 * moments when the schedule raises the resolution. */
int dvgo_grid_resample(const float* src, const int32_t G_src[3], void* dst, int dst_dtype,
                       const int32_t G_dst[3], int32_t C, void* stream);

/* Occupancy mask (Sec. 1): mask[v] = alpha(density[v]) >= alpha_thres with
 * alpha = 1 - exp(-interval softplus(raw + shift)).  density is bricked
 * (dtype F32 or BF16); mask is dense uint8 [Gz][Gy][Gx]. */
int dvgo_build_mask(const void* density, int dtype, const dvgo_grid_desc* grid, float shift,
                    float interval, float alpha_thres, uint8_t* mask, void* stream);

/* Progressive occupancy-mask update (Sec. 1: the mask is updated as training
 * goes, deactivating space whose density has become low): mask[v] =
 * alpha(density[v]) >= alpha_thres, as dvgo_build_mask decides it, re-evaluated
 * for the grid points of the listed bricks only (brick_list int32 [*brick_count],
 * both device; both NULL = every brick).  Given the bricks an optimizer step
 * changed (the compacted touched list of dvgo_touched_compact), it keeps the
 * mask equal to dvgo_build_mask of the current density. */
int dvgo_update_mask(const void* density, int dtype, const dvgo_grid_desc* grid, float shift, float interval,
                     float alpha_thres, const int32_t* brick_list, const int32_t* brick_count, uint8_t* mask,
                     void* stream);

/* Trilinear query (Sec. 1, "constant time" grid query) of a bricked grid
 * with C channels at points xyz[n][3] (f32).  u_a = (x_a - lo_a) (G_a - 1) /
 * (hi_a - lo_a) is clamped to [0, G_a - 1].  If idx (int32, may be NULL) is
 * given, thread j queries sample idx[j] and writes row idx[j] of out;
 * otherwise sample j.  out: f32 [.., C] rows at the sample index. */
int dvgo_sample_grid_fwd(const void* grid, int dtype, const dvgo_grid_desc* gd, int32_t C,
                         const float* xyz, const int32_t* idx, int64_t n_cap,
                         const int64_t* n_dev, float* out, void* stream);

/* Adjoint of dvgo_sample_grid_fwd: g_grid (bricked f32, C channels) +=
 * trilinear weights x g_out[row]; touched (uint8 per brick, may be NULL) is
 * set to 1 for every brick that received a contribution.  Uses atomics
 * (summation order is not deterministic). */
int dvgo_sample_grid_bwd(const float* g_out, const dvgo_grid_desc* gd, int32_t C, const float* xyz,
                         const int32_t* idx, int64_t n_cap, const int64_t* n_dev, float* g_grid,
                         uint8_t* touched, void* stream);

/* Both adjoints at once for two grids of the same geometry queried at the
 * same samples (the density grid, C_a channels, and the feature grid, C_b
 * channels): each sample's corners are located once.  Same result as the
 * two dvgo_sample_grid_bwd calls (g_out_a / g_grid_a / touched_a, then
 * g_out_b / g_grid_b / touched_b). */
int dvgo_sample_grid_bwd2(const float* g_out_a, int32_t C_a, float* g_grid_a, uint8_t* touched_a,
                          const float* g_out_b, int32_t C_b, float* g_grid_b, uint8_t* touched_b,
                          const dvgo_grid_desc* gd, const float* xyz, const int32_t* idx,
                          int64_t n_cap, const int64_t* n_dev, void* stream);

/* ---------------------------------------------------------------- sampler */
size_t dvgo_sample_rays_workspace_size(int64_t R);

/* Ray sampling (see dvgo_sampler_desc).  rays_o/rays_d: f32 [R][3].  mask:
 * dense uint8 grid (may be NULL).  Outputs (capacity S_cap >= R*max_steps
 * is required, so the list never overflows): ray_off [R+1] (ray_off[R] is
 * the sample count S), xyz [S_cap][3], ray_id, step_k [S_cap] int32,
 * s_mid, s_len [S_cap] f32.  ws: dvgo_sample_rays_workspace_size(R) bytes of
 * device scratch owned by the caller (per-ray counts, then per-ray keep bits
 * of the first 1024 steps, which the second pass reads instead of repeating
 * the occupancy lookups; longer marches repeat them).  Needs no clearing. */
int dvgo_sample_rays(const float* rays_o, const float* rays_d, int64_t R,
                     const dvgo_grid_desc* grid, const dvgo_sampler_desc* smp,
                     const uint8_t* mask, int64_t S_cap, int64_t* ray_off, float* xyz,
                     int32_t* ray_id, int32_t* step_k, float* s_mid, float* s_len, void* ws,
                     size_t ws_bytes, void* stream);

/* dvgo_sample_rays for callers that cannot allocate device memory (for
 * instance a host application that owns the whole memory budget and does not
 * let libraries allocate, so no workspace can be passed).  The paper has no
 * counterpart; this is a deployment variant.  Same arguments and results as
 * dvgo_sample_rays without ws/ws_bytes.  Its scratch is a fixed array inside
 * the library, present on every GPU that loads the library until the
 * process exits, limited to R <= dvgo_sample_rays_noalloc_max_rays()
 * (1,048,576 rays; larger R returns DVGO_ERR_SHAPE).  The first call in a
 * context (per device, and again after that device's context was destroyed
 * and re-created, e.g. by cudaDeviceReset) looks the array's device address
 * up (cudaGetSymbolAddress) and caches it with the context's identity, so
 * make the first call on a device, and the first call after a reset, before
 * any stream capture.  The array needs no clearing: each call writes every
 * count it reads.  All calls share the one array: calls that overlap on the
 * GPU (other streams, other threads) race and must be serialised by the
 * caller.  No allocation of any kind is made. */
int64_t dvgo_sample_rays_noalloc_max_rays(void);
int dvgo_sample_rays_noalloc(const float* rays_o, const float* rays_d, int64_t R,
                             const dvgo_grid_desc* grid, const dvgo_sampler_desc* smp,
                             const uint8_t* mask, int64_t S_cap, int64_t* ray_off, float* xyz,
                             int32_t* ray_id, int32_t* step_k, float* s_mid, float* s_len,
                             void* stream);

/* Live-sample list after early stop: live_idx lists, ray by ray, the first
 * seg_len[r] samples of every ray (the samples with nonzero weight), and
 * *live_count their number.  live_idx: int32 [capacity ray_off total].
 * ws: dvgo_live_samples_workspace_size(R) bytes. */
size_t dvgo_live_samples_workspace_size(int64_t R);

/* The colour-query list with low-weight samples skipped (a variant; DVGO's
 * implementations skip colour queries of points with negligible compositing
 * weight): the first seg_len[r] samples of every ray whose weight w[s] >=
 * w_min, in ray order, and *live_count their number.  The rows of the skipped
 * samples (before the halt, w < w_min) are set to zero in rgb [S][3] and g_k0
 * [S][12] (each may be NULL; g_k0 16-byte aligned): their colour contributes
 * nothing to the render and their features receive no gradient, so the
 * compositing, its adjoint and the grid adjoints can keep using the full
 * live list.  ws: dvgo_live_samples_workspace_size(R) bytes. */
int dvgo_live_samples_cull(const int64_t* ray_off, const int32_t* seg_len, const float* w, float w_min,
                           int64_t R, int32_t* live_idx, int64_t* live_count, float* rgb, float* g_k0,
                           void* ws, size_t ws_bytes, void* stream);
int dvgo_live_samples(const int64_t* ray_off, const int32_t* seg_len, int64_t R,
                      int32_t* live_idx, int64_t* live_count, void* ws, size_t ws_bytes,
                      void* stream);

/* -------------------------------------------------------------- rendering */
/* Per-sample intervals: the calls that turn raw into alpha take the common
 * alpha interval (voxel units) and an optional per-sample array delta [S]
 * (f32, may be NULL); sample s uses delta[s] when it is given (a sample that
 * stands for the stretch up to the next one, as the learned proposal's picks
 * do), else interval.  "interval" below means that per-sample value.
 *
 * raw -> alpha and transmittance (Sec. 3 "Re-implement rendering utils",
 * fused): per ray, alpha_i = 1 - exp(-interval softplus(raw_i + shift)),
 * T_i = prod_{j<i}(1 - alpha_j) carried as an FP32 log-sum with compensated
 * carries, w_i = T_i alpha_i; the ray halts at the first i with T_i < T_stop
 * (that sample is not composited).  Writes w[S], T[S] (T_end beyond the
 * stop), n_live[R] (halting index) and T_end[R]. */
int dvgo_alpha_weights_fwd(const float* raw, const int64_t* ray_off, int64_t R, float shift,
                           float interval, const float* delta, float T_stop, float* w, float* T,
                           int32_t* n_live, float* T_end, void* stream);

/* The whole compositing forward of a ray batch in one call:
 * dvgo_alpha_weights_fwd (raw -> w, T, n_live, T_end) followed by
 * dvgo_composite_rgb_fwd (color).  Its adjoint is dvgo_composite_bwd. */
int dvgo_composite_fwd(const float* raw, const float* rgb, const int64_t* ray_off, int64_t R,
                       float shift, float interval, const float* delta, float T_stop, const float bg[3],
                       float* color, float* w, float* T, int32_t* n_live, float* T_end, void* stream);

/* dvgo_sample_grid_fwd of a one-channel density grid fused with
 * dvgo_alpha_weights_fwd: raw[S], w[S], T[S], n_live[R], T_end[R] as those
 * two calls define them, except that samples at or past a ray's halting
 * index are not queried (their raw is written as 0; nothing downstream reads
 * it).  xyz [S][3] f32 in ray order (the sampler's output). */
int dvgo_density_alpha_fwd(const void* grid, int dtype, const dvgo_grid_desc* gd, const float* xyz,
                           const int64_t* ray_off, int64_t R, float shift, float interval,
                           const float* delta, float T_stop, float* raw, float* w, float* T,
                           int32_t* n_live, float* T_end, void* stream);

/* Colour accumulation: color[r] = sum_{i < n_live[r]} w_i rgb_i + T_end[r] bg. */
int dvgo_composite_rgb_fwd(const float* w, const float* rgb, const int64_t* ray_off,
                           const int32_t* n_live, const float* T_end, int64_t R, const float bg[3],
                           float* color, void* stream);

/* Backward of raw->alpha + compositing: with g_i = <rgb_i, g_color[r]> +
 * g_w[i] (rgb and g_w may be NULL: that term is 0) and g_T = <bg,
 * g_color[r]>, the reverse recurrence over the live samples
 * R_k = g_{k+1} alpha_{k+1} + (1 - alpha_{k+1}) R_{k+1}, R_{n-1} = g_T, gives
 * g_raw[k] = interval sigmoid(raw_k + shift) T_{k+1} (g_k - R_k).  It is
 * evaluated as T_{k+1} g_k - S_k with the suffix sum S_k = T_{k+1} R_k =
 * sum_{j>k} g_j w_j + g_T T_end (compensated FP32 sums, so the error does not
 * grow with the ray's length).  g_rgb (may be NULL) receives w_k g_color[r].
 * Samples past the halting index get zero gradients. */
int dvgo_composite_bwd(const float* g_color, const float* g_w, const float* raw, const float* T,
                       const float* rgb, const int64_t* ray_off, const int32_t* n_live, int64_t R,
                       float shift, float interval, const float* delta, const float bg[3], float* g_raw,
                       float* g_rgb, void* stream);

/* Distortion loss (Sec. 2, Eq. dist_loss, O(N) prefix-sum form) per ray:
 * L_r = 2 sum_i w_i (m_i W_{<i} - WM_{<i}) + 1/3 sum_i w_i^2 ds_i over the
 * ray's first seg_len[r] samples (all samples if seg_len is NULL); the
 * running sums of w and w m are Kahan-compensated FP32. */
int dvgo_distortion_fwd(const float* w, const float* m, const float* ds, const int64_t* ray_off,
                        const int32_t* seg_len, int64_t R, float* L_r, void* stream);

/* Gradient (Sec. 2): g_w[k] = g_L[r] (2 (m_k W_{<k} - WM_{<k} + WM_{>k} -
 * m_k W_{>k}) + 2/3 w_k ds_k); g_L is per ray, or (g_L == NULL) the scalar
 * g_L_scalar for every ray.  Samples beyond seg_len get 0. */
int dvgo_distortion_bwd(const float* g_L, float g_L_scalar, const float* w, const float* m,
                        const float* ds, const int64_t* ray_off, const int32_t* seg_len, int64_t R,
                        float* g_w, void* stream);

/* The two per-ray forward tails in one pass over each ray's live samples:
 * dvgo_composite_rgb_fwd (color) and dvgo_distortion_fwd with seg_len =
 * n_live (L_r), m = sample midpoints, ds = interval lengths. */
int dvgo_composite_distortion_fwd(const float* w, const float* rgb, const float* m, const float* ds,
                                  const int64_t* ray_off, const int32_t* n_live, const float* T_end,
                                  int64_t R, const float bg[3], float* color, float* L_r,
                                  void* stream);

/* dvgo_composite_bwd (g_rgb not written) with g_w = the distortion gradient
 * of dvgo_distortion_bwd for the scalar upstream g_L and seg_len = n_live,
 * formed inside the compositing adjoint's reverse scan (never stored). */
int dvgo_composite_distortion_bwd(const float* g_color, float g_L, const float* w, const float* raw,
                                  const float* T, const float* rgb, const float* m, const float* ds,
                                  const int64_t* ray_off, const int32_t* n_live, int64_t R,
                                  float shift, float interval, const float* delta, const float bg[3],
                                  float* g_raw, void* stream);

/* dvgo_composite_distortion_fwd and dvgo_rgb_loss (with L_r) in one launch:
 * color, L_r, g_color and loss_out exactly as those two calls define them
 * (the loss sums are added in a different but fixed order: deterministic).
 * ws: dvgo_composite_loss_workspace_size(R) bytes, 16-byte aligned, zeroed
 * by the caller before its first use; every call leaves it zeroed again. */
size_t dvgo_composite_loss_workspace_size(int64_t R);
int dvgo_composite_distortion_loss_fwd(const float* w, const float* rgb, const float* m,
                                       const float* ds, const int64_t* ray_off,
                                       const int32_t* n_live, const float* T_end, int64_t R,
                                       const float bg[3], const float* target, float lambda_dist,
                                       float* color, float* L_r, float* g_color, float* loss_out,
                                       void* ws, void* stream);

/* dvgo_composite_distortion_loss_fwd and then, for each ray in the same warp
 * with the g_color just formed, dvgo_composite_distortion_bwd (g_L, raw, T,
 * shift, interval as that call takes them): color, L_r, g_color, loss_out
 * and g_raw [S] bit-equal to the two calls, in one launch (one pass of the
 * per-ray tail of a training step).  ws as for the forward call. */
int dvgo_composite_distortion_loss_fwd_bwd(const float* w, const float* rgb, const float* m,
                                           const float* ds, const int64_t* ray_off,
                                           const int32_t* n_live, const float* T_end, int64_t R,
                                           const float bg[3], const float* target,
                                           float lambda_dist, float g_L, const float* raw,
                                           const float* T, float shift, float interval,
                                           const float* delta, float* color, float* L_r,
                                           float* g_color, float* loss_out, float* g_raw, void* ws,
                                           void* stream);

/* Photometric loss and its gradient: loss_out[0] = mean over R x 3 of
 * (color - target)^2, loss_out[1] = mean_r L_r (0 if L_r is NULL),
 * loss_out[2] = loss_out[0] + lambda_dist loss_out[1]; g_color =
 * 2 (color - target)/(3R).  Deterministic single-pass reduction. */
int dvgo_rgb_loss(const float* color, const float* target, const float* L_r, int64_t R,
                  float lambda_dist, float* loss_out, float* g_color, void* stream);

/* -------------------------------------------------------------- colour MLP */
/* rgbnet (Tab. 1 "hybrid" colour): input [k0 (12 features), view-direction
 * encoding [d, sin(2^f d_a), cos(2^f d_a)], f < 4, axis major] = 39 ->
 * ReLU 128 -> ReLU 128 -> sigmoid 3.  params: f32 flat W1[128][39], b1,
 * W2[128][128], b2, W3[3][128], b3 (22019 values).  Processes samples
 * idx[j] (j < *n_dev or n_cap); k0 rows and rgb rows are at the sample
 * index; the direction is rays_d[ray_id[sample]].  precision:
 *   DVGO_F32     exact FP32 on the CUDA cores;
 *   DVGO_F32_TC  FP32 accuracy on the tensor cores: every operand, after an
 *                exact power-of-two scale, is split into two FP16 terms
 *                hi + lo and each product is taken as hi*hi + hi*lo + lo*hi
 *                with FP32 accumulation (relative error about 2^-22 per
 *                product, like FP32 arithmetic).  Inputs must stay below
 *                512 in magnitude and hidden activations below 2048, else
 *                dvgo_device_status reports DVGO_ERR_RANGE;
 *   DVGO_BF16    the BF16 form: the parameters are used as their BF16
 *                values (the stored precision of this form) and every
 *                tensor-core operand is BF16 with FP32 accumulation; weight
 *                matrices are one BF16 term, every other operand (layer
 *                inputs, hidden activations, gradient rows) two BF16 terms
 *                hi + lo (16 significant bits), so no value is rounded to
 *                BF16 between layers.  Same kernels and workspace as
 *                DVGO_F32_TC; no range limit.
 * act: DVGO_F32 may be NULL, else see dvgo_rgbnet_bwd; DVGO_F32_TC and
 * DVGO_BF16 required, dvgo_rgbnet_act_bytes(n_cap, precision) bytes,
 * 16-byte aligned (the forward stores each 128-sample tile's split layer
 * inputs for the backward). */
int dvgo_rgbnet_fwd(const float* k0, const float* rays_d, const int32_t* ray_id,
                    const int32_t* idx, int64_t n_cap, const int64_t* n_dev, const float* params,
                    int precision, float* rgb, float* act, void* stream);

/* Backward: the upstream colour gradient of sample s is g_rgb[s] (f32
 * [.., 3] at the sample index) when g_rgb is given, else w[s] *
 * g_color[ray_id[s]] (the colour part of the compositing gradient).
 * Accumulates g_params (+=, f32) and writes g_k0 [.., 12] rows at the
 * sample index.  act (FP32 form, may be NULL): f32 [n_cap][256] written by
 * dvgo_rgbnet_fwd for the same list, row j = [h1 (128) | h2 (128)] of list
 * position j; with it (and rgb, the forward's output, may be NULL) the
 * backward reads the hidden activations instead of recomputing them.
 * DVGO_F32_TC and DVGO_BF16: act is the buffer its forward filled for the
 * same list and count, and rgb that forward's output (both required: the
 * output layer's sigmoid derivative is y (1 - y) with y = rgb[s], not
 * recomputed); the backward also writes the per-CTA partial gradients
 * stored after the tile images, and sums those partials in a fixed order
 * (deterministic). */
int dvgo_rgbnet_bwd(const float* g_rgb, const float* g_color, const float* w, const float* k0,
                    const float* rays_d, const int32_t* ray_id, const int32_t* idx, int64_t n_cap,
                    const int64_t* n_dev, const float* params, int precision, const float* act,
                    const float* rgb, float* g_params, float* g_k0, void* stream);

/* Bytes of the act buffer dvgo_rgbnet_fwd / _bwd need for n_cap list
 * positions: n_cap * 1024 for DVGO_F32 (optional there); for DVGO_F32_TC and
 * DVGO_BF16 256 + 90112 per 128-position tile + 152 * 22019 * 4 (one partial
 * parameter gradient per SM); -1 for a bad precision or n_cap < 0. */
int64_t dvgo_rgbnet_act_bytes(int64_t n_cap, int precision);

/* ------------------------------------------------------- learned proposal */
/* Not in the paper: a small network that predicts where each ray's
 * compositing weight lies, so that far fewer samples are rendered.  It is
 * trained on the plain renderer's own weights and the plain dense render
 * stays the fallback.  Network: position encoding [x, sin(2^f x_a),
 * cos(2^f x_a)], f < 6 (39 values) -> ReLU 64 -> ReLU 64 -> 1 logit, in the
 * BF16 form of dvgo_rgbnet_fwd: parameters used as their BF16 values, BF16
 * tensor-core operands (weights one term, inputs, activations and gradient
 * rows two terms) with FP32 accumulation.  params: f32 flat W1[64][39], b1,
 * W2[64][64], b2, W3[1][64], b3 (6785 values). */
int dvgo_proposal_fwd(const float* xyz, const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                      const float* params, float* logits, void* stream);
/* Accumulates g_params (+=) from the per-sample logit gradients. */
int dvgo_proposal_bwd(const float* g_logits, const float* xyz, const int32_t* idx, int64_t n_cap,
                      const int64_t* n_dev, const float* params, float* g_params, void* stream);
/* Per ray (CSR ray_off): q = softmax(logits); with w_target (the plain
 * renderer's weights over the same samples, may be NULL) the target is
 * p_j = (w_j / W + eps_u) / (1 + N eps_u), W = sum w (uniform if W = 0),
 * loss_r = -sum p_j log q_j and g_logits = g_scale (q - p).  q, loss_r and
 * g_logits may each be NULL. */
int dvgo_proposal_xent(const float* logits, const float* w_target, const int64_t* ray_off, int64_t R,
                       float eps_u, float g_scale, float* loss_r, float* g_logits, float* q,
                       void* stream);
/* Inverse-CDF selection per ray: for u_k = (k + 0.5)/n_draw, k < n_draw, the
 * first candidate j whose running FP32 sum of q (in candidate order)
 * exceeds u_k; repeated picks collapse.  sel [R][n_draw] holds candidate
 * indices relative to the ray start (ascending, -1 past n_sel[r]). */
int dvgo_proposal_select(const float* q, const int64_t* ray_off, int64_t R, int32_t n_draw,
                         int32_t* sel, int32_t* n_sel, void* stream);
/* Gathers the selected samples into a new ragged list (out_ray_off [R+1]
 * from a scan of n_sel; per-sample arrays copied; out_src, may be NULL,
 * receives each kept sample's index in the input list).
 * out_delta (f32 [n], may be NULL): each pick then stands for the candidates
 * from itself up to the next pick of its ray (the last pick: up to the ray's
 * last candidate), so that the picks cover the same depth range as the
 * candidates.  For pick j with next pick j' (j' = the ray's candidate count
 * after the last pick) the kernel writes, in FP32 round-to-nearest,
 *   out_delta = interval * (j' - j)   (the per-sample alpha interval of
 *                                      dvgo_alpha_weights_fwd, voxel units)
 *   start = s_mid[j] - 0.5 s_len[j]; end = s_mid[j'] - 0.5 s_len[j'], or
 *   s_mid[last] + 0.5 s_len[last] after the last pick;
 *   out_s_mid = 0.5 (start + end); out_s_len = end - start.
 * (The candidates are contiguous spans.)  interval > 0 when out_delta is
 * given, else ignored. */
int dvgo_compact_samples(const int32_t* sel, const int32_t* n_sel, int32_t n_draw,
                         const int64_t* ray_off, int64_t R, const float* xyz, const int32_t* ray_id,
                         const int32_t* step_k, const float* s_mid, const float* s_len,
                         int64_t* out_ray_off, float* out_xyz, int32_t* out_ray_id,
                         int32_t* out_step_k, float* out_s_mid, float* out_s_len, int32_t* out_src,
                         float interval, float* out_delta, void* stream);

/* ------------------------------------------------------------ regularisers */
/* TV gradient (Sec. 2, "Efficient total variation (TV) loss"), added into
 * g_grid without a forward pass: for each grid point v and channel c,
 * g += weight * 2/(N C) sum_{u in 6-nbr(v)} clamp(grid[v,c] - grid[u,c],
 * -delta, delta), N = number of grid points.  dense_mode != 0: every entry;
 * otherwise only entries whose incoming gradient is nonzero, and only in
 * bricks flagged in touched (uint8 per brick, may be NULL = all bricks).  In
 * dense mode every flag of touched (if given) is set to 1.  grid and g_grid
 * are bricked; grid dtype F32 or BF16, g_grid f32. */
int dvgo_tv_add_grad(const void* grid, int dtype, const int32_t G[3], int32_t C, float weight,
                     float delta, int dense_mode, uint8_t* touched, float* g_grid, void* stream);

/* Several grids of the same shape G in one launch (the density and the
 * feature grid of a step): grid i behaves as dvgo_tv_add_grad(grids[i].grid,
 * grids[i].dtype, G, grids[i].C, grids[i].weight, delta, dense_mode,
 * grids[i].touched, grids[i].g_grid).  count <= 4; grids is a host array. */
typedef struct {
  const void* grid;
  int32_t dtype;
  int32_t C;
  float weight;
  uint8_t* touched;
  float* g_grid;
} dvgo_tv_grid;

int dvgo_tv_add_grad_multi(const dvgo_tv_grid* grids, int32_t count, const int32_t G[3], float delta,
                           int dense_mode, const int32_t* brick_list, const int32_t* brick_count,
                           void* stream);

/* Compacted list of the flagged bricks: list[0 .. *count) = the indices b
 * with touched[b] != 0, in no particular order (list holds nb entries;
 * count is one int32 on the device, written here).  Given to
 * dvgo_tv_add_grad_multi (brick_list / brick_count, sparse mode; NULL =
 * visit every brick and test its flag) and to dvgo_adam_step_multi
 * (block_list / block_count of a bricked array), the kernels visit only those
 * bricks, spread evenly over persistent blocks. */
int dvgo_touched_compact(const uint8_t* touched, int64_t nb, int32_t* list, int32_t* count,
                         void* stream);

/* ------------------------------------------------------------------ Adam */
/* Fused Adam (Sec. 3 "Re-implement Adam optimizer"): for each entry with a
 * nonzero gradient, m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps); entries with g == 0 are
 * left untouched.  With touched (uint8 per block of block_elems entries,
 * may be NULL) only flagged blocks are visited.  zero_grad != 0 clears the
 * visited gradients and the visited flags.  p_shadow (may be NULL) receives
 * a BF16 copy of every updated p. */
int dvgo_adam_step(float* p, uint16_t* p_shadow, float* g, float* m, float* v, int64_t n,
                   uint8_t* touched, int64_t block_elems, float lr, float beta1, float beta2,
                   float eps, int64_t step, int zero_grad, void* stream);

/* The sparse Adam step of a bricked grid (Sec. 3): dvgo_adam_step with the
 * grid's brick flags (one uint8 per brick of 512 voxels, C channels each, so
 * block_elems = 512 C); a NULL touched visits every brick and skips g == 0. */
int dvgo_grid_adam_step(float* p, uint16_t* p_shadow, float* g, float* m, float* v,
                        const int32_t G[3], int32_t C, uint8_t* touched, float lr, float beta1,
                        float beta2, float eps, int64_t step, int zero_grad, void* stream);

/* Several parameter arrays in one launch (density grid, feature grid, colour
 * MLP): params[i] behaves as dvgo_adam_step(params[i].p, .p_shadow, .g, .m,
 * .v, .n, .touched, .block_elems, .lr, beta1, beta2, eps, step, zero_grad).
 * count <= 4; params is a host array; p, g, m, v 16-byte aligned (p_shadow
 * 8-byte aligned) and, with touched, block_elems a multiple of 4. */
typedef struct {
  float* p;
  uint16_t* p_shadow;
  float* g;
  float* m;
  float* v;
  int64_t n;
  uint8_t* touched;
  int64_t block_elems;
  float lr;
  const int32_t* block_list;   /* optional (with touched): the flagged blocks, see dvgo_touched_compact */
  const int32_t* block_count;
} dvgo_adam_param;

int dvgo_adam_step_multi(const dvgo_adam_param* params, int32_t count, float beta1, float beta2,
                         float eps, int64_t step, int zero_grad, void* stream);

/* Same, with the step count on the device: step points to two int64 words;
 * step[0] (t) is incremented by one and used, step[1] receives the two FP32
 * bias corrections of the new t (scratch).  A captured CUDA graph of a
 * training step can then be replayed step after step. */
int dvgo_adam_step_multi_dev(const dvgo_adam_param* params, int32_t count, float beta1, float beta2,
                             float eps, int64_t* step, int zero_grad, void* stream);

/* Reads and clears the device status word that kernels with bounded waits
 * set (DVGO_ERR_TIMEOUT) instead of hanging.  Synchronises the stream. */
int dvgo_device_status(void* stream);

/* ------------------------------------------------------ measurement aid */
/* Not a step of the method (the benchmark's L2 read-rate probe): sink_len
 * blocks of 512 threads each read the first bytes/16 float4 of buf (16-byte
 * aligned) reps times and
 * add a checksum into sink[block] (f32 [sink_len], caller-zeroed).  A buffer
 * well inside L2 gives the L2 read rate the gathers' corner reads see. */
int dvgo_read_probe(const void* buf, int64_t bytes, int32_t reps, float* sink, int32_t sink_len,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DVGO_H_ */
