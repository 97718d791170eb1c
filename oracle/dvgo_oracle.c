/*
 * FP64 CPU oracle for the DVGOv2 volume-rendering training step
 * (Sun, Sun, Chen: "Improved Direct Voxel Grid Optimization for Radiance
 * Fields Reconstruction", arXiv 2206.05085).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA library; each function below writes out
 * the plain definition the paper gives (or, where the paper is silent, the
 * documented reading of it) with plain loops, one ray or one grid point at a
 * time, with no blocking and no fusion.
 *
 * Precision: FP64 for every value.  The only exceptions are the integer
 * decisions of the ray sampler (which samples exist, their step index and
 * the occupancy lookup).  Those are taken in IEEE FP32 with the fixed
 * operation order stated at each function, so that both implementations
 * reach the same integers; this file must be compiled with
 * -ffp-contract=off and without -ffast-math.
 *
 * Layouts (all arrays are caller-owned):
 *   dense grid   g[((z*Gy + y)*Gx + x)*C + c]   (x fastest, channel innermost)
 *   ragged lists CSR: ray_off[R+1], samples of ray r are
 *                [ray_off[r], ray_off[r+1]); an optional seg_len[r] limits a
 *                ray to its first seg_len[r] samples.
 *
 * Parity status per function is listed in the Python wrapper's docstring.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* raw -> alpha (Sec. 3 "Re-implement rendering utils"; alpha_init of Sec.  */
/* 5.3).  alpha = 1 - (1 + exp(raw + shift))^(-interval)                     */
/*              = 1 - exp(-interval * softplus(raw + shift)),                */
/* with shift = log(1/(1 - alpha_init) - 1) so that raw = 0 gives            */
/* alpha = 1 - (1 - alpha_init)^interval.                                    */
/* ------------------------------------------------------------------------ */
static double softplus(double x) { return (x > 0 ? x : 0.0) + log1p(exp(-fabs(x))); }
static double sigmoid(double x) { return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x)); }

OR_API double or_alpha_shift(double alpha_init) { return log(1.0 / (1.0 - alpha_init) - 1.0); }

OR_API void or_raw2alpha(const double* raw, int64_t n, double shift, double interval,
                         double* alpha, double* dalpha_draw) {
  for (int64_t i = 0; i < n; ++i) {
    double sp = softplus(raw[i] + shift);
    double a = -expm1(-interval * sp);
    alpha[i] = a;
    /* d alpha / d raw = interval * (1 - alpha) * sigmoid(raw + shift) */
    if (dalpha_draw) dalpha_draw[i] = interval * (1.0 - a) * sigmoid(raw[i] + shift);
  }
}

/* Occupancy mask (Sec. 1): a grid point is on iff its alpha >= thres. */
OR_API void or_build_mask(const float* density, int64_t n, double shift, double interval,
                          double thres, uint8_t* mask) {
  for (int64_t i = 0; i < n; ++i) {
    double a = -expm1(-interval * softplus((double)density[i] + shift));
    mask[i] = (uint8_t)(a >= thres);
  }
}

/* ------------------------------------------------------------------------ */
/* Ray sampling inside the scene bbox (Sec. 3 "Re-implement rendering        */
/* utils": sample only where the ray meets the bbox) with occupancy culling  */
/* (Sec. 1).  FP32 decisions, operation order:                               */
/*   slab (use_slab): for each axis a with d_a != 0:                         */
/*       ta = (lo_a - o_a) / d_a ; tb = (hi_a - o_a) / d_a                   */
/*       tlo = max(tlo, min(ta,tb)) ; thi = min(thi, max(ta,tb))             */
/*     starting from tlo = near, thi = far; an axis with d_a == 0 and o_a    */
/*     outside [lo_a, hi_a] empties the ray.                                 */
/*   n = thi > tlo ? min(max_steps, ceil((thi - tlo) / step - off)) : 0      */
/*   t_k = tlo + ((float)k + off) * step ;  x_a = o_a + t_k * d_a            */
/*   keep iff lo_a <= x_a <= hi_a for all a, and (no mask or                 */
/*   mask[nearest] != 0) with nearest_a = clamp(floor(u_a + 0.5), 0, G_a-1),  */
/*   u_a = (x_a - lo_a) * ((float)(G_a - 1) / (hi_a - lo_a)).                 */
/* The normalised distance of Eq. (dist_loss) is s = (t - tlo)/(thi - tlo);  */
/* the sample is the interval centred at t_k of length step, so              */
/* s_mid = (k + off) * step / (thi - tlo) and s_len = step / (thi - tlo).    */
/* Returns the total sample count S; writes at most cap samples.             */
/* ------------------------------------------------------------------------ */
static int nearest_index(float x, float lo, float hi, int G) {
  float scale = (float)(G - 1) / (hi - lo);
  float u = (x - lo) * scale;
  float f = floorf(u + 0.5f);
  int n = (int)f;
  if (!(f >= 0.0f)) n = 0;
  if (f > (float)(G - 1)) n = G - 1;
  return n;
}

static int mask_on(const uint8_t* mask, const int32_t G[3], const float lo[3], const float hi[3],
                   const float x[3]) {
  if (!mask) return 1;
  int ix = nearest_index(x[0], lo[0], hi[0], G[0]);
  int iy = nearest_index(x[1], lo[1], hi[1], G[1]);
  int iz = nearest_index(x[2], lo[2], hi[2], G[2]);
  return mask[((int64_t)iz * G[1] + iy) * G[0] + ix] != 0;
}

OR_API int64_t or_sample_rays_bbox(const float* o, const float* d, int64_t R,
                                   const float lo[3], const float hi[3], const int32_t G[3],
                                   float near, float far, float step, float off, int use_slab,
                                   int32_t max_steps, const uint8_t* mask,
                                   int64_t* ray_off, float* xyz, int32_t* ray_id, int32_t* step_k,
                                   double* s_mid, double* s_len, int64_t cap) {
  int64_t S = 0;
  ray_off[0] = 0;
  for (int64_t r = 0; r < R; ++r) {
    const float* ro = o + 3 * r;
    const float* rd = d + 3 * r;
    float tlo = near, thi = far;
    int empty = 0;
    if (use_slab) {
      for (int a = 0; a < 3; ++a) {
        if (rd[a] == 0.0f) {
          if (ro[a] < lo[a] || ro[a] > hi[a]) empty = 1;
        } else {
          float ta = (lo[a] - ro[a]) / rd[a];
          float tb = (hi[a] - ro[a]) / rd[a];
          float tn = ta < tb ? ta : tb;
          float tf = ta < tb ? tb : ta;
          if (tn > tlo) tlo = tn;
          if (tf < thi) thi = tf;
        }
      }
    }
    int32_t n = 0;
    if (!empty && thi > tlo) {
      float u = (thi - tlo) / step;
      float nf = ceilf(u - off);
      if (nf > (float)max_steps) n = max_steps;
      else if (nf > 0.0f) n = (int32_t)nf;
    }
    for (int32_t k = 0; k < n; ++k) {
      float t = tlo + ((float)k + off) * step;
      float x[3];
      int inside = 1;
      for (int a = 0; a < 3; ++a) {
        x[a] = ro[a] + t * rd[a];
        if (!(x[a] >= lo[a] && x[a] <= hi[a])) inside = 0;
      }
      if (!inside || !mask_on(mask, G, lo, hi, x)) continue;
      if (S < cap) {
        xyz[3 * S + 0] = x[0];
        xyz[3 * S + 1] = x[1];
        xyz[3 * S + 2] = x[2];
        ray_id[S] = (int32_t)r;
        step_k[S] = k;
        double span = (double)thi - (double)tlo;
        s_mid[S] = ((double)k + (double)off) * (double)step / span;
        s_len[S] = (double)step / span;
      }
      ++S;
    }
    ray_off[r + 1] = S;
  }
  return S;
}

/* ------------------------------------------------------------------------ */
/* Forward-facing scenes (Sec. 5.3 "Points parameterization and sampling"):  */
/* NeRF's normalized device coordinates warp the frustum in front of a       */
/* camera looking down -z to a box; the grid is D depth layers over the      */
/* box's z extent (multiplane images) and the samples are the ray's          */
/* crossings of the layer planes, one every `step` layers.                   */
/* Per ray (d_z < 0, else no samples), in FP32 with this operation order:    */
/*   t  = -(near + o_z)/d_z ; p_a = o_a + t*d_a  (the ray moved to z = -near) */
/*   rx = p_x/p_z ; ry = p_y/p_z  (no samples unless p_z < 0)                 */
/*   o' = (-(fx*rx), -(fy*ry), 1 + (2*near)/p_z)                             */
/*   d' = (-(fx*(d_x/d_z - rx)), -(fy*(d_y/d_z - ry)), -((2*near)/p_z))       */
/*   K  = min(max_steps, floor((G_z - 1)/step) + 1)                          */
/*   layer k < K: dz = (hi_z - lo_z)/(G_z - 1) ; z = lo_z + (k*step)*dz ;     */
/*                t = (z - o'_z)/d'_z ; x = (o'_x + t*d'_x, o'_y + t*d'_y, z) */
/* A crossing exists iff it lies in the box and the mask is on at its        */
/* nearest grid point.  Distortion coordinates: s_mid = (k + 0.5)/K,         */
/* s_len = 1/K (uniform in layer index, i.e. in inverse depth).              */
/* ------------------------------------------------------------------------ */
OR_API int64_t or_sample_rays_ndc(const float* o, const float* d, int64_t R, const float lo[3],
                                  const float hi[3], const int32_t G[3], float fx, float fy,
                                  float near, float step, int32_t max_steps, const uint8_t* mask,
                                  int64_t* ray_off, float* xyz, int32_t* ray_id, int32_t* step_k,
                                  double* s_mid, double* s_len, int64_t cap) {
  int64_t S = 0;
  ray_off[0] = 0;
  for (int64_t r = 0; r < R; ++r) {
    const float* ro = o + 3 * r;
    const float* rd = d + 3 * r;
    int32_t K = 0;
    float qo[3] = {0, 0, 0}, qd[3] = {0, 0, 0};
    if (rd[2] < 0.0f) {
      float t = -(near + ro[2]) / rd[2];
      float px = ro[0] + t * rd[0], py = ro[1] + t * rd[1], pz = ro[2] + t * rd[2];
      if (pz < 0.0f) {
        float rx = px / pz, ry = py / pz, two_n = 2.0f * near;
        qo[0] = -(fx * rx);
        qo[1] = -(fy * ry);
        qo[2] = 1.0f + two_n / pz;
        qd[0] = -(fx * (rd[0] / rd[2] - rx));
        qd[1] = -(fy * (rd[1] / rd[2] - ry));
        qd[2] = -(two_n / pz);
        float nf = floorf((float)(G[2] - 1) / step);
        K = (int32_t)nf + 1;
        if (K > max_steps) K = max_steps;
      }
    }
    float dz = (hi[2] - lo[2]) / (float)(G[2] - 1);
    for (int32_t k = 0; k < K; ++k) {
      float z = lo[2] + ((float)k * step) * dz;
      float t = (z - qo[2]) / qd[2];
      float x[3] = {qo[0] + t * qd[0], qo[1] + t * qd[1], z};
      int inside = 1;
      for (int a = 0; a < 3; ++a)
        if (!(x[a] >= lo[a] && x[a] <= hi[a])) inside = 0;
      if (!inside || !mask_on(mask, G, lo, hi, x)) continue;
      if (S < cap) {
        xyz[3 * S + 0] = x[0];
        xyz[3 * S + 1] = x[1];
        xyz[3 * S + 2] = x[2];
        ray_id[S] = (int32_t)r;
        step_k[S] = k;
        s_mid[S] = ((double)k + 0.5) / (double)K;
        s_len[S] = 1.0 / (double)K;
      }
      ++S;
    }
    ray_off[r + 1] = S;
  }
  return S;
}

/* ------------------------------------------------------------------------ */
/* Unbounded scenes, Eq. (ub) of Sec. 5.4:                                   */
/*   x' = x                                      if ||x||_p <= 1             */
/*   x' = (1 + b - b/||x||_p) (x / ||x||_p)      otherwise,  p in {2, inf}.  */
/* FP64 form, used by the pins.                                              */
/* ------------------------------------------------------------------------ */
OR_API void or_contract(const double* x, int64_t n, double b, int p_inf, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    const double* p = x + 3 * i;
    double r;
    if (p_inf) {
      r = fabs(p[0]);
      if (fabs(p[1]) > r) r = fabs(p[1]);
      if (fabs(p[2]) > r) r = fabs(p[2]);
    } else {
      r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    }
    double s = r <= 1.0 ? 1.0 : (1.0 + b - b / r) / r;
    for (int a = 0; a < 3; ++a) out[3 * i + a] = s * p[a];
  }
}

/* Sampling with the step measured in the contracted space (Sec. 5.4).       */
/* Reading: march in world space, x_{k+1} = x_k + h_k d, where h_k is the    */
/* world length that advances the contracted point by step_c to first order: */
/* h_k = step_c / ||J(x_k) d||_2, J the Jacobian of Eq. (ub).  With          */
/* r = ||x||_p and g(r) = (1 + b)/r - b/r^2 (so x' = g(r) x for r > 1):       */
/*   J d = g d + g'(r) (grad r . d) x,   g'(r) = -(1 + b)/r^2 + 2b/r^3,       */
/*   grad r . d = (x . d)/r (p = 2) or sign(x_m) d_m, m = first argmax |x_a|  */
/*   (p = inf);  J d = d when r <= 1.                                         */
/* The march starts at x_0 = o + near d, emits x'_k for k < max_steps and     */
/* stops before a point whose contracted p-norm radius reaches (1 + b) -     */
/* step_c (a NaN radius also stops), or when h_k is not finite and positive. */
/* FP32, order:                                                              */
/*   r (p=inf): max(max(|x0|,|x1|),|x2|) ; (p=2): sqrtf((x0*x0 + x1*x1) + x2*x2) */
/*   gr = (1+b)/r - b/(r*r) ; x'_a = gr * x_a ; contracted radius = the same  */
/*   p-norm formula applied to x'                                             */
/*   gp = (2*b)/((r*r)*r) - (1+b)/(r*r)                                       */
/*   rd = ((x0*d0 + x1*d1) + x2*d2)/r  (p=2)  or  (x_m < 0 ? -d_m : d_m)      */
/*   j_a = gr*d_a + (gp*rd)*x_a ; nj = sqrtf((j0*j0 + j1*j1) + j2*j2)          */
/*   h = step_c / nj ; x_a = x_a + h*d_a                                      */
/* Distortion coordinates: s_mid = (k + 0.5)/max_steps, s_len = 1/max_steps.  */
/* ------------------------------------------------------------------------ */
OR_API int64_t or_sample_rays_contracted(const float* o, const float* d, int64_t R, float b,
                                         int p_inf, float near, float step_c, int32_t max_steps,
                                         const float lo[3], const float hi[3], const int32_t G[3],
                                         const uint8_t* mask, int64_t* ray_off, float* xyz,
                                         int32_t* ray_id, int32_t* step_k, double* s_mid,
                                         double* s_len, int64_t cap) {
  int64_t S = 0;
  ray_off[0] = 0;
  const float opb = 1.0f + b;
  const float rmax = opb - step_c;
  for (int64_t r = 0; r < R; ++r) {
    const float* rd = d + 3 * r;
    float x[3];
    for (int a = 0; a < 3; ++a) x[a] = o[3 * r + a] + near * rd[a];
    for (int32_t k = 0; k < max_steps; ++k) {
      float rad;
      int m = 0;
      if (p_inf) {
        float a0 = fabsf(x[0]), a1 = fabsf(x[1]), a2 = fabsf(x[2]);
        rad = a0;
        if (a1 > rad) { rad = a1; m = 1; }
        if (a2 > rad) { rad = a2; m = 2; }
      } else {
        rad = sqrtf((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
      }
      float xc[3], j[3];
      if (rad <= 1.0f) {
        for (int a = 0; a < 3; ++a) { xc[a] = x[a]; j[a] = rd[a]; }
      } else {
        float r2 = rad * rad;
        float gr = opb / rad - b / r2;
        float gp = (2.0f * b) / (r2 * rad) - opb / r2;
        float rdot;
        if (p_inf) rdot = x[m] < 0.0f ? -rd[m] : rd[m];
        else rdot = ((x[0] * rd[0] + x[1] * rd[1]) + x[2] * rd[2]) / rad;
        float gq = gp * rdot;
        for (int a = 0; a < 3; ++a) {
          xc[a] = gr * x[a];
          j[a] = gr * rd[a] + gq * x[a];
        }
      }
      float cr;
      if (p_inf) {
        cr = fabsf(xc[0]);
        if (fabsf(xc[1]) > cr) cr = fabsf(xc[1]);
        if (fabsf(xc[2]) > cr) cr = fabsf(xc[2]);
      } else {
        cr = sqrtf((xc[0] * xc[0] + xc[1] * xc[1]) + xc[2] * xc[2]);
      }
      if (!(cr < rmax)) break;
      int inside = 1;
      for (int a = 0; a < 3; ++a)
        if (!(xc[a] >= lo[a] && xc[a] <= hi[a])) inside = 0;
      if (inside && mask_on(mask, G, lo, hi, xc)) {
        if (S < cap) {
          xyz[3 * S + 0] = xc[0];
          xyz[3 * S + 1] = xc[1];
          xyz[3 * S + 2] = xc[2];
          ray_id[S] = (int32_t)r;
          step_k[S] = k;
          s_mid[S] = ((double)k + 0.5) / (double)max_steps;
          s_len[S] = 1.0 / (double)max_steps;
        }
        ++S;
      }
      float nj = sqrtf((j[0] * j[0] + j[1] * j[1]) + j[2] * j[2]);
      float h = step_c / nj;
      if (!(h > 0.0f) || isinf(h)) break;
      for (int a = 0; a < 3; ++a) x[a] = x[a] + h * rd[a];
    }
    ray_off[r + 1] = S;
  }
  return S;
}

/* ------------------------------------------------------------------------ */
/* Trilinear interpolation of a dense, corner-aligned grid (the explicit     */
/* grid query of Sec. 1, "constant time"): u_a = (x_a - lo_a)/(hi_a - lo_a)  */
/* * (G_a - 1), clamped to [0, G_a - 1]; i_a = min(floor(u_a), G_a - 2);     */
/* f_a = u_a - i_a; value = sum over the 8 corners of the product of         */
/* (1 - f_a) or f_a times the corner value.                                  */
/* ------------------------------------------------------------------------ */
static void tri_setup(const float* p, const float lo[3], const float hi[3], const int32_t G[3],
                      int64_t i0[3], double f[3]) {
  for (int a = 0; a < 3; ++a) {
    double u = ((double)p[a] - (double)lo[a]) / ((double)hi[a] - (double)lo[a]) * (double)(G[a] - 1);
    if (u < 0) u = 0;
    if (u > G[a] - 1) u = G[a] - 1;
    int64_t i = (int64_t)floor(u);
    if (i > G[a] - 2) i = G[a] - 2;
    if (i < 0) i = 0;
    i0[a] = i;
    f[a] = u - (double)i;
  }
}

OR_API void or_trilinear(const float* grid, const int32_t G[3], int C, const float lo[3],
                         const float hi[3], const float* xyz, int64_t n, double* out) {
  for (int64_t s = 0; s < n; ++s) {
    int64_t i0[3];
    double f[3];
    tri_setup(xyz + 3 * s, lo, hi, G, i0, f);
    for (int c = 0; c < C; ++c) out[s * C + c] = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          double wgt = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
          int64_t v = ((i0[2] + dz) * G[1] + (i0[1] + dy)) * G[0] + (i0[0] + dx);
          for (int c = 0; c < C; ++c) out[s * C + c] += wgt * (double)grid[v * C + c];
        }
  }
}

/* Progressive grid scaling (Sec. 5.4, grid-scaling schedule): the dense    */
/* grid src (Gs points per axis, C channels) resampled to Gd points per axis */
/* over the same box by trilinear interpolation of corner-aligned grids:     */
/* destination point x of axis a sits at source index u = x (Gs-1)/(Gd-1).   */
OR_API void or_grid_resample(const float* src, const int32_t Gs[3], int C, const int32_t Gd[3],
                             double* dst) {
  for (int64_t z = 0; z < Gd[2]; ++z)
    for (int64_t y = 0; y < Gd[1]; ++y)
      for (int64_t x = 0; x < Gd[0]; ++x) {
        const int64_t p[3] = {x, y, z};
        int64_t i0[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
          double u = (double)p[a] * (double)(Gs[a] - 1) / (double)(Gd[a] - 1);
          int64_t i = (int64_t)floor(u);
          if (i > Gs[a] - 2) i = Gs[a] - 2;
          if (i < 0) i = 0;
          i0[a] = i;
          f[a] = u - (double)i;
        }
        double* o = dst + ((z * Gd[1] + y) * Gd[0] + x) * C;
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              double wgt = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
              int64_t v = ((i0[2] + dz) * Gs[1] + (i0[1] + dy)) * Gs[0] + (i0[0] + dx);
              for (int c = 0; c < C; ++c) o[c] += wgt * (double)src[v * C + c];
            }
      }
}

/* Adjoint of or_trilinear: g_grid += sum_s weights(s) * g_out[s]. */
OR_API void or_trilinear_adjoint(const double* g_out, const int32_t G[3], int C, const float lo[3],
                                 const float hi[3], const float* xyz, int64_t n, double* g_grid) {
  for (int64_t s = 0; s < n; ++s) {
    int64_t i0[3];
    double f[3];
    tri_setup(xyz + 3 * s, lo, hi, G, i0, f);
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          double wgt = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
          int64_t v = ((i0[2] + dz) * G[1] + (i0[1] + dy)) * G[0] + (i0[0] + dx);
          for (int c = 0; c < C; ++c) g_grid[v * C + c] += wgt * g_out[s * C + c];
        }
  }
}

/* ------------------------------------------------------------------------ */
/* Front-to-back alpha compositing with early stop (Sec. 3 "Re-implement     */
/* rendering utils": halt a ray once the accumulated transmittance is below  */
/* T_stop = 1e-3).  Per ray, over its samples i = 0..N-1:                    */
/*   T_0 = 1 ; if T_i < T_stop the ray halts at i (n = i) ;                  */
/*   w_i = T_i alpha_i ; T_{i+1} = T_i (1 - alpha_i).                        */
/*   C = sum_{i<n} w_i c_i + T_n bg ; samples i >= n get w_i = 0.            */
/* The halting sample itself is not composited (T is tested before use).     */
/* alpha_i = 1 - exp(-delta_i softplus(raw_i + shift)) (Eq. 1 with the      */
/* softplus density), delta_i = interval for every sample, or the caller's   */
/* per-sample interval delta[i] when delta is given.                         */
/* ------------------------------------------------------------------------ */
static int64_t seg_end(const int64_t* ray_off, const int32_t* seg_len, int64_t r) {
  int64_t e = ray_off[r + 1];
  if (seg_len && ray_off[r] + seg_len[r] < e) e = ray_off[r] + seg_len[r];
  return e;
}

OR_API void or_composite(const double* raw, const double* rgb, const int64_t* ray_off, int64_t R,
                         double shift, double interval, const double* delta, double T_stop,
                         const double bg[3],
                         double* w, double* T, int32_t* n_live, double* T_end, double* color) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = ray_off[r + 1];
    double t = 1.0;
    int64_t stop = e;
    double acc[3] = {0, 0, 0};
    for (int64_t i = b; i < e; ++i) {
      if (t < T_stop) { stop = i; break; }
      double a = -expm1(-(delta ? delta[i] : interval) * softplus(raw[i] + shift));
      T[i] = t;
      w[i] = t * a;
      if (rgb)
        for (int c = 0; c < 3; ++c) acc[c] += w[i] * rgb[3 * i + c];
      t = t * (1.0 - a);
    }
    for (int64_t i = stop; i < e; ++i) { w[i] = 0.0; T[i] = t; }
    n_live[r] = (int32_t)(stop - b);
    T_end[r] = t;
    if (color)
      for (int c = 0; c < 3; ++c) color[3 * r + c] = acc[c] + t * bg[c];
  }
}

/* Gradient of the compositing above, by the chain rule on the product form. */
/* With g_i = dL/dw_i = <c_i, dL/dC> + g_w_extra_i and g_T = <bg, dL/dC>,    */
/* for k < n:                                                                */
/*   dL/dalpha_k = g_k T_k - (sum_{k<i<n} g_i w_i + g_T T_n) / (1 - alpha_k) */
/*   dL/draw_k   = dL/dalpha_k * interval (1 - alpha_k) sigmoid(raw_k+shift) */
/*               = interval sigmoid(.) (g_k T_{k+1} - sum_{k<i<n} g_i w_i    */
/*                 - g_T T_n)          (the (1 - alpha_k) factors cancel)    */
/*   dL/dc_k = w_k dL/dC ;  samples k >= n get zero gradient.                */
/* ------------------------------------------------------------------------ */
OR_API void or_composite_bwd(const double* raw, const double* rgb, const int64_t* ray_off, int64_t R,
                             double shift, double interval, const double* delta, double T_stop,
                             const double bg[3],
                             const double* g_color, const double* g_w_extra, double* g_raw,
                             double* g_rgb) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = ray_off[r + 1];
    int64_t N = e - b;
    double* a = (double*)malloc(sizeof(double) * (N + 1));
    double* T = (double*)malloc(sizeof(double) * (N + 2));
    double t = 1.0;
    int64_t n = N;
    for (int64_t i = 0; i < N; ++i) {
      if (t < T_stop) { n = i; break; }
      a[i] = -expm1(-(delta ? delta[b + i] : interval) * softplus(raw[b + i] + shift));
      T[i] = t;
      t = t * (1.0 - a[i]);
    }
    T[n] = t;
    const double* gC = g_color + 3 * r;
    double gT = gC[0] * bg[0] + gC[1] * bg[1] + gC[2] * bg[2];
    for (int64_t k = 0; k < N; ++k) {
      int64_t s = b + k;
      if (k >= n) {
        g_raw[s] = 0.0;
        if (g_rgb) for (int c = 0; c < 3; ++c) g_rgb[3 * s + c] = 0.0;
        continue;
      }
      double tail = gT * T[n];
      for (int64_t i = k + 1; i < n; ++i) {
        double gi = (rgb ? rgb[3 * (b + i)] * gC[0] + rgb[3 * (b + i) + 1] * gC[1] +
                           rgb[3 * (b + i) + 2] * gC[2] : 0.0) +
                    (g_w_extra ? g_w_extra[b + i] : 0.0);
        tail += gi * T[i] * a[i];
      }
      double gk = (rgb ? rgb[3 * s] * gC[0] + rgb[3 * s + 1] * gC[1] + rgb[3 * s + 2] * gC[2] : 0.0) +
                  (g_w_extra ? g_w_extra[s] : 0.0);
      double Tk1 = T[k] * (1.0 - a[k]);
      g_raw[s] = (delta ? delta[s] : interval) * sigmoid(raw[s] + shift) * (gk * Tk1 - tail);
      if (g_rgb) for (int c = 0; c < 3; ++c) g_rgb[3 * s + c] = T[k] * a[k] * gC[c];
    }
    free(a);
    free(T);
  }
}

/* ------------------------------------------------------------------------ */
/* Distortion loss, Eq. (dist_loss) of Sec. 2, per ray:                      */
/*   L = sum_i sum_j w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2 ds_i              */
/* with m_i the interval midpoint and ds_i its length.                       */
/* ------------------------------------------------------------------------ */
/* O(N^2) double sum, exactly as defined. */
OR_API void or_distortion_naive(const double* w, const double* m, const double* ds,
                                const int64_t* ray_off, const int32_t* seg_len, int64_t R,
                                double* L) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = seg_end(ray_off, seg_len, r);
    double acc = 0.0;
    for (int64_t i = b; i < e; ++i)
      for (int64_t j = b; j < e; ++j) acc += w[i] * w[j] * fabs(m[i] - m[j]);
    for (int64_t i = b; i < e; ++i) acc += w[i] * w[i] * ds[i] / 3.0;
    L[r] = acc;
  }
}

/* O(N) form of Sec. 2: with m increasing along the ray and the prefix sums  */
/* W_{<i} = sum_{j<i} w_j, WM_{<i} = sum_{j<i} w_j m_j,                      */
/*   L^{1st} = 2 sum_i w_i m_i W_{<i} - 2 sum_i w_i WM_{<i}.                 */
OR_API void or_distortion(const double* w, const double* m, const double* ds,
                          const int64_t* ray_off, const int32_t* seg_len, int64_t R, double* L) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = seg_end(ray_off, seg_len, r);
    double W = 0.0, WM = 0.0, first = 0.0, second = 0.0;
    for (int64_t i = b; i < e; ++i) {
      first += 2.0 * (w[i] * m[i] * W - w[i] * WM);
      second += w[i] * w[i] * ds[i] / 3.0;
      W += w[i];
      WM += w[i] * m[i];
    }
    L[r] = first + second;
  }
}

/* Derivative of Sec. 2 (with the third term read as 2 sum_{i>k} w_i m_i,    */
/* as the line before it in the paper implies), plus the derivative of the  */
/* second term, 2/3 w_k ds_k, which the paper does not print:                */
/*   dL/dw_k = 2 (m_k W_{<k} - WM_{<k} + WM_{>k} - m_k W_{>k})               */
/*             + 2/3 w_k ds_k                                                */
/* g_w = g_L[r] * dL_r/dw for the samples of ray r; 0 beyond seg_len.        */
OR_API void or_distortion_grad(const double* g_L, const double* w, const double* m,
                               const double* ds, const int64_t* ray_off, const int32_t* seg_len,
                               int64_t R, double* g_w) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = seg_end(ray_off, seg_len, r), ee = ray_off[r + 1];
    double Wt = 0.0, WMt = 0.0;
    for (int64_t i = b; i < e; ++i) { Wt += w[i]; WMt += w[i] * m[i]; }
    double W = 0.0, WM = 0.0;
    for (int64_t k = b; k < e; ++k) {
      double Wg = Wt - W - w[k], WMg = WMt - WM - w[k] * m[k];
      double d = 2.0 * (m[k] * W - WM + WMg - m[k] * Wg) + 2.0 / 3.0 * w[k] * ds[k];
      g_w[k] = g_L[r] * d;
      W += w[k];
      WM += w[k] * m[k];
    }
    for (int64_t k = e; k < ee; ++k) g_w[k] = 0.0;
  }
}

/* Direct derivative of the O(N^2) definition: 2 sum_j w_j |m_k - m_j|       */
/* + 2/3 w_k ds_k (no ordering of m assumed).                                */
OR_API void or_distortion_grad_naive(const double* g_L, const double* w, const double* m,
                                     const double* ds, const int64_t* ray_off,
                                     const int32_t* seg_len, int64_t R, double* g_w) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = seg_end(ray_off, seg_len, r), ee = ray_off[r + 1];
    for (int64_t k = b; k < e; ++k) {
      double acc = 0.0;
      for (int64_t j = b; j < e; ++j) acc += w[j] * fabs(m[k] - m[j]);
      g_w[k] = g_L[r] * (2.0 * acc + 2.0 / 3.0 * w[k] * ds[k]);
    }
    for (int64_t k = e; k < ee; ++k) g_w[k] = 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Multilayer perceptron with ReLU hidden layers (the shallow colour MLP of  */
/* the hybrid representation, Tab. 1 / Sec. 1).  dims[0..L]; the flat FP32   */
/* parameter vector holds, per layer l, W_l[dims[l+1]][dims[l]] then         */
/* b_l[dims[l+1]].  Output activation: 1 = sigmoid (colour), 0 = identity.   */
/* ------------------------------------------------------------------------ */
static int64_t mlp_offset(const int32_t* dims, int l) {
  int64_t off = 0;
  for (int i = 0; i < l; ++i) off += (int64_t)dims[i + 1] * dims[i] + dims[i + 1];
  return off;
}

OR_API void or_mlp_fwd(const int32_t* dims, int L, const double* params, const double* x, int64_t n,
                       int out_sigmoid, double* out) {
  int maxw = 0;
  for (int l = 0; l <= L; ++l) if (dims[l] > maxw) maxw = dims[l];
  double* h = (double*)malloc(sizeof(double) * maxw);
  double* h2 = (double*)malloc(sizeof(double) * maxw);
  for (int64_t s = 0; s < n; ++s) {
    for (int i = 0; i < dims[0]; ++i) h[i] = x[s * dims[0] + i];
    for (int l = 0; l < L; ++l) {
      const double* W = params + mlp_offset(dims, l);
      const double* bias = W + (int64_t)dims[l + 1] * dims[l];
      for (int o = 0; o < dims[l + 1]; ++o) {
        double acc = bias[o];
        for (int i = 0; i < dims[l]; ++i) acc += W[(int64_t)o * dims[l] + i] * h[i];
        if (l < L - 1) acc = acc > 0 ? acc : 0.0;
        else if (out_sigmoid) acc = sigmoid(acc);
        h2[o] = acc;
      }
      double* tmp = h; h = h2; h2 = tmp;
    }
    for (int o = 0; o < dims[L]; ++o) out[s * dims[L] + o] = h[o];
  }
  free(h);
  free(h2);
}

/* Backward of or_mlp_fwd (reverse-mode chain rule, one sample at a time):   */
/* g_params += sum_s dL/dparams, g_x[s] = dL/dx[s] (if non-NULL).            */
OR_API void or_mlp_bwd(const int32_t* dims, int L, const double* params, const double* x, int64_t n,
                       int out_sigmoid, const double* g_out, double* g_params, double* g_x) {
  int64_t tot = 0;
  for (int l = 0; l <= L; ++l) tot += dims[l];
  double* act = (double*)malloc(sizeof(double) * tot);  /* post-activation per layer */
  double* pre = (double*)malloc(sizeof(double) * tot);
  int maxw = 0;
  for (int l = 0; l <= L; ++l) if (dims[l] > maxw) maxw = dims[l];
  double* g = (double*)malloc(sizeof(double) * maxw);
  double* gp = (double*)malloc(sizeof(double) * maxw);
  for (int64_t s = 0; s < n; ++s) {
    int64_t base[16];
    base[0] = 0;
    for (int l = 0; l < L; ++l) base[l + 1] = base[l] + dims[l];
    for (int i = 0; i < dims[0]; ++i) act[i] = x[s * dims[0] + i];
    for (int l = 0; l < L; ++l) {
      const double* W = params + mlp_offset(dims, l);
      const double* bias = W + (int64_t)dims[l + 1] * dims[l];
      for (int o = 0; o < dims[l + 1]; ++o) {
        double acc = bias[o];
        for (int i = 0; i < dims[l]; ++i) acc += W[(int64_t)o * dims[l] + i] * act[base[l] + i];
        pre[base[l + 1] + o] = acc;
        double y = acc;
        if (l < L - 1) y = acc > 0 ? acc : 0.0;
        else if (out_sigmoid) y = sigmoid(acc);
        act[base[l + 1] + o] = y;
      }
    }
    /* gradient w.r.t. the last pre-activation */
    for (int o = 0; o < dims[L]; ++o) {
      double y = act[base[L] + o];
      g[o] = g_out[s * dims[L] + o] * (out_sigmoid ? y * (1.0 - y) : 1.0);
    }
    for (int l = L - 1; l >= 0; --l) {
      const double* W = params + mlp_offset(dims, l);
      double* gW = g_params + mlp_offset(dims, l);
      double* gb = gW + (int64_t)dims[l + 1] * dims[l];
      for (int o = 0; o < dims[l + 1]; ++o) {
        gb[o] += g[o];
        for (int i = 0; i < dims[l]; ++i) gW[(int64_t)o * dims[l] + i] += g[o] * act[base[l] + i];
      }
      for (int i = 0; i < dims[l]; ++i) {
        double acc = 0.0;
        for (int o = 0; o < dims[l + 1]; ++o) acc += W[(int64_t)o * dims[l] + i] * g[o];
        gp[i] = acc;
      }
      if (l > 0)
        for (int i = 0; i < dims[l]; ++i) g[i] = pre[base[l] + i] > 0 ? gp[i] : 0.0;
      else if (g_x)
        for (int i = 0; i < dims[0]; ++i) g_x[s * dims[0] + i] = gp[i];
    }
  }
  free(act);
  free(pre);
  free(g);
  free(gp);
}

/* Per sample, the smallest |pre-activation| over the hidden (ReLU) layers of */
/* or_mlp_fwd.  A ReLU whose input is this close to 0 takes its on/off      */
/* decision at the rounding level of the arithmetic, so implementations in   */
/* different precisions may legitimately disagree there.                     */
OR_API void or_mlp_min_abs_preact(const int32_t* dims, int L, const double* params, const double* x,
                                  int64_t n, double* out) {
  int maxw = 0;
  for (int l = 0; l <= L; ++l) if (dims[l] > maxw) maxw = dims[l];
  double* h = (double*)malloc(sizeof(double) * maxw);
  double* h2 = (double*)malloc(sizeof(double) * maxw);
  for (int64_t s = 0; s < n; ++s) {
    double mn = INFINITY;
    for (int i = 0; i < dims[0]; ++i) h[i] = x[s * dims[0] + i];
    for (int l = 0; l < L - 1; ++l) {
      const double* W = params + mlp_offset(dims, l);
      const double* bias = W + (int64_t)dims[l + 1] * dims[l];
      for (int o = 0; o < dims[l + 1]; ++o) {
        double acc = bias[o];
        for (int i = 0; i < dims[l]; ++i) acc += W[(int64_t)o * dims[l] + i] * h[i];
        if (fabs(acc) < mn) mn = fabs(acc);
        h2[o] = acc > 0 ? acc : 0.0;
      }
      double* tmp = h; h = h2; h2 = tmp;
    }
    out[s] = mn;
  }
  free(h);
  free(h2);
}

/* Frequency encoding: [v, sin(2^f v_a) for a in 0..2, f in 0..F-1 (axis    */
/* major), cos(same order)] -> 3 + 6F values.                                */
OR_API void or_freq_encode(const float* v, int64_t n, int F, double* out) {
  int D = 3 + 6 * F;
  for (int64_t s = 0; s < n; ++s) {
    double* o = out + s * D;
    for (int a = 0; a < 3; ++a) o[a] = v[3 * s + a];
    for (int a = 0; a < 3; ++a)
      for (int f = 0; f < F; ++f) {
        double e = (double)v[3 * s + a] * ldexp(1.0, f);
        o[3 + a * F + f] = sin(e);
        o[3 + 3 * F + a * F + f] = cos(e);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Total variation, Sec. 2 "Efficient total variation (TV) loss": for each   */
/* grid point, the Huber loss to each of its six nearest neighbours (both    */
/* orders of every pair are counted; neighbours outside the grid are         */
/* skipped), averaged over grid points and channels:                         */
/*   L_tv = 1/(N C) sum_v sum_c sum_{u in nbr6(v)} H_delta(g[v,c] - g[u,c])  */
/*   H_delta(x) = x^2/2 if |x| <= delta else delta (|x| - delta/2).          */
/* ------------------------------------------------------------------------ */
static double huber(double x, double dl) { double a = fabs(x); return a <= dl ? 0.5 * x * x : dl * (a - 0.5 * dl); }
static double huber_d(double x, double dl) { return x > dl ? dl : (x < -dl ? -dl : x); }

OR_API double or_tv_loss(const double* g, const int32_t G[3], int C, double delta) {
  double acc = 0.0;
  int64_t N = (int64_t)G[0] * G[1] * G[2];
  for (int64_t z = 0; z < G[2]; ++z)
    for (int64_t y = 0; y < G[1]; ++y)
      for (int64_t x = 0; x < G[0]; ++x) {
        int64_t v = (z * G[1] + y) * G[0] + x;
        const int64_t nb[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z},
                                  {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
        for (int q = 0; q < 6; ++q) {
          if (nb[q][0] < 0 || nb[q][0] >= G[0] || nb[q][1] < 0 || nb[q][1] >= G[1] ||
              nb[q][2] < 0 || nb[q][2] >= G[2]) continue;
          int64_t u = (nb[q][2] * G[1] + nb[q][1]) * G[0] + nb[q][0];
          for (int c = 0; c < C; ++c) acc += huber(g[v * C + c] - g[u * C + c], delta);
        }
      }
  return acc / ((double)N * C);
}

/* TV gradient added into grad (the paper skips the forward and adds the    */
/* gradient between backward and the optimizer step).  dense_mode != 0: all */
/* grid points; otherwise only entries whose incoming gradient is non-zero  */
/* (Sec. 2: after 10k iterations only the points involved in the iteration).*/
/*   d L_tv / d g[v,c] = 2/(N C) sum_{u in nbr6(v)} H'_delta(g[v,c]-g[u,c])  */
OR_API void or_tv_add_grad(const double* g, const int32_t G[3], int C, double weight, double delta,
                           int dense_mode, const double* grad_in, double* grad_out) {
  int64_t N = (int64_t)G[0] * G[1] * G[2];
  double scale = weight * 2.0 / ((double)N * C);
  for (int64_t z = 0; z < G[2]; ++z)
    for (int64_t y = 0; y < G[1]; ++y)
      for (int64_t x = 0; x < G[0]; ++x) {
        int64_t v = (z * G[1] + y) * G[0] + x;
        const int64_t nb[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z},
                                  {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
        for (int c = 0; c < C; ++c) {
          int64_t e = v * C + c;
          grad_out[e] = grad_in[e];
          if (!dense_mode && grad_in[e] == 0.0) continue;
          double acc = 0.0;
          for (int q = 0; q < 6; ++q) {
            if (nb[q][0] < 0 || nb[q][0] >= G[0] || nb[q][1] < 0 || nb[q][1] >= G[1] ||
                nb[q][2] < 0 || nb[q][2] >= G[2]) continue;
            int64_t u = (nb[q][2] * G[1] + nb[q][1]) * G[0] + nb[q][0];
            acc += huber_d(g[e] - g[u * C + c], delta);
          }
          grad_out[e] += scale * acc;
        }
      }
}

/* ------------------------------------------------------------------------ */
/* Adam (Sec. 3 "Re-implement Adam optimizer"): the textbook update with a   */
/* global step t for bias correction; entries whose gradient is exactly zero */
/* are skipped (parameter and both moments left as they are) when skip_zero.*/
/*   m = b1 m + (1-b1) g ; v = b2 v + (1-b2) g^2                             */
/*   p = p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)            */
/* ------------------------------------------------------------------------ */
OR_API void or_adam(double* p, const double* g, double* m, double* v, int64_t n, double lr,
                    double b1, double b2, double eps, int64_t t, int skip_zero) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    if (skip_zero && g[i] == 0.0) continue;
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* ------------------------------------------------------------------------ */
/* Learned proposal (not in the paper; the sample-reduction network of the   */
/* build's precision/proposal configuration).  Per ray with K candidates:    */
/*   q = softmax(logits over the ray's candidates)                           */
/*   loss_r = -sum_j p_j log q_j ;  d loss_r / d logit_j = q_j - p_j         */
/* (p sums to one).  Selection: inverse CDF of q at u_k = (k + 0.5)/n_draw,  */
/* the candidate j with CDF_{j-1} <= u_k < CDF_j (CDF in FP32, summed in     */
/* candidate order), duplicates removed, indices ascending.                  */
/* ------------------------------------------------------------------------ */
OR_API void or_softmax_xent(const double* logits, const double* p, int64_t R, int K, double* loss,
                            double* g_logits, double* q_out) {
  for (int64_t r = 0; r < R; ++r) {
    const double* z = logits + r * K;
    double mx = z[0];
    for (int j = 1; j < K; ++j) if (z[j] > mx) mx = z[j];
    double se = 0.0;
    for (int j = 0; j < K; ++j) se += exp(z[j] - mx);
    double lse = mx + log(se);
    double l = 0.0;
    for (int j = 0; j < K; ++j) {
      double q = exp(z[j] - lse);
      l -= p[r * K + j] * (z[j] - lse);
      if (g_logits) g_logits[r * K + j] = q - p[r * K + j];
      if (q_out) q_out[r * K + j] = q;
    }
    loss[r] = l;
  }
}

OR_API void or_inverse_cdf_select(const float* q, int64_t R, int K, int n_draw, int32_t* sel,
                                  int32_t* n_sel) {
  for (int64_t r = 0; r < R; ++r) {
    int cnt = 0, j = 0;
    float cdf = q[r * K];
    for (int k = 0; k < n_draw; ++k) {
      float u = ((float)k + 0.5f) / (float)n_draw;
      while (j < K - 1 && !(u < cdf)) { ++j; cdf = cdf + q[r * K + j]; }
      if (cnt == 0 || sel[r * n_draw + cnt - 1] != j) sel[r * n_draw + cnt++] = j;
    }
    n_sel[r] = cnt;
    for (int k = cnt; k < n_draw; ++k) sel[r * n_draw + k] = -1;
  }
}

/* Ragged forms of the two functions above, over a CSR list of candidates.  */
/* Target: p_j = (w_j / W + eps_u) / (1 + N eps_u) with W = sum_j w_j (the   */
/* plain renderer's weights, plus a uniform floor), uniform if W = 0.       */
OR_API void or_proposal_xent_ragged(const double* logits, const double* w, const int64_t* ray_off,
                                    int64_t R, double eps_u, double* loss, double* g_logits,
                                    double* q_out) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r], e = ray_off[r + 1];
    int64_t N = e - b;
    loss[r] = 0.0;
    if (N == 0) continue;
    double mx = logits[b], W = 0.0;
    for (int64_t i = b; i < e; ++i) {
      if (logits[i] > mx) mx = logits[i];
      W += w[i];
    }
    double se = 0.0;
    for (int64_t i = b; i < e; ++i) se += exp(logits[i] - mx);
    double lse = mx + log(se);
    for (int64_t i = b; i < e; ++i) {
      double q = exp(logits[i] - lse);
      double p = W > 0 ? (w[i] / W + eps_u) / (1.0 + (double)N * eps_u) : 1.0 / (double)N;
      loss[r] -= p * (logits[i] - lse);
      if (g_logits) g_logits[i] = q - p;
      if (q_out) q_out[i] = q;
    }
  }
}

OR_API void or_inverse_cdf_select_ragged(const float* q, const int64_t* ray_off, int64_t R,
                                         int n_draw, int32_t* sel, int32_t* n_sel) {
  for (int64_t r = 0; r < R; ++r) {
    int64_t b = ray_off[r];
    int N = (int)(ray_off[r + 1] - b);
    int32_t* out = sel + r * n_draw;
    int cnt = 0;
    if (N > 0) {
      int j = 0;
      float cdf = q[b];
      for (int k = 0; k < n_draw; ++k) {
        float u = ((float)k + 0.5f) / (float)n_draw;
        while (j < N - 1 && !(u < cdf)) { ++j; cdf = cdf + q[b + j]; }
        if (cnt == 0 || out[cnt - 1] != j) out[cnt++] = j;
      }
    }
    n_sel[r] = cnt;
    for (int k = cnt; k < n_draw; ++k) out[k] = -1;
  }
}
