// Ray sampling (Sec. 3 "Re-implement rendering utils": sample only inside
// the scene bbox; Sec. 1 occupancy mask; Sec. 5.4 contracted step for
// unbounded scenes) and the live-sample list used after early stop.
//
// Every decision that creates or drops a sample is IEEE FP32 with explicit
// round-to-nearest intrinsics (no FMA contraction), in the operation order
// stated in dvgo.h / below, so the integer results are reproducible bit for
// bit by any IEEE FP32 implementation of the same formulas.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace dvgo {

struct SamplerArgs {
  float lo[3], hi[3];
  int G[3];
  float scale[3];  // (G-1)/(hi-lo), FP32
  dvgo_sampler_desc s;
};

__device__ __forceinline__ int nearest_idx(float x, float lo, float scale, int G) {
  float u = __fmul_rn(__fsub_rn(x, lo), scale);
  float f = floorf(__fadd_rn(u, 0.5f));
  int n = (int)f;
  if (!(f >= 0.0f)) n = 0;
  if (f > (float)(G - 1)) n = G - 1;
  return n;
}

__device__ __forceinline__ bool keep_point(const SamplerArgs& A, const uint8_t* __restrict__ mask,
                                           const float x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (!(x[a] >= A.lo[a] && x[a] <= A.hi[a])) return false;
  if (!mask) return true;
  int ix = nearest_idx(x[0], A.lo[0], A.scale[0], A.G[0]);
  int iy = nearest_idx(x[1], A.lo[1], A.scale[1], A.G[1]);
  int iz = nearest_idx(x[2], A.lo[2], A.scale[2], A.G[2]);
  return __ldg(mask + ((int64_t)iz * A.G[1] + iy) * A.G[0] + ix) != 0;
}

struct RaySpan {
  float tlo, thi;
  int n;
};

// Ray/bbox slab and step count (mode 0).
__device__ __forceinline__ RaySpan ray_span(const SamplerArgs& A, const float o[3], const float d[3]) {
  float tlo = A.s.near, thi = A.s.far;
  bool empty = false;
  if (A.s.use_slab) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (d[a] == 0.0f) {
        if (o[a] < A.lo[a] || o[a] > A.hi[a]) empty = true;
      } else {
        float ta = __fdiv_rn(__fsub_rn(A.lo[a], o[a]), d[a]);
        float tb = __fdiv_rn(__fsub_rn(A.hi[a], o[a]), d[a]);
        float tn = ta < tb ? ta : tb;
        float tf = ta < tb ? tb : ta;
        if (tn > tlo) tlo = tn;
        if (tf < thi) thi = tf;
      }
    }
  }
  int n = 0;
  if (!empty && thi > tlo) {
    float u = __fdiv_rn(__fsub_rn(thi, tlo), A.s.step);
    float nf = ceilf(__fsub_rn(u, A.s.step_offset));
    if (nf > (float)A.s.max_steps) n = A.s.max_steps;
    else if (nf > 0.0f) n = (int)nf;
  }
  return {tlo, thi, n};
}

__device__ __forceinline__ void point_at(const SamplerArgs& A, const float o[3], const float d[3],
                                         float tlo, int k, float x[3]) {
  float t = __fadd_rn(tlo, __fmul_rn(__fadd_rn((float)k, A.s.step_offset), A.s.step));
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(t, d[a]));
}

__device__ __forceinline__ void load_ray(const float* __restrict__ ro, const float* __restrict__ rd,
                                         int64_t r, float o[3], float d[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o[a] = __ldg(ro + 3 * r + a);
    d[a] = __ldg(rd + 3 * r + a);
  }
}

// Mode 2: the ray in normalized device coordinates (forward-facing scenes);
// ok is false for a ray that does not look down -z.
struct NdcRay {
  float o[3], d[3];
  int n;   // layer crossings
};

__device__ __forceinline__ NdcRay ndc_ray(const SamplerArgs& A, const float o[3], const float d[3]) {
  NdcRay q;
  q.n = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) q.o[a] = q.d[a] = 0.0f;
  if (!(d[2] < 0.0f)) return q;
  const float nr = A.s.ndc_near;
  const float t = __fdiv_rn(-__fadd_rn(nr, o[2]), d[2]);
  const float ox = __fadd_rn(o[0], __fmul_rn(t, d[0]));
  const float oy = __fadd_rn(o[1], __fmul_rn(t, d[1]));
  const float oz = __fadd_rn(o[2], __fmul_rn(t, d[2]));
  if (!(oz < 0.0f)) return q;
  const float rx = __fdiv_rn(ox, oz), ry = __fdiv_rn(oy, oz);
  const float two_n = __fmul_rn(2.0f, nr);
  q.o[0] = -__fmul_rn(A.s.ndc_fx, rx);
  q.o[1] = -__fmul_rn(A.s.ndc_fy, ry);
  q.o[2] = __fadd_rn(1.0f, __fdiv_rn(two_n, oz));
  q.d[0] = -__fmul_rn(A.s.ndc_fx, __fsub_rn(__fdiv_rn(d[0], d[2]), rx));
  q.d[1] = -__fmul_rn(A.s.ndc_fy, __fsub_rn(__fdiv_rn(d[1], d[2]), ry));
  q.d[2] = -__fdiv_rn(two_n, oz);
  const float nf = floorf(__fdiv_rn((float)(A.G[2] - 1), A.s.step));
  const int K = (int)nf + 1;
  q.n = K < A.s.max_steps ? K : A.s.max_steps;
  return q;
}

// Crossing of layer plane k: z_k = lo_z + (k step) dz, dz = (hi_z - lo_z)/(G_z - 1).
__device__ __forceinline__ void ndc_point(const SamplerArgs& A, const NdcRay& q, int k, float x[3]) {
  const float dz = __fdiv_rn(__fsub_rn(A.hi[2], A.lo[2]), (float)(A.G[2] - 1));
  const float z = __fadd_rn(A.lo[2], __fmul_rn(__fmul_rn((float)k, A.s.step), dz));
  const float t = __fdiv_rn(__fsub_rn(z, q.o[2]), q.d[2]);
  x[0] = __fadd_rn(q.o[0], __fmul_rn(t, q.d[0]));
  x[1] = __fadd_rn(q.o[1], __fmul_rn(t, q.d[1]));
  x[2] = z;
}

// Steps per ray whose keep bits pass 1 records for pass 2: one word of 32
// steps per lane of the ray's warp (1024 steps).  Longer marches recompute
// the keep test in pass 2.
constexpr int kBitWords = 32;

// Mode 0, pass 1: one warp per ray counts the kept samples.  With bits,
// the warp also stores each 32-step chunk's keep ballot (lane j holds chunk
// j's word; one coalesced store per ray), so that pass 2 need not repeat the
// occupancy lookups.
// kNdc: mode 2 (layer crossings of the warped ray) instead of mode 0.
template <bool kNdc>
__global__ void __launch_bounds__(256, 8) bbox_count_kernel(SamplerArgs A, const float* __restrict__ ro,
                                  const float* __restrict__ rd, int64_t R,
                                  const uint8_t* __restrict__ mask, int32_t* __restrict__ counts,
                                  uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < R; r += nwarps) {
    float o[3], d[3];
    load_ray(ro, rd, r, o, d);
    RaySpan sp{0.0f, 0.0f, 0};
    NdcRay q;
    if (kNdc) {
      q = ndc_ray(A, o, d);
      sp.n = q.n;
    } else {
      sp = ray_span(A, o, d);
    }
    int cnt = 0;
    uint32_t mine = 0;
    // four 32-step chunks per round, so that their occupancy lookups are in
    // flight together
    for (int k0 = 0; k0 < sp.n; k0 += 128) {
      bool keep[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + 32 * u + lane;
        keep[u] = false;
        if (k < sp.n) {
          float x[3];
          if (kNdc) ndc_point(A, q, k, x);
          else point_at(A, o, d, sp.tlo, k, x);
          keep[u] = keep_point(A, mask, x);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned bal = __ballot_sync(0xffffffffu, keep[u]);
        if (lane == (k0 >> 5) + u) mine = bal;
        cnt += __popc(bal);
      }
    }
    if (lane == 0) counts[r] = cnt;
    if (bits && 32 * lane < sp.n) bits[r * kBitWords + lane] = mine;
  }
}

// Mode 0, pass 2: one warp per ray writes the kept samples in step order.
// With bits (only when max_steps <= 32 kBitWords = 1024) the keep decisions are
// pass 1's ballots; without, the keep test is evaluated again (same FP32
// operations, same result).
template <bool kNdc>
__global__ void bbox_fill_kernel(SamplerArgs A, const float* __restrict__ ro,
                                 const float* __restrict__ rd, int64_t R,
                                 const uint8_t* __restrict__ mask,
                                 const uint32_t* __restrict__ bits,
                                 const int64_t* __restrict__ ray_off, float* __restrict__ xyz,
                                 int32_t* __restrict__ ray_id, int32_t* __restrict__ step_k,
                                 float* __restrict__ s_mid, float* __restrict__ s_len) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < R; r += nwarps) {
    float o[3], d[3];
    load_ray(ro, rd, r, o, d);
    RaySpan sp{0.0f, 0.0f, 0};
    NdcRay q;
    float span, slen;
    if (kNdc) {
      q = ndc_ray(A, o, d);
      sp.n = q.n;
      span = (float)q.n;                 // s = (k + 0.5)/K, length 1/K
      slen = __fdiv_rn(1.0f, span);
    } else {
      sp = ray_span(A, o, d);
      span = __fsub_rn(sp.thi, sp.tlo);
      slen = __fdiv_rn(A.s.step, span);
    }
    int64_t pos = ray_off[r];
    uint32_t mine = 0;
    if (bits && 32 * lane < sp.n) mine = bits[r * kBitWords + lane];
    for (int k0 = 0; k0 < sp.n; k0 += 32) {
      int k = k0 + lane;
      bool keep = false;
      float x[3];
      unsigned bal;
      if (bits) {
        bal = __shfl_sync(0xffffffffu, mine, k0 >> 5);
        keep = (bal >> lane) & 1u;
        if (keep) {
          if (kNdc) ndc_point(A, q, k, x);
          else point_at(A, o, d, sp.tlo, k, x);
        }
      } else {
        if (k < sp.n) {
          if (kNdc) ndc_point(A, q, k, x);
          else point_at(A, o, d, sp.tlo, k, x);
          keep = keep_point(A, mask, x);
        }
        bal = __ballot_sync(0xffffffffu, keep);
      }
      if (keep) {
        int64_t s = pos + __popc(bal & lt_mask);
        xyz[3 * s + 0] = x[0];
        xyz[3 * s + 1] = x[1];
        xyz[3 * s + 2] = x[2];
        ray_id[s] = (int32_t)r;
        step_k[s] = k;
        s_mid[s] = kNdc ? __fdiv_rn(__fadd_rn((float)k, 0.5f), span)
                        : __fdiv_rn(__fmul_rn(__fadd_rn((float)k, A.s.step_offset), A.s.step), span);
        s_len[s] = slen;
      }
      pos += __popc(bal);
    }
  }
}

// Mode 1: contracted-space march (Eq. ub).  One step at world point x: the
// contracted point xc and the Jacobian-mapped direction j (false when xc's
// contracted radius has reached rmax: the march ends before xc), then the
// advance of x by the contracted step (false when the step is not finite).
struct CMarch {
  float b, opb, rmax, two_b;
  bool p_inf;
};

__device__ __forceinline__ CMarch cmarch_consts(const SamplerArgs& A) {
  CMarch M;
  M.b = A.s.contract_b;
  M.opb = __fadd_rn(1.0f, M.b);
  M.rmax = __fsub_rn(M.opb, A.s.step_c);
  M.two_b = __fmul_rn(2.0f, M.b);
  M.p_inf = A.s.p_inf != 0;
  return M;
}

__device__ __forceinline__ bool cmarch_point(const CMarch& M, const float x[3], const float d[3], float xc[3],
                                             float j[3], bool& inside) {
  float rad;
  int m = 0;
  if (M.p_inf) {
    float a0 = fabsf(x[0]), a1 = fabsf(x[1]), a2 = fabsf(x[2]);
    rad = a0;
    if (a1 > rad) { rad = a1; m = 1; }
    if (a2 > rad) { rad = a2; m = 2; }
  } else {
    rad = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x[0], x[0]), __fmul_rn(x[1], x[1])),
                               __fmul_rn(x[2], x[2])));
  }
  inside = rad <= 1.0f;
  if (inside) {
#pragma unroll
    for (int a = 0; a < 3; ++a) { xc[a] = x[a]; j[a] = d[a]; }
    // xc = x: its contracted radius is rad itself (the same operations on
    // the same values)
    return rad < M.rmax;
  } else {
    float r2 = __fmul_rn(rad, rad);
    float gr = __fsub_rn(__fdiv_rn(M.opb, rad), __fdiv_rn(M.b, r2));
    float gp = __fsub_rn(__fdiv_rn(M.two_b, __fmul_rn(r2, rad)), __fdiv_rn(M.opb, r2));
    float rdot;
    if (M.p_inf) {
      float xm = m == 0 ? x[0] : (m == 1 ? x[1] : x[2]);
      float dm = m == 0 ? d[0] : (m == 1 ? d[1] : d[2]);
      rdot = xm < 0.0f ? -dm : dm;
    } else {
      rdot = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(x[0], d[0]), __fmul_rn(x[1], d[1])),
                                 __fmul_rn(x[2], d[2])), rad);
    }
    float gq = __fmul_rn(gp, rdot);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xc[a] = __fmul_rn(gr, x[a]);
      j[a] = __fadd_rn(__fmul_rn(gr, d[a]), __fmul_rn(gq, x[a]));
    }
  }
  float cr;
  if (M.p_inf) {
    cr = fabsf(xc[0]);
    if (fabsf(xc[1]) > cr) cr = fabsf(xc[1]);
    if (fabsf(xc[2]) > cr) cr = fabsf(xc[2]);
  } else {
    cr = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(xc[0], xc[0]), __fmul_rn(xc[1], xc[1])),
                              __fmul_rn(xc[2], xc[2])));
  }
  return cr < M.rmax;
}

// step_c / |j|, the contracted step along j
__device__ __forceinline__ float cmarch_step_len(const SamplerArgs& A, const float j[3]) {
  const float nj = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(j[0], j[0]), __fmul_rn(j[1], j[1])),
                                        __fmul_rn(j[2], j[2])));
  return __fdiv_rn(A.s.step_c, nj);
}

// Inside the unit ball j = d, so the step is the ray's constant h_in =
// cmarch_step_len(A, d), formed once per ray (the same value bit for bit).
__device__ __forceinline__ bool cmarch_advance(const SamplerArgs& A, float x[3], const float d[3],
                                               const float j[3], bool inside, float h_in) {
  const float h = inside ? h_in : cmarch_step_len(A, j);
  if (!(h > 0.0f) || isinf(h)) return false;
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(x[a], __fmul_rn(h, d[a]));
  return true;
}

// Checkpoints of the march for the parallel second pass: the march of a ray
// is cut into kCkpt chunks of L = ceil(max_steps / kCkpt) steps; record c of
// the ray holds x at step c L (3 floats) and the kept samples of chunk c
// (int32, -1 for a chunk the march never reaches).  kCkpt x 4 words per ray
// fit the per-ray keep-bit words of the workspace.
constexpr int kCkpt = 8;

__device__ __forceinline__ int ckpt_len(const SamplerArgs& A) {
  return (A.s.max_steps + kCkpt - 1) / kCkpt;
}

// Mode 1, one thread per ray: the whole march.  Pass 1 (kWrite false)
// counts, and with ckpt records the checkpoints; pass 2 without checkpoints
// (kWrite) repeats the march and writes.
template <bool kWrite>
__global__ void contracted_kernel(SamplerArgs A, const float* __restrict__ ro,
                                  const float* __restrict__ rd, int64_t R,
                                  const uint8_t* __restrict__ mask, int32_t* __restrict__ counts,
                                  uint32_t* __restrict__ ckpt,
                                  const int64_t* __restrict__ ray_off, float* __restrict__ xyz,
                                  int32_t* __restrict__ ray_id, int32_t* __restrict__ step_k,
                                  float* __restrict__ s_mid, float* __restrict__ s_len) {
  const CMarch M = cmarch_consts(A);
  const float inv_steps = __fdiv_rn(1.0f, (float)A.s.max_steps);
  const int L = ckpt_len(A);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    float o[3], d[3];
    load_ray(ro, rd, r, o, d);
    const float h_in = cmarch_step_len(A, d);
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(A.s.near, d[a]));
    int cnt = 0, chunk_start = 0, c = -1;
    int64_t pos = kWrite ? ray_off[r] : 0;
    uint32_t* rec = ckpt ? ckpt + r * (4 * kCkpt) : nullptr;
    for (int k = 0; k < A.s.max_steps; ++k) {
      if (!kWrite && rec && k % L == 0) {   // a new chunk: close the previous one, record x
        if (c >= 0) rec[4 * c + 3] = (uint32_t)(cnt - chunk_start);
        ++c;
        chunk_start = cnt;
        rec[4 * c] = __float_as_uint(x[0]);
        rec[4 * c + 1] = __float_as_uint(x[1]);
        rec[4 * c + 2] = __float_as_uint(x[2]);
      }
      float xc[3], j[3];
      bool inside;
      if (!cmarch_point(M, x, d, xc, j, inside)) break;
      if (keep_point(A, mask, xc)) {
        if (kWrite) {
          int64_t s = pos + cnt;
          xyz[3 * s + 0] = xc[0];
          xyz[3 * s + 1] = xc[1];
          xyz[3 * s + 2] = xc[2];
          ray_id[s] = (int32_t)r;
          step_k[s] = k;
          s_mid[s] = __fmul_rn(__fadd_rn((float)k, 0.5f), inv_steps);
          s_len[s] = inv_steps;
        }
        ++cnt;
      }
      if (!cmarch_advance(A, x, d, j, inside, h_in)) break;
    }
    if (!kWrite) {
      counts[r] = cnt;
      if (rec) {
        if (c >= 0) rec[4 * c + 3] = (uint32_t)(cnt - chunk_start);
        for (int cc = c + 1; cc < kCkpt; ++cc) rec[4 * cc + 3] = 0xffffffffu;
      }
    }
  }
}

// Mode 1, pass 2 from the checkpoints: a block of 256 threads takes 32 rays,
// warp c of it chunk c of each of them (the lanes of a warp march the same
// part of 32 rays, so they take the same branches); each thread repeats the
// march of its chunk from the recorded x (the same FP32 operations as pass
// 1, so the same points) and writes its kept samples after those of the
// ray's earlier chunks.
__global__ void __launch_bounds__(32 * kCkpt) contracted_fill_kernel(
    SamplerArgs A, const float* __restrict__ rd, int64_t R, const uint8_t* __restrict__ mask,
    const uint32_t* __restrict__ ckpt, const int64_t* __restrict__ ray_off, float* __restrict__ xyz,
    int32_t* __restrict__ ray_id, int32_t* __restrict__ step_k, float* __restrict__ s_mid,
    float* __restrict__ s_len) {
  __shared__ int kept[kCkpt][32];
  const CMarch M = cmarch_consts(A);
  const float inv_steps = __fdiv_rn(1.0f, (float)A.s.max_steps);
  const int L = ckpt_len(A);
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * 32 + lane;
  const bool ray_ok = r < R;
  const uint32_t* rec = ckpt + (ray_ok ? r : 0) * (4 * kCkpt) + 4 * c;
  const uint32_t n_c = ray_ok ? rec[3] : 0xffffffffu;
  const int mine = n_c == 0xffffffffu ? 0 : (int)n_c;
  kept[c][lane] = mine;
  __syncthreads();
  int before = 0;   // kept samples of the ray's earlier chunks
  for (int q = 0; q < c; ++q) before += kept[q][lane];
  if (mine == 0) return;
  float d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = __ldg(rd + 3 * r + a);
  const float h_in = cmarch_step_len(A, d);
  float x[3] = {__uint_as_float(rec[0]), __uint_as_float(rec[1]), __uint_as_float(rec[2])};
  int64_t s = ray_off[r] + before;
  const bool vec = ((reinterpret_cast<uintptr_t>(xyz) | reinterpret_cast<uintptr_t>(ray_id) |
                     reinterpret_cast<uintptr_t>(step_k) | reinterpret_cast<uintptr_t>(s_mid) |
                     reinterpret_cast<uintptr_t>(s_len)) & 15u) == 0;
  // samples are written in groups of four consecutive list positions (16-byte
  // stores; xyz as three), one at a time before the first aligned position
  float bx[4][3] = {};
  int bk[4] = {};
  int nb = 0;
  auto put1 = [&](const float* p, int k) {
    xyz[3 * s] = p[0];
    xyz[3 * s + 1] = p[1];
    xyz[3 * s + 2] = p[2];
    ray_id[s] = (int32_t)r;
    step_k[s] = k;
    s_mid[s] = __fmul_rn(__fadd_rn((float)k, 0.5f), inv_steps);
    s_len[s] = inv_steps;
    ++s;
  };
  auto flush4 = [&]() {
    float4* xq = reinterpret_cast<float4*>(xyz + 3 * s);
    xq[0] = make_float4(bx[0][0], bx[0][1], bx[0][2], bx[1][0]);
    xq[1] = make_float4(bx[1][1], bx[1][2], bx[2][0], bx[2][1]);
    xq[2] = make_float4(bx[2][2], bx[3][0], bx[3][1], bx[3][2]);
    *reinterpret_cast<int4*>(ray_id + s) = make_int4((int)r, (int)r, (int)r, (int)r);
    *reinterpret_cast<int4*>(step_k + s) = make_int4(bk[0], bk[1], bk[2], bk[3]);
    *reinterpret_cast<float4*>(s_mid + s) = make_float4(
        __fmul_rn(__fadd_rn((float)bk[0], 0.5f), inv_steps), __fmul_rn(__fadd_rn((float)bk[1], 0.5f), inv_steps),
        __fmul_rn(__fadd_rn((float)bk[2], 0.5f), inv_steps), __fmul_rn(__fadd_rn((float)bk[3], 0.5f), inv_steps));
    *reinterpret_cast<float4*>(s_len + s) = make_float4(inv_steps, inv_steps, inv_steps, inv_steps);
    s += 4;
  };
  const int k_end = min((c + 1) * L, A.s.max_steps);
  for (int k = c * L; k < k_end; ++k) {
    float xc[3], j[3];
    bool inside;
    if (!cmarch_point(M, x, d, xc, j, inside)) break;
    if (keep_point(A, mask, xc)) {
      if (!vec || ((s & 3) != 0 && nb == 0)) {
        put1(xc, k);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)   // static slots, so that the buffer stays in registers
          if (q == nb) {
            bx[q][0] = xc[0];
            bx[q][1] = xc[1];
            bx[q][2] = xc[2];
            bk[q] = k;
          }
        if (++nb == 4) {
          flush4();
          nb = 0;
        }
      }
    }
    if (!cmarch_advance(A, x, d, j, inside, h_in)) break;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < nb) put1(bx[q], bk[q]);
}

// Exclusive scan of int32 counts into int64 offsets off[0..n] (one block of
// 1024 threads).  Each pass covers 8192 counts: thread t takes 8 consecutive
// ones (two 16-byte loads when aligned), scans them in registers, and the
// block scans the per-thread totals; a running carry joins the passes.
__global__ void __launch_bounds__(1024) scan_counts_kernel(const int32_t* __restrict__ counts, int64_t n,
                                                           int64_t* __restrict__ off,
                                                           int64_t* __restrict__ total_out) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t pass_total;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const bool vec = (reinterpret_cast<uintptr_t>(counts) & 15u) == 0;
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += 8 * (int64_t)blockDim.x) {
    const int64_t i0 = base + 8 * (int64_t)t;
    int32_t c[8];
    if (vec && i0 + 8 <= n) {
      const int4 a = __ldg(reinterpret_cast<const int4*>(counts + i0));
      const int4 b = __ldg(reinterpret_cast<const int4*>(counts + i0 + 4));
      c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
      c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) c[k] = i0 + k < n ? __ldg(counts + i0 + k) : 0;
    }
    int64_t loc[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      loc[k] = s;
      s += c[k];
    }
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int nw = (int)(blockDim.x >> 5);
      int64_t v = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      if (lane < nw) warp_tot[lane] = v;   // inclusive warp totals
      if (lane == nw - 1) pass_total = v;
    }
    __syncthreads();
    const int64_t ex = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + incl - s;
    if (i0 + 8 <= n && (reinterpret_cast<uintptr_t>(off + i0) & 15u) == 0) {
#pragma unroll
      for (int k = 0; k < 8; k += 2)
        *reinterpret_cast<longlong2*>(off + i0 + k) = make_longlong2(ex + loc[k], ex + loc[k + 1]);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (i0 + k < n) off[i0 + k] = ex + loc[k];
    }
    carry += pass_total;
    __syncthreads();   // warp_tot and pass_total are rewritten by the next pass
  }
  if (t == 0) {
    off[n] = carry;
    if (total_out) *total_out = carry;
  }
}

// Live list: live_idx[live_off[r] + i] = ray_off[r] + i for i < seg_len[r].
__global__ void live_fill_kernel(const int64_t* __restrict__ ray_off,
                                 const int32_t* __restrict__ seg_len, int64_t R,
                                 const int64_t* __restrict__ live_off, int32_t* __restrict__ live_idx) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < R; r += nwarps) {
    int64_t b = ray_off[r];
    int64_t dst = live_off[r];
    int n = seg_len[r];
    for (int i = lane; i < n; i += 32) live_idx[dst + i] = (int32_t)(b + i);
  }
}

// Low-weight cull of the colour-query list: warp per ray, the first
// seg_len[r] samples, kept iff w >= w_min (one ballot per 32 samples).  With
// fill, kept samples are listed in ray order and the rgb and g_k0 rows of the
// culled ones are zeroed; without, only the count per ray is written.
template <bool kFill>
__global__ void cull_kernel(const int64_t* __restrict__ ray_off, const int32_t* __restrict__ seg_len,
                            const float* __restrict__ w, float w_min, int64_t R, int32_t* __restrict__ counts,
                            const int64_t* __restrict__ off, int32_t* __restrict__ live_idx,
                            float* __restrict__ rgb, float* __restrict__ g_k0) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R; r += nw) {
    const int64_t b = ray_off[r];
    const int n = seg_len[r];
    int64_t dst = kFill ? off[r] : 0;
    int cnt = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const bool valid = i < n;
      const bool keep = valid && __ldg(w + b + i) >= w_min;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (kFill) {
        if (keep) live_idx[dst + __popc(bal & lt)] = (int32_t)(b + i);
        if (valid && !keep) {
          const int64_t s = b + i;
          if (rgb) {
            rgb[3 * s] = 0.0f;
            rgb[3 * s + 1] = 0.0f;
            rgb[3 * s + 2] = 0.0f;
          }
          if (g_k0) {
            float4* q = reinterpret_cast<float4*>(g_k0 + s * 12);
            q[0] = q[1] = q[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
        }
        dst += __popc(bal);
      } else {
        cnt += __popc(bal);
      }
    }
    if (!kFill && lane == 0) counts[r] = cnt;
  }
}

static bool fill_args(SamplerArgs& A, const dvgo_grid_desc* g, const dvgo_sampler_desc* s) {
  for (int a = 0; a < 3; ++a) {
    A.lo[a] = g->lo[a];
    A.hi[a] = g->hi[a];
    A.G[a] = g->G[a];
    if (g->G[a] < 2 || !(g->hi[a] > g->lo[a])) return false;
    // FP32: (float)(G-1) / (hi - lo)
    volatile float num = (float)(g->G[a] - 1);
    volatile float den = g->hi[a] - g->lo[a];
    A.scale[a] = num / den;
  }
  A.s = *s;
  return true;
}

}  // namespace dvgo

using namespace dvgo;

// Workspace: per-ray counts ((R+1) int32, padded to 256 bytes), then R x
// kBitWords uint32 per-ray words: the keep bits of pass 1 (modes 0 and 2) or
// the march checkpoints of pass 1 (mode 1).
static size_t counts_bytes(int64_t R) {
  return (size_t)((R + 1) * sizeof(int32_t) + 255) / 256 * 256;
}

extern "C" size_t dvgo_sample_rays_workspace_size(int64_t R) {
  return counts_bytes(R) + (size_t)R * kBitWords * sizeof(uint32_t);
}

extern "C" int dvgo_sample_rays(const float* rays_o, const float* rays_d, int64_t R,
                                const dvgo_grid_desc* grid, const dvgo_sampler_desc* smp,
                                const uint8_t* mask, int64_t S_cap, int64_t* ray_off, float* xyz,
                                int32_t* ray_id, int32_t* step_k, float* s_mid, float* s_len,
                                void* ws, size_t ws_bytes, void* stream) {
  DVGO_CHECK_ARG(grid && smp && ray_off && R >= 0);
  DVGO_CHECK_ARG(R == 0 || (rays_o && rays_d && xyz && ray_id && step_k && s_mid && s_len && ws));
  DVGO_CHECK_ARG(smp->mode >= 0 && smp->mode <= 2);
  DVGO_CHECK_ARG(smp->max_steps >= 0);
  if (smp->mode == 0 || smp->mode == 2) DVGO_CHECK_ARG(smp->step > 0.0f);
  if (smp->mode == 1) DVGO_CHECK_ARG(smp->step_c > 0.0f && smp->contract_b > 0.0f);
  if (smp->mode == 2) DVGO_CHECK_ARG(smp->ndc_near > 0.0f && smp->ndc_fx > 0.0f && smp->ndc_fy > 0.0f);
  if (S_cap < R * (int64_t)smp->max_steps || S_cap > INT32_MAX) return DVGO_ERR_SHAPE;
  if (ws_bytes < dvgo_sample_rays_workspace_size(R)) return DVGO_ERR_WORKSPACE;
  SamplerArgs A;
  DVGO_CHECK_ARG(fill_args(A, grid, smp));
  cudaStream_t st = as_stream(stream);
  if (R == 0) {
    cudaMemsetAsync(ray_off, 0, sizeof(int64_t), st);
    return launch_status();
  }
  int32_t* counts = reinterpret_cast<int32_t*>(ws);
  if (smp->mode == 0 || smp->mode == 2) {
    const int block = 256;
    int g = grid_for(R * 32, block, 16);
    uint32_t* bits = smp->max_steps <= 32 * kBitWords
                         ? reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + counts_bytes(R))
                         : nullptr;
    if (smp->mode == 0) {
      bbox_count_kernel<false><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, counts, bits);
      scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, ray_off, nullptr);
      bbox_fill_kernel<false><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, bits, ray_off, xyz, ray_id,
                                                   step_k, s_mid, s_len);
    } else {
      bbox_count_kernel<true><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, counts, bits);
      scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, ray_off, nullptr);
      bbox_fill_kernel<true><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, bits, ray_off, xyz, ray_id,
                                                  step_k, s_mid, s_len);
    }
  } else {
    // one warp of rays per block, so that the sequential marches spread over
    // every SM (8192 rays: 256 blocks)
    const int block = 32;
    int g = (int)ceil_div(R, block);
    // pass 1 records the march's checkpoints in the keep-bit words, so that
    // pass 2 runs kCkpt chunks of each march in parallel
    uint32_t* ckpt = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + counts_bytes(R));
    contracted_kernel<false><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, counts, ckpt,
                                                  nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, ray_off, nullptr);
    contracted_fill_kernel<<<(int)ceil_div(R, 32), 32 * kCkpt, 0, st>>>(A, rays_d, R, mask, ckpt, ray_off,
                                                                        xyz, ray_id, step_k, s_mid, s_len);
  }
  return launch_status();
}

extern "C" size_t dvgo_live_samples_workspace_size(int64_t R) {
  // offsets [R + 1] int64, then (the cull) counts [R] int32
  return (size_t)((R + 1) * sizeof(int64_t) + 255) / 256 * 256 + (size_t)(R * sizeof(int32_t) + 255) / 256 * 256;
}

extern "C" int dvgo_live_samples_cull(const int64_t* ray_off, const int32_t* seg_len, const float* w,
                                      float w_min, int64_t R, int32_t* live_idx, int64_t* live_count,
                                      float* rgb, float* g_k0, void* ws, size_t ws_bytes, void* stream) {
  DVGO_CHECK_ARG(ray_off && seg_len && w && live_idx && live_count && ws && R >= 0 && w_min >= 0.0f);
  DVGO_CHECK_ARG(((uintptr_t)g_k0 % 16) == 0);
  if (ws_bytes < dvgo_live_samples_workspace_size(R)) return DVGO_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  if (R == 0) {
    cudaMemsetAsync(live_count, 0, sizeof(int64_t), st);
    return launch_status();
  }
  int64_t* off = reinterpret_cast<int64_t*>(ws);
  int32_t* counts = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(ws) +
                                               (size_t)((R + 1) * sizeof(int64_t) + 255) / 256 * 256);
  const int g = grid_for(R * 32, 256, 16);
  cull_kernel<false><<<g, 256, 0, st>>>(ray_off, seg_len, w, w_min, R, counts, nullptr, nullptr, nullptr, nullptr);
  scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, off, live_count);
  cull_kernel<true><<<g, 256, 0, st>>>(ray_off, seg_len, w, w_min, R, nullptr, off, live_idx, rgb, g_k0);
  return launch_status();
}

extern "C" int dvgo_live_samples(const int64_t* ray_off, const int32_t* seg_len, int64_t R,
                                 int32_t* live_idx, int64_t* live_count, void* ws, size_t ws_bytes,
                                 void* stream) {
  DVGO_CHECK_ARG(ray_off && seg_len && live_idx && live_count && ws && R >= 0);
  if (ws_bytes < dvgo_live_samples_workspace_size(R)) return DVGO_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  if (R == 0) {
    cudaMemsetAsync(live_count, 0, sizeof(int64_t), st);
    return launch_status();
  }
  int64_t* live_off = reinterpret_cast<int64_t*>(ws);
  scan_counts_kernel<<<1, 1024, 0, st>>>(seg_len, R, live_off, live_count);
  live_fill_kernel<<<grid_for(R * 32, 256, 16), 256, 0, st>>>(ray_off, seg_len, R, live_off,
                                                              live_idx);
  return launch_status();
}

// ------------------------------------------------------------------------
// Ray sampling that allocates nothing.  Some callers cannot call cudaMalloc
// at all -- for example a host application that owns the device's whole
// memory budget and does not let libraries allocate, or code running where
// allocation is not permitted -- so they cannot provide the workspace that
// dvgo_sample_rays needs.  For them the per-ray count scratch lives in a
// fixed-size array in this library's own device memory: every GPU that
// loads the library holds it (4 MiB) until the process exits.
namespace dvgo {

constexpr int64_t kNoAllocMaxRays = 1 << 20;
static __device__ __align__(256) int32_t g_noalloc_counts[kNoAllocMaxRays + 1];

constexpr int kNoAllocMaxDevices = 64;

// The array's device address, cached per device together with the identity
// of the context it was looked up in.  A context that is torn down and
// created again (cudaDeviceReset, or a driver-API context switch) gets a new
// identity, so the address is looked up again there instead of being reused.
struct NoAllocSlot {
  int32_t* ptr = nullptr;
  unsigned long long ctx_id = 0;
};
static NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identity of the calling thread's current context (false if there is none
// or the driver does not provide the query).
static bool current_ctx_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_counts in the current context.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// (cudaGetSymbolAddress, with the device current) on the first call in a
// context and cached; later calls in the same context reuse it.
static int noalloc_counts(int32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DVGO_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return DVGO_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocSlot& slot = g_noalloc_slot[dev];
  unsigned long long id = 0;
  if (slot.ptr && current_ctx_id(&id) && id == slot.ctx_id) {
    *out = slot.ptr;
    return DVGO_OK;
  }
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_noalloc_counts) != cudaSuccess || !addr) return DVGO_ERR_CUDA;
  // without a context identity the address is not cached (looked up every call)
  slot.ptr = current_ctx_id(&id) ? static_cast<int32_t*>(addr) : nullptr;
  slot.ctx_id = id;
  *out = static_cast<int32_t*>(addr);
  return DVGO_OK;
}

}  // namespace dvgo

extern "C" int64_t dvgo_sample_rays_noalloc_max_rays(void) { return dvgo::kNoAllocMaxRays; }

extern "C" int dvgo_sample_rays_noalloc(const float* rays_o, const float* rays_d, int64_t R,
                                        const dvgo_grid_desc* grid, const dvgo_sampler_desc* smp,
                                        const uint8_t* mask, int64_t S_cap, int64_t* ray_off,
                                        float* xyz, int32_t* ray_id, int32_t* step_k,
                                        float* s_mid, float* s_len, void* stream) {
  DVGO_CHECK_ARG(grid && smp && ray_off && R >= 0);
  DVGO_CHECK_ARG(R == 0 || (rays_o && rays_d && xyz && ray_id && step_k && s_mid && s_len));
  DVGO_CHECK_ARG(smp->mode >= 0 && smp->mode <= 2);
  DVGO_CHECK_ARG(smp->max_steps >= 0);
  if (smp->mode == 0 || smp->mode == 2) DVGO_CHECK_ARG(smp->step > 0.0f);
  if (smp->mode == 1) DVGO_CHECK_ARG(smp->step_c > 0.0f && smp->contract_b > 0.0f);
  if (smp->mode == 2) DVGO_CHECK_ARG(smp->ndc_near > 0.0f && smp->ndc_fx > 0.0f && smp->ndc_fy > 0.0f);
  if (R > kNoAllocMaxRays) return DVGO_ERR_SHAPE;
  if (S_cap < R * (int64_t)smp->max_steps || S_cap > INT32_MAX) return DVGO_ERR_SHAPE;
  SamplerArgs A;
  DVGO_CHECK_ARG(fill_args(A, grid, smp));
  int32_t* counts = nullptr;
  int rc = noalloc_counts(&counts);
  if (rc != DVGO_OK) return rc;
  cudaStream_t st = as_stream(stream);
  if (R == 0) {
    cudaMemsetAsync(ray_off, 0, sizeof(int64_t), st);
    return launch_status();
  }
  // the count kernel writes counts[0, R) before the scan reads them, so the
  // shared array needs no clearing between calls
  if (smp->mode == 0) {
    const int block = 256;
    int g = grid_for(R * 32, block, 16);
    bbox_count_kernel<false><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, counts, nullptr);
    scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, ray_off, nullptr);
    bbox_fill_kernel<false><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, nullptr, ray_off, xyz,
                                                 ray_id, step_k, s_mid, s_len);
  } else if (smp->mode == 2) {
    const int block = 256;
    int g = grid_for(R * 32, block, 16);
    bbox_count_kernel<true><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, counts, nullptr);
    scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, ray_off, nullptr);
    bbox_fill_kernel<true><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, nullptr, ray_off, xyz,
                                                ray_id, step_k, s_mid, s_len);
  } else {
    // one warp of rays per block, so that the sequential marches spread over
    // every SM (8192 rays: 256 blocks)
    const int block = 32;
    int g = (int)ceil_div(R, block);
    contracted_kernel<false><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, counts, nullptr,
                                                  nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    scan_counts_kernel<<<1, 1024, 0, st>>>(counts, R, ray_off, nullptr);
    contracted_kernel<true><<<g, block, 0, st>>>(A, rays_o, rays_d, R, mask, nullptr, nullptr, ray_off, xyz,
                                                 ray_id, step_k, s_mid, s_len);
  }
  return launch_status();
}
