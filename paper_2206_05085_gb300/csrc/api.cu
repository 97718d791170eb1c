// C-ABI entry points of the colour MLP and library-wide helpers.
#include "common.cuh"
#include "mlp_common.cuh"

int dvgo_rgbnet_fwd_f32(const float*, const float*, const int32_t*, const int32_t*, int64_t,
                        const int64_t*, const float*, float*, float*, cudaStream_t);
int dvgo_rgbnet_bwd_f32(const float*, const float*, const float*, const float*, const float*,
                        const int32_t*, const int32_t*, int64_t, const int64_t*, const float*,
                        const float*, const float*, float*, float*, cudaStream_t);
int dvgo_mlp_status_read_and_clear(cudaStream_t);
int dvgo_rgbnet_fwd_tc(const float*, const float*, const int32_t*, const int32_t*, int64_t, const int64_t*,
                       const float*, float*, float*, bool, cudaStream_t);
int dvgo_rgbnet_bwd_tc(const float*, const float*, const float*, const float*, const int32_t*, const int32_t*,
                       int64_t, const int64_t*, const float*, float*, float*, float*, bool, cudaStream_t);
int64_t rgbnet_act_bytes_tc(int64_t);
int dvgo_mlp_tc_status_read_and_clear(cudaStream_t);

using namespace dvgo;

extern "C" int dvgo_version(void) { return 100; }

extern "C" const char* dvgo_status_string(int status) {
  switch (status) {
    case DVGO_OK: return "ok";
    case DVGO_ERR_INVALID_ARG: return "invalid argument";
    case DVGO_ERR_SHAPE: return "inconsistent sizes or capacity too small";
    case DVGO_ERR_CUDA: return "CUDA runtime error";
    case DVGO_ERR_BOUNDS: return "device-side bounds check failed";
    case DVGO_ERR_TIMEOUT: return "bounded device-side wait gave up";
    case DVGO_ERR_UNSUPPORTED: return "unsupported combination";
    case DVGO_ERR_WORKSPACE: return "workspace too small";
    case DVGO_ERR_RANGE: return "value outside the range of a split-FP16 operand";
    default: return "unknown status";
  }
}

extern "C" int dvgo_rgbnet_fwd(const float* k0, const float* rays_d, const int32_t* ray_id,
                               const int32_t* idx, int64_t n_cap, const int64_t* n_dev,
                               const float* params, int precision, float* rgb, float* act,
                               void* stream) {
  DVGO_CHECK_ARG(n_cap >= 0);
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG(k0 && rays_d && ray_id && params && rgb);
  DVGO_CHECK_ARG(((uintptr_t)k0 % 16) == 0 && ((uintptr_t)act % 16) == 0);
  cudaStream_t st = as_stream(stream);
  if (precision == DVGO_F32)
    return dvgo_rgbnet_fwd_f32(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb, act, st);
  if (precision == DVGO_F32_TC || precision == DVGO_BF16) {
    DVGO_CHECK_ARG(act != nullptr);
    return dvgo_rgbnet_fwd_tc(k0, rays_d, ray_id, idx, n_cap, n_dev, params, rgb, act,
                              precision == DVGO_BF16, st);
  }
  return DVGO_ERR_INVALID_ARG;
}

extern "C" int dvgo_rgbnet_bwd(const float* g_rgb, const float* g_color, const float* w, const float* k0,
                               const float* rays_d, const int32_t* ray_id, const int32_t* idx,
                               int64_t n_cap, const int64_t* n_dev, const float* params,
                               int precision, const float* act, const float* rgb, float* g_params,
                               float* g_k0, void* stream) {
  DVGO_CHECK_ARG(n_cap >= 0);
  if (n_cap == 0) return DVGO_OK;
  DVGO_CHECK_ARG((g_rgb || (g_color && w)) && k0 && rays_d && ray_id && params && g_params && g_k0);
  DVGO_CHECK_ARG(((uintptr_t)k0 % 16) == 0 && ((uintptr_t)g_k0 % 16) == 0 &&
                 ((uintptr_t)act % 16) == 0);
  cudaStream_t st = as_stream(stream);
  if (precision == DVGO_F32)
    return dvgo_rgbnet_bwd_f32(g_rgb, g_color, w, k0, rays_d, ray_id, idx, n_cap, n_dev, params, act,
                               rgb, g_params, g_k0, st);
  if (precision == DVGO_F32_TC || precision == DVGO_BF16) {
    // act: the forward's tile images (read) and the per-CTA partial rows
    // (written); rgb: the forward's output, for the sigmoid derivative
    DVGO_CHECK_ARG(act != nullptr && rgb != nullptr);
    return dvgo_rgbnet_bwd_tc(g_rgb, g_color, w, rgb, ray_id, idx, n_cap, n_dev, params,
                              const_cast<float*>(act), g_params, g_k0, precision == DVGO_BF16, st);
  }
  return DVGO_ERR_INVALID_ARG;
}

extern "C" int64_t dvgo_rgbnet_act_bytes(int64_t n_cap, int precision) {
  if (n_cap < 0) return -1;
  if (precision == DVGO_F32) return n_cap * 1024;
  if (precision == DVGO_F32_TC || precision == DVGO_BF16) return rgbnet_act_bytes_tc(n_cap);
  return -1;
}

// Read-bandwidth probe: every block reads buf[0 .. n4) (float4) reps times
// with coalesced 16-byte loads and folds the values into sink[block] (so the
// loads are kept).  With n4 * 16 bytes well inside L2 it measures the L2 read
// rate that the gathers' repeated corner reads see.
__global__ void __launch_bounds__(512) read_probe_kernel(const float4* __restrict__ buf, int64_t n4,
                                                         int reps, float* __restrict__ sink) {
  float acc = 0.0f;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
      const float4 v = __ldcg(buf + i);   // cached in L2 only
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sink + blockIdx.x, acc);
}

extern "C" int dvgo_read_probe(const void* buf, int64_t bytes, int32_t reps, float* sink,
                               int32_t sink_len, void* stream) {
  DVGO_CHECK_ARG(buf && sink && bytes >= 16 && reps >= 1 && sink_len >= 1);
  DVGO_CHECK_ARG((reinterpret_cast<uintptr_t>(buf) & 15u) == 0);
  read_probe_kernel<<<sink_len, 512, 0, as_stream(stream)>>>(reinterpret_cast<const float4*>(buf),
                                                            bytes / 16, reps, sink);
  return launch_status();
}

extern "C" int dvgo_device_status(void* stream) {
  const int a = dvgo_mlp_status_read_and_clear(as_stream(stream));
  const int b = dvgo_mlp_tc_status_read_and_clear(as_stream(stream));
  return a != DVGO_OK ? a : b;
}
