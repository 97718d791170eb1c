"""ctypes binding of libdvgo.so (declared in include/dvgo.h).

Argument marshalling only: every function here takes torch tensors (device
memory), turns them into raw pointers plus the current CUDA stream, and
calls the C entry point of the same name.  A nonzero status raises
DvgoError.  The library is loaded on first use; if it has not been built
(``paper_2206_05085_gb300.build``), loading fails loudly -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdvgo.so")

F32, BF16, F32_TC = 0, 1, 2

P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int32
F = ctypes.c_float
INT = ctypes.c_int
SZ = ctypes.c_size_t


class GridDesc(ctypes.Structure):
    _fields_ = [("lo", F * 3), ("hi", F * 3), ("G", I32 * 3)]

    @staticmethod
    def make(lo, hi, G):
        d = GridDesc()
        lo = [float(v) for v in (lo if hasattr(lo, "__len__") else (lo,) * 3)]
        hi = [float(v) for v in (hi if hasattr(hi, "__len__") else (hi,) * 3)]
        G = [int(v) for v in (G if hasattr(G, "__len__") else (G,) * 3)]
        for a in range(3):
            d.lo[a], d.hi[a], d.G[a] = lo[a], hi[a], G[a]
        return d


class SamplerDesc(ctypes.Structure):
    _fields_ = [("mode", I32), ("near", F), ("far", F), ("step", F), ("step_offset", F),
                ("use_slab", I32), ("max_steps", I32), ("contract_b", F), ("p_inf", I32),
                ("step_c", F), ("ndc_fx", F), ("ndc_fy", F), ("ndc_near", F)]


class TvGrid(ctypes.Structure):
    _fields_ = [("grid", P), ("dtype", I32), ("C", I32), ("weight", F), ("touched", P),
                ("g_grid", P)]


class AdamParam(ctypes.Structure):
    _fields_ = [("p", P), ("p_shadow", P), ("g", P), ("m", P), ("v", P), ("n", I64),
                ("touched", P), ("block_elems", I64), ("lr", F), ("block_list", P),
                ("block_count", P)]


class DvgoError(RuntimeError):
    pass


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise DvgoError(f"{LIB_PATH} not built; run paper_2206_05085_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    sig = {
        "dvgo_version": ([], INT),
        "dvgo_status_string": ([INT], ctypes.c_char_p),
        "dvgo_grid_bricked_elems": ([P, I32], I64),
        "dvgo_grid_num_bricks": ([P], I64),
        "dvgo_grid_pack": ([P, P, P, I32, INT, P], INT),
        "dvgo_grid_unpack": ([P, P, P, I32, INT, P], INT),
        "dvgo_build_mask": ([P, INT, P, F, F, F, P, P], INT),
        "dvgo_sample_grid_fwd": ([P, INT, P, I32, P, P, I64, P, P, P], INT),
        "dvgo_sample_grid_bwd": ([P, P, I32, P, P, I64, P, P, P, P], INT),
        "dvgo_sample_grid_bwd2": ([P, I32, P, P, P, I32, P, P, P, P, P, I64, P, P], INT),
        "dvgo_sample_rays_workspace_size": ([I64], SZ),
        "dvgo_sample_rays": ([P, P, I64, P, P, P, I64, P, P, P, P, P, P, P, SZ, P], INT),
        "dvgo_live_samples_workspace_size": ([I64], SZ),
        "dvgo_live_samples": ([P, P, I64, P, P, P, SZ, P], INT),
        "dvgo_alpha_weights_fwd": ([P, P, I64, F, F, P, F, P, P, P, P, P], INT),
        "dvgo_composite_rgb_fwd": ([P, P, P, P, P, I64, P, P, P], INT),
        "dvgo_composite_fwd": ([P, P, P, I64, F, F, P, F, P, P, P, P, P, P, P], INT),
        "dvgo_grid_adam_step": ([P, P, P, P, P, P, I32, P, F, F, F, F, I64, INT, P], INT),
        "dvgo_composite_bwd": ([P, P, P, P, P, P, P, I64, F, F, P, P, P, P, P], INT),
        "dvgo_distortion_fwd": ([P, P, P, P, P, I64, P, P], INT),
        "dvgo_distortion_bwd": ([P, F, P, P, P, P, P, I64, P, P], INT),
        "dvgo_rgb_loss": ([P, P, P, I64, F, P, P, P], INT),
        "dvgo_composite_distortion_fwd": ([P, P, P, P, P, P, P, I64, P, P, P, P], INT),
        "dvgo_composite_loss_workspace_size": ([I64], SZ),
        "dvgo_read_probe": ([P, I64, I32, P, I32, P], INT),
        "dvgo_density_alpha_fwd": ([P, INT, P, P, P, I64, F, F, P, F, P, P, P, P, P, P], INT),
        "dvgo_composite_distortion_loss_fwd": ([P, P, P, P, P, P, P, I64, P, P, F, P, P, P, P, P, P], INT),
        "dvgo_composite_distortion_bwd": ([P, F, P, P, P, P, P, P, P, P, I64, F, F, P, P, P, P], INT),
        "dvgo_composite_distortion_loss_fwd_bwd": ([P, P, P, P, P, P, P, I64, P, P, F, F, P, P, F, F,
                                                    P, P, P, P, P, P, P, P], INT),
        "dvgo_rgbnet_fwd": ([P, P, P, P, I64, P, P, INT, P, P, P], INT),
        "dvgo_rgbnet_bwd": ([P, P, P, P, P, P, P, I64, P, P, INT, P, P, P, P, P], INT),
        "dvgo_rgbnet_act_bytes": ([I64, INT], I64),
        "dvgo_tv_add_grad": ([P, INT, P, I32, F, F, INT, P, P, P], INT),
        "dvgo_adam_step": ([P, P, P, P, P, I64, P, I64, F, F, F, F, I64, INT, P], INT),
        "dvgo_tv_add_grad_multi": ([P, I32, P, F, INT, P, P, P], INT),
        "dvgo_touched_compact": ([P, I64, P, P, P], INT),
        "dvgo_adam_step_multi": ([P, I32, F, F, F, I64, INT, P], INT),
        "dvgo_adam_step_multi_dev": ([P, I32, F, F, F, P, INT, P], INT),
        "dvgo_device_status": ([P], INT),
        "dvgo_proposal_fwd": ([P, P, I64, P, P, P, P], INT),
        "dvgo_proposal_bwd": ([P, P, P, I64, P, P, P, P], INT),
        "dvgo_proposal_xent": ([P, P, P, I64, F, F, P, P, P, P], INT),
        "dvgo_proposal_select": ([P, P, I64, I32, P, P, P], INT),
        "dvgo_compact_samples": ([P, P, I32, P, I64, P, P, P, P, P, P, P, P, P, P, P, P, F, P, P], INT),
        "dvgo_sample_rays_noalloc_max_rays": ([], I64),
        "dvgo_sample_rays_noalloc": ([P, P, I64, P, P, P, I64, P, P, P, P, P, P, P], INT),
        "dvgo_grid_resample": ([P, P, P, INT, P, I32, P], INT),
        "dvgo_update_mask": ([P, INT, P, F, F, F, P, P, P, P], INT),
        "dvgo_live_samples_cull": ([P, P, P, F, I64, P, P, P, P, P, SZ, P], INT),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res


def exported_names():
    """Names this binding expects the library to export."""
    return [
        "dvgo_version", "dvgo_status_string", "dvgo_grid_bricked_elems", "dvgo_grid_num_bricks",
        "dvgo_grid_pack", "dvgo_grid_unpack", "dvgo_build_mask", "dvgo_sample_grid_fwd",
        "dvgo_sample_grid_bwd", "dvgo_sample_rays_workspace_size", "dvgo_sample_rays",
        "dvgo_live_samples_workspace_size", "dvgo_live_samples", "dvgo_alpha_weights_fwd",
        "dvgo_composite_rgb_fwd", "dvgo_composite_bwd", "dvgo_distortion_fwd",
        "dvgo_distortion_bwd", "dvgo_rgb_loss", "dvgo_rgbnet_fwd", "dvgo_rgbnet_bwd",
        "dvgo_tv_add_grad", "dvgo_adam_step", "dvgo_device_status", "dvgo_proposal_fwd",
        "dvgo_proposal_bwd", "dvgo_proposal_xent", "dvgo_proposal_select", "dvgo_compact_samples",
        "dvgo_sample_rays_noalloc_max_rays", "dvgo_sample_rays_noalloc", "dvgo_rgbnet_act_bytes",
        "dvgo_sample_grid_bwd2", "dvgo_composite_distortion_fwd", "dvgo_composite_distortion_bwd",
        "dvgo_composite_distortion_loss_fwd_bwd",
        "dvgo_tv_add_grad_multi", "dvgo_adam_step_multi", "dvgo_touched_compact",
        "dvgo_adam_step_multi_dev", "dvgo_composite_fwd", "dvgo_grid_adam_step",
        "dvgo_composite_loss_workspace_size", "dvgo_composite_distortion_loss_fwd",
        "dvgo_read_probe", "dvgo_density_alpha_fwd"]


def ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    assert t.is_cuda or not torch.cuda.is_available(), "expected a device tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(name, rc):
    if rc != 0:
        msg = lib().dvgo_status_string(rc).decode()
        raise DvgoError(f"{name} failed: {msg} ({rc})")


def _call(name, *args):
    _check(name, getattr(lib(), name)(*args))


def _vec3(v, ctype):
    return (ctype * 3)(*v)


# ---------------------------------------------------------------- grid
def grid_bricked_elems(G, C):
    return int(lib().dvgo_grid_bricked_elems(_vec3(G, I32), C))


def grid_num_bricks(G):
    return int(lib().dvgo_grid_num_bricks(_vec3(G, I32)))


def grid_pack(dense, bricked, G, C, dtype, stream=None):
    _call("dvgo_grid_pack", ptr(dense), ptr(bricked), _vec3(G, I32), C, dtype, _stream(stream))


def grid_unpack(bricked, dense, G, C, dtype, stream=None):
    _call("dvgo_grid_unpack", ptr(bricked), ptr(dense), _vec3(G, I32), C, dtype, _stream(stream))


def grid_resample(src, G_src, dst, dst_dtype, G_dst, C, stream=None):
    _call("dvgo_grid_resample", ptr(src), _vec3(G_src, I32), ptr(dst), dst_dtype, _vec3(G_dst, I32), C,
          _stream(stream))


def update_mask(density, dtype, gd, shift, interval, thres, brick_list, brick_count, mask, stream=None):
    _call("dvgo_update_mask", ptr(density), dtype, ctypes.byref(gd), shift, interval, thres, ptr(brick_list),
          ptr(brick_count), ptr(mask), _stream(stream))


def build_mask(density, dtype, gd, shift, interval, thres, mask, stream=None):
    _call("dvgo_build_mask", ptr(density), dtype, ctypes.byref(gd), shift, interval, thres,
          ptr(mask), _stream(stream))


def sample_grid_fwd(grid, dtype, gd, C, xyz, idx, n_cap, n_dev, out, stream=None):
    _call("dvgo_sample_grid_fwd", ptr(grid), dtype, ctypes.byref(gd), C, ptr(xyz), ptr(idx),
          n_cap, ptr(n_dev), ptr(out), _stream(stream))


def sample_grid_bwd(g_out, gd, C, xyz, idx, n_cap, n_dev, g_grid, touched, stream=None):
    _call("dvgo_sample_grid_bwd", ptr(g_out), ctypes.byref(gd), C, ptr(xyz), ptr(idx), n_cap,
          ptr(n_dev), ptr(g_grid), ptr(touched), _stream(stream))


def sample_grid_bwd2(g_out_a, C_a, g_grid_a, touched_a, g_out_b, C_b, g_grid_b, touched_b, gd, xyz,
                     idx, n_cap, n_dev, stream=None):
    _call("dvgo_sample_grid_bwd2", ptr(g_out_a), C_a, ptr(g_grid_a), ptr(touched_a), ptr(g_out_b),
          C_b, ptr(g_grid_b), ptr(touched_b), ctypes.byref(gd), ptr(xyz), ptr(idx), n_cap,
          ptr(n_dev), _stream(stream))


# -------------------------------------------------------------- sampler
def sample_rays_workspace_size(R):
    return int(lib().dvgo_sample_rays_workspace_size(R))


def sample_rays(rays_o, rays_d, R, gd, sd, mask, S_cap, ray_off, xyz, ray_id, step_k, s_mid,
                s_len, ws, stream=None):
    _call("dvgo_sample_rays", ptr(rays_o), ptr(rays_d), R, ctypes.byref(gd), ctypes.byref(sd),
          ptr(mask), S_cap, ptr(ray_off), ptr(xyz), ptr(ray_id), ptr(step_k), ptr(s_mid),
          ptr(s_len), ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


def sample_rays_noalloc_max_rays():
    return int(lib().dvgo_sample_rays_noalloc_max_rays())


def sample_rays_noalloc(rays_o, rays_d, R, gd, sd, mask, S_cap, ray_off, xyz, ray_id, step_k,
                        s_mid, s_len, stream=None):
    """dvgo_sample_rays without a workspace, for callers that cannot allocate."""
    _call("dvgo_sample_rays_noalloc", ptr(rays_o), ptr(rays_d), R, ctypes.byref(gd),
          ctypes.byref(sd), ptr(mask), S_cap, ptr(ray_off), ptr(xyz), ptr(ray_id), ptr(step_k),
          ptr(s_mid), ptr(s_len), _stream(stream))


def live_samples_workspace_size(R):
    return int(lib().dvgo_live_samples_workspace_size(R))


def live_samples_cull(ray_off, seg_len, w, w_min, R, live_idx, live_count, rgb, g_k0, ws, stream=None):
    _call("dvgo_live_samples_cull", ptr(ray_off), ptr(seg_len), ptr(w), w_min, R, ptr(live_idx),
          ptr(live_count), ptr(rgb), ptr(g_k0), ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


def live_samples(ray_off, seg_len, R, live_idx, live_count, ws, stream=None):
    _call("dvgo_live_samples", ptr(ray_off), ptr(seg_len), R, ptr(live_idx), ptr(live_count),
          ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


# ------------------------------------------------------------ rendering
def density_alpha_fwd(grid, dtype, gd, xyz, ray_off, R, shift, interval, T_stop, raw, w, T, n_live,
                      T_end, stream=None, delta=None):
    _call("dvgo_density_alpha_fwd", ptr(grid), dtype, ctypes.byref(gd), ptr(xyz), ptr(ray_off), R,
          shift, interval, ptr(delta), T_stop, ptr(raw), ptr(w), ptr(T), ptr(n_live), ptr(T_end),
          _stream(stream))


def alpha_weights_fwd(raw, ray_off, R, shift, interval, T_stop, w, T, n_live, T_end, stream=None,
                      delta=None):
    _call("dvgo_alpha_weights_fwd", ptr(raw), ptr(ray_off), R, shift, interval, ptr(delta), T_stop,
          ptr(w), ptr(T), ptr(n_live), ptr(T_end), _stream(stream))


def composite_rgb_fwd(w, rgb, ray_off, n_live, T_end, R, bg, color, stream=None):
    _call("dvgo_composite_rgb_fwd", ptr(w), ptr(rgb), ptr(ray_off), ptr(n_live), ptr(T_end), R,
          _vec3(bg, F), ptr(color), _stream(stream))


def composite_fwd(raw, rgb, ray_off, R, shift, interval, T_stop, bg, color, w, T, n_live, T_end,
                  stream=None, delta=None):
    _call("dvgo_composite_fwd", ptr(raw), ptr(rgb), ptr(ray_off), R, shift, interval, ptr(delta), T_stop,
          _vec3(bg, F), ptr(color), ptr(w), ptr(T), ptr(n_live), ptr(T_end), _stream(stream))


def grid_adam_step(p, p_shadow, g, m, v, G, C, touched, lr, beta1, beta2, eps, step, zero_grad,
                   stream=None):
    _call("dvgo_grid_adam_step", ptr(p), ptr(p_shadow), ptr(g), ptr(m), ptr(v), _vec3(G, I32), C,
          ptr(touched), lr, beta1, beta2, eps, step, int(zero_grad), _stream(stream))


def composite_bwd(g_color, g_w, raw, T, rgb, ray_off, n_live, R, shift, interval, bg, g_raw,
                  g_rgb=None, stream=None, delta=None):
    _call("dvgo_composite_bwd", ptr(g_color), ptr(g_w), ptr(raw), ptr(T), ptr(rgb), ptr(ray_off),
          ptr(n_live), R, shift, interval, ptr(delta), _vec3(bg, F), ptr(g_raw), ptr(g_rgb),
          _stream(stream))


def composite_distortion_fwd(w, rgb, m, ds, ray_off, n_live, T_end, R, bg, color, L_r, stream=None):
    _call("dvgo_composite_distortion_fwd", ptr(w), ptr(rgb), ptr(m), ptr(ds), ptr(ray_off),
          ptr(n_live), ptr(T_end), R, _vec3(bg, F), ptr(color), ptr(L_r), _stream(stream))


def composite_loss_workspace_size(R):
    return int(lib().dvgo_composite_loss_workspace_size(R))


def composite_distortion_loss_fwd(w, rgb, m, ds, ray_off, n_live, T_end, R, bg, target, lambda_dist,
                                  color, L_r, g_color, loss_out, ws, stream=None):
    _call("dvgo_composite_distortion_loss_fwd", ptr(w), ptr(rgb), ptr(m), ptr(ds), ptr(ray_off),
          ptr(n_live), ptr(T_end), R, _vec3(bg, F), ptr(target), lambda_dist, ptr(color), ptr(L_r),
          ptr(g_color), ptr(loss_out), ptr(ws), _stream(stream))


def composite_distortion_loss_fwd_bwd(w, rgb, m, ds, ray_off, n_live, T_end, R, bg, target,
                                      lambda_dist, g_L, raw, T, shift, interval, color, L_r,
                                      g_color, loss_out, g_raw, ws, stream=None, delta=None):
    _call("dvgo_composite_distortion_loss_fwd_bwd", ptr(w), ptr(rgb), ptr(m), ptr(ds), ptr(ray_off),
          ptr(n_live), ptr(T_end), R, _vec3(bg, F), ptr(target), lambda_dist, g_L, ptr(raw), ptr(T),
          shift, interval, ptr(delta), ptr(color), ptr(L_r), ptr(g_color), ptr(loss_out), ptr(g_raw),
          ptr(ws), _stream(stream))


def composite_distortion_bwd(g_color, g_L, w, raw, T, rgb, m, ds, ray_off, n_live, R, shift,
                             interval, bg, g_raw, stream=None, delta=None):
    _call("dvgo_composite_distortion_bwd", ptr(g_color), g_L, ptr(w), ptr(raw), ptr(T), ptr(rgb),
          ptr(m), ptr(ds), ptr(ray_off), ptr(n_live), R, shift, interval, ptr(delta), _vec3(bg, F),
          ptr(g_raw), _stream(stream))


def distortion_fwd(w, m, ds, ray_off, seg_len, R, L_r, stream=None):
    _call("dvgo_distortion_fwd", ptr(w), ptr(m), ptr(ds), ptr(ray_off), ptr(seg_len), R, ptr(L_r),
          _stream(stream))


def distortion_bwd(g_L, g_L_scalar, w, m, ds, ray_off, seg_len, R, g_w, stream=None):
    _call("dvgo_distortion_bwd", ptr(g_L), g_L_scalar, ptr(w), ptr(m), ptr(ds), ptr(ray_off),
          ptr(seg_len), R, ptr(g_w), _stream(stream))


def rgb_loss(color, target, L_r, R, lambda_dist, loss_out, g_color, stream=None):
    _call("dvgo_rgb_loss", ptr(color), ptr(target), ptr(L_r), R, lambda_dist, ptr(loss_out),
          ptr(g_color), _stream(stream))


# ------------------------------------------------------------ colour MLP
def rgbnet_fwd(k0, rays_d, ray_id, idx, n_cap, n_dev, params, precision, rgb, act=None,
               stream=None):
    _call("dvgo_rgbnet_fwd", ptr(k0), ptr(rays_d), ptr(ray_id), ptr(idx), n_cap, ptr(n_dev),
          ptr(params), precision, ptr(rgb), ptr(act), _stream(stream))


def rgbnet_act_bytes(n_cap, precision):
    return int(lib().dvgo_rgbnet_act_bytes(n_cap, precision))


def rgbnet_bwd(g_rgb, g_color, w, k0, rays_d, ray_id, idx, n_cap, n_dev, params, precision,
               g_params, g_k0, act=None, rgb=None, stream=None):
    _call("dvgo_rgbnet_bwd", ptr(g_rgb), ptr(g_color), ptr(w), ptr(k0), ptr(rays_d), ptr(ray_id),
          ptr(idx), n_cap, ptr(n_dev), ptr(params), precision, ptr(act), ptr(rgb), ptr(g_params),
          ptr(g_k0), _stream(stream))


# ------------------------------------------------------- regularisation
def tv_add_grad(grid, dtype, G, C, weight, delta, dense_mode, touched, g_grid, stream=None):
    _call("dvgo_tv_add_grad", ptr(grid), dtype, _vec3(G, I32), C, weight, delta, int(dense_mode),
          ptr(touched), ptr(g_grid), _stream(stream))


def tv_add_grad_multi(grids, G, delta, dense_mode, brick_list=None, brick_count=None, stream=None):
    """grids: list of (grid, dtype, C, weight, touched, g_grid)."""
    arr = (TvGrid * len(grids))(*[TvGrid(ptr(g), dt, C, w, ptr(t), ptr(gg))
                                  for g, dt, C, w, t, gg in grids])
    _call("dvgo_tv_add_grad_multi", arr, len(grids), _vec3(G, I32), delta, int(dense_mode),
          ptr(brick_list), ptr(brick_count), _stream(stream))


def touched_compact(touched, nb, brick_list, brick_count, stream=None):
    _call("dvgo_touched_compact", ptr(touched), nb, ptr(brick_list), ptr(brick_count),
          _stream(stream))


def adam_step_multi(params, beta1, beta2, eps, step, zero_grad, stream=None):
    """params: list of (p, p_shadow, g, m, v, n, touched, block_elems, lr[, block_list,
    block_count])."""
    def one(t):
        p, sh, g, m, v, n, tch, be, lr = t[:9]
        bl, bc = (t[9], t[10]) if len(t) > 9 else (None, None)
        return AdamParam(ptr(p), ptr(sh), ptr(g), ptr(m), ptr(v), n, ptr(tch), be, lr, ptr(bl), ptr(bc))
    arr = (AdamParam * len(params))(*[one(t) for t in params])
    _call("dvgo_adam_step_multi", arr, len(params), beta1, beta2, eps, step, int(zero_grad),
          _stream(stream))


def adam_step_multi_dev(params, beta1, beta2, eps, step_dev, zero_grad, stream=None):
    """adam_step_multi with the step count in device memory (incremented here)."""
    def one(t):
        p, sh, g, m, v, n, tch, be, lr = t[:9]
        bl, bc = (t[9], t[10]) if len(t) > 9 else (None, None)
        return AdamParam(ptr(p), ptr(sh), ptr(g), ptr(m), ptr(v), n, ptr(tch), be, lr, ptr(bl), ptr(bc))
    arr = (AdamParam * len(params))(*[one(t) for t in params])
    _call("dvgo_adam_step_multi_dev", arr, len(params), beta1, beta2, eps, ptr(step_dev),
          int(zero_grad), _stream(stream))


def adam_step(p, p_shadow, g, m, v, n, touched, block_elems, lr, beta1, beta2, eps, step,
              zero_grad, stream=None):
    _call("dvgo_adam_step", ptr(p), ptr(p_shadow), ptr(g), ptr(m), ptr(v), n, ptr(touched),
          block_elems, lr, beta1, beta2, eps, step, int(zero_grad), _stream(stream))


def read_probe(buf, nbytes, reps, sink, stream=None):
    _call("dvgo_read_probe", ptr(buf), nbytes, reps, ptr(sink), sink.numel(), _stream(stream))


def device_status(stream=None):
    return int(lib().dvgo_device_status(_stream(stream)))


# ------------------------------------------------------ learned proposal
def proposal_fwd(xyz, idx, n_cap, n_dev, params, logits, stream=None):
    _call("dvgo_proposal_fwd", ptr(xyz), ptr(idx), n_cap, ptr(n_dev), ptr(params), ptr(logits),
          _stream(stream))


def proposal_bwd(g_logits, xyz, idx, n_cap, n_dev, params, g_params, stream=None):
    _call("dvgo_proposal_bwd", ptr(g_logits), ptr(xyz), ptr(idx), n_cap, ptr(n_dev), ptr(params),
          ptr(g_params), _stream(stream))


def proposal_xent(logits, w_target, ray_off, R, eps_u, g_scale, loss_r, g_logits, q, stream=None):
    _call("dvgo_proposal_xent", ptr(logits), ptr(w_target), ptr(ray_off), R, eps_u, g_scale,
          ptr(loss_r), ptr(g_logits), ptr(q), _stream(stream))


def proposal_select(q, ray_off, R, n_draw, sel, n_sel, stream=None):
    _call("dvgo_proposal_select", ptr(q), ptr(ray_off), R, n_draw, ptr(sel), ptr(n_sel),
          _stream(stream))


def compact_samples(sel, n_sel, n_draw, ray_off, R, xyz, ray_id, step_k, s_mid, s_len, out_ray_off,
                    out_xyz, out_ray_id, out_step_k, out_s_mid, out_s_len, out_src=None, stream=None,
                    interval=0.0, out_delta=None):
    _call("dvgo_compact_samples", ptr(sel), ptr(n_sel), n_draw, ptr(ray_off), R, ptr(xyz),
          ptr(ray_id), ptr(step_k), ptr(s_mid), ptr(s_len), ptr(out_ray_off), ptr(out_xyz),
          ptr(out_ray_id), ptr(out_step_k), ptr(out_s_mid), ptr(out_s_len), ptr(out_src),
          interval, ptr(out_delta), _stream(stream))
