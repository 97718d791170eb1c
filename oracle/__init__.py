"""FP64 CPU oracle for the DVGOv2 training step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``dvgo_oracle.c`` (plain
loops, FP64, one ray / one grid point at a time) through ctypes and shares
nothing with the CUDA library.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):

* ``distortion`` / ``distortion_naive`` / ``distortion_grad``: pinned (O(N)
  form equals the O(N^2) double sum; closed forms for N = 1, 2; gradient
  equals central finite differences and the direct O(N^2) derivative).
* ``composite`` / ``composite_bwd``: pinned (sum of weights = 1 - T_end,
  alpha = 0 gives the background, an opaque sample gives its colour, halting
  index, finite differences, closed form for two samples).
* ``raw2alpha``: pinned (raw = 0 closed form, finite differences, torch's
  softplus as a library routine).
* ``trilinear`` / ``trilinear_adjoint``: pinned (corners, affine fields,
  adjoint dot-product identity, torch grid_sample as a library routine).
* ``mlp_fwd`` / ``mlp_bwd`` / ``freq_encode``: pinned (torch fp64 autograd as
  a library routine; the BF16-operand variant against torch with bfloat16
  rounding of the same operands and gradient hooks).
* ``tv_loss`` / ``tv_add_grad``: pinned (torch huber_loss, finite
  differences, sparse-mode support).
* ``adam``: pinned (torch.optim.Adam as a library routine; skipped entries
  bit-unchanged).
* ``sample_rays_bbox``: pinned (closed-form slab intersections for
  axis-aligned rays, brute-force nearest-voxel culling).
* ``sample_rays_contracted`` / ``contract``: pinned (identity inside the unit
  ball, limit 1 + b, continuity, monotone along rays, finite-difference
  Jacobian step).
* ``softmax_xent`` / ``inverse_cdf_select`` and their ragged forms: pinned
  (torch cross-entropy, numpy searchsorted, ragged = per-ray dense call).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvgo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP32 decisions need -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fvisibility=hidden", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int32
D = ctypes.c_double
F = ctypes.c_float
INT = ctypes.c_int


def _declare(L):
    L.or_alpha_shift.restype = D
    L.or_alpha_shift.argtypes = [D]
    L.or_raw2alpha.argtypes = [P, I64, D, D, P, P]
    L.or_build_mask.argtypes = [P, I64, D, D, D, P]
    L.or_sample_rays_bbox.restype = I64
    L.or_sample_rays_bbox.argtypes = [P, P, I64, P, P, P, F, F, F, F, INT, I32, P,
                                      P, P, P, P, P, P, I64]
    L.or_sample_rays_ndc.restype = I64
    L.or_sample_rays_ndc.argtypes = [P, P, I64, P, P, P, F, F, F, F, I32, P, P, P, P, P, P, P, I64]
    L.or_contract.argtypes = [P, I64, D, INT, P]
    L.or_sample_rays_contracted.restype = I64
    L.or_sample_rays_contracted.argtypes = [P, P, I64, F, INT, F, F, I32, P, P, P, P,
                                            P, P, P, P, P, P, I64]
    L.or_trilinear.argtypes = [P, P, INT, P, P, P, I64, P]
    L.or_trilinear_adjoint.argtypes = [P, P, INT, P, P, P, I64, P]
    L.or_composite.argtypes = [P, P, P, I64, D, D, P, D, P, P, P, P, P, P]
    L.or_composite_bwd.argtypes = [P, P, P, I64, D, D, P, D, P, P, P, P, P]
    for nm in ("or_distortion_naive", "or_distortion"):
        getattr(L, nm).argtypes = [P, P, P, P, P, I64, P]
    for nm in ("or_distortion_grad", "or_distortion_grad_naive"):
        getattr(L, nm).argtypes = [P, P, P, P, P, P, I64, P]
    L.or_grid_resample.argtypes = [P, P, INT, P, P]
    L.or_mlp_fwd.argtypes = [P, INT, P, P, I64, INT, P]
    L.or_mlp_bwd.argtypes = [P, INT, P, P, I64, INT, P, P, P]
    L.or_mlp_min_abs_preact.argtypes = [P, INT, P, P, I64, P]
    L.or_freq_encode.argtypes = [P, I64, INT, P]
    L.or_tv_loss.restype = D
    L.or_tv_loss.argtypes = [P, P, INT, D]
    L.or_tv_add_grad.argtypes = [P, P, INT, D, D, INT, P, P]
    L.or_adam.argtypes = [P, P, P, P, I64, D, D, D, D, I64, INT]
    L.or_softmax_xent.argtypes = [P, P, I64, INT, P, P, P]
    L.or_inverse_cdf_select.argtypes = [P, I64, INT, INT, P, P]
    L.or_proposal_xent_ragged.argtypes = [P, P, P, I64, D, P, P, P]
    L.or_inverse_cdf_select_ragged.argtypes = [P, P, I64, INT, P, P]


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _vec3f(v):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float32), (3,)))


def _vec3i(v):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.int32), (3,)))


# --------------------------------------------------------------------------
def alpha_shift(alpha_init: float) -> float:
    """shift = log(1/(1 - alpha_init) - 1) (alpha_init of Sec. 5.4)."""
    return lib().or_alpha_shift(alpha_init)


def raw2alpha(raw, shift, interval):
    raw = _f64(raw)
    a = np.empty_like(raw)
    da = np.empty_like(raw)
    lib().or_raw2alpha(_p(raw), raw.size, shift, interval, _p(a), _p(da))
    return a, da


def build_mask(density, shift, interval, thres=1e-4):
    density = _f32(density)
    m = np.empty(density.shape, dtype=np.uint8)
    lib().or_build_mask(_p(density), density.size, shift, interval, thres, _p(m))
    return m


class Samples:
    """Ragged sample list: ray_off [R+1], xyz [S,3] f32, ray_id, step_k [S]
    int32, s_mid, s_len [S] f64."""

    def __init__(self, ray_off, xyz, ray_id, step_k, s_mid, s_len):
        self.ray_off, self.xyz, self.ray_id = ray_off, xyz, ray_id
        self.step_k, self.s_mid, self.s_len = step_k, s_mid, s_len

    @property
    def S(self):
        return int(self.ray_off[-1])


def sample_rays_bbox(o, d, lo, hi, G, near, far, step, off, use_slab, max_steps, mask=None):
    o, d = _f32(o), _f32(d)
    R = o.shape[0]
    cap = R * max_steps
    ray_off = np.zeros(R + 1, np.int64)
    xyz = np.zeros((cap, 3), np.float32)
    rid = np.zeros(cap, np.int32)
    sk = np.zeros(cap, np.int32)
    sm = np.zeros(cap, np.float64)
    sl = np.zeros(cap, np.float64)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    S = lib().or_sample_rays_bbox(_p(o), _p(d), R, _p(_vec3f(lo)), _p(_vec3f(hi)),
                                  _p(_vec3i(G)), near, far, step, off, int(use_slab),
                                  max_steps, _p(mask), _p(ray_off), _p(xyz), _p(rid),
                                  _p(sk), _p(sm), _p(sl), cap)
    return Samples(ray_off, xyz[:S], rid[:S], sk[:S], sm[:S], sl[:S])


def sample_rays_ndc(o, d, lo, hi, G, fx, fy, near, step, max_steps, mask=None):
    """Forward-facing sampling: NDC warp of each ray, crossings of the depth
    layers (see or_sample_rays_ndc)."""
    o, d = _f32(o), _f32(d)
    R = o.shape[0]
    cap = R * max_steps
    ray_off = np.zeros(R + 1, np.int64)
    xyz = np.zeros((cap, 3), np.float32)
    rid = np.zeros(cap, np.int32)
    sk = np.zeros(cap, np.int32)
    sm = np.zeros(cap, np.float64)
    sl = np.zeros(cap, np.float64)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    S = lib().or_sample_rays_ndc(_p(o), _p(d), R, _p(_vec3f(lo)), _p(_vec3f(hi)), _p(_vec3i(G)), fx, fy,
                                 near, step, max_steps, _p(mask), _p(ray_off), _p(xyz), _p(rid), _p(sk),
                                 _p(sm), _p(sl), cap)
    return Samples(ray_off, xyz[:S], rid[:S], sk[:S], sm[:S], sl[:S])


def contract(x, b, p_inf):
    x = _f64(x).reshape(-1, 3)
    out = np.empty_like(x)
    lib().or_contract(_p(x), x.shape[0], b, int(p_inf), _p(out))
    return out


def sample_rays_contracted(o, d, b, p_inf, near, step_c, max_steps, lo, hi, G, mask=None):
    o, d = _f32(o), _f32(d)
    R = o.shape[0]
    cap = R * max_steps
    ray_off = np.zeros(R + 1, np.int64)
    xyz = np.zeros((cap, 3), np.float32)
    rid = np.zeros(cap, np.int32)
    sk = np.zeros(cap, np.int32)
    sm = np.zeros(cap, np.float64)
    sl = np.zeros(cap, np.float64)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    S = lib().or_sample_rays_contracted(_p(o), _p(d), R, b, int(p_inf), near, step_c,
                                        max_steps, _p(_vec3f(lo)), _p(_vec3f(hi)),
                                        _p(_vec3i(G)), _p(mask), _p(ray_off), _p(xyz),
                                        _p(rid), _p(sk), _p(sm), _p(sl), cap)
    return Samples(ray_off, xyz[:S], rid[:S], sk[:S], sm[:S], sl[:S])


def trilinear(grid, lo, hi, xyz):
    """grid: dense float32 [Gz,Gy,Gx] or [Gz,Gy,Gx,C]; returns [n,C] f64."""
    grid = _f32(grid)
    C = 1 if grid.ndim == 3 else grid.shape[3]
    G = _vec3i((grid.shape[2], grid.shape[1], grid.shape[0]))
    xyz = _f32(xyz).reshape(-1, 3)
    out = np.zeros((xyz.shape[0], C), np.float64)
    lib().or_trilinear(_p(grid), _p(G), C, _p(_vec3f(lo)), _p(_vec3f(hi)), _p(xyz),
                       xyz.shape[0], _p(out))
    return out


def grid_resample(grid, G_dst):
    """grid: dense [Gz, Gy, Gx] or [Gz, Gy, Gx, C] f32; G_dst (x, y, z).
    Returns the trilinear resampling to G_dst points per axis (FP64)."""
    g = _f32(grid)
    squeeze = g.ndim == 3
    if squeeze:
        g = g[..., None]
    Gs = _vec3i((g.shape[2], g.shape[1], g.shape[0]))
    Gd = _vec3i(G_dst)
    C = g.shape[3]
    out = np.zeros((int(Gd[2]), int(Gd[1]), int(Gd[0]), C))
    lib().or_grid_resample(_p(g), _p(Gs), C, _p(Gd), _p(out))
    return out[..., 0] if squeeze else out


def trilinear_adjoint(g_out, grid_shape, lo, hi, xyz):
    """Returns the dense f64 gradient of the grid (shape grid_shape)."""
    C = 1 if len(grid_shape) == 3 else int(grid_shape[3])
    g_out = _f64(g_out).reshape(xyz.shape[0], C)
    Gz, Gy, Gx = grid_shape[:3]
    G = _vec3i((Gx, Gy, Gz))
    xyz = _f32(xyz).reshape(-1, 3)
    gg = np.zeros((Gz, Gy, Gx, C), np.float64)
    lib().or_trilinear_adjoint(_p(g_out), _p(G), C, _p(_vec3f(lo)), _p(_vec3f(hi)), _p(xyz),
                               xyz.shape[0], _p(gg))
    return gg.reshape(grid_shape)


def composite(raw, rgb, ray_off, shift, interval, T_stop, bg, delta=None):
    """Returns dict(w, T, n_live, T_end, color).  delta: optional per-sample
    intervals (voxel units) in place of the scalar interval."""
    raw = _f64(raw)
    S = raw.size
    rgb = None if rgb is None else _f64(rgb).reshape(S, 3)
    ray_off = _i64(ray_off)
    R = ray_off.size - 1
    w = np.zeros(S)
    T = np.zeros(S)
    n_live = np.zeros(R, np.int32)
    T_end = np.zeros(R)
    color = np.zeros((R, 3))
    dl = None if delta is None else _f64(delta)
    lib().or_composite(_p(raw), _p(rgb), _p(ray_off), R, shift, interval, _p(dl), T_stop,
                       _p(_f64(np.broadcast_to(bg, (3,)))), _p(w), _p(T), _p(n_live),
                       _p(T_end), _p(color))
    return dict(w=w, T=T, n_live=n_live, T_end=T_end, color=color)


def composite_bwd(raw, rgb, ray_off, shift, interval, T_stop, bg, g_color, g_w_extra=None,
                  delta=None):
    raw = _f64(raw)
    S = raw.size
    rgb = None if rgb is None else _f64(rgb).reshape(S, 3)
    ray_off = _i64(ray_off)
    R = ray_off.size - 1
    g_color = _f64(g_color).reshape(R, 3)
    gwe = None if g_w_extra is None else _f64(g_w_extra)
    g_raw = np.zeros(S)
    g_rgb = np.zeros((S, 3))
    dl = None if delta is None else _f64(delta)
    lib().or_composite_bwd(_p(raw), _p(rgb), _p(ray_off), R, shift, interval, _p(dl), T_stop,
                           _p(_f64(np.broadcast_to(bg, (3,)))), _p(g_color), _p(gwe),
                           _p(g_raw), _p(g_rgb))
    return g_raw, g_rgb


def _dist_call(fn, w, m, ds, ray_off, seg_len):
    w, m, ds, ray_off = _f64(w), _f64(m), _f64(ds), _i64(ray_off)
    R = ray_off.size - 1
    L = np.zeros(R)
    fn(_p(w), _p(m), _p(ds), _p(ray_off), _p(_i32(seg_len)), R, _p(L))
    return L


def distortion(w, m, ds, ray_off, seg_len=None):
    """Per-ray distortion loss by the O(N) prefix-sum form (Sec. 2)."""
    return _dist_call(lib().or_distortion, w, m, ds, ray_off, seg_len)


def distortion_naive(w, m, ds, ray_off, seg_len=None):
    """Per-ray distortion loss by the O(N^2) definition, Eq. (dist_loss)."""
    return _dist_call(lib().or_distortion_naive, w, m, ds, ray_off, seg_len)


def _dist_grad_call(fn, g_L, w, m, ds, ray_off, seg_len):
    w, m, ds, ray_off = _f64(w), _f64(m), _f64(ds), _i64(ray_off)
    R = ray_off.size - 1
    g_L = _f64(np.broadcast_to(g_L, (R,)))
    g = np.zeros(w.size)
    fn(_p(g_L), _p(w), _p(m), _p(ds), _p(ray_off), _p(_i32(seg_len)), R, _p(g))
    return g


def distortion_grad(g_L, w, m, ds, ray_off, seg_len=None):
    return _dist_grad_call(lib().or_distortion_grad, g_L, w, m, ds, ray_off, seg_len)


def distortion_grad_naive(g_L, w, m, ds, ray_off, seg_len=None):
    return _dist_grad_call(lib().or_distortion_grad_naive, g_L, w, m, ds, ray_off, seg_len)


def mlp_fwd(dims, params, x, out_sigmoid=True):
    dims = _i32(dims)
    params, x = _f64(params), _f64(x)
    n = x.shape[0]
    out = np.zeros((n, int(dims[-1])))
    lib().or_mlp_fwd(_p(dims), dims.size - 1, _p(params), _p(x), n, int(out_sigmoid), _p(out))
    return out


def mlp_bwd(dims, params, x, g_out, out_sigmoid=True):
    """Returns (g_params [P], g_x [n, dims[0]])."""
    dims = _i32(dims)
    params, x, g_out = _f64(params), _f64(x), _f64(g_out)
    n = x.shape[0]
    gp = np.zeros(params.size)
    gx = np.zeros((n, int(dims[0])))
    lib().or_mlp_bwd(_p(dims), dims.size - 1, _p(params), _p(x), n, int(out_sigmoid),
                     _p(g_out), _p(gp), _p(gx))
    return gp, gx


def mlp_min_abs_preact(dims, params, x):
    """Per sample, min |pre-activation| over the hidden ReLU layers."""
    dims = _i32(dims)
    params, x = _f64(params), _f64(x)
    out = np.zeros(x.shape[0])
    lib().or_mlp_min_abs_preact(_p(dims), dims.size - 1, _p(params), _p(x), x.shape[0], _p(out))
    return out


def freq_encode(v, F):
    v = _f32(v).reshape(-1, 3)
    out = np.zeros((v.shape[0], 3 + 6 * F))
    lib().or_freq_encode(_p(v), v.shape[0], F, _p(out))
    return out


def rgbnet_input(k0, dirs):
    """[k0 (12), view-direction encoding (3 + 6*4 = 27)] -> [n, 39]."""
    return np.concatenate([_f64(k0), freq_encode(dirs, 4)], axis=1)


def tv_loss(grid, delta=1.0):
    """grid: dense [Gz,Gy,Gx] or [Gz,Gy,Gx,C]."""
    g = _f64(grid)
    C = 1 if g.ndim == 3 else g.shape[3]
    G = _vec3i((g.shape[2], g.shape[1], g.shape[0]))
    return lib().or_tv_loss(_p(g), _p(G), C, delta)


def tv_add_grad(grid, grad, weight, delta=1.0, dense_mode=True):
    g = _f64(grid)
    C = 1 if g.ndim == 3 else g.shape[3]
    G = _vec3i((g.shape[2], g.shape[1], g.shape[0]))
    gin = _f64(grad)
    gout = np.zeros_like(gin)
    lib().or_tv_add_grad(_p(g), _p(G), C, weight, delta, int(dense_mode), _p(gin), _p(gout))
    return gout


def adam(p, g, m, v, lr, b1, b2, eps, t, skip_zero=True):
    """Returns updated (p, m, v) as new f64 arrays."""
    p, m, v = _f64(p).copy(), _f64(m).copy(), _f64(v).copy()
    g = _f64(g)
    lib().or_adam(_p(p), _p(g), _p(m), _p(v), p.size, lr, b1, b2, eps, t, int(skip_zero))
    return p, m, v


def softmax_xent(logits, p):
    logits, p = _f64(logits), _f64(p)
    R, K = logits.shape
    loss = np.zeros(R)
    g = np.zeros_like(logits)
    q = np.zeros_like(logits)
    lib().or_softmax_xent(_p(logits), _p(p), R, K, _p(loss), _p(g), _p(q))
    return loss, g, q


def inverse_cdf_select(q32, n_draw):
    q32 = _f32(q32)
    R, K = q32.shape
    sel = np.zeros((R, n_draw), np.int32)
    n_sel = np.zeros(R, np.int32)
    lib().or_inverse_cdf_select(_p(q32), R, K, n_draw, _p(sel), _p(n_sel))
    return sel, n_sel


def proposal_xent_ragged(logits, w, ray_off, eps_u):
    """Per-ray softmax cross-entropy against p = normalised w + uniform floor."""
    logits, w, ray_off = _f64(logits), _f64(w), _i64(ray_off)
    R = ray_off.size - 1
    loss = np.zeros(R)
    g = np.zeros_like(logits)
    q = np.zeros_like(logits)
    lib().or_proposal_xent_ragged(_p(logits), _p(w), _p(ray_off), R, eps_u, _p(loss), _p(g), _p(q))
    return loss, g, q


def inverse_cdf_select_ragged(q32, ray_off, n_draw):
    q32, ray_off = _f32(q32), _i64(ray_off)
    R = ray_off.size - 1
    sel = np.zeros((R, n_draw), np.int32)
    n_sel = np.zeros(R, np.int32)
    lib().or_inverse_cdf_select_ragged(_p(q32), _p(ray_off), R, n_draw, _p(sel), _p(n_sel))
    return sel, n_sel
