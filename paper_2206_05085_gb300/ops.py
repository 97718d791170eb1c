"""The forward/backward kernel pairs as ``torch.autograd.Function``s.

Each ``forward`` calls a forward entry point of ``libdvgo.so`` and each
``backward`` its hand-written adjoint (no PyTorch arithmetic on the data
path; tensors only carry device pointers and the stream).  Chaining the
functions gives the volume-rendering loss of one training iteration, whose
``backward()`` runs the same adjoint kernels that ``train.Trainer`` calls
directly:

  raw = sample_grid(density, xyz)                      (trilinear, Sec. 1)
  color, w = composite(raw, rgb, ray_off, ...)         (raw->alpha, T, w, C; Sec. 3)
  L_r = distortion(w, m, ds, ray_off, n_live)          (Eq. dist_loss, Sec. 2)
  rgb = rgbnet(k0, params, rays_d, ray_id)             (Tab. 1 colour MLP)

Ragged samples are CSR (``ray_off`` int64 [R+1]); every count is a host
integer here (the functions are for composing and testing; the training
step keeps its counts on the device).
"""
from __future__ import annotations

import torch

from . import _lib as L


def _zeros_like(t):
    return torch.zeros_like(t, memory_format=torch.contiguous_format)


class SampleGrid(torch.autograd.Function):
    """out[s] = trilinear(grid, xyz[s]), grid bricked FP32 with C channels.
    Backward: the trilinear adjoint scattered into a bricked FP32 gradient."""

    @staticmethod
    def forward(ctx, grid, xyz, gd, C):
        S = xyz.shape[0]
        out = torch.empty(S, C, dtype=torch.float32, device=xyz.device)
        L.sample_grid_fwd(grid, L.F32, gd, C, xyz, None, S, None, out)
        ctx.save_for_backward(xyz)
        ctx.gd, ctx.C, ctx.grid_shape = gd, C, grid.shape
        return out

    @staticmethod
    def backward(ctx, g_out):
        (xyz,) = ctx.saved_tensors
        g_grid = torch.zeros(ctx.grid_shape, dtype=torch.float32, device=xyz.device)
        L.sample_grid_bwd(g_out.contiguous(), ctx.gd, ctx.C, xyz, None, xyz.shape[0], None, g_grid,
                          None)
        return g_grid, None, None, None


class Composite(torch.autograd.Function):
    """Per ray: alpha_i = 1 - exp(-interval softplus(raw_i + shift)),
    T_i = prod_{j<i} (1 - alpha_j), w_i = T_i alpha_i, halt at T_i < T_stop,
    color = sum w_i rgb_i + T_end bg.  Outputs (color [R,3], w [S]).
    Backward: the reverse affine scan (g_w enters as the weights' gradient)."""

    @staticmethod
    def forward(ctx, raw, rgb, ray_off, shift, interval, T_stop, bg):
        R, S = ray_off.numel() - 1, raw.numel()
        dev = raw.device
        color = torch.empty(R, 3, dtype=torch.float32, device=dev)
        w = torch.empty(S, dtype=torch.float32, device=dev)
        T = torch.empty(S, dtype=torch.float32, device=dev)
        n_live = torch.empty(R, dtype=torch.int32, device=dev)
        T_end = torch.empty(R, dtype=torch.float32, device=dev)
        L.composite_fwd(raw, rgb, ray_off, R, shift, interval, T_stop, bg, color, w, T, n_live, T_end)
        ctx.save_for_backward(raw, rgb, ray_off, T, n_live)
        ctx.shift, ctx.interval, ctx.bg = shift, interval, bg
        ctx.mark_non_differentiable(n_live)
        return color, w, n_live

    @staticmethod
    def backward(ctx, g_color, g_w, _g_n_live):
        raw, rgb, ray_off, T, n_live = ctx.saved_tensors
        R = ray_off.numel() - 1
        if g_color is None:
            g_color = torch.zeros(R, 3, dtype=torch.float32, device=raw.device)
        g_raw = torch.empty_like(raw)
        g_rgb = torch.empty_like(rgb)
        L.composite_bwd(g_color.contiguous(), None if g_w is None else g_w.contiguous(), raw, T, rgb,
                        ray_off, n_live, R, ctx.shift, ctx.interval, ctx.bg, g_raw, g_rgb)
        return g_raw, g_rgb, None, None, None, None, None


class Distortion(torch.autograd.Function):
    """L_r = 2 sum_i w_i (m_i W_<i - WM_<i) + 1/3 sum_i w_i^2 ds_i over the
    first seg_len[r] samples of each ray (the O(N) form of Eq. dist_loss).
    Backward: dL_r/dw by the same prefix sums."""

    @staticmethod
    def forward(ctx, w, m, ds, ray_off, seg_len):
        R = ray_off.numel() - 1
        L_r = torch.empty(R, dtype=torch.float32, device=w.device)
        L.distortion_fwd(w, m, ds, ray_off, seg_len, R, L_r)
        ctx.save_for_backward(w, m, ds, ray_off, seg_len)
        return L_r

    @staticmethod
    def backward(ctx, g_L):
        w, m, ds, ray_off, seg_len = ctx.saved_tensors
        g_w = torch.empty_like(w)
        L.distortion_bwd(g_L.contiguous(), 0.0, w, m, ds, ray_off, seg_len, ray_off.numel() - 1, g_w)
        return g_w, None, None, None, None


class RGBNet(torch.autograd.Function):
    """Colour MLP (39 -> ReLU 128 -> ReLU 128 -> sigmoid 3) of every sample:
    input [k0 (12), view-direction encoding of rays_d[ray_id]].  precision:
    "f32tc" (FP32 accuracy on the tensor cores, the default), "f32" (CUDA
    cores) or "bf16" (stored BF16 parameters, BF16 tensor-core operands).
    Backward: the fused adjoint kernel (parameter and k0 gradients)."""

    PREC = {"f32": L.F32, "f32tc": L.F32_TC, "bf16": L.BF16}

    @staticmethod
    def forward(ctx, k0, params, rays_d, ray_id, precision="f32tc"):
        S = k0.shape[0]
        prec = RGBNet.PREC[precision]
        rgb = torch.empty(S, 3, dtype=torch.float32, device=k0.device)
        act = None
        if prec == L.F32:
            act = torch.empty(S, 256, dtype=torch.float32, device=k0.device)
        else:   # tensor-core forms: tile images of the split layer inputs
            act = torch.empty(L.rgbnet_act_bytes(S, prec), dtype=torch.uint8, device=k0.device)
        L.rgbnet_fwd(k0, rays_d, ray_id, None, S, None, params, prec, rgb, act)
        ctx.save_for_backward(k0, params, rays_d, ray_id, rgb)
        ctx.act, ctx.prec = act, prec
        return rgb

    @staticmethod
    def backward(ctx, g_rgb):
        k0, params, rays_d, ray_id, rgb = ctx.saved_tensors
        S = k0.shape[0]
        g_params = torch.zeros_like(params)
        g_k0 = torch.empty_like(k0)
        L.rgbnet_bwd(g_rgb.contiguous(), None, None, k0, rays_d, ray_id, None, S, None, params,
                     ctx.prec, g_params, g_k0, ctx.act, rgb)
        return g_k0, g_params, None, None, None


def sample_grid(grid, xyz, gd, C):
    return SampleGrid.apply(grid, xyz, gd, C)


def composite(raw, rgb, ray_off, shift, interval, T_stop, bg):
    return Composite.apply(raw, rgb, ray_off, shift, interval, T_stop, bg)


def distortion(w, m, ds, ray_off, seg_len=None):
    return Distortion.apply(w, m, ds, ray_off, seg_len)


def rgbnet(k0, params, rays_d, ray_id, precision="f32tc"):
    return RGBNet.apply(k0, params, rays_d, ray_id, precision)
