"""Learned proposal: fewer samples per ray, chosen by a small network.

Not part of the paper.  Candidates are up to 512 uniformly spaced points per
ray inside the scene bbox (no occupancy mask).  The plain renderer's own
compositing weights over the candidates (raw->alpha, transmittance, early
stop) are the training target of a BF16 tensor-core MLP on the candidates'
position encoding; at render time the network's per-ray softmax is inverted
at 64 evenly spaced quantiles (duplicates collapsed), each pick stands for
the candidates from itself up to the next pick (its alpha interval and
distortion span cover that gap), and the plain training step runs on them.
The plain dense render over all candidates stays the fallback.  Every step
runs in the library's kernels (dvgo_proposal_*, dvgo_compact_samples, the
renderer).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import _lib as L
from .synth import PROPOSAL_DIMS, RenderParams, SceneConfig, grid_dims, mlp_num_params, voxel_size
from .train import Trainer, alpha_shift

N_CAND = 512
N_DRAW = 64


def candidate_params(cfg: SceneConfig, rp: RenderParams) -> RenderParams:
    """Up to 512 midpoint candidates per ray over its bbox slab: the step is
    the box diagonal / 512, so every slab fits."""
    diag = math.sqrt(3.0) * (cfg.bbox_max - cfg.bbox_min)
    step = np.float32(diag / N_CAND)
    return dataclasses.replace(rp, step=float(step), step_offset=0.5, use_slab=True,
                               max_steps=N_CAND, interval=float(step / voxel_size(cfg)),
                               mask_thres=None)


class Proposal:
    def __init__(self, cfg: SceneConfig, rp: RenderParams, density_view, density_dtype,
                 params: np.ndarray, n_rays: int, lr: float = 1e-2, eps_u: float = 1e-3,
                 device: str = "cuda"):
        self.cfg, self.R = cfg, int(n_rays)
        self.rp = candidate_params(cfg, rp)
        self.dev = torch.device(device)
        self.eps_u, self.lr = eps_u, lr
        self.density, self.density_dtype = density_view, density_dtype
        assert params.size == mlp_num_params(PROPOSAL_DIMS)
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.params = torch.tensor(params, **f32)
        self.g = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.it = 0
        self.gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, list(grid_dims(cfg)))
        sd = L.SamplerDesc()
        sd.mode, sd.near, sd.far, sd.step = 0, self.rp.near, self.rp.far, self.rp.step
        sd.step_offset, sd.use_slab, sd.max_steps = self.rp.step_offset, 1, N_CAND
        self.sd = sd
        R, S = self.R, self.R * N_CAND
        self.S_cap = S
        i32 = dict(dtype=torch.int32, device=self.dev)
        self.ray_off = torch.zeros(R + 1, dtype=torch.int64, device=self.dev)
        self.xyz = torch.empty(S, 3, **f32)
        self.ray_id = torch.empty(S, **i32)
        self.step_k = torch.empty(S, **i32)
        self.s_mid = torch.empty(S, **f32)
        self.s_len = torch.empty(S, **f32)
        self.raw = torch.empty(S, **f32)
        self.w = torch.empty(S, **f32)
        self.T = torch.empty(S, **f32)
        self.n_live = torch.empty(R, **i32)
        self.T_end = torch.empty(R, **f32)
        self.logits = torch.empty(S, **f32)
        self.g_logits = torch.empty(S, **f32)
        self.q = torch.empty(S, **f32)
        self.loss_r = torch.empty(R, **f32)
        self.sel = torch.empty(R * N_DRAW, **i32)
        self.n_sel = torch.empty(R, **i32)
        self.ws = torch.empty(L.sample_rays_workspace_size(R), dtype=torch.uint8, device=self.dev)
        self.shift = alpha_shift(self.rp.alpha_init)

    def candidates(self, rays_o, rays_d):
        L.sample_rays(rays_o, rays_d, self.R, self.gd, self.sd, None, self.S_cap, self.ray_off,
                      self.xyz, self.ray_id, self.step_k, self.s_mid, self.s_len, self.ws)

    def target_weights(self):
        """The plain renderer's compositing weights over the candidates."""
        S_dev = self.ray_off[self.R:]
        L.sample_grid_fwd(self.density, self.density_dtype, self.gd, 1, self.xyz, None, self.S_cap,
                          S_dev, self.raw)
        L.alpha_weights_fwd(self.raw, self.ray_off, self.R, self.shift, self.rp.interval,
                            self.rp.T_stop, self.w, self.T, self.n_live, self.T_end)

    def train_step(self, rays_o, rays_d):
        """One proposal update on the plain renderer's weights; returns the
        per-ray cross-entropy (device)."""
        self.candidates(rays_o, rays_d)
        self.target_weights()
        S_dev = self.ray_off[self.R:]
        L.proposal_fwd(self.xyz, None, self.S_cap, S_dev, self.params, self.logits)
        L.proposal_xent(self.logits, self.w, self.ray_off, self.R, self.eps_u, 1.0 / self.R,
                        self.loss_r, self.g_logits, self.q)
        L.proposal_bwd(self.g_logits, self.xyz, None, self.S_cap, S_dev, self.params, self.g)
        self.it += 1
        L.adam_step(self.params, None, self.g, self.m, self.v, self.params.numel(), None, 0, self.lr,
                    0.9, 0.99, 1e-15, self.it, True)
        return self.loss_r

    def select_into(self, tr: Trainer, rays_o, rays_d, uniform: bool = False, spans: bool = True):
        """Candidates -> proposal softmax -> inverse-CDF picks -> the picked
        samples written into the trainer's sample buffers.  uniform=True picks
        with a flat distribution instead (the baseline without the network).
        spans=False keeps each pick's own one-candidate interval."""
        self.candidates(rays_o, rays_d)
        S_dev = self.ray_off[self.R:]
        if uniform:
            self.logits.zero_()
        else:
            L.proposal_fwd(self.xyz, None, self.S_cap, S_dev, self.params, self.logits)
        L.proposal_xent(self.logits, None, self.ray_off, self.R, 0.0, 0.0, None, None, self.q)
        L.proposal_select(self.q, self.ray_off, self.R, N_DRAW, self.sel, self.n_sel)
        if spans and tr.delta is None:
            tr.delta = torch.empty(tr.S_cap, dtype=torch.float32, device=self.dev)
        elif not spans:
            tr.delta = None
        L.compact_samples(self.sel, self.n_sel, N_DRAW, self.ray_off, self.R, self.xyz,
                          self.ray_id, self.step_k, self.s_mid, self.s_len, tr.ray_off, tr.xyz,
                          tr.ray_id, tr.step_k, tr.s_mid, tr.s_len,
                          interval=self.rp.interval, out_delta=tr.delta)


def psnr(a: torch.Tensor, b: torch.Tensor) -> float:
    mse = torch.mean((a.double() - b.double()) ** 2).item()
    return float("inf") if mse == 0 else -10.0 * math.log10(mse)


def make_forms(cfg, rp, density, feature, mlp_params, prop_params, n_rays, precision="f32"):
    """The plain dense-candidate trainer, the proposal-form trainer (<= 64
    samples per ray, same grids and MLP) and the proposal itself."""
    rp_c = candidate_params(cfg, rp)
    dense = Trainer(cfg, rp_c, density, feature, mlp_params, n_rays, precision)
    prop_tr = Trainer(cfg, dataclasses.replace(rp_c, max_steps=N_DRAW), density, feature,
                      mlp_params, n_rays, precision)
    grid, dt = dense.density.render_view
    prop = Proposal(cfg, rp, grid, dt, prop_params, n_rays)
    return dense, prop_tr, prop
