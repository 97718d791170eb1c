"""One DVGOv2 training iteration on the GPU, driven through the C ABI.

The order follows the paper's training loop (Sec. 2 listing: zero_grad ->
loss -> backward -> TV add-grad -> optimizer step) with the rendering
utilities of Sec. 3:

  forward : sample rays (bbox + occupancy mask, or contracted march) ->
            density query -> raw->alpha, transmittance, early stop ->
            live-sample list -> feature query -> colour MLP -> colour
            accumulation -> distortion loss -> photometric loss
  backward: distortion grad -> compositing adjoint -> colour-MLP adjoint ->
            grid scatters -> TV gradient -> sparse Adam (grids) + Adam (MLP)

Only samples in front of the halting point (T >= 1e-3) reach the colour
MLP: past it every weight and gradient is exactly zero.  Every buffer is
allocated once here (torch is used for device memory and the stream); the
step itself reads nothing back to the host.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import _lib as L
from .synth import RenderParams, SceneConfig

FEAT = 12


def alpha_shift(alpha_init: float) -> float:
    """shift = log(1/(1 - alpha_init) - 1), rounded to FP32 (Sec. 5.4 alpha_init)."""
    return float(np.float32(math.log(1.0 / (1.0 - alpha_init) - 1.0)))


@dataclasses.dataclass
class GridParam:
    """A bricked grid parameter with its optimizer state."""
    C: int
    p: torch.Tensor            # FP32 master (bricked)
    g: torch.Tensor            # FP32 gradient (bricked)
    m: torch.Tensor
    v: torch.Tensor
    touched: torch.Tensor      # uint8 per brick
    shadow: torch.Tensor | None  # BF16 copy read by the renderer (BF16 form)

    @property
    def render_view(self):
        return (self.shadow, L.BF16) if self.shadow is not None else (self.p, L.F32)


class Trainer:
    def __init__(self, cfg: SceneConfig, rp: RenderParams, density: np.ndarray,
                 feature: np.ndarray, mlp_params: np.ndarray, n_rays: int,
                 precision: str = "f32", device: str = "cuda", mask_update: bool = False,
                 w_min: float | None = None):
        self.cfg, self.rp, self.R = cfg, rp, int(n_rays)
        # mask_update: the occupancy mask follows the density (re-evaluated in the
        # bricks each optimizer step changed); w_min: samples in front of the halt
        # whose compositing weight is below w_min skip the colour query (feature
        # gather and colour MLP)
        self.mask_update = bool(mask_update)
        self.w_min = w_min
        self.dev = torch.device(device)
        # "f32": colour MLP in FP32 on the CUDA cores; "f32tc": FP32-accurate on
        # the tensor cores (split-FP16 operands); "bf16": BF16 grids and MLP
        self.precision = {"f32": L.F32, "f32tc": L.F32_TC, "bf16": L.BF16}[precision]
        from .synth import grid_dims
        G = list(grid_dims(cfg))
        self.G = G
        self.gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, G)
        self.shift = alpha_shift(rp.alpha_init)
        self.density = self._grid_param(density, 1)
        self.feature = self._grid_param(feature, FEAT)
        # colour MLP (flat FP32) and its Adam state
        self.mlp = torch.tensor(mlp_params, dtype=torch.float32, device=self.dev)
        self.mlp_g = torch.zeros_like(self.mlp)
        self.mlp_m = torch.zeros_like(self.mlp)
        self.mlp_v = torch.zeros_like(self.mlp)
        # occupancy mask (Sec. 1), built from the initial density
        self.mask = None
        if rp.mask_thres is not None:
            self.mask = torch.empty(G[2], G[1], G[0], dtype=torch.uint8, device=self.dev)
            grid, dt = self.density.render_view
            L.build_mask(grid, dt, self.gd, self.shift, rp.interval, rp.mask_thres, self.mask)
        # sampler
        sd = L.SamplerDesc()
        if rp.ndc:
            sd.mode, sd.step, sd.max_steps = 2, rp.step, rp.max_steps
            sd.ndc_fx, sd.ndc_fy, sd.ndc_near = rp.ndc_fx, rp.ndc_fy, rp.ndc_near
        elif rp.contracted:
            sd.mode, sd.near, sd.max_steps = 1, rp.near, rp.max_steps
            sd.contract_b, sd.p_inf, sd.step_c = rp.contract_b, int(rp.contract_p_inf), rp.step_c
        else:
            sd.mode, sd.near, sd.far, sd.step = 0, rp.near, rp.far, rp.step
            sd.step_offset, sd.use_slab, sd.max_steps = rp.step_offset, int(rp.use_slab), rp.max_steps
        self.sd = sd
        self.S_cap = self.R * rp.max_steps
        self._alloc_step_buffers()
        self.it = 0

    # ------------------------------------------------------------------ setup
    def _grid_param(self, dense: np.ndarray, C: int) -> GridParam:
        G = self.G
        n = L.grid_bricked_elems(G, C)
        d = torch.tensor(np.ascontiguousarray(dense, dtype=np.float32), device=self.dev)
        p = torch.empty(n, dtype=torch.float32, device=self.dev)
        L.grid_pack(d, p, G, C, L.F32)
        nb = L.grid_num_bricks(G)
        shadow = None
        if self.precision == L.BF16:
            shadow = torch.empty(n, dtype=torch.bfloat16, device=self.dev)
            L.grid_pack(d.to(torch.bfloat16), shadow, G, C, L.BF16)
        return GridParam(C, p, torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p),
                         torch.zeros(nb, dtype=torch.uint8, device=self.dev), shadow)

    def _alloc_step_buffers(self):
        S, R, dev = self.S_cap, self.R, self.dev
        f32 = dict(dtype=torch.float32, device=dev)
        i32 = dict(dtype=torch.int32, device=dev)
        self.ray_off = torch.zeros(R + 1, dtype=torch.int64, device=dev)
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
        self.live_idx = torch.empty(S, **i32)
        self.live_count = torch.zeros(1, dtype=torch.int64, device=dev)
        if self.w_min is not None:   # the colour-query list after the low-weight cull
            self.query_idx = torch.empty(S, **i32)
            self.query_count = torch.zeros(1, dtype=torch.int64, device=dev)
        else:
            self.query_idx, self.query_count = self.live_idx, self.live_count
        self.k0 = torch.empty(S, FEAT, **f32)
        self.rgb = torch.zeros(S, 3, **f32)
        self.color = torch.empty(R, 3, **f32)
        self.L_r = torch.empty(R, **f32)
        self.loss = torch.zeros(3, **f32)
        self.g_color = torch.empty(R, 3, **f32)
        self.g_raw = torch.empty(S, **f32)
        self.g_k0 = torch.zeros(S, FEAT, **f32)
        # FP32 forms: what the colour-MLP forward saves for its backward (hidden
        # activations, or the split layer inputs of each 128-sample tile)
        # (BF16 form: the backward's per-CTA partial gradients)
        if self.precision == L.F32:
            self.act = torch.empty(S, 256, **f32)
        else:
            self.act = torch.empty(L.rgbnet_act_bytes(S, self.precision), dtype=torch.uint8, device=dev)
        self.ws_sample = torch.empty(L.sample_rays_workspace_size(R), dtype=torch.uint8, device=dev)
        self.ws_live = torch.empty(L.live_samples_workspace_size(R), dtype=torch.uint8, device=dev)
        # zeroed once: the loss pass leaves its ticket counter at zero after every call
        self.ws_loss = torch.zeros(L.composite_loss_workspace_size(R), dtype=torch.uint8, device=dev)
        nb = self.density.touched.numel()
        self.brick_list = torch.empty(nb, **i32)
        self.brick_count = torch.zeros(1, **i32)
        self.step_dev = torch.zeros(2, dtype=torch.int64, device=dev)   # Adam's t (+ scratch)
        # per-sample alpha intervals of a given sample list (a proposal's picks,
        # each covering the span up to the next pick); None = the scalar interval
        self.delta = None
        self._delta = None

    # --------------------------------------------------------------- forward
    def sample(self, rays_o, rays_d):
        L.sample_rays(rays_o, rays_d, self.R, self.gd, self.sd, self.mask, self.S_cap, self.ray_off,
                      self.xyz, self.ray_id, self.step_k, self.s_mid, self.s_len, self.ws_sample)

    def forward(self, rays_o, rays_d, target, sample: bool = True, tail_adjoint: bool = False):
        """Forward pass.  sample=False renders the sample list already in the
        buffers (ray_off, xyz, ray_id, step_k, s_mid, s_len, and delta when it
        is set), e.g. the samples a proposal network selected.  tail_adjoint: the compositing adjoint of
        each ray (g_raw) runs in the same pass as its loss (then backward takes
        tail_done=True)."""
        rp, R, S = self.rp, self.R, self.S_cap
        if sample:
            self.sample(rays_o, rays_d)
        self._delta = None if sample else self.delta
        # density query and weights in one pass over each ray, up to its halt
        dgrid, ddt = self.density.render_view
        L.density_alpha_fwd(dgrid, ddt, self.gd, self.xyz, self.ray_off, R, self.shift, rp.interval,
                            rp.T_stop, self.raw, self.w, self.T, self.n_live, self.T_end,
                            delta=self._delta)
        L.live_samples(self.ray_off, self.n_live, R, self.live_idx, self.live_count, self.ws_live)
        if self.w_min is not None:
            L.live_samples_cull(self.ray_off, self.n_live, self.w, self.w_min, R, self.query_idx,
                                self.query_count, self.rgb, self.g_k0, self.ws_live)
        fgrid, fdt = self.feature.render_view
        L.sample_grid_fwd(fgrid, fdt, self.gd, FEAT, self.xyz, self.query_idx, S, self.query_count,
                          self.k0)
        L.rgbnet_fwd(self.k0, rays_d, self.ray_id, self.query_idx, S, self.query_count, self.mlp,
                     self.precision, self.rgb, self.act)
        # colour accumulation, distortion loss and the photometric loss in one pass
        # over each ray (with tail_adjoint, followed in the same warp by the ray's
        # compositing adjoint)
        if tail_adjoint:
            L.composite_distortion_loss_fwd_bwd(
                self.w, self.rgb, self.s_mid, self.s_len, self.ray_off, self.n_live, self.T_end, R,
                rp.bg, target, rp.lambda_dist, rp.lambda_dist / R, self.raw, self.T, self.shift,
                rp.interval, self.color, self.L_r, self.g_color, self.loss, self.g_raw, self.ws_loss,
                delta=self._delta)
        else:
            L.composite_distortion_loss_fwd(self.w, self.rgb, self.s_mid, self.s_len, self.ray_off,
                                            self.n_live, self.T_end, R, rp.bg, target,
                                            rp.lambda_dist, self.color, self.L_r, self.g_color,
                                            self.loss, self.ws_loss)

    # -------------------------------------------------------------- backward
    def backward(self, rays_d, tail_done: bool = False):
        rp, R, S = self.rp, self.R, self.S_cap
        # compositing adjoint with the distortion gradient formed inside its reverse scan
        if not tail_done:
            L.composite_distortion_bwd(self.g_color, rp.lambda_dist / R, self.w, self.raw, self.T,
                                       self.rgb, self.s_mid, self.s_len, self.ray_off, self.n_live,
                                       R, self.shift, rp.interval, rp.bg, self.g_raw,
                                       delta=self._delta)
        L.rgbnet_bwd(None, self.g_color, self.w, self.k0, rays_d, self.ray_id, self.query_idx, S,
                     self.query_count, self.mlp, self.precision, self.mlp_g, self.g_k0,
                     self.act, self.rgb)
        # both grid adjoints in one pass over the live samples
        L.sample_grid_bwd2(self.g_raw, 1, self.density.g, self.density.touched, self.g_k0, FEAT,
                           self.feature.g, self.feature.touched, self.gd, self.xyz, self.live_idx, S,
                           self.live_count)

    # ----------------------------------------------------------- optimizer
    def regularize_and_step(self, tv_dense: bool):
        rp = self.rp
        self.it += 1
        grids = ((self.density, rp.tv_w_density), (self.feature, rp.tv_w_feature))
        nb = self.density.touched.numel()
        # The trilinear adjoints flag the same bricks in both grids; their
        # compacted list drives the sparse TV and Adam (dense TV flags every
        # brick, so then the list is taken after it).
        if not tv_dense:
            L.touched_compact(self.density.touched, nb, self.brick_list, self.brick_count)
        # TV of both grids in one launch (they share the geometry), then one
        # Adam launch for both grids and the colour MLP
        tv = [(*gp.render_view, gp.C, tvw, gp.touched, gp.g) for gp, tvw in grids if tvw > 0]
        if tv:
            L.tv_add_grad_multi(tv, self.G, rp.tv_delta, tv_dense, self.brick_list, self.brick_count)
        if tv_dense:
            L.touched_compact(self.density.touched, nb, self.brick_list, self.brick_count)
        params = [(gp.p, gp.shadow, gp.g, gp.m, gp.v, gp.p.numel(), gp.touched, 512 * gp.C,
                   rp.lr_grid, self.brick_list, self.brick_count) for gp, _ in grids]
        params.append((self.mlp, None, self.mlp_g, self.mlp_m, self.mlp_v, self.mlp.numel(), None, 0,
                       rp.lr_mlp))
        # the step count t lives on the device (so that a captured step can be replayed)
        L.adam_step_multi_dev(params, rp.beta1, rp.beta2, rp.eps, self.step_dev, True)
        if self.mask_update and self.mask is not None:
            # the density changed only in the listed bricks
            dgrid, ddt = self.density.render_view
            L.update_mask(dgrid, ddt, self.gd, self.shift, rp.interval, rp.mask_thres, self.brick_list,
                          self.brick_count, self.mask)

    def step(self, rays_o, rays_d, target, tv_dense: bool = False, sample: bool = True):
        """One full training iteration; returns the device loss tensor [3]."""
        self.forward(rays_o, rays_d, target, sample=sample, tail_adjoint=True)
        self.backward(rays_d, tail_done=True)
        self.regularize_and_step(tv_dense)
        return self.loss

    def capture(self, rays_o, rays_d, target, tv_dense: bool = False):
        """Record one training step (sampling through the optimizer) as a CUDA
        graph over fixed device input buffers.  Returns (graph, inputs): copy a
        batch into inputs = (rays_o, rays_d, target), then graph.replay() runs
        one step (the Adam step count advances on the device).  Two eager
        warm-up steps on the given batch run first (they update the state)."""
        self.g_in = tuple(torch.empty_like(x) for x in (rays_o, rays_d, target))
        for dst, src in zip(self.g_in, (rays_o, rays_d, target)):
            dst.copy_(src)
        side = torch.cuda.Stream(device=self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            for _ in range(2):
                self.step(*self.g_in, tv_dense=tv_dense)
        torch.cuda.current_stream(self.dev).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.step(*self.g_in, tv_dense=tv_dense)
        return graph, self.g_in

    # ------------------------------------------------- progressive scaling
    def upscale(self, grid: int, moments: str = "resample"):
        """Progressive grid scaling (Sec. 5.4, grid-scaling schedule): both grids
        resampled to `grid` points per axis over the same box (trilinear,
        corner aligned), with the Adam moments m and v resampled the same way
        (moments="reset": zeroed instead).  Gradients and touched flags start
        empty, the renderer's BF16 copies are rebuilt, the sampler step is
        re-derived for the new voxel size (half a voxel) and the occupancy mask
        rebuilt from the new density.  The Adam step count carries on."""
        import dataclasses
        from . import synth
        G_old, G_new = self.G, [int(grid)] * 3
        for gp in (self.density, self.feature):
            n = L.grid_bricked_elems(G_new, gp.C)
            fresh = {}
            for name in ("p", "m", "v"):
                t = torch.empty(n, dtype=torch.float32, device=self.dev)
                if name == "p" or moments == "resample":
                    L.grid_resample(getattr(gp, name), G_old, t, L.F32, G_new, gp.C)
                else:
                    t.zero_()
                fresh[name] = t
            if gp.shadow is not None:
                gp.shadow = torch.empty(n, dtype=torch.bfloat16, device=self.dev)
                L.grid_resample(gp.p, G_old, gp.shadow, L.BF16, G_new, gp.C)
            gp.p, gp.m, gp.v = fresh["p"], fresh["m"], fresh["v"]
            gp.g = torch.zeros_like(gp.p)
            gp.touched = torch.zeros(L.grid_num_bricks(G_new), dtype=torch.uint8, device=self.dev)
        self.cfg = dataclasses.replace(self.cfg, grid=int(grid))
        fine = synth.render_params(self.cfg)
        self.rp = dataclasses.replace(self.rp, step=fine.step, max_steps=fine.max_steps, step_c=fine.step_c,
                                      interval=fine.interval)
        self.G = G_new
        self.gd = L.GridDesc.make(self.cfg.bbox_min, self.cfg.bbox_max, G_new)
        if self.rp.mask_thres is not None:
            self.mask = torch.empty(G_new[2], G_new[1], G_new[0], dtype=torch.uint8, device=self.dev)
            dgrid, dt = self.density.render_view
            L.build_mask(dgrid, dt, self.gd, self.shift, self.rp.interval, self.rp.mask_thres, self.mask)
        sd = self.sd
        if self.rp.contracted:
            sd.max_steps, sd.step_c = self.rp.max_steps, self.rp.step_c
        else:
            sd.step, sd.max_steps = self.rp.step, self.rp.max_steps
        self.S_cap = self.R * self.rp.max_steps
        step_dev = self.step_dev
        self._alloc_step_buffers()
        self.step_dev = step_dev

    # ------------------------------------------------------------- helpers
    def dense(self, gp: GridParam, which: str = "p") -> torch.Tensor:
        src = getattr(gp, which)
        out = torch.empty(self.G[2], self.G[1], self.G[0], gp.C, dtype=src.dtype, device=self.dev)
        L.grid_unpack(src, out, self.G, gp.C, L.BF16 if src.dtype == torch.bfloat16 else L.F32)
        return out


# ------------------------------------------------------ quality reference
TRUTH_DETAIL_STD = 1.6


def heldout_truth_render(cfg: SceneConfig, rp: RenderParams, density: np.ndarray,
                         feature: np.ndarray, mlp_params: np.ndarray, rays_o, rays_d, target,
                         detail_std: float = TRUTH_DETAIL_STD, seed: int = 0,
                         step_factor: int = 4) -> torch.Tensor:
    """Colours of a held-out truth scene on the given rays, the reference of
    the PSNR comparisons between forms of the step.  The truth holds what the
    model's grids cannot: both grids refined to the 2x lattice (2G-1 points
    per axis over the same box, corner aligned, so that the refined trilinear
    field is the model's own) plus i.i.d. Gaussian detail of std detail_std
    in raw density and in every feature channel.  It is rendered with a
    `step_factor` times finer step (the converged integral), its densities
    kept in the model's voxel units (the alpha interval scales with the
    step only), no occupancy mask, the same colour MLP."""
    from . import synth
    assert not rp.contracted and not rp.ndc, "bounded scenes only"
    G = synth.grid_dims(cfg)
    G2 = [2 * g - 1 for g in G]
    dev = rays_o.device
    grids = []
    for slot, (arr, C) in enumerate(((density, 1), (feature, feature.shape[-1]))):
        src = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).to(dev)
        packed = torch.empty(L.grid_bricked_elems(G, C), dtype=torch.float32, device=dev)
        L.grid_pack(src, packed, G, C, L.F32)
        fine = torch.empty(L.grid_bricked_elems(G2, C), dtype=torch.float32, device=dev)
        L.grid_resample(packed, G, fine, L.F32, G2, C)
        out = torch.empty(G2[2], G2[1], G2[0], C, dtype=torch.float32, device=dev)
        L.grid_unpack(fine, out, G2, C, L.F32)
        arr2 = out.cpu().numpy()
        arr2 += synth.truth_detail(arr2.shape, detail_std, seed=seed + slot)
        grids.append(arr2 if C > 1 else arr2[..., 0])
        del src, packed, fine, out
    cfg2 = dataclasses.replace(cfg, grid=G2[0], dims=tuple(G2) if cfg.dims is not None else None)
    rp2 = dataclasses.replace(rp, step=float(np.float32(rp.step / step_factor)),
                              max_steps=rp.max_steps * step_factor,
                              interval=float(np.float32(rp.interval / step_factor)),
                              mask_thres=None)
    R = int(rays_o.shape[0])
    tr = Trainer(cfg2, rp2, grids[0], grids[1], mlp_params, n_rays=R, precision="f32tc")
    tr.forward(rays_o, rays_d, target)
    color = tr.color.clone()
    del tr
    torch.cuda.empty_cache()
    return color
