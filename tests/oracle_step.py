"""A full training iteration composed from the FP64 oracle (test helper).

Follows the same order as the paper's training loop (Sec. 2 listing) and
rendering utilities (Sec. 3); every piece is an oracle function.  Only
``oracle`` and the seeded generators are used here.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2206_05085_gb300 import synth


def shift32(alpha_init):
    return float(np.float32(oracle.alpha_shift(alpha_init)))


def sample(cfg, rp, o, d, mask):
    if rp.ndc:
        return oracle.sample_rays_ndc(o, d, cfg.bbox_min, cfg.bbox_max, synth.grid_dims(cfg), rp.ndc_fx,
                                      rp.ndc_fy, rp.ndc_near, rp.step, rp.max_steps, mask)
    if rp.contracted:
        return oracle.sample_rays_contracted(o, d, rp.contract_b, rp.contract_p_inf, rp.near,
                                             rp.step_c, rp.max_steps, cfg.bbox_min, cfg.bbox_max,
                                             synth.grid_dims(cfg), mask)
    return oracle.sample_rays_bbox(o, d, cfg.bbox_min, cfg.bbox_max, synth.grid_dims(cfg), rp.near, rp.far,
                                   rp.step, rp.step_offset, rp.use_slab, rp.max_steps, mask)


def live_of(ray_off, n_live):
    """Boolean [S]: sample is before its ray's halting index."""
    S = int(ray_off[-1])
    live = np.zeros(S, bool)
    for r in range(len(n_live)):
        live[ray_off[r]:ray_off[r] + n_live[r]] = True
    return live


def forward_backward(cfg, rp, density, feature, params, o, d, target, grads=True, w_min=None,
                     smp=None, delta=None):
    """density [G,G,G] f32, feature [G,G,G,12] f32, params flat f32 (the values
    the renderer reads: BF16-rounded already for the BF16 form).  w_min: the
    low-weight cull -- samples in front of the halt whose compositing weight
    is below w_min get no colour query (their colour is 0, their features no
    gradient); out["query"] marks the queried samples.  smp: a given sample
    list (e.g. a proposal's picks) in place of the sampler's, with delta its
    per-sample alpha intervals (None: rp.interval for every sample)."""
    lo, hi = cfg.bbox_min, cfg.bbox_max
    sh = shift32(rp.alpha_init)
    mask = None
    if smp is None:
        if rp.mask_thres is not None:
            mask = oracle.build_mask(density, sh, rp.interval, rp.mask_thres)
        smp = sample(cfg, rp, o, d, mask)
    R = o.shape[0]
    raw = oracle.trilinear(density, lo, hi, smp.xyz)[:, 0]
    c0 = oracle.composite(raw, None, smp.ray_off, sh, rp.interval, rp.T_stop, rp.bg, delta=delta)
    live = live_of(smp.ray_off, c0["n_live"])
    query = live & (c0["w"] >= w_min) if w_min is not None else live
    k0 = oracle.trilinear(feature, lo, hi, smp.xyz[query])
    x = oracle.rgbnet_input(k0, d[smp.ray_id[query]])
    p64 = params.astype(np.float64)
    rgb_q = oracle.mlp_fwd(synth.RGBNET_DIMS, p64, x, True)
    rgb = np.zeros((smp.S, 3))
    rgb[query] = rgb_q
    comp = oracle.composite(raw, rgb, smp.ray_off, sh, rp.interval, rp.T_stop, rp.bg, delta=delta)
    L_r = oracle.distortion(comp["w"], smp.s_mid, smp.s_len, smp.ray_off, comp["n_live"])
    tgt = target.astype(np.float64)
    loss_rgb = np.mean((comp["color"] - tgt) ** 2)
    loss_dist = np.mean(L_r)
    out = dict(mask=mask, smp=smp, raw=raw, live=live, query=query, k0=k0, rgb=rgb, L_r=L_r, x=x,
               loss=np.array([loss_rgb, loss_dist, loss_rgb + rp.lambda_dist * loss_dist]), **comp)
    if not grads:
        return out
    g_color = 2.0 * (comp["color"] - tgt) / (3 * R)
    g_w = oracle.distortion_grad(rp.lambda_dist / R, comp["w"], smp.s_mid, smp.s_len, smp.ray_off,
                                 comp["n_live"])
    g_raw, g_rgb = oracle.composite_bwd(raw, rgb, smp.ray_off, sh, rp.interval, rp.T_stop, rp.bg,
                                        g_color, g_w, delta=delta)
    g_params, g_x = oracle.mlp_bwd(synth.RGBNET_DIMS, p64, x, g_rgb[query], True)
    g_density = oracle.trilinear_adjoint(g_raw[live], density.shape, lo, hi, smp.xyz[live])
    g_feature = oracle.trilinear_adjoint(g_x[:, :12], feature.shape, lo, hi, smp.xyz[query])
    out.update(g_color=g_color, g_w=g_w, g_raw=g_raw, g_rgb=g_rgb, g_params=g_params,
               g_k0=g_x[:, :12], g_density=g_density, g_feature=g_feature)
    return out


def proposal_picks(cfg, rp_c, prop_params, o, d, n_draw=64):
    """The learned proposal's sample list: the candidates (the bbox sampler
    with the candidate step, no mask), the network's per-ray softmax over
    them (FP64 MLP on the parameters' stored values), inverse-CDF picks at
    u_k = (k + 0.5)/n_draw over the FP32 CDF (duplicates collapsed), and the
    picked samples, each standing for the candidates from itself up to the
    next pick (the last: up to the ray's last candidate): its interval
    delta = interval * gap, its distortion span from its own start to the
    next pick's start.  Returns (picks Samples, delta [S], sel, n_sel)."""
    cand = sample(cfg, rp_c, o, d, None)
    x = oracle.freq_encode(cand.xyz, 6)
    logits = oracle.mlp_fwd(synth.PROPOSAL_DIMS, prop_params.astype(np.float64), x, False)[:, 0]
    _, _, q = oracle.proposal_xent_ragged(logits, np.zeros(cand.S), cand.ray_off, 0.0)
    sel, n_sel = oracle.inverse_cdf_select_ragged(q.astype(np.float32), cand.ray_off, n_draw)
    R = len(n_sel)
    src, delta, mid, length = [], [], [], []
    for r in range(R):
        b = int(cand.ray_off[r])
        n_c = int(cand.ray_off[r + 1]) - b
        picks = [int(j) for j in sel[r, :n_sel[r]]]
        for i, j in enumerate(picks):
            nxt = picks[i + 1] if i + 1 < len(picks) else n_c
            start = cand.s_mid[b + j] - 0.5 * cand.s_len[b + j]
            if nxt < n_c:
                end = cand.s_mid[b + nxt] - 0.5 * cand.s_len[b + nxt]
            else:
                end = cand.s_mid[b + n_c - 1] + 0.5 * cand.s_len[b + n_c - 1]
            src.append(b + j)
            delta.append(rp_c.interval * (nxt - j))
            mid.append(0.5 * (start + end))
            length.append(end - start)
    src = np.array(src, np.int64)
    ray_off = np.concatenate([[0], np.cumsum(n_sel)]).astype(np.int64)
    picks = oracle.Samples(ray_off, cand.xyz[src], cand.ray_id[src], cand.step_k[src],
                           np.array(mid), np.array(length))
    return picks, np.array(delta), sel, n_sel


def optimizer(rp, it, density_master, feature_master, params_master, fb, tv_dense,
              density_render, feature_render):
    """TV add-grad + Adam from zero moments (step `it`).  Returns updated
    masters and the gradients after TV."""
    gd = oracle.tv_add_grad(density_render, fb["g_density"], rp.tv_w_density, rp.tv_delta,
                            tv_dense) if rp.tv_w_density > 0 else fb["g_density"]
    gf = oracle.tv_add_grad(feature_render, fb["g_feature"], rp.tv_w_feature, rp.tv_delta,
                            tv_dense) if rp.tv_w_feature > 0 else fb["g_feature"]
    z = np.zeros
    pd, _, _ = oracle.adam(density_master, gd, z(gd.shape), z(gd.shape), rp.lr_grid, rp.beta1,
                           rp.beta2, rp.eps, it)
    pf, _, _ = oracle.adam(feature_master, gf, z(gf.shape), z(gf.shape), rp.lr_grid, rp.beta1,
                           rp.beta2, rp.eps, it)
    gp = fb["g_params"]
    pp, _, _ = oracle.adam(params_master, gp, z(gp.shape), z(gp.shape), rp.lr_mlp, rp.beta1,
                           rp.beta2, rp.eps, it)
    return dict(density=pd, feature=pf, params=pp, g_density_tv=gd, g_feature_tv=gf)
