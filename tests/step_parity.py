"""One training iteration on the GPU and the same iteration composed from
the FP64 oracle, on the same rays, and the relative error of every output
and gradient between the two (helper of the step parity tests and of the
benchmark's oracle leg).

Relative error of a tensor: max|x - ref| / max|ref| (conftest.rel_err).
Entries where the two precisions may legitimately take different discrete
decisions are compared separately and counted: samples whose smallest ReLU
input lies within rounding of 0 (|z| < tau), and, after the first Adam step
(which moves every entry by about lr * sign(g)), entries whose gradient is
at the rounding-noise level.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from conftest import rel_err
from oracle_step import forward_backward, optimizer, proposal_picks
from paper_2206_05085_gb300 import synth

MLP_TENSORS = ("W1", "b1", "W2", "b2", "W3", "b3")


def _host(t):
    torch.cuda.synchronize()
    return t.detach().float().cpu().numpy()


def gpu_step(cfg, rp, D, Fg, P, o, d, tgt, precision, tv_dense, w_min=None):
    """Forward, backward, TV and Adam of one batch through the library; the
    outputs and gradients before the optimizer and the parameters after it."""
    from paper_2206_05085_gb300 import train
    tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=len(o), precision=precision, w_min=w_min)
    to, td, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (o, d, tgt))
    tr.forward(to, td, tt)
    tr.backward(td)
    return _gpu_outputs(tr, tv_dense)


def _gpu_outputs(tr, tv_dense):
    S = int(_host(tr.ray_off)[-1])
    gpu = dict(loss=_host(tr.loss), color=_host(tr.color), L_r=_host(tr.L_r), n_live=_host(tr.n_live),
               S=S, ray_off=tr.ray_off.cpu().numpy(), w=_host(tr.w[:S]), rgb=_host(tr.rgb[:S]), g_raw=_host(tr.g_raw[:S]),
               g_k0=_host(tr.g_k0[:S]), g_mlp=_host(tr.mlp_g),
               g_density=_host(tr.dense(tr.density, "g"))[..., 0],
               g_feature=_host(tr.dense(tr.feature, "g")))
    tr.regularize_and_step(tv_dense)
    gpu.update(density=_host(tr.dense(tr.density, "p"))[..., 0], feature=_host(tr.dense(tr.feature, "p")),
               params=_host(tr.mlp))
    from paper_2206_05085_gb300 import _lib as L
    gpu["device_status"] = L.device_status()
    return gpu


def gpu_proposal_step(cfg, rp, D, Fg, P, PP, o, d, tgt, precision, tv_dense):
    """The learned-proposal form of one iteration through the library: the
    proposal (parameters PP) picks <= 64 of the <= 512 candidates per ray, the
    plain step runs on the picks with their spans.  Also returns the picks
    (sel [R][64], n_sel)."""
    import dataclasses
    from paper_2206_05085_gb300 import proposal, train
    R = len(o)
    rp_c = proposal.candidate_params(cfg, rp)
    tr = train.Trainer(cfg, dataclasses.replace(rp_c, max_steps=proposal.N_DRAW), D, Fg, P,
                       n_rays=R, precision=precision)
    grid, dt = tr.density.render_view
    prop = proposal.Proposal(cfg, rp, grid, dt, PP, R)
    to, td, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (o, d, tgt))
    prop.select_into(tr, to, td)
    tr.forward(to, td, tt, sample=False)
    tr.backward(td)
    sel = _host(prop.sel).astype(np.int64).reshape(R, proposal.N_DRAW)
    n_sel = _host(prop.n_sel).astype(np.int64)
    S = int(_host(tr.ray_off)[-1])
    delta = _host(tr.delta)[:S]
    gpu = _gpu_outputs(tr, tv_dense)
    gpu.update(sel=sel, n_sel=n_sel, delta=delta)
    return gpu


def oracle_proposal_step(cfg, rp, D, Fg, P, PP, o, d, tgt, precision, tv_dense):
    """The same from the oracle: its own picks (proposal network in FP64 on
    the BF16-stored proposal parameters), the spans, then the step.  Returns
    (fb, opt, params the renderer read, sel, n_sel)."""
    import dataclasses
    from paper_2206_05085_gb300 import proposal
    bf = precision == "bf16"
    Dr = synth.bf16_round(D) if bf else D
    Fr = synth.bf16_round(Fg) if bf else Fg
    Pr = synth.bf16_round(P) if bf else P
    rp_c = proposal.candidate_params(cfg, rp)
    picks, delta, sel, n_sel = proposal_picks(cfg, rp_c, synth.bf16_round(PP), o, d, proposal.N_DRAW)
    rp_p = dataclasses.replace(rp_c, max_steps=proposal.N_DRAW)
    fb = forward_backward(cfg, rp_p, Dr, Fr, Pr, o, d, tgt, smp=picks, delta=delta)
    fb["density0"], fb["feature0"], fb["params0"] = D, Fg, P
    fb["delta"] = delta
    opt = optimizer(rp_p, 1, D, Fg, P, fb, tv_dense, Dr, Fr)
    return fb, opt, Pr, sel, n_sel


def oracle_step(cfg, rp, D, Fg, P, o, d, tgt, precision, tv_dense, w_min=None):
    """The same iteration from the oracle.  The BF16 form's stored values
    (grids and MLP parameters) are the BF16-rounded ones; the Adam masters
    stay FP32.  Returns (fb, opt, params the renderer read)."""
    bf = precision == "bf16"
    Dr = synth.bf16_round(D) if bf else D
    Fr = synth.bf16_round(Fg) if bf else Fg
    Pr = synth.bf16_round(P) if bf else P
    fb = forward_backward(cfg, rp, Dr, Fr, Pr, o, d, tgt, w_min=w_min)
    fb["density0"], fb["feature0"], fb["params0"] = D, Fg, P
    opt = optimizer(rp, 1, D, Fg, P, fb, tv_dense, Dr, Fr)
    return fb, opt, Pr


def mlp_grad_errors(dims, params, x, g_out, gpu_gp, tau, out_sigmoid=True, names=MLP_TENSORS):
    """Per weight / bias tensor of an MLP: the relative error of the parameter
    gradient, and the same with the share of samples whose smallest ReLU
    input lies within tau of 0 set aside (each such sample may switch a unit
    in one precision and not the other; twice its own gradient is allowed).
    Returns (errors, errors_beyond_ambiguous, number of such samples)."""
    zmin = oracle.mlp_min_abs_preact(dims, params, x)
    amb = np.nonzero(zmin < tau)[0]
    gp, _ = oracle.mlp_bwd(dims, params, x, g_out, out_sigmoid)
    slack = np.zeros_like(gp)
    for s in amb:
        gps, _ = oracle.mlp_bwd(dims, params, x[s:s + 1], g_out[s:s + 1], out_sigmoid)
        slack += 2 * np.abs(gps)
    offs = [0]
    for i in range(len(dims) - 1):
        offs += [offs[-1] + dims[i + 1] * dims[i], offs[-1] + dims[i + 1] * dims[i] + dims[i + 1]]
    raw, adj = {}, {}
    for nm, a, b in zip(names, offs[:-1], offs[1:]):
        err = np.abs(np.asarray(gpu_gp[a:b], np.float64) - gp[a:b])
        scale = max(float(np.max(np.abs(gp[a:b]))), 1e-30)
        raw[nm] = float(np.max(err) / scale)
        adj[nm] = float(np.max(np.maximum(err - slack[a:b], 0.0)) / scale)
    return raw, adj, int(len(amb))


def cell_voxels(cfg, xyz):
    """Dense indices (z, y, x) of the 8 corners of each point's trilinear cell."""
    G = np.array(synth.grid_dims(cfg))
    u = (xyz.astype(np.float64) - cfg.bbox_min) / (cfg.bbox_max - cfg.bbox_min) * (G - 1)
    i0 = np.clip(np.floor(np.clip(u, 0, G - 1)).astype(int), 0, G - 2)
    out = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                out.append(np.stack([i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx], 1))
    return np.concatenate(out, 0)


def error_table(gpu, fb, opt, cfg, rp, params, tau):
    """Relative error of every output and gradient of the step (and of the
    parameters after the optimizer) against the oracle.  Returns a dict:
    per-tensor errors, plus the counts of the entries compared separately."""
    e = {"samples": int(gpu["S"]), "halting_index_mismatches": int(np.sum(gpu["n_live"] != fb["n_live"]))}
    same_list = gpu["S"] == fb["smp"].S
    e["sample_list_equal"] = bool(same_list)
    e["color"] = rel_err(gpu["color"], fb["color"])
    e["loss"] = rel_err(gpu["loss"], fb["loss"])
    e["L_r"] = rel_err(gpu["L_r"], fb["L_r"])
    live = fb["query"]       # the samples that reached the colour MLP
    zmin = oracle.mlp_min_abs_preact(synth.RGBNET_DIMS, params.astype(np.float64), fb["x"])
    amb = zmin < tau
    e["relu_ambiguous_samples"] = int(amb.sum())
    e["live_samples"] = int(fb["live"].sum())
    e["colour_query_samples"] = int(live.sum())
    if same_list:
        e["w"] = rel_err(gpu["w"], fb["w"])
        e["rgb"] = rel_err(gpu["rgb"][live], fb["rgb"][live])
        e["g_raw"] = rel_err(gpu["g_raw"], fb["g_raw"])
        e["g_k0"] = rel_err(gpu["g_k0"][live][~amb], fb["g_k0"][~amb])
    raw, adj, _ = mlp_grad_errors(synth.RGBNET_DIMS, params.astype(np.float64), fb["x"],
                                  fb["g_rgb"][live], gpu["g_mlp"], tau)
    for nm in MLP_TENSORS:
        e["g_mlp_" + nm] = adj[nm]           # ambiguous samples' share set aside
        e["g_mlp_" + nm + "_raw"] = raw[nm]
    e["g_density"] = rel_err(gpu["g_density"], fb["g_density"])
    gf = gpu["g_feature"]
    rf = fb["g_feature"].reshape(gf.shape)
    keep = np.ones(gf.shape[:3], bool)
    if amb.any():
        v = cell_voxels(cfg, fb["smp"].xyz[live][amb])
        keep[v[:, 0], v[:, 1], v[:, 2]] = False
    touched = np.abs(rf).sum(-1) > 0
    e["g_feature"] = float(np.max(np.abs(gf - rf)[keep]) / max(np.max(np.abs(rf)), 1e-30))
    e["g_feature_voxels_set_aside"] = int((~keep & touched).sum())
    e["g_feature_voxels_touched"] = int(touched.sum())
    for name, gname in (("density", "g_density_tv"), ("feature", "g_feature_tv"), ("params", None)):
        ref = opt[name].reshape(gpu[name].shape)
        g_ref = (opt[gname] if gname else fb["g_params"]).reshape(gpu[name].shape)
        clear = np.abs(g_ref) > 1e-3 * np.max(np.abs(g_ref))
        if name == "feature":
            clear &= np.broadcast_to(keep[..., None], clear.shape)
        e["adam_" + name] = float(np.max(np.abs(gpu[name] - ref)[clear]) / np.max(np.abs(ref)))
        start = {"density": fb["density0"], "feature": fb["feature0"], "params": fb["params0"]}[name]
        e["adam_" + name + "_max_step"] = float(np.max(np.abs(gpu[name] - start.reshape(gpu[name].shape))))
    return e
