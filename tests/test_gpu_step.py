"""GPU parity of a whole training iteration (forward, backward, TV, Adam)
against the same iteration composed from the FP64 oracle, on the seeded
synthetic workloads."""
import dataclasses

import numpy as np
import pytest
import torch

from conftest import rel_err
from paper_2206_05085_gb300 import synth
from step_parity import (error_table, gpu_proposal_step, gpu_step, oracle_proposal_step,
                         oracle_step)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2206_05085_gb300 import build
    build.build()
    from paper_2206_05085_gb300 import train
    return train


def host(t):
    torch.cuda.synchronize()
    return t.detach().float().cpu().numpy()


def _run(T, cfg, n_rays, precision, tv_dense, ray_stride=1):
    rp = synth.render_params(cfg)
    D = synth.density_grid(cfg)
    Fg = synth.feature_grid(cfg)
    P = synth.mlp_params()
    o, d = synth.rays(cfg)
    tgt = synth.target_rgb(cfg)
    o, d, tgt = o[::ray_stride][:n_rays], d[::ray_stride][:n_rays], tgt[::ray_stride][:n_rays]
    gpu = gpu_step(cfg, rp, D, Fg, P, o, d, tgt, precision, tv_dense)
    fb, opt, Pr = oracle_step(cfg, rp, D, Fg, P, o, d, tgt, precision, tv_dense)
    return gpu, fb, opt, cfg, rp, Pr


def _compare(gpu, fb, opt, tol, cfg, rp, params, bf16=False):
    import oracle
    assert gpu["S"] == fb["smp"].S
    assert gpu["device_status"] == 0
    bad = np.nonzero(gpu["n_live"] != fb["n_live"])[0]
    assert len(bad) == 0, f"halting index differs on rays {bad[:10]}"
    # ReLU inputs within rounding of 0 (tau: the operand precision's reach)
    tau = 1e-5 if bf16 else 1e-6
    e = error_table(gpu, fb, opt, cfg, rp, params, tau)
    for k in ("color", "loss", "L_r", "w", "rgb", "g_raw", "g_k0", "g_density", "g_feature",
              "adam_density", "adam_feature", "adam_params"):
        assert e[k] < tol, (k, e[k])
    from conftest import check_mlp_grads
    check_mlp_grads(oracle, synth.RGBNET_DIMS, params.astype(np.float64), fb["x"],
                    fb["g_rgb"][fb["query"]], gpu["g_mlp"], None, tol, tau=tau)
    # voxels of samples with an ambiguous ReLU unit are few
    assert e["g_feature_voxels_set_aside"] <= 0.05 * e["g_feature_voxels_touched"] + 8
    # elsewhere the first Adam step is bounded by the learning rate
    for name, lr in (("density", rp.lr_grid), ("feature", rp.lr_grid), ("params", rp.lr_mlp)):
        assert e["adam_" + name + "_max_step"] <= lr * (1 + 1e-3) + 1e-6


def test_step_small_fp32(T):
    gpu, fb, opt, cfg, rp, P = _run(T, synth.CFG1, 512, "f32", tv_dense=False, ray_stride=4)
    assert fb["live"].sum() > 10000
    _compare(gpu, fb, opt, 1e-5, cfg, rp, P)


def test_step_dvgo160_fp32_sparse_tv(T):
    gpu, fb, opt, cfg, rp, P = _run(T, synth.CFG2, 1024, "f32", tv_dense=False, ray_stride=8)
    assert (fb["n_live"] < np.diff(fb["smp"].ray_off)).sum() > 50   # early stop is exercised
    _compare(gpu, fb, opt, 1e-5, cfg, rp, P)


@pytest.mark.parametrize("cfg_name", ["small_64", "dvgo_160"])
def test_step_fp32_tensor_core_mlp(T, cfg_name):
    # the colour MLP on the tensor cores with split-FP16 operands: same FP32 bar
    cfg = synth.CONFIGS[cfg_name]
    gpu, fb, opt, cfg, rp, P = _run(T, cfg, 1024, "f32tc", tv_dense=False, ray_stride=8)
    _compare(gpu, fb, opt, 1e-5, cfg, rp, P)


@pytest.mark.parametrize("precision,tv_dense,tol", [("f32tc", False, 1e-5), ("f32", True, 1e-5)])
def test_step_ragged_grid(T, precision, tv_dense, tol):
    """A grid whose sides are no multiple of the 8-voxel brick (61 x 47 x 53
    points): padded bricks in the queries, the adjoints, the touched list,
    TV and Adam, and a non-cubic occupancy mask, against the oracle."""
    cfg = dataclasses.replace(synth.CFG1, name="small_ragged", grid=61, dims=(61, 47, 53))
    gpu, fb, opt, cfg, rp, P = _run(T, cfg, 1024, precision, tv_dense=tv_dense, ray_stride=2)
    assert fb["live"].sum() > 5000
    _compare(gpu, fb, opt, tol, cfg, rp, P)


def test_step_empty_sample_list(T):
    """Degenerate batch: a density so low that the occupancy mask is empty and
    no ray has a sample.  The colour is the background and the loss the
    oracle's, every gradient is zero and the optimizer leaves every parameter
    as it was."""
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    assert rp.mask_thres is not None
    D = np.full(synth.density_grid(cfg).shape, -100.0, np.float32)
    Fg, P = synth.feature_grid(cfg), synth.mlp_params()
    o, d = synth.rays(cfg)
    tgt = synth.target_rgb(cfg)
    o, d, tgt = o[:256], d[:256], tgt[:256]
    gpu = gpu_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False)
    fb, opt, _ = oracle_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False)
    assert gpu["S"] == 0 == fb["smp"].S
    assert gpu["device_status"] == 0
    assert np.all(gpu["n_live"] == 0)
    assert rel_err(gpu["color"], fb["color"]) < 1e-6
    assert rel_err(gpu["loss"], fb["loss"]) < 1e-6
    assert not np.any(gpu["g_mlp"]) and not np.any(gpu["g_density"]) and not np.any(gpu["g_feature"])
    assert np.array_equal(gpu["density"], D) and np.array_equal(gpu["feature"], Fg)
    assert np.array_equal(gpu["params"], P)


def test_step_opaque_scene(T):
    """Degenerate batch: a density so high that every ray halts after its
    first sample (alpha = 1 in FP32), so that the live list holds one sample
    per non-empty ray: the whole step against the oracle."""
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    D = np.full(synth.density_grid(cfg).shape, 50.0, np.float32)
    Fg, P = synth.feature_grid(cfg), synth.mlp_params()
    o, d = synth.rays(cfg)
    tgt = synth.target_rgb(cfg)
    o, d, tgt = o[::16][:512], d[::16][:512], tgt[::16][:512]
    gpu = gpu_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False)
    fb, opt, Pr = oracle_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False)
    counts = np.diff(fb["smp"].ray_off)
    assert np.array_equal(fb["n_live"], np.minimum(counts, 1)) and counts.max() > 10
    _compare(gpu, fb, opt, 1e-5, cfg, rp, Pr)


def test_step_dvgo160_fp32_dense_tv(T):
    gpu, fb, opt, cfg, rp, P = _run(T, synth.CFG2, 256, "f32", tv_dense=True, ray_stride=32)
    _compare(gpu, fb, opt, 1e-5, cfg, rp, P)


def test_step_dvgo160_bf16(T):
    gpu, fb, opt, cfg, rp, P = _run(T, synth.CFG4, 1024, "bf16", tv_dense=False, ray_stride=16)
    _compare(gpu, fb, opt, 2e-3, cfg, rp, P, bf16=True)


def test_step_low_weight_cull(T):
    """The colour query skips samples whose compositing weight is below 1e-4:
    the step equals the oracle's step with the same cull (colour 0 and no
    feature gradient for the skipped samples, density gradient for all), and
    the render stays close to the uncull render."""
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    o, d = synth.rays(cfg)
    tgt = synth.target_rgb(cfg)
    o, d, tgt = o[::8][:1024], d[::8][:1024], tgt[::8][:1024]
    gpu = gpu_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False, w_min=1e-4)
    fb, opt, Pr = oracle_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False, w_min=1e-4)
    skipped = fb["live"] & ~fb["query"]
    assert skipped.sum() > 0.05 * fb["live"].sum()     # the cull does something here
    # no weight sits so close to the threshold that FP32 and FP64 could disagree
    w = fb["w"][fb["live"]]
    assert np.min(np.abs(w - 1e-4)) > 1e-5 * 1e-4
    _compare(gpu, fb, opt, 1e-5, cfg, rp, Pr)
    full = oracle_step(cfg, rp, D, Fg, P, o, d, tgt, "f32tc", False)[0]
    mse = np.mean((gpu["color"].astype(np.float64) - full["color"]) ** 2)
    psnr = -10 * np.log10(mse)
    print(f"low-weight cull: {int(skipped.sum())} of {int(fb['live'].sum())} live samples skipped, "
          f"render vs full render {psnr:.1f} dB")
    assert psnr > 50


@pytest.mark.parametrize("precision,tol", [("f32tc", 1e-5), ("bf16", 2e-3)])
def test_step_learned_proposal(T, precision, tol):
    """The learned-proposal form: the proposal network picks <= 64 of the
    <= 512 candidates of each ray and the step runs on the picks, each with
    the span up to the next pick.  The picks equal the oracle's (its FP64
    network on the same stored parameters) except on rays where a CDF value
    sits within the network's rounding of a quantile; on the rays whose
    picks agree, the spans and the whole step match the oracle's."""
    import dataclasses as dc
    from paper_2206_05085_gb300 import proposal
    cfg = synth.CFG5 if precision == "f32tc" else synth.CFG4
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    PP = (synth.proposal_params() * 3.0).astype(np.float32)
    o, d = synth.rays(cfg)
    tgt = synth.target_rgb(cfg)
    o, d, tgt = o[::16][:384], d[::16][:384], tgt[::16][:384]
    args = (cfg, rp, D, Fg, P, PP)
    gpu = gpu_proposal_step(*args, o, d, tgt, precision, False)
    fb, opt, Pr, sel, n_sel = oracle_proposal_step(*args, o, d, tgt, precision, False)
    R = len(o)
    agree = np.array([n_sel[r] == gpu["n_sel"][r] and
                      np.array_equal(sel[r, :n_sel[r]], gpu["sel"][r, :n_sel[r]]) for r in range(R)])
    print(f"picks equal on {int(agree.sum())} of {R} rays; {int(n_sel.sum())} picks")
    assert agree.mean() > 0.9
    if not agree.all():
        o, d, tgt = o[agree], d[agree], tgt[agree]
        gpu = gpu_proposal_step(*args, o, d, tgt, precision, False)
        fb, opt, Pr, sel, n_sel = oracle_proposal_step(*args, o, d, tgt, precision, False)
        assert np.array_equal(gpu["n_sel"], n_sel)
    assert np.array_equal(gpu["sel"], np.where(sel >= 0, sel, gpu["sel"]))
    assert n_sel.mean() > 20 and (n_sel < 64).any()        # spans longer than one candidate
    assert rel_err(gpu["delta"], fb["delta"]) < 1e-6
    assert np.max(fb["delta"]) > 4 * np.min(fb["delta"])
    rp_p = dc.replace(proposal.candidate_params(cfg, rp), max_steps=proposal.N_DRAW)
    _compare(gpu, fb, opt, tol, cfg, rp_p, Pr, bf16=precision == "bf16")


def test_full_size_learned_proposal(T):
    """The learned-proposal form at the benchmark's size (16384 rays of the
    dvgo_160 scene, <= 512 candidates per ray): for 48 sampled rays the picks
    equal the oracle's (except where a CDF value sits within the network's
    rounding of a quantile), and on the rays whose picks agree the spans,
    the colour and loss terms, and the per-sample weights, colours and raw
    gradients (rescaled from 1/48 to the batch's 1/R) match the oracle's."""
    cfg = synth.CFG5
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    PP = (synth.proposal_params() * 3.0).astype(np.float32)
    o, d = synth.rays(cfg)
    tgt = synth.target_rgb(cfg)
    R = len(o)
    args = (cfg, rp, D, Fg, P, PP)
    gpu = gpu_proposal_step(*args, o, d, tgt, "f32tc", False)
    rays = np.sort(np.random.default_rng(9).choice(R, 48, replace=False))
    fb, _, _, sel, n_sel = oracle_proposal_step(*args, o[rays], d[rays], tgt[rays], "f32tc", False)
    agree = np.array([n_sel[i] == gpu["n_sel"][r] and
                      np.array_equal(sel[i, :n_sel[i]], gpu["sel"][r, :n_sel[i]])
                      for i, r in enumerate(rays)])
    assert agree.mean() > 0.9 and n_sel.mean() > 20
    scale = len(rays) / R
    off_g, off_o = gpu["ray_off"], fb["smp"].ray_off
    g_rows, o_rows = [], []
    for i in np.nonzero(agree)[0]:
        r = rays[i]
        assert off_g[r + 1] - off_g[r] == off_o[i + 1] - off_o[i]
        assert gpu["n_live"][r] == fb["n_live"][i]
        g_rows.append(np.arange(off_g[r], off_g[r + 1]))
        o_rows.append(np.arange(off_o[i], off_o[i + 1]))
    g_rows, o_rows = np.concatenate(g_rows), np.concatenate(o_rows)
    live = fb["live"][o_rows]
    assert live.sum() > 500
    assert rel_err(gpu["delta"][g_rows], fb["delta"][o_rows]) < 1e-6
    assert rel_err(gpu["w"][g_rows], fb["w"][o_rows]) < 1e-5
    assert rel_err(gpu["rgb"][g_rows][live], fb["rgb"][o_rows][live]) < 1e-5
    assert rel_err(gpu["g_raw"][g_rows][live], fb["g_raw"][o_rows][live] * scale) < 1e-5
    a = rays[agree]
    assert rel_err(gpu["color"][a], fb["color"][agree]) < 1e-5
    assert rel_err(gpu["L_r"][a], fb["L_r"][agree]) < 1e-5


def test_step_forward_facing_ndc(T):
    """Forward-facing capture: NDC warp and depth-layer sampling (96 x 96 x 64
    layers standing in for 384^2 x 256), the full step against the oracle."""
    cfg = dataclasses.replace(synth.CFG6, grid=96, dims=(96, 96, 64))
    gpu, fb, opt, cfg, rp, P = _run(T, cfg, 512, "f32tc", tv_dense=False, ray_stride=8)
    assert fb["live"].sum() > 5000
    _compare(gpu, fb, opt, 1e-5, cfg, rp, P)


def test_step_unbounded_contracted(T):
    # the 320^3 grids of the workload are exercised by the benchmark; a 96^3
    # grid keeps the FP64 oracle's TV/Adam pass small here
    cfg = dataclasses.replace(synth.CFG3, grid=96)
    gpu, fb, opt, cfg, rp, P = _run(T, cfg, 256, "f32", tv_dense=False, ray_stride=32)
    _compare(gpu, fb, opt, 1e-5, cfg, rp, P)


def test_captured_step_replays_like_eager(T):
    """A training step captured as a CUDA graph and replayed on new batches
    leaves the same state as the same steps launched one by one."""
    cfg = synth.CFG1
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    batches = []
    for seed in (1, 2, 3):
        o, d = synth.rays(cfg, seed=seed, n_rays=1024)
        t = synth.target_rgb(cfg, seed=seed, n_rays=1024)
        batches.append(tuple(torch.from_numpy(a).cuda() for a in (o, d, t)))
    eager = T.Trainer(cfg, rp, D, Fg, P, n_rays=1024, precision="f32tc")
    for b in (batches[0], batches[0], batches[1], batches[2]):
        eager.step(*b)
    graphed = T.Trainer(cfg, rp, D, Fg, P, n_rays=1024, precision="f32tc")
    graph, inputs = graphed.capture(*batches[0])       # two eager steps on batch 0
    for b in batches[1:]:
        for dst, src in zip(inputs, b):
            dst.copy_(src)
        graph.replay()
    torch.cuda.synchronize()
    assert int(graphed.step_dev[0].item()) == 4 == int(eager.step_dev[0].item())
    # the grid adjoints sum with atomics, so the two runs differ only by that
    # summation order: the loss and the MLP to FP32 rounding; grid entries by
    # far less than one Adam step (lr = 0.1), except the very few whose tiny
    # gradient (a near-cancelling sum) changes sign with the order - Adam
    # moves those by up to lr either way
    for a, b in ((eager.loss, graphed.loss), (eager.mlp, graphed.mlp)):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-5 * max(np.max(np.abs(a)), 1e-30)
    for a, b in ((eager.density.p, graphed.density.p), (eager.feature.p, graphed.feature.p)):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        d = np.abs(a - b)
        assert np.mean(d > 1e-3 * rp.lr_grid) < 1e-4
        assert np.max(d) <= 2 * rp.lr_grid


def test_full_size_step_sampled_outputs(T):
    """The benchmark's own configuration - dvgo_160 at 8192 rays, the FP32 form
    with the colour MLP on the tensor cores, one replay of the captured step -
    checked where the oracle can follow it: the whole sample list (bit-exact
    against the oracle's sampler), the per-ray and per-sample outputs of 48
    sampled rays (oracle run on those rays, gradients rescaled to the batch's
    1/R), the grids after the step's TV + Adam on the voxels only those rays
    reach, and the loss as the mean of the per-ray terms."""
    import oracle
    from oracle_step import forward_backward, sample, shift32
    from paper_2206_05085_gb300 import _lib as L
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    o, d = synth.rays(cfg, seed=0)
    tgt = synth.target_rgb(cfg, seed=0)
    R = cfg.n_rays
    tr = T.Trainer(cfg, rp, D, Fg, P, n_rays=R, precision="f32tc")
    to, td, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (o, d, tgt))
    graph, _ = tr.capture(to, td, tt)        # its two eager warm-up steps change the state
    for gp, dense, C in ((tr.density, D, 1), (tr.feature, Fg, 12)):
        L.grid_pack(torch.from_numpy(np.ascontiguousarray(dense, np.float32)).cuda(), gp.p, tr.G, C, L.F32)
        gp.m.zero_()
        gp.v.zero_()
    tr.mlp.copy_(torch.from_numpy(P).cuda())
    tr.mlp_m.zero_()
    tr.mlp_v.zero_()
    tr.step_dev.zero_()
    graph.replay()
    ray_off = host(tr.ray_off)
    S = int(ray_off[-1])
    n_live = host(tr.n_live)
    color, L_r, loss = host(tr.color), host(tr.L_r), host(tr.loss)
    w, rgb, g_raw, g_k0, xyz = (host(x[:S]) for x in (tr.w, tr.rgb, tr.g_raw, tr.g_k0, tr.xyz))
    ray_id = tr.ray_id[:S].cpu().numpy()
    p_d = host(tr.dense(tr.density, "p"))[..., 0]
    p_f = host(tr.dense(tr.feature, "p"))
    # the whole sample list
    mask = oracle.build_mask(D, shift32(rp.alpha_init), rp.interval, rp.mask_thres)
    smp = sample(cfg, rp, o, d, mask)
    assert np.array_equal(ray_off, smp.ray_off)
    assert np.array_equal(xyz, smp.xyz)
    # the loss from the per-ray terms (FP64 on the host)
    mse = np.mean((color.astype(np.float64) - tgt) ** 2)
    ld = np.mean(L_r.astype(np.float64))
    assert rel_err(loss, np.array([mse, ld, mse + rp.lambda_dist * ld])) < 1e-5
    # 48 sampled rays against the oracle on those rays alone
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(R, 48, replace=False))
    fb = forward_backward(cfg, rp, D, Fg, P, o[sel], d[sel], tgt[sel])
    assert np.array_equal(n_live[sel], fb["n_live"])
    assert rel_err(color[sel], fb["color"]) < 1e-5
    assert rel_err(L_r[sel], fb["L_r"]) < 1e-5
    rows = np.concatenate([np.arange(ray_off[r], ray_off[r + 1]) for r in sel]).astype(np.int64)
    live = fb["live"]
    scale = len(sel) / R                     # the oracle's gradients carry 1/48, the batch's 1/8192
    assert rel_err(w[rows], fb["w"]) < 1e-5
    assert rel_err(rgb[rows][live], fb["rgb"][live]) < 1e-5
    assert rel_err(g_raw[rows][live], fb["g_raw"][live] * scale) < 1e-5
    # g_k0 per live sample, except samples whose ReLU input sits within rounding of 0
    zmin = oracle.mlp_min_abs_preact(synth.RGBNET_DIMS, P.astype(np.float64), fb["x"])
    keep = zmin >= 1e-6
    assert rel_err(g_k0[rows][live][keep], fb["g_k0"][keep] * scale) < 1e-5
    # the grids after the step's TV + Adam on the voxels only those rays reach
    live_all = np.zeros(S, bool)
    for r in range(R):
        a = int(ray_off[r])
        live_all[a:a + int(n_live[r])] = True
    _check_exclusive_voxels(cfg, rp, D, Fg, P, fb, scale, xyz, live_all, ray_id, sel, p_d, p_f)


def _exclusive_voxels(cfg, xyz_all, live_all, ray_all, sel):
    """Dense voxel indices reached by the trilinear corners of the live samples
    of the rays in sel and by no other ray's live samples (on those voxels the
    batch's grid gradient is the selected rays' gradient alone)."""
    from step_parity import cell_voxels
    G = np.array(synth.grid_dims(cfg))
    pts = xyz_all[live_all]
    rays = ray_all[live_all]
    v = cell_voxels(cfg, pts)                          # [8 n, 3] (corner-major)
    lin = (v[:, 0] * G[1] + v[:, 1]) * G[0] + v[:, 2]
    mine = np.isin(np.tile(rays, 8), sel)
    return np.setdiff1d(np.unique(lin[mine]), np.unique(lin[~mine]))


def _check_exclusive_voxels(cfg, rp, D, Fg, P, fb, scale, xyz, live_all, ray_id, sel, p_d, p_f,
                            g_d=None, g_f=None, tol=1e-5, tau=1e-6, tv_grids=None, min_voxels=500):
    """On the voxels that only the selected rays reach: the grid gradients
    (when given) and the grids after TV + Adam (first step from zero moments)
    against the oracle run on those rays, its gradients rescaled by scale.
    P: the parameters the renderer read; tv_grids: the grids TV reads (the
    BF16 copies in the BF16 form; default D, Fg)."""
    import oracle
    from oracle_step import optimizer
    excl = _exclusive_voxels(cfg, xyz, live_all, ray_id, sel)
    assert len(excl) > min_voxels
    fb_g = dict(fb, g_density=fb["g_density"] * scale, g_feature=fb["g_feature"] * scale,
                g_params=np.zeros_like(fb["g_params"]))
    ref_d = fb_g["g_density"].reshape(-1)[excl]
    ref_f = fb_g["g_feature"].reshape(-1, 12)[excl]
    if g_d is not None:
        assert rel_err(g_d.reshape(-1)[excl], ref_d) < tol
    # feature voxels of samples with a ReLU input within rounding of 0 are set aside
    zmin = oracle.mlp_min_abs_preact(synth.RGBNET_DIMS, P.astype(np.float64), fb["x"])
    amb = zmin < tau
    keep = np.ones(len(excl), bool)
    if amb.any():
        from step_parity import cell_voxels
        G = np.array(synth.grid_dims(cfg))
        v = cell_voxels(cfg, fb["smp"].xyz[fb["live"]][amb])
        bad = (v[:, 0] * G[1] + v[:, 1]) * G[0] + v[:, 2]
        keep = ~np.isin(excl, bad)
    if g_f is not None:
        assert rel_err(g_f.reshape(-1, 12)[excl][keep], ref_f[keep]) < tol
    # TV + Adam (first step from zero moments) on those voxels, where the
    # gradient is clear of rounding noise
    Dt, Ft = tv_grids if tv_grids is not None else (D, Fg)
    opt = optimizer(rp, 1, D, Fg, P, fb_g, False, Dt, Ft)
    for got, ref, g in ((p_d.reshape(-1)[excl], opt["density"].reshape(-1)[excl],
                         opt["g_density_tv"].reshape(-1)[excl]),
                        (p_f.reshape(-1, 12)[excl][keep], opt["feature"].reshape(-1, 12)[excl][keep],
                         opt["g_feature_tv"].reshape(-1, 12)[excl][keep])):
        clear = np.abs(g) > 1e-3 * np.max(np.abs(g))
        assert np.max(np.abs(got - ref)[clear]) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("name", ["dvgo_160", "unbounded_320", "forward_facing_384", "dvgo_160_bf16"])
def test_full_size_grid_gradients_and_adam(T, name):
    """At the benchmark's full size (the workload's grids and ray count): the
    per-ray and per-sample outputs of 48 sampled rays, and the grid gradients
    and the parameters after TV + Adam on the voxels that only those rays
    reach, against the oracle run on those rays (its gradients rescaled from
    1/48 to the batch's 1/R).  The BF16 form (16384 rays) against the oracle
    on the BF16-stored grids and weights, at its 2e-3 bar."""
    from oracle_step import forward_backward
    cfg = synth.CONFIGS[name]
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    bf = name.endswith("_bf16")
    tol, tau = (2e-3, 1e-5) if bf else (1e-5, 1e-6)
    Dr, Fr, Pr = (synth.bf16_round(x) for x in (D, Fg, P)) if bf else (D, Fg, P)
    o, d = synth.rays(cfg, seed=0)
    tgt = synth.target_rgb(cfg, seed=0)
    R = cfg.n_rays
    tr = T.Trainer(cfg, rp, D, Fg, P, n_rays=R, precision="bf16" if bf else "f32tc")
    to, td, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (o, d, tgt))
    tr.forward(to, td, tt, tail_adjoint=True)
    tr.backward(td, tail_done=True)
    torch.cuda.synchronize()
    ray_off = tr.ray_off.cpu().numpy()
    S = int(ray_off[-1])
    n_live = tr.n_live.cpu().numpy()
    xyz, ray_id = host(tr.xyz[:S]), tr.ray_id[:S].cpu().numpy()
    live_all = np.zeros(S, bool)
    for r in range(R):
        live_all[ray_off[r]:ray_off[r] + n_live[r]] = True
    color, L_r = host(tr.color), host(tr.L_r)
    w, rgb, g_raw = (host(x[:S]) for x in (tr.w, tr.rgb, tr.g_raw))
    g_d = host(tr.dense(tr.density, "g"))[..., 0]
    g_f = host(tr.dense(tr.feature, "g"))
    tr.regularize_and_step(False)
    p_d = host(tr.dense(tr.density, "p"))[..., 0]
    p_f = host(tr.dense(tr.feature, "p"))
    rng = np.random.default_rng(8)
    sel = np.sort(rng.choice(np.nonzero(n_live > 0)[0], 48, replace=False))
    fb = forward_backward(cfg, rp, Dr, Fr, Pr, o[sel], d[sel], tgt[sel])
    assert np.array_equal(n_live[sel], fb["n_live"])
    # per-ray and per-sample outputs of the selected rays
    rows = np.concatenate([np.arange(ray_off[r], ray_off[r + 1]) for r in sel]).astype(np.int64)
    live = fb["live"]
    scale = len(sel) / R
    assert np.array_equal(xyz[rows], fb["smp"].xyz)
    assert rel_err(color[sel], fb["color"]) < tol
    assert rel_err(L_r[sel], fb["L_r"]) < tol
    assert rel_err(w[rows], fb["w"]) < tol
    assert rel_err(rgb[rows][live], fb["rgb"][live]) < tol
    assert rel_err(g_raw[rows][live], fb["g_raw"][live] * scale) < tol
    _check_exclusive_voxels(cfg, rp, D, Fg, Pr, fb, scale, xyz, live_all, ray_id, sel, p_d, p_f,
                            g_d, g_f, tol=tol, tau=tau, tv_grids=(Dr, Fr),
                            min_voxels=100 if R > 8192 else 500)   # denser rays: fewer voxels of their own
