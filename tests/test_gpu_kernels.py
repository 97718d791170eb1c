"""GPU parity of each C-ABI kernel against the FP64 oracle on seeded inputs.

Tolerances: integer/index outputs bit-exact; FP32 form 1e-5 relative
(max|x - ref| / max|ref| per tensor); BF16 form 2e-3 relative.  The BF16
form is compared with the plain FP64 oracle on the stored (BF16-rounded)
parameters and grids; nothing in the oracle copies the kernels' rounding.
"""
import numpy as np
import pytest
import torch

import oracle
from conftest import rel_err
from paper_2206_05085_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 2e-3


@pytest.fixture(scope="module")
def L():
    from paper_2206_05085_gb300 import build
    build.build()
    from paper_2206_05085_gb300 import _lib
    _lib.lib()
    return _lib


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def shift32():
    return float(np.float32(oracle.alpha_shift(1e-4)))


# ----------------------------------------------------------------- grids
@pytest.mark.parametrize("G,C", [((16, 16, 16), 1), ((19, 9, 13), 12), ((8, 24, 17), 5)])
def test_pack_unpack_roundtrip(L, G, C):
    rng = np.random.default_rng(0)
    dense = rng.normal(size=(G[2], G[1], G[0], C)).astype(np.float32)
    for dt, tdt in ((L.F32, torch.float32), (L.BF16, torch.bfloat16)):
        d = dev(dense).to(tdt)
        b = torch.empty(L.grid_bricked_elems(G, C), dtype=tdt, device="cuda")
        L.grid_pack(d, b, G, C, dt)
        back = torch.empty_like(d)
        L.grid_unpack(b, back, G, C, dt)
        assert torch.equal(back, d)


def _bricked(L, dense, G, C, dtype=torch.float32):
    b = torch.empty(L.grid_bricked_elems(G, C), dtype=dtype, device="cuda")
    L.grid_pack(dev(dense).to(dtype), b, G, C, L.BF16 if dtype == torch.bfloat16 else L.F32)
    return b


@pytest.mark.parametrize("C", [1, 12, 5])
@pytest.mark.parametrize("bf16", [False, True])
def test_trilinear_fwd_bwd(L, C, bf16):
    rng = np.random.default_rng(C)
    G = (21, 18, 26)
    lo, hi = np.array([-1.0, -0.5, -2.0]), np.array([1.0, 1.5, 2.0])
    dense = rng.normal(size=(G[2], G[1], G[0], C)).astype(np.float32)
    if bf16:
        dense = synth.bf16_round(dense)
    n = 10000
    xyz = (lo + (hi - lo) * rng.uniform(-0.02, 1.02, (n, 3))).astype(np.float32)  # some clamp
    gd = L.GridDesc.make(lo, hi, G)
    grid = _bricked(L, dense, G, C, torch.bfloat16 if bf16 else torch.float32)
    out = torch.full((n, C), -7.0, device="cuda")
    # subset through idx, count on the device
    idx = np.sort(rng.choice(n, 6000, replace=False)).astype(np.int32)
    n_dev = torch.tensor([5000], dtype=torch.int64, device="cuda")
    L.sample_grid_fwd(grid, L.BF16 if bf16 else L.F32, gd, C, dev(xyz), dev(idx), len(idx), n_dev, out)
    got = host(out)
    ref = oracle.trilinear(dense.reshape(G[2], G[1], G[0], C), lo, hi, xyz)
    sel = idx[:5000]
    assert rel_err(got[sel], ref[sel]) < TOL32
    untouched = np.setdiff1d(np.arange(n), sel)
    assert np.all(got[untouched] == -7.0)
    # adjoint
    g_out = rng.normal(size=(n, C)).astype(np.float32)
    g_grid = torch.zeros(L.grid_bricked_elems(G, C), device="cuda")
    touched = torch.zeros(L.grid_num_bricks(G), dtype=torch.uint8, device="cuda")
    L.sample_grid_bwd(dev(g_out), gd, C, dev(xyz), dev(idx), len(idx), n_dev, g_grid, touched)
    gg = torch.empty(G[2], G[1], G[0], C, device="cuda")
    L.grid_unpack(g_grid, gg, G, C, L.F32)
    ref_g = oracle.trilinear_adjoint(g_out[sel], (G[2], G[1], G[0], C), lo, hi, xyz[sel])
    assert rel_err(host(gg), ref_g) < TOL32
    # touched bricks = bricks holding a nonzero adjoint entry (or none)
    nz = np.abs(ref_g).sum(-1) > 0
    nb = [(g + 7) // 8 for g in G]
    tb = np.zeros((nb[2], nb[1], nb[0]), bool)
    zz, yy, xx = np.nonzero(nz)
    tb[zz // 8, yy // 8, xx // 8] = True
    got_t = host(touched).reshape(nb[2], nb[1], nb[0]).astype(bool)
    assert np.all(got_t[tb])


@pytest.mark.parametrize("C", [1, 12])
@pytest.mark.parametrize("bf16", [False, True])
def test_trilinear_fwd_many_samples_per_thread(L, C, bf16):
    """The specialised gathers loop over a resident wave of blocks with the
    next sample's index and position prefetched: enough listed samples that
    every thread takes several steps (and a ragged last one), through an
    index list in random order, count on the device."""
    rng = np.random.default_rng(100 + C + bf16)
    G = (37, 29, 33)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    dense = rng.normal(size=(G[2], G[1], G[0], C)).astype(np.float32)
    if bf16:
        dense = synth.bf16_round(dense)
    n = 1_300_003
    xyz = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    gd = L.GridDesc.make(lo, hi, G)
    grid = _bricked(L, dense, G, C, torch.bfloat16 if bf16 else torch.float32)
    idx = rng.permutation(n).astype(np.int32)
    m = n - 7
    n_dev = torch.tensor([m], dtype=torch.int64, device="cuda")
    out = torch.full((n, C), -7.0, device="cuda")
    L.sample_grid_fwd(grid, L.BF16 if bf16 else L.F32, gd, C, dev(xyz), dev(idx), n, n_dev, out)
    got = host(out)
    ref = oracle.trilinear(dense, lo, hi, xyz)
    sel = idx[:m]
    assert rel_err(got[sel], ref[sel]) < TOL32
    assert np.all(got[idx[m:]] == -7.0)


@pytest.mark.parametrize("C", [1, 12])
def test_trilinear_adjoint_along_rays(L, C):
    """Ray-ordered samples (the layout the renderer produces): consecutive list
    positions share corner voxels, so the scatter's per-warp aggregation table
    sums most contributions before the global reductions; rays of 1-3 samples
    mixed with long ones also fill the table past its capacity."""
    rng = np.random.default_rng(40 + C)
    G = (40, 33, 37)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    vs = 2.0 / 32
    pts = []
    for r in range(300):
        o = rng.uniform(-0.9, 0.9, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        k = int(rng.choice([1, 2, 3, 40, 90]))
        step = vs * rng.choice([0.25, 0.5, 1.0])
        pts.append(np.clip(o + d * step * np.arange(k)[:, None], -1.05, 1.05))
    xyz = np.concatenate(pts).astype(np.float32)
    n = len(xyz)
    live = np.sort(rng.choice(n, int(0.8 * n), replace=False)).astype(np.int32)
    g_out = rng.normal(size=(n, C)).astype(np.float32)
    gd = L.GridDesc.make(lo, hi, G)
    g_grid = torch.zeros(L.grid_bricked_elems(G, C), device="cuda")
    touched = torch.zeros(L.grid_num_bricks(G), dtype=torch.uint8, device="cuda")
    n_dev = torch.tensor([len(live)], dtype=torch.int64, device="cuda")
    L.sample_grid_bwd(dev(g_out), gd, C, dev(xyz), dev(live), n, n_dev, g_grid, touched)
    gg = torch.empty(G[2], G[1], G[0], C, device="cuda")
    L.grid_unpack(g_grid, gg, G, C, L.F32)
    ref_g = oracle.trilinear_adjoint(g_out[live], (G[2], G[1], G[0], C), lo, hi, xyz[live])
    assert rel_err(host(gg), ref_g) < TOL32
    nz = np.abs(ref_g).sum(-1) > 0
    nb = [(g + 7) // 8 for g in G]
    tb = np.zeros((nb[2], nb[1], nb[0]), bool)
    zz, yy, xx = np.nonzero(nz)
    tb[zz // 8, yy // 8, xx // 8] = True
    got_t = host(touched).reshape(nb[2], nb[1], nb[0]).astype(bool)
    assert np.all(got_t[tb])


def test_trilinear_adjoint_pair_along_rays(L):
    """The paired adjoint on ray-ordered samples (neighbouring list positions
    often share a cell, so the warp merges them) against the oracle."""
    rng = np.random.default_rng(45)
    G = (40, 33, 37)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    vs = 2.0 / 32
    pts = []
    for r in range(400):
        o = rng.uniform(-0.9, 0.9, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        k = int(rng.choice([1, 2, 3, 33, 90]))
        step = vs * rng.choice([0.1, 0.25, 0.5, 1.0])
        pts.append(np.clip(o + d * step * np.arange(k)[:, None], -1.05, 1.05))
    xyz = np.concatenate(pts).astype(np.float32)
    n = len(xyz)
    live = np.sort(rng.choice(n, int(0.9 * n), replace=False)).astype(np.int32)
    ga = rng.normal(size=(n, 1)).astype(np.float32)
    gb = rng.normal(size=(n, 12)).astype(np.float32)
    gd = L.GridDesc.make(lo, hi, G)
    nb = L.grid_num_bricks(G)
    outs = [(torch.zeros(L.grid_bricked_elems(G, C), device="cuda"),
             torch.zeros(nb, dtype=torch.uint8, device="cuda")) for C in (1, 12)]
    n_dev = torch.tensor([len(live)], dtype=torch.int64, device="cuda")
    L.sample_grid_bwd2(dev(ga), 1, outs[0][0], outs[0][1], dev(gb), 12, outs[1][0], outs[1][1], gd,
                       dev(xyz), dev(live), n, n_dev)
    for (g_grid, touched), C, g in zip(outs, (1, 12), (ga, gb)):
        gg = torch.empty(G[2], G[1], G[0], C, device="cuda")
        L.grid_unpack(g_grid, gg, G, C, L.F32)
        ref = oracle.trilinear_adjoint(g[live], (G[2], G[1], G[0], C), lo, hi, xyz[live])
        assert rel_err(host(gg), ref) < TOL32
        nz = np.abs(ref).sum(-1) > 0
        nbv = [(q + 7) // 8 for q in G]
        tb = np.zeros((nbv[2], nbv[1], nbv[0]), bool)
        zz, yy, xx = np.nonzero(nz)
        tb[zz // 8, yy // 8, xx // 8] = True
        assert np.all(host(touched).reshape(nbv[2], nbv[1], nbv[0]).astype(bool)[tb])


@pytest.mark.parametrize("bf16", [False, True])
def test_trilinear_fwd_along_rays(L, bf16):
    """The feature query on ray-ordered samples: neighbouring list positions
    often share a cell (runs of up to ten at 0.1-voxel steps) and then share
    one set of corner loads; against the oracle, with a list count that
    leaves a partial last warp."""
    rng = np.random.default_rng(46)
    G = (40, 33, 37)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    vs = 2.0 / 32
    pts = []
    for r in range(700):
        o = rng.uniform(-0.9, 0.9, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        k = int(rng.choice([1, 2, 3, 33, 90]))
        step = vs * rng.choice([0.1, 0.25, 0.5, 1.0])
        pts.append(np.clip(o + d * step * np.arange(k)[:, None], -1.05, 1.05))
    xyz = np.concatenate(pts).astype(np.float32)
    n = len(xyz)
    live = np.sort(rng.choice(n, int(0.9 * n), replace=False)).astype(np.int32)
    m = len(live) - 13
    dense = rng.normal(size=(G[2], G[1], G[0], 12)).astype(np.float32)
    if bf16:
        dense = synth.bf16_round(dense)
    gd = L.GridDesc.make(lo, hi, G)
    grid = _bricked(L, dense, G, 12, torch.bfloat16 if bf16 else torch.float32)
    out = torch.full((n, 12), -7.0, device="cuda")
    n_dev = torch.tensor([m], dtype=torch.int64, device="cuda")
    L.sample_grid_fwd(grid, L.BF16 if bf16 else L.F32, gd, 12, dev(xyz), dev(live), n, n_dev, out)
    got = host(out)
    ref = oracle.trilinear(dense, lo, hi, xyz[live[:m]])
    assert rel_err(got[live[:m]], ref) < TOL32
    rest = np.setdiff1d(np.arange(n), live[:m])
    assert np.all(got[rest] == -7.0)


def test_trilinear_adjoint_pair(L):
    """The paired density / feature adjoint equals the two single ones."""
    rng = np.random.default_rng(44)
    G = (30, 27, 33)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    n = 20000
    xyz = rng.uniform(-1.02, 1.02, (n, 3)).astype(np.float32)
    live = np.sort(rng.choice(n, 15000, replace=False)).astype(np.int32)
    ga = rng.normal(size=(n, 1)).astype(np.float32)
    gb = rng.normal(size=(n, 12)).astype(np.float32)
    gd = L.GridDesc.make(lo, hi, G)
    nb = L.grid_num_bricks(G)
    outs = []
    for C in (1, 12):
        outs.append((torch.zeros(L.grid_bricked_elems(G, C), device="cuda"),
                     torch.zeros(nb, dtype=torch.uint8, device="cuda")))
    n_dev = torch.tensor([len(live)], dtype=torch.int64, device="cuda")
    L.sample_grid_bwd2(dev(ga), 1, outs[0][0], outs[0][1], dev(gb), 12, outs[1][0], outs[1][1], gd,
                       dev(xyz), dev(live), n, n_dev)
    for (g_grid, touched), C, g in zip(outs, (1, 12), (ga, gb)):
        gg = torch.empty(G[2], G[1], G[0], C, device="cuda")
        L.grid_unpack(g_grid, gg, G, C, L.F32)
        ref = oracle.trilinear_adjoint(g[live], (G[2], G[1], G[0], C), lo, hi, xyz[live])
        assert rel_err(host(gg), ref) < TOL32
        one = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        g1 = torch.zeros(L.grid_bricked_elems(G, C), device="cuda")
        L.sample_grid_bwd(dev(g), gd, C, dev(xyz), dev(live), n, n_dev, g1, one)
        assert np.array_equal(host(touched), host(one))


def test_build_mask_bit_exact(L):
    cfg = synth.CFG2
    D = synth.density_grid(cfg)
    G = [cfg.grid] * 3
    gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, G)
    m = torch.empty(G[2], G[1], G[0], dtype=torch.uint8, device="cuda")
    L.build_mask(_bricked(L, D, G, 1), L.F32, gd, shift32(), 0.5, 1e-4, m)
    ref = oracle.build_mask(D, shift32(), 0.5, 1e-4)
    assert np.array_equal(host(m), ref)


# --------------------------------------------------------------- sampler
def _gpu_sample(L, cfg, rp, o, d, mask=None):
    R = o.shape[0]
    S_cap = R * rp.max_steps
    gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, list(synth.grid_dims(cfg)))
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
    out = dict(ray_off=torch.zeros(R + 1, dtype=torch.int64, device="cuda"),
               xyz=torch.empty(S_cap, 3, device="cuda"),
               ray_id=torch.empty(S_cap, dtype=torch.int32, device="cuda"),
               step_k=torch.empty(S_cap, dtype=torch.int32, device="cuda"),
               s_mid=torch.empty(S_cap, device="cuda"), s_len=torch.empty(S_cap, device="cuda"))
    ws = torch.empty(L.sample_rays_workspace_size(R), dtype=torch.uint8, device="cuda")
    L.sample_rays(dev(o), dev(d), R, gd, sd, mask, S_cap, out["ray_off"], out["xyz"],
                  out["ray_id"], out["step_k"], out["s_mid"], out["s_len"], ws)
    res = {k: host(v) for k, v in out.items()}
    S = int(res["ray_off"][-1])
    for k in ("xyz", "ray_id", "step_k", "s_mid", "s_len"):
        res[k] = res[k][:S]
    return res


def _check_samples(got, ref):
    assert np.array_equal(got["ray_off"], ref.ray_off)
    assert np.array_equal(got["ray_id"], ref.ray_id)
    assert np.array_equal(got["step_k"], ref.step_k)
    assert np.array_equal(got["xyz"], ref.xyz)          # FP32 positions bit for bit
    assert rel_err(got["s_mid"], ref.s_mid) < TOL32
    assert rel_err(got["s_len"], ref.s_len) < TOL32


def _forward_facing_small():
    """The forward-facing workload on a 96 x 96 x 64 layer stack (the oracle's
    passes over the full 384^2 x 256 stack would take minutes)."""
    import dataclasses
    return dataclasses.replace(synth.CFG6, name="forward_facing_96", grid=96, dims=(96, 96, 64))


@pytest.mark.parametrize("name", ["small_64", "dvgo_160", "unbounded_320", "forward_facing_96",
                                  "forward_facing_96_wide"])
def test_sampler_bit_exact(L, name):
    import dataclasses
    if name.startswith("forward_facing_96"):
        cfg = _forward_facing_small()
        if name.endswith("wide"):   # a 400 x 240 image at focal 300: fx != fy
            cfg = dataclasses.replace(cfg, name=name, img_w=400, img_h=240, focal=300.0)
    else:
        cfg = synth.CONFIGS[name]
    rp = synth.render_params(cfg)
    if name.endswith("wide"):
        rp = dataclasses.replace(rp, ndc_near=0.5)
        assert rp.ndc_fx != rp.ndc_fy
    o, d = synth.rays(cfg)            # full ray count of the workload
    mask_np = mask_t = None
    if rp.mask_thres is not None:
        D = synth.density_grid(cfg)
        mask_np = oracle.build_mask(D, shift32(), rp.interval, rp.mask_thres)
        mask_t = dev(mask_np)
    got = _gpu_sample(L, cfg, rp, o, d, mask_t)
    from oracle_step import sample
    ref = sample(cfg, rp, o, d, mask_np)
    assert ref.S > 0
    _check_samples(got, ref)


@pytest.mark.parametrize("step_scale", [0.55, 0.45])
def test_sampler_long_march(L, step_scale):
    """Step caps either side of the 1024-step limit of the recorded keep bits
    (0.55: max_steps 1010, kept samples up to step ~640, so about 20 bit words
    per ray; 0.45: max_steps 1232, the second pass evaluates the keep test
    again)."""
    import dataclasses
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    step = float(np.float32(rp.step * step_scale))
    diag = np.sqrt(3.0) * (cfg.bbox_max - cfg.bbox_min)
    rp = dataclasses.replace(rp, step=step, max_steps=int(np.ceil(diag / step)) + 8)
    assert (rp.max_steps <= 1024) == (step_scale > 0.5)
    o, d = synth.rays(cfg, n_rays=400)
    D = synth.density_grid(cfg)
    mask_np = oracle.build_mask(D, shift32(), rp.interval, rp.mask_thres)
    got = _gpu_sample(L, cfg, rp, o, d, dev(mask_np))
    from oracle_step import sample
    ref = sample(cfg, rp, o, d, mask_np)
    assert ref.S > 0 and int(np.max(ref.step_k)) > 512
    _check_samples(got, ref)


@pytest.mark.parametrize("max_steps", [1, 7, 13, 100, 600])
def test_contracted_march_chunks(L, max_steps):
    """The contracted march's second pass runs eight chunks of each march in
    parallel from checkpoints that the first pass records: step caps that
    leave one-step chunks, a partial last chunk, and marches that end (at the
    contracted boundary) before the cap, on rays from inside and outside the
    unit ball, bit-exact against the oracle's sequential march."""
    import dataclasses
    cfg = synth.CFG3
    rp = dataclasses.replace(synth.render_params(cfg), max_steps=max_steps)
    o, d = synth.rays(cfg, n_rays=300)
    o = o.copy()
    o[::3] *= np.float32(1.6)      # a third of the rays start outside the unit ball
    mask_np = mask_t = None
    if max_steps >= 100:   # with occupancy culling (the first steps near the origin are empty)
        D = synth.density_grid(cfg)
        mask_np = oracle.build_mask(D, shift32(), rp.interval, 1e-4)
        mask_t = dev(mask_np)
    got = _gpu_sample(L, cfg, rp, o, d, mask_t)
    from oracle_step import sample
    ref = sample(cfg, rp, o, d, mask_np)
    assert ref.S > 0
    _check_samples(got, ref)
    if max_steps == 600:   # some marches end at the contracted boundary before the cap
        last = np.array([ref.step_k[b:e].max() if e > b else -1
                         for b, e in zip(ref.ray_off[:-1], ref.ray_off[1:])])
        assert (last < max_steps - 1).sum() > 10


@pytest.mark.parametrize("b", [1.0, 0.5])
def test_contracted_march_euclidean(L, b):
    """The contraction with the Euclidean norm (p = 2; the workloads use the
    max norm) and two contraction parameters b: the march's samples bit-exact
    against the oracle's sequential march, with occupancy culling, on rays
    from inside and outside the unit ball."""
    import dataclasses
    cfg = synth.CFG3
    rp = dataclasses.replace(synth.render_params(cfg), contract_p_inf=False, contract_b=b, max_steps=300)
    o, d = synth.rays(cfg, n_rays=300)
    o = o.copy()
    o[::3] *= np.float32(1.6)
    D = synth.density_grid(cfg)
    mask_np = oracle.build_mask(D, shift32(), rp.interval, 1e-4)
    got = _gpu_sample(L, cfg, rp, o, d, dev(mask_np))
    from oracle_step import sample
    ref = sample(cfg, rp, o, d, mask_np)
    assert ref.S > 1000
    _check_samples(got, ref)


def test_sampler_edge_cases(L):
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    # rays that miss the box, start inside it, run along an axis, zero components
    o = np.array([[-4, 3, 0], [0.1, 0.2, 0.3], [-4, 0, 0], [0, -4, 0.5], [4, 4, 4]], np.float32)
    d = np.array([[1, 0, 0], [0, 0, 1], [1, 0, 0], [0, 1, 0], [-1, -1, -1]], np.float32)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = _gpu_sample(L, cfg, rp, o, d)
    from oracle_step import sample
    ref = sample(cfg, rp, o, d, None)
    _check_samples(got, ref)
    assert got["ray_off"][1] == 0
    # empty ray batch
    got0 = _gpu_sample(L, cfg, rp, o[:0], d[:0])
    assert got0["ray_off"].tolist() == [0]


# ------------------------------------------------------------- rendering
def _ragged_case(seed, counts, scale=3.0, bias=8.0):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    raw = (rng.normal(0, scale, S) + bias).astype(np.float32)
    rgb = rng.uniform(0, 1, (S, 3)).astype(np.float32)
    return off, raw, rgb


COUNTS = [0, 1, 2, 31, 32, 33, 64, 100, 300, 559] + list(np.random.default_rng(9).integers(0, 260, 500))


@pytest.mark.parametrize("T_stop", [1e-3, 0.0])
def test_alpha_weights_and_composite(L, T_stop):
    off, raw, rgb = _ragged_case(1, COUNTS)
    R, S = len(off) - 1, int(off[-1])
    bg = np.array([1.0, 0.5, 0.25], np.float32)
    sh = shift32()
    w, T = torch.empty(S, device="cuda"), torch.empty(S, device="cuda")
    n_live = torch.empty(R, dtype=torch.int32, device="cuda")
    T_end = torch.empty(R, device="cuda")
    L.alpha_weights_fwd(dev(raw), dev(off), R, sh, 0.5, T_stop, w, T, n_live, T_end)
    color = torch.empty(R, 3, device="cuda")
    L.composite_rgb_fwd(w, dev(rgb), dev(off), n_live, T_end, R, bg, color)
    ref = oracle.composite(raw, rgb, off, sh, 0.5, T_stop, bg)
    nl = host(n_live)
    # halting index: exact except where T sits on the threshold within FP32 rounding
    diff = np.nonzero(nl != ref["n_live"])[0]
    for r in diff:
        k = min(nl[r], ref["n_live"][r])
        assert abs(ref["T"][off[r] + k] / T_stop - 1) < 1e-5, (r, nl[r], ref["n_live"][r])
    ok = np.setdiff1d(np.arange(R), diff)
    okS = np.concatenate([np.arange(off[r], off[r + 1]) for r in ok])
    assert rel_err(host(w)[okS], ref["w"][okS]) < TOL32
    assert rel_err(host(T)[okS], ref["T"][okS]) < TOL32
    assert rel_err(host(T_end)[ok], ref["T_end"][ok]) < TOL32
    assert rel_err(host(color)[ok], ref["color"][ok]) < TOL32
    assert (nl < np.diff(off)).sum() > 10 or T_stop == 0.0


def test_composite_backward(L):
    off, raw, rgb = _ragged_case(2, COUNTS, scale=2.0, bias=7.0)
    R, S = len(off) - 1, int(off[-1])
    bg = np.array([0.2, 0.9, 0.4], np.float32)
    sh = shift32()
    rng = np.random.default_rng(3)
    g_color = rng.normal(size=(R, 3)).astype(np.float32)
    g_w = rng.normal(size=S).astype(np.float32)
    for T_stop in (1e-3, 0.0):
        w, T = torch.empty(S, device="cuda"), torch.empty(S, device="cuda")
        n_live = torch.empty(R, dtype=torch.int32, device="cuda")
        T_end = torch.empty(R, device="cuda")
        L.alpha_weights_fwd(dev(raw), dev(off), R, sh, 0.5, T_stop, w, T, n_live, T_end)
        g_raw = torch.empty(S, device="cuda")
        g_rgb = torch.empty(S, 3, device="cuda")
        L.composite_bwd(dev(g_color), dev(g_w), dev(raw), T, dev(rgb), dev(off), n_live, R, sh,
                        0.5, bg, g_raw, g_rgb)
        ref = oracle.composite(raw, rgb, off, sh, 0.5, T_stop, bg)
        assert np.array_equal(host(n_live), ref["n_live"])
        gr, gc = oracle.composite_bwd(raw, rgb, off, sh, 0.5, T_stop, bg, g_color, g_w)
        assert rel_err(host(g_raw), gr) < TOL32
        assert rel_err(host(g_rgb), gc) < TOL32


def test_composite_distortion_fused(L):
    """The fused per-ray tails equal compositing + distortion (forward) and the
    compositing adjoint fed with the distortion gradient (backward)."""
    off, raw, rgb = _ragged_case(2, COUNTS, scale=2.0, bias=7.0)
    R, S = len(off) - 1, int(off[-1])
    bg = np.array([0.2, 0.9, 0.4], np.float32)
    sh = shift32()
    rng = np.random.default_rng(31)
    m = np.zeros(S, np.float32)
    for r in range(R):
        m[off[r]:off[r + 1]] = np.sort(rng.uniform(2, 6, off[r + 1] - off[r]))
    ds = rng.uniform(0.001, 0.01, S).astype(np.float32)
    g_color = rng.normal(size=(R, 3)).astype(np.float32)
    gL = 0.37
    for T_stop in (1e-3, 0.0):
        w, T = torch.empty(S, device="cuda"), torch.empty(S, device="cuda")
        n_live = torch.empty(R, dtype=torch.int32, device="cuda")
        T_end = torch.empty(R, device="cuda")
        L.alpha_weights_fwd(dev(raw), dev(off), R, sh, 0.5, T_stop, w, T, n_live, T_end)
        ref = oracle.composite(raw, rgb, off, sh, 0.5, T_stop, bg)
        assert np.array_equal(host(n_live), ref["n_live"])
        color = torch.empty(R, 3, device="cuda")
        L_r = torch.empty(R, device="cuda")
        L.composite_distortion_fwd(w, dev(rgb), dev(m), dev(ds), dev(off), n_live, T_end, R, bg,
                                   color, L_r)
        assert rel_err(host(color), ref["color"]) < TOL32
        L_ref = oracle.distortion(ref["w"], m, ds, off, ref["n_live"])
        assert rel_err(host(L_r), L_ref) < TOL32
        g_raw = torch.full((S,), 5.0, device="cuda")
        L.composite_distortion_bwd(dev(g_color), gL, w, dev(raw), T, dev(rgb), dev(m), dev(ds),
                                   dev(off), n_live, R, sh, 0.5, bg, g_raw)
        g_w = oracle.distortion_grad(gL, ref["w"], m, ds, off, ref["n_live"])
        gr, _ = oracle.composite_bwd(raw, rgb, off, sh, 0.5, T_stop, bg, g_color, g_w)
        assert rel_err(host(g_raw), gr) < TOL32


@pytest.mark.parametrize("bf16,per_sample", [(False, False), (True, False), (False, True)])
def test_density_alpha_fused(L, bf16, per_sample):
    """Density query + weights in one pass = dvgo_sample_grid_fwd then
    dvgo_alpha_weights_fwd (bit-equal w, T, n_live, T_end; raw equal before
    each ray's halt), on rays sampled through a blob scene so that many halt;
    per_sample: with per-sample intervals."""
    rng = np.random.default_rng(50 + bf16)
    G = (40, 40, 40)
    lo, hi = np.array([-1.0] * 3), np.array([1.0] * 3)
    ax = np.linspace(-1, 1, 40)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    dense = (30.0 * np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / 0.1) - 3.0).astype(np.float32)[..., None]
    if bf16:
        dense = synth.bf16_round(dense)
    R = 700
    counts = rng.integers(0, 100, R)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    pts = []
    for r in range(R):
        o = rng.uniform(-0.5, 0.5, 3) * np.array([1, 1, 0]) + np.array([0, 0, -0.99])
        d = np.array([0.0, 0.0, 1.0]) + rng.normal(0, 0.2, 3)
        d /= np.linalg.norm(d)
        pts.append(np.clip(o + d * 0.02 * np.arange(counts[r])[:, None], -1, 1))
    xyz = np.concatenate(pts).astype(np.float32)
    S = len(xyz)
    gd = L.GridDesc.make(lo, hi, G)
    grid = _bricked(L, dense, G, 1, torch.bfloat16 if bf16 else torch.float32)
    dt = L.BF16 if bf16 else L.F32
    sh = shift32()
    dl = dev(0.5 * rng.integers(1, 6, S).astype(np.float32)) if per_sample else None
    outs = []
    for fused in (False, True):
        raw, w, T = (torch.full((S,), -9.0, device="cuda") for _ in range(3))
        n_live = torch.empty(R, dtype=torch.int32, device="cuda")
        T_end = torch.empty(R, device="cuda")
        if fused:
            L.density_alpha_fwd(grid, dt, gd, dev(xyz), dev(off), R, sh, 0.5, 1e-3, raw, w, T, n_live,
                                T_end, delta=dl)
        else:
            L.sample_grid_fwd(grid, dt, gd, 1, dev(xyz), None, S, None, raw)
            L.alpha_weights_fwd(raw, dev(off), R, sh, 0.5, 1e-3, w, T, n_live, T_end, delta=dl)
        outs.append([host(x) for x in (raw, w, T, n_live, T_end)])
    (r0, w0, T0, n0, e0), (r1, w1, T1, n1, e1) = outs
    assert np.array_equal(n0, n1) and np.array_equal(e0, e1)
    assert np.array_equal(w0, w1) and np.array_equal(T0, T1)
    halted = int(np.sum(n0 < np.diff(off)))
    assert halted > 50   # (93 of the 700 rays halt in the FP64 oracle)
    for r in range(R):
        k = slice(off[r], off[r] + n0[r])
        assert np.array_equal(r0[k], r1[k])


def test_per_sample_intervals(L):
    """Every compositing entry with a per-sample interval array (the spans of
    a proposal's picks) against the oracle given the same intervals: weights,
    halting, colour, the compositing adjoint, and the fused tails (forward,
    distortion adjoint, loss + adjoint) bit-equal to the unfused calls."""
    off, raw, rgb = _ragged_case(12, COUNTS, scale=2.0, bias=4.0)
    R, S = len(off) - 1, int(off[-1])
    rng = np.random.default_rng(13)
    delta = (0.5 * rng.integers(1, 24, S)).astype(np.float32)
    bg = np.array([0.2, 0.9, 0.4], np.float32)
    sh = shift32()
    m = np.zeros(S, np.float32)
    for r in range(R):
        m[off[r]:off[r + 1]] = np.sort(rng.uniform(0, 1, off[r + 1] - off[r]))
    ds = rng.uniform(0.001, 0.01, S).astype(np.float32)
    g_color = rng.normal(size=(R, 3)).astype(np.float32)
    target = rng.uniform(0, 1, (R, 3)).astype(np.float32)
    gL, lam = 0.37, 0.01
    dl = dev(delta)
    for T_stop in (1e-3, 0.0):
        w, T = torch.empty(S, device="cuda"), torch.empty(S, device="cuda")
        n_live = torch.empty(R, dtype=torch.int32, device="cuda")
        T_end = torch.empty(R, device="cuda")
        L.alpha_weights_fwd(dev(raw), dev(off), R, sh, 0.5, T_stop, w, T, n_live, T_end, delta=dl)
        ref = oracle.composite(raw, rgb, off, sh, 0.5, T_stop, bg, delta=delta)
        nl = host(n_live)
        diff = np.nonzero(nl != ref["n_live"])[0]
        for r in diff:
            k = min(nl[r], ref["n_live"][r])
            assert abs(ref["T"][off[r] + k] / T_stop - 1) < 1e-5, (r, nl[r], ref["n_live"][r])
        ok = np.setdiff1d(np.arange(R), diff)
        okS = np.concatenate([np.arange(off[r], off[r + 1]) for r in ok])
        assert rel_err(host(w)[okS], ref["w"][okS]) < TOL32
        assert rel_err(host(T_end)[ok], ref["T_end"][ok]) < TOL32
        assert (nl < np.diff(off)).sum() > 100 or T_stop == 0.0
        # colour through the one-pass compositing forward
        c_one = torch.empty(R, 3, device="cuda")
        w2, T2 = torch.empty(S, device="cuda"), torch.empty(S, device="cuda")
        n2, e2 = torch.empty(R, dtype=torch.int32, device="cuda"), torch.empty(R, device="cuda")
        L.composite_fwd(dev(raw), dev(rgb), dev(off), R, sh, 0.5, T_stop, bg, c_one, w2, T2, n2, e2,
                        delta=dl)
        assert torch.equal(w, w2) and torch.equal(n_live, n2)
        assert rel_err(host(c_one)[ok], ref["color"][ok]) < TOL32
        # compositing adjoint (with the live counts of the oracle where they agree)
        g_w = rng.normal(size=S).astype(np.float32)
        g_raw = torch.empty(S, device="cuda")
        L.composite_bwd(dev(g_color), dev(g_w), dev(raw), T, dev(rgb), dev(off), n_live, R, sh, 0.5,
                        bg, g_raw, None, delta=dl)
        gr, _ = oracle.composite_bwd(raw, rgb, off, sh, 0.5, T_stop, bg, g_color, g_w, delta=delta)
        assert rel_err(host(g_raw)[okS], gr[okS]) < TOL32
        # distortion adjoint inside the reverse scan
        gd_raw = torch.empty(S, device="cuda")
        L.composite_distortion_bwd(dev(g_color), gL, w, dev(raw), T, dev(rgb), dev(m), dev(ds),
                                   dev(off), n_live, R, sh, 0.5, bg, gd_raw, delta=dl)
        g_wd = oracle.distortion_grad(gL, ref["w"], m, ds, off, ref["n_live"])
        grd, _ = oracle.composite_bwd(raw, rgb, off, sh, 0.5, T_stop, bg, g_color, g_wd, delta=delta)
        assert rel_err(host(gd_raw)[okS], grd[okS]) < TOL32
        # loss + adjoint in one pass: bit-equal to the loss pass then the adjoint
        args = (w, dev(rgb), dev(m), dev(ds), dev(off), n_live, T_end, R, bg)
        ws = torch.zeros(L.composite_loss_workspace_size(R), dtype=torch.uint8, device="cuda")
        c1, l1 = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
        loss1, g1 = torch.empty(3, device="cuda"), torch.empty(R, 3, device="cuda")
        L.composite_distortion_loss_fwd(*args, dev(target), lam, c1, l1, g1, loss1, ws)
        gr1 = torch.empty(S, device="cuda")
        L.composite_distortion_bwd(g1, lam / R, w, dev(raw), T, dev(rgb), dev(m), dev(ds), dev(off),
                                   n_live, R, sh, 0.5, bg, gr1, delta=dl)
        c3, l3 = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
        loss3, g3, gr3 = (torch.empty(3, device="cuda"), torch.empty(R, 3, device="cuda"),
                          torch.empty(S, device="cuda"))
        L.composite_distortion_loss_fwd_bwd(*args, dev(target), lam, lam / R, dev(raw), T, sh, 0.5,
                                            c3, l3, g3, loss3, gr3, ws, delta=dl)
        assert torch.equal(c1, c3) and torch.equal(g1, g3) and torch.equal(gr1, gr3)


@pytest.mark.parametrize("R_rays", [37, 5000])
def test_composite_distortion_loss_fused(L, R_rays):
    """One launch = compositing + distortion + photometric loss: colour, L_r
    and g_color bit-equal to the separate calls, the loss against the oracle's
    mean squared error; repeated calls give the same bits and leave the
    workspace's ticket at zero (several blocks reach the last-block sum)."""
    rng = np.random.default_rng(R_rays)
    counts = rng.integers(0, 40, R_rays)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    raw = (rng.normal(size=S) * 2.0 + 1.0).astype(np.float32)
    rgb = rng.uniform(0, 1, (S, 3)).astype(np.float32)
    m = np.zeros(S, np.float32)
    for r in range(R_rays):
        m[off[r]:off[r + 1]] = np.sort(rng.uniform(0, 1, counts[r]))
    ds = rng.uniform(0.001, 0.01, S).astype(np.float32)
    target = rng.uniform(0, 1, (R_rays, 3)).astype(np.float32)
    bg = np.array([1.0, 1.0, 1.0], np.float32)
    sh, lam = shift32(), 0.01
    w, T = torch.empty(S, device="cuda"), torch.empty(S, device="cuda")
    n_live = torch.empty(R_rays, dtype=torch.int32, device="cuda")
    T_end = torch.empty(R_rays, device="cuda")
    L.alpha_weights_fwd(dev(raw), dev(off), R_rays, sh, 0.5, 1e-3, w, T, n_live, T_end)
    args = (w, dev(rgb), dev(m), dev(ds), dev(off), n_live, T_end, R_rays, bg)
    c1, l1 = torch.empty(R_rays, 3, device="cuda"), torch.empty(R_rays, device="cuda")
    L.composite_distortion_fwd(*args, c1, l1)
    loss1, g1 = torch.empty(3, device="cuda"), torch.empty(R_rays, 3, device="cuda")
    L.rgb_loss(c1, dev(target), l1, R_rays, lam, loss1, g1)
    ws = torch.zeros(L.composite_loss_workspace_size(R_rays), dtype=torch.uint8, device="cuda")
    outs = []
    for _ in range(3):
        c2, l2 = torch.empty(R_rays, 3, device="cuda"), torch.empty(R_rays, device="cuda")
        loss2, g2 = torch.empty(3, device="cuda"), torch.empty(R_rays, 3, device="cuda")
        L.composite_distortion_loss_fwd(*args, dev(target), lam, c2, l2, g2, loss2, ws)
        outs.append(host(loss2))
        assert torch.equal(c1, c2) and torch.equal(l1, l2) and torch.equal(g1, g2)
        assert int(host(ws[:4].view(torch.int32))[0]) == 0
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    # with the compositing adjoint in the same pass: every output bit-equal to the two calls
    gr1 = torch.empty(S, device="cuda")
    L.composite_distortion_bwd(g1, lam / R_rays, w, dev(raw), T, dev(rgb), dev(m), dev(ds), dev(off),
                               n_live, R_rays, sh, 0.5, bg, gr1)
    c3, l3 = torch.empty(R_rays, 3, device="cuda"), torch.empty(R_rays, device="cuda")
    loss3, g3, gr3 = torch.empty(3, device="cuda"), torch.empty(R_rays, 3, device="cuda"), torch.empty(S, device="cuda")
    L.composite_distortion_loss_fwd_bwd(*args, dev(target), lam, lam / R_rays, dev(raw), T, sh, 0.5,
                                        c3, l3, g3, loss3, gr3, ws)
    assert torch.equal(c1, c3) and torch.equal(l1, l3) and torch.equal(g1, g3)
    assert torch.equal(gr1, gr3)
    assert np.array_equal(outs[0], host(loss3))
    ref = oracle.composite(raw, rgb, off, sh, 0.5, 1e-3, bg)
    mse = np.mean((ref["color"] - target) ** 2)
    Ld = np.mean(oracle.distortion(ref["w"], m, ds, off, ref["n_live"]))
    assert rel_err(outs[0], np.array([mse, Ld, mse + lam * Ld])) < TOL32
    assert rel_err(outs[0], host(loss1)) < 1e-6


def test_distortion(L):
    rng = np.random.default_rng(4)
    counts = COUNTS
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    R, S = len(counts), int(off[-1])
    w = rng.uniform(0, 0.05, S).astype(np.float32)
    m = np.zeros(S, np.float32)
    for r in range(R):
        m[off[r]:off[r + 1]] = np.sort(rng.uniform(0, 1, counts[r]))
    ds = rng.uniform(0.001, 0.01, S).astype(np.float32)
    seg = np.array([min(c, int(rng.integers(0, c + 1))) if r % 3 == 0 else c
                    for r, c in enumerate(counts)], np.int32)
    for seg_len in (None, seg):
        L_r = torch.empty(R, device="cuda")
        sl = None if seg_len is None else dev(seg_len)
        L.distortion_fwd(dev(w), dev(m), dev(ds), dev(off), sl, R, L_r)
        ref = oracle.distortion(w, m, ds, off, seg_len)
        assert rel_err(host(L_r), ref) < TOL32
        gL = rng.normal(size=R).astype(np.float32)
        g_w = torch.full((S,), 9.0, device="cuda")
        L.distortion_bwd(dev(gL), 0.0, dev(w), dev(m), dev(ds), dev(off), sl, R, g_w)
        assert rel_err(host(g_w), oracle.distortion_grad(gL, w, m, ds, off, seg_len)) < TOL32
        L.distortion_bwd(None, 0.25, dev(w), dev(m), dev(ds), dev(off), sl, R, g_w)
        assert rel_err(host(g_w), oracle.distortion_grad(0.25, w, m, ds, off, seg_len)) < TOL32


def test_rgb_loss(L):
    rng = np.random.default_rng(5)
    R = 3000
    color = rng.uniform(0, 1, (R, 3)).astype(np.float32)
    target = rng.uniform(0, 1, (R, 3)).astype(np.float32)
    L_r = rng.uniform(0, 0.1, R).astype(np.float32)
    loss = torch.empty(3, device="cuda")
    g = torch.empty(R, 3, device="cuda")
    L.rgb_loss(dev(color), dev(target), dev(L_r), R, 0.01, loss, g)
    c64, t64 = color.astype(np.float64), target.astype(np.float64)
    ref = np.mean((c64 - t64) ** 2)
    got = host(loss)
    assert abs(got[0] - ref) / ref < TOL32
    assert abs(got[1] - L_r.astype(np.float64).mean()) / L_r.mean() < TOL32
    assert abs(got[2] - (ref + 0.01 * L_r.astype(np.float64).mean())) / ref < TOL32
    assert rel_err(host(g), 2 * (c64 - t64) / (3 * R)) < TOL32


# ------------------------------------------------------------ colour MLP
def _mlp_case(n, seed=6):
    rng = np.random.default_rng(seed)
    k0 = rng.normal(0, 0.3, (n, 12)).astype(np.float32)
    R = 97
    d = rng.normal(size=(R, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    ray_id = rng.integers(0, R, n).astype(np.int32)
    params = synth.mlp_params()
    params = (params * 2.0).astype(np.float32)   # larger activations than init
    g_rgb = rng.normal(size=(n, 3)).astype(np.float32)
    return k0, d, ray_id, params, g_rgb


@pytest.mark.parametrize("precision", ["f32", "f32tc", "bf16"])
@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000])
def test_rgbnet_fwd_bwd(L, precision, n):
    from conftest import check_mlp_grads
    k0, d, ray_id, params, g_rgb = _mlp_case(n)
    bf = precision == "bf16"
    prec = {"f32": L.F32, "f32tc": L.F32_TC, "bf16": L.BF16}[precision]
    tol = TOL16 if bf else TOL32
    act_tc = None
    if precision in ("f32tc", "bf16"):
        act_tc = torch.empty(L.rgbnet_act_bytes(n, prec), dtype=torch.uint8, device="cuda")
    p_ref = synth.bf16_round(params) if bf else params
    # every other sample through idx, count on the device
    idx = np.arange(0, n, 2 if n > 2 else 1).astype(np.int32)
    m = len(idx)
    rgb = torch.full((n, 3), -1.0, device="cuda")
    n_dev = torch.tensor([m], dtype=torch.int64, device="cuda")
    L.rgbnet_fwd(dev(k0), dev(d), dev(ray_id), dev(idx), n, n_dev, dev(params), prec, rgb, act_tc)
    x = oracle.rgbnet_input(k0[idx], d[ray_id[idx]])
    ref = oracle.mlp_fwd(synth.RGBNET_DIMS, p_ref, x, True)
    got = host(rgb)
    assert rel_err(got[idx], ref) < tol
    rest = np.setdiff1d(np.arange(n), idx)
    assert np.all(got[rest] == -1.0)
    # backward recomputing the forward, and (FP32 form) from stored activations
    for use_act in ((False, True) if precision == "f32" else (True,)):
        act = act_tc
        if use_act and precision == "f32":
            act = torch.empty(n, 256, device="cuda")
            L.rgbnet_fwd(dev(k0), dev(d), dev(ray_id), dev(idx), n, n_dev, dev(params), prec, rgb,
                         act)
        g_params = torch.zeros(len(params), device="cuda")
        g_k0 = torch.zeros(n, 12, device="cuda")
        L.rgbnet_bwd(dev(g_rgb), None, None, dev(k0), dev(d), dev(ray_id), dev(idx), n, n_dev,
                     dev(params), prec, g_params, g_k0, act, rgb if use_act else None)
        check_mlp_grads(oracle, synth.RGBNET_DIMS, p_ref, x, g_rgb[idx], host(g_params),
                        host(g_k0)[idx], tol, tau=2e-5 if bf else 1e-6)
    assert L.device_status() == 0


def test_rgbnet_bwd_from_compositing_gradient(L):
    # upstream colour gradient formed in-kernel as w[s] * g_color[ray_id[s]]
    n = 3000
    k0, d, ray_id, params, _ = _mlp_case(n, 8)
    rng = np.random.default_rng(8)
    w = rng.uniform(0, 1, n).astype(np.float32)
    g_color = rng.normal(size=(d.shape[0], 3)).astype(np.float32)
    g_params = torch.zeros(len(params), device="cuda")
    g_k0 = torch.zeros(n, 12, device="cuda")
    L.rgbnet_bwd(None, dev(g_color), dev(w), dev(k0), dev(d), dev(ray_id), None, n, None,
                 dev(params), L.F32, g_params, g_k0)
    # the stored activations of the forward give the same gradients
    rgb = torch.empty(n, 3, device="cuda")
    act = torch.empty(n, 256, device="cuda")
    L.rgbnet_fwd(dev(k0), dev(d), dev(ray_id), None, n, None, dev(params), L.F32, rgb, act)
    g2 = torch.zeros(len(params), device="cuda")
    gk2 = torch.zeros(n, 12, device="cuda")
    L.rgbnet_bwd(None, dev(g_color), dev(w), dev(k0), dev(d), dev(ray_id), None, n, None,
                 dev(params), L.F32, g2, gk2, act, rgb)
    assert rel_err(host(g2), host(g_params)) < 1e-6
    assert rel_err(host(gk2), host(g_k0)) < 1e-6
    x = oracle.rgbnet_input(k0, d[ray_id])
    from conftest import check_mlp_grads
    check_mlp_grads(oracle, synth.RGBNET_DIMS, params, x, w[:, None] * g_color[ray_id],
                    host(g_params), host(g_k0), TOL32)


def test_rgbnet_tc_compositing_gradient_wide_range(L):
    """Tensor-core FP32 form with the in-kernel upstream w[s] * g_color[ray]:
    weights spanning 1e-9..1 exercise the per-sample power-of-two gradient
    scales: every sample's input gradient keeps FP32 relative accuracy."""
    n = 4000
    k0, d, ray_id, params, _ = _mlp_case(n, 9)
    rng = np.random.default_rng(9)
    w = (10.0 ** rng.uniform(-9, 0, n)).astype(np.float32)
    g_color = (rng.normal(size=(d.shape[0], 3)) * 1e-4).astype(np.float32)
    act = torch.empty(L.rgbnet_act_bytes(n, L.F32_TC), dtype=torch.uint8, device="cuda")
    rgb = torch.empty(n, 3, device="cuda")
    L.rgbnet_fwd(dev(k0), dev(d), dev(ray_id), None, n, None, dev(params), L.F32_TC, rgb, act)
    g_params = torch.zeros(len(params), device="cuda")
    g_k0 = torch.zeros(n, 12, device="cuda")
    L.rgbnet_bwd(None, dev(g_color), dev(w), dev(k0), dev(d), dev(ray_id), None, n, None,
                 dev(params), L.F32_TC, g_params, g_k0, act, rgb)
    assert L.device_status() == 0
    x = oracle.rgbnet_input(k0, d[ray_id])
    assert rel_err(host(rgb), oracle.mlp_fwd(synth.RGBNET_DIMS, params, x, True)) < TOL32
    from conftest import check_mlp_grads
    g_up = w[:, None] * g_color[ray_id]
    check_mlp_grads(oracle, synth.RGBNET_DIMS, params, x, g_up, host(g_params), host(g_k0), TOL32)
    _, gx = oracle.mlp_bwd(synth.RGBNET_DIMS, params, x, g_up, True)
    gx = gx[:, :12]
    zmin = oracle.mlp_min_abs_preact(synth.RGBNET_DIMS, params, x)
    got = host(g_k0)
    keep = np.nonzero(zmin > 1e-6)[0]
    assert len(keep) > 0.9 * n
    err = np.linalg.norm(got[keep] - gx[keep], axis=1) / np.linalg.norm(gx[keep], axis=1)
    worst = int(np.argmax(err))
    assert err[worst] < TOL32, (int(keep[worst]), float(w[keep[worst]]), float(err[worst]))


def test_rgbnet_tc_range_status(L):
    """Inputs the split-FP16 operands cannot hold are reported (no fault)."""
    n = 300
    k0, d, ray_id, params, _ = _mlp_case(n, 10)
    k0[17, 3] = 1.0e4
    act = torch.empty(L.rgbnet_act_bytes(n, L.F32_TC), dtype=torch.uint8, device="cuda")
    rgb = torch.empty(n, 3, device="cuda")
    L.device_status()
    L.rgbnet_fwd(dev(k0), dev(d), dev(ray_id), None, n, None, dev(params), L.F32_TC, rgb, act)
    assert L.device_status() == -8
    assert L.device_status() == 0


# --------------------------------------------------------- TV and Adam
@pytest.mark.parametrize("C", [1, 12, 3])
@pytest.mark.parametrize("dense_mode", [True, False])
@pytest.mark.parametrize("bf16", [False, True])
def test_tv_add_grad(L, C, dense_mode, bf16):
    rng = np.random.default_rng(10 + C)
    G = (20, 17, 11)
    grid = rng.normal(0, 1.2, (G[2], G[1], G[0], C)).astype(np.float32)
    if bf16:
        grid = synth.bf16_round(grid)
    g0 = np.where(rng.uniform(size=grid.shape) < 0.2, rng.normal(size=grid.shape), 0.0).astype(np.float32)
    gb = _bricked(L, g0, G, C)
    touched = torch.zeros(L.grid_num_bricks(G), dtype=torch.uint8, device="cuda")
    if not dense_mode:
        nb = [(g + 7) // 8 for g in G]
        t = np.zeros((nb[2], nb[1], nb[0]), np.uint8)
        zz, yy, xx = np.nonzero(np.abs(g0).sum(-1) > 0)
        t[zz // 8, yy // 8, xx // 8] = 1
        touched = dev(t.reshape(-1))
    if bf16:
        L.tv_add_grad(_bricked(L, grid, G, C, torch.bfloat16), L.BF16, G, C, 0.5, 1.0, dense_mode,
                      touched, gb)
    else:
        L.tv_add_grad(_bricked(L, grid, G, C), L.F32, G, C, 0.5, 1.0, dense_mode, touched, gb)
    out = torch.empty(G[2], G[1], G[0], C, device="cuda")
    L.grid_unpack(gb, out, G, C, L.F32)
    ref = oracle.tv_add_grad(grid, g0, 0.5, 1.0, dense_mode)
    assert rel_err(host(out), ref) < TOL32
    if dense_mode:
        assert np.all(host(touched) == 1)


def test_touched_compact(L):
    rng = np.random.default_rng(23)
    for nb in (1, 31, 1000, 70001):
        flags = (rng.uniform(size=nb) < 0.3).astype(np.uint8)
        lst = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), 77, dtype=torch.int32, device="cuda")
        L.touched_compact(dev(flags), nb, lst, cnt)
        c = int(host(cnt)[0])
        assert c == int(flags.sum())
        assert np.array_equal(np.sort(host(lst)[:c]), np.nonzero(flags)[0])


@pytest.mark.parametrize("use_list", [False, True])
@pytest.mark.parametrize("dense_mode", [True, False])
def test_tv_add_grad_multi(L, dense_mode, use_list):
    """Two grids of one shape in one launch = two single TV calls (oracle)."""
    rng = np.random.default_rng(21)
    G = (19, 23, 10)
    nb = [(g + 7) // 8 for g in G]
    cases = []
    for C, bf16, w in ((1, False, 0.7), (12, True, 0.3)):
        grid = rng.normal(0, 1.2, (G[2], G[1], G[0], C)).astype(np.float32)
        if bf16:
            grid = synth.bf16_round(grid)
        g0 = np.where(rng.uniform(size=grid.shape) < 0.2, rng.normal(size=grid.shape), 0.0).astype(np.float32)
        t = np.zeros((nb[2], nb[1], nb[0]), np.uint8)
        zz, yy, xx = np.nonzero(np.abs(g0).sum(-1) > 0)
        t[zz // 8, yy // 8, xx // 8] = 1
        gb = _bricked(L, g0, G, C)
        tb = dev(t.reshape(-1))
        gridb = _bricked(L, grid, G, C, torch.bfloat16 if bf16 else torch.float32)
        cases.append((grid, g0, C, w, bf16, gridb, gb, tb))
    lst = cnt = None
    if use_list:   # the two grids' flags are the same here only by chance; list from the union
        union = np.maximum(host(cases[0][7]), host(cases[1][7]))
        lst = torch.empty(len(union), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        L.touched_compact(dev(union), len(union), lst, cnt)
    L.tv_add_grad_multi([(gridb, L.BF16 if bf16 else L.F32, C, w, tb, gb)
                         for grid, g0, C, w, bf16, gridb, gb, tb in cases], G, 1.0, dense_mode,
                        lst, cnt)
    for grid, g0, C, w, bf16, gridb, gb, tb in cases:
        out = torch.empty(G[2], G[1], G[0], C, device="cuda")
        L.grid_unpack(gb, out, G, C, L.F32)
        assert rel_err(host(out), oracle.tv_add_grad(grid, g0, w, 1.0, dense_mode)) < TOL32
        if dense_mode:
            assert np.all(host(tb) == 1)


@pytest.mark.parametrize("use_list", [False, True])
def test_adam_step_multi(L, use_list):
    """Two bricked grids (flagged blocks) and a flat odd-length vector in one
    launch = three single Adam calls (oracle)."""
    rng = np.random.default_rng(12)
    arrays = []
    for C, nb in ((1, 30), (12, 17)):
        n = nb * 512 * C
        p = rng.normal(size=n).astype(np.float32)
        m = rng.normal(0, 0.1, n).astype(np.float32)
        v = rng.uniform(0, 0.1, n).astype(np.float32)
        g = np.zeros(n, np.float32)
        flags = (rng.uniform(size=nb) < 0.5).astype(np.uint8)
        for b in np.nonzero(flags)[0]:
            blk = slice(b * 512 * C, (b + 1) * 512 * C)
            g[blk] = np.where(rng.uniform(size=512 * C) < 0.7, rng.normal(size=512 * C), 0.0)
        arrays.append((p, g, m, v, flags, 512 * C, 0.1))
    n = 22019
    arrays.append((rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32),
                   rng.normal(0, 0.1, n).astype(np.float32), rng.uniform(0, 0.1, n).astype(np.float32),
                   None, 0, 1e-3))
    dev_arrays = [(dev(p), dev(g), dev(m), dev(v), None if f is None else dev(f))
                  for p, g, m, v, f, be, lr in arrays]
    params = []
    for (tp, tg, tm, tv, tf), (p, g, m, v, f, be, lr) in zip(dev_arrays, arrays):
        entry = [tp, None, tg, tm, tv, tp.numel(), tf, be, lr]
        if use_list and f is not None:
            lst = torch.empty(len(f), dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            L.touched_compact(tf, len(f), lst, cnt)
            entry += [lst, cnt]
        params.append(tuple(entry))
    if use_list:   # the device-side step count: 4 -> 5
        step = torch.tensor([4, 0], dtype=torch.int64, device="cuda")
        L.adam_step_multi_dev(params, 0.9, 0.99, 1e-15, step, True)
        assert int(host(step)[0]) == 5
    else:
        L.adam_step_multi(params, 0.9, 0.99, 1e-15, 5, True)
    for (tp, tg, tm, tv, tf), (p, g, m, v, f, be, lr) in zip(dev_arrays, arrays):
        rp, rm, rv = oracle.adam(p, g, m, v, lr, 0.9, 0.99, 1e-15, 5)
        assert rel_err(host(tp), rp) < TOL32
        assert rel_err(host(tm), rm) < TOL32
        assert rel_err(host(tv), rv) < TOL32
        z = g == 0
        assert np.array_equal(host(tp)[z], p[z])
        assert np.all(host(tg) == 0)
        if f is not None:
            assert np.all(host(tf) == 0)


@pytest.mark.parametrize("sparse", [True, False])
def test_adam_step(L, sparse):
    rng = np.random.default_rng(11)
    C, nb = 12, 40
    n = nb * 512 * C
    p = rng.normal(size=n).astype(np.float32)
    m = rng.normal(0, 0.1, n).astype(np.float32)
    v = rng.uniform(0, 0.1, n).astype(np.float32)
    g = np.zeros(n, np.float32)
    flags = (rng.uniform(size=nb) < 0.5).astype(np.uint8)
    for b in np.nonzero(flags)[0]:
        blk = slice(b * 512 * C, (b + 1) * 512 * C)
        g[blk] = np.where(rng.uniform(size=512 * C) < 0.7, rng.normal(size=512 * C), 0.0)
    tp, tg, tm, tv = dev(p), dev(g), dev(m), dev(v)
    sh = torch.zeros(n, dtype=torch.bfloat16, device="cuda")
    touched = dev(flags) if sparse else None
    L.adam_step(tp, sh, tg, tm, tv, n, touched, 512 * C, 0.1, 0.9, 0.99, 1e-15, 7, True)
    rp, rm, rv = oracle.adam(p, g, m, v, 0.1, 0.9, 0.99, 1e-15, 7)
    assert rel_err(host(tp), rp) < TOL32
    assert rel_err(host(tm), rm) < TOL32
    assert rel_err(host(tv), rv) < TOL32
    z = g == 0
    assert np.array_equal(host(tp)[z], p[z])          # skipped entries bit-unchanged
    assert np.all(host(tg) == 0)
    upd = ~z
    assert np.array_equal(host(sh.float())[upd], synth.bf16_round(host(tp))[upd])
    if sparse:
        assert np.all(host(touched) == 0)
    # odd-length flat vector (MLP parameters)
    q = rng.normal(size=22019).astype(np.float32)
    gq = rng.normal(size=22019).astype(np.float32)
    tq, tgq = dev(q), dev(gq)
    tmq, tvq = torch.zeros_like(tq), torch.zeros_like(tq)
    L.adam_step(tq, None, tgq, tmq, tvq, 22019, None, 0, 1e-3, 0.9, 0.99, 1e-15, 1, True)
    rq, _, _ = oracle.adam(q, gq, np.zeros(22019), np.zeros(22019), 1e-3, 0.9, 0.99, 1e-15, 1)
    assert rel_err(host(tq), rq) < TOL32


def test_grid_adam_step(L):
    """dvgo_grid_adam_step: the bricked-grid form (geometry instead of a
    flat length; one flag per brick) = the oracle's Adam on the same data."""
    rng = np.random.default_rng(13)
    G, C = (21, 9, 17), 12
    n = L.grid_bricked_elems(G, C)
    nb = L.grid_num_bricks(G)
    assert n == nb * 512 * C
    p = rng.normal(size=n).astype(np.float32)
    m = rng.normal(0, 0.1, n).astype(np.float32)
    v = rng.uniform(0, 0.1, n).astype(np.float32)
    g = np.zeros(n, np.float32)
    flags = (rng.uniform(size=nb) < 0.5).astype(np.uint8)
    for b in np.nonzero(flags)[0]:
        blk = slice(b * 512 * C, (b + 1) * 512 * C)
        g[blk] = np.where(rng.uniform(size=512 * C) < 0.7, rng.normal(size=512 * C), 0.0)
    tp, tg, tm, tv, tf = dev(p), dev(g), dev(m), dev(v), dev(flags)
    L.grid_adam_step(tp, None, tg, tm, tv, G, C, tf, 0.1, 0.9, 0.99, 1e-15, 3, True)
    rp, rm, rv = oracle.adam(p, g, m, v, 0.1, 0.9, 0.99, 1e-15, 3)
    assert rel_err(host(tp), rp) < TOL32
    assert rel_err(host(tm), rm) < TOL32
    assert rel_err(host(tv), rv) < TOL32
    assert np.array_equal(host(tp)[g == 0], p[g == 0])
    assert np.all(host(tg) == 0) and np.all(host(tf) == 0)


def test_invalid_arguments_raise(L):
    with pytest.raises(L.DvgoError):
        L.distortion_fwd(None, None, None, None, None, 5, None)
    with pytest.raises(L.DvgoError):
        L.rgbnet_fwd(None, None, None, None, 10, None, None, 7, None)
    assert L.device_status() == 0


# ------------------------------------------------------- grid scaling
@pytest.mark.parametrize("Gs,Gd", [((13, 10, 17), (25, 19, 33)), ((13, 10, 17), (7, 6, 9)),
                                   ((16, 16, 16), (16, 16, 16))])
def test_grid_resample(L, Gs, Gd):
    rng = np.random.default_rng(80)
    C = 5
    dense = rng.normal(size=(Gs[2], Gs[1], Gs[0], C)).astype(np.float32)
    src = _bricked(L, dense, Gs, C)
    out = torch.empty(L.grid_bricked_elems(Gd, C), device="cuda")
    L.grid_resample(src, Gs, out, L.F32, Gd, C)
    got = torch.empty(Gd[2], Gd[1], Gd[0], C, device="cuda")
    L.grid_unpack(out, got, Gd, C, L.F32)
    ref = oracle.grid_resample(dense, Gd)
    assert rel_err(host(got), ref) < TOL32
    if Gs == Gd:
        assert np.array_equal(host(got), dense)
    # the BF16 copy is the FP32 result rounded to nearest
    outb = torch.empty(L.grid_bricked_elems(Gd, C), dtype=torch.bfloat16, device="cuda")
    L.grid_resample(src, Gs, outb, L.BF16, Gd, C)
    gotb = torch.empty(Gd[2], Gd[1], Gd[0], C, dtype=torch.bfloat16, device="cuda")
    L.grid_unpack(outb, gotb, Gd, C, L.BF16)     # (brick padding is not written)
    assert np.array_equal(host(gotb.float()), synth.bf16_round(host(got)))


@pytest.mark.parametrize("precision", ["f32tc", "bf16"])
def test_trainer_upscale_then_step(L, precision):
    """A trainer whose grids are raised from 48^3 to 80^3 (moments resampled
    with them) takes a step that matches the oracle's step on the resampled
    grids."""
    import dataclasses
    from paper_2206_05085_gb300 import train
    cfg = dataclasses.replace(synth.CFG2, grid=48)
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    o, d = synth.rays(cfg, n_rays=256)
    tgt = synth.target_rgb(cfg, n_rays=256)
    to, td, tt = (dev(a) for a in (o, d, tgt))
    tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=256, precision=precision)
    tr.step(to, td, tt)                       # moments and t are no longer zero
    m_before = host(tr.dense(tr.feature, "m"))
    tr.upscale(80)
    assert tr.G == [80, 80, 80] and int(tr.step_dev[0].item()) == 1
    Dn = host(tr.dense(tr.density, "p"))[..., 0]
    Fn = host(tr.dense(tr.feature, "p"))
    # the moments were resampled with the grids
    assert rel_err(host(tr.dense(tr.feature, "m")), oracle.grid_resample(m_before, (80, 80, 80))) < TOL32
    Pn = host(tr.mlp)
    cfg2, rp2 = tr.cfg, tr.rp
    assert rp2.max_steps > rp.max_steps
    # one forward/backward on the new grids against the oracle's on the same stored values
    tr.forward(to, td, tt)
    tr.backward(td)
    S = int(host(tr.ray_off)[-1])
    gpu = dict(loss=host(tr.loss), color=host(tr.color), L_r=host(tr.L_r), n_live=host(tr.n_live), S=S)
    from oracle_step import forward_backward
    bf = precision == "bf16"
    fb = forward_backward(cfg2, rp2, synth.bf16_round(Dn) if bf else Dn, synth.bf16_round(Fn) if bf else Fn,
                          synth.bf16_round(Pn) if bf else Pn, o, d, tgt, grads=False)
    assert S == fb["smp"].S
    assert np.array_equal(gpu["n_live"], fb["n_live"])
    tol = 2e-3 if bf else TOL32
    assert rel_err(gpu["color"], fb["color"]) < tol
    assert rel_err(gpu["loss"], fb["loss"]) < tol


# ---------------------------------------------- progressive occupancy mask
def test_update_mask_follows_density(L):
    """After the density changes in some bricks, re-evaluating the mask in
    those bricks gives the mask built from scratch (bit-exact against the
    oracle's mask of the new density)."""
    cfg = synth.CFG2
    G = [cfg.grid] * 3
    gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, G)
    D0 = synth.density_grid(cfg)
    rng = np.random.default_rng(90)
    nbx = (cfg.grid + 7) // 8
    bricks = np.sort(rng.choice(nbx ** 3, 400, replace=False)).astype(np.int32)
    D1 = D0.copy()
    for b in bricks:
        bx, by, bz = b % nbx, (b // nbx) % nbx, b // (nbx * nbx)
        sl = np.s_[bz * 8:bz * 8 + 8, by * 8:by * 8 + 8, bx * 8:bx * 8 + 8]
        D1[sl] += rng.normal(0, 6.0, D1[sl].shape).astype(np.float32)
    m = torch.empty(G[2], G[1], G[0], dtype=torch.uint8, device="cuda")
    L.build_mask(_bricked(L, D0, G, 1), L.F32, gd, shift32(), 0.5, 1e-4, m)
    L.update_mask(_bricked(L, D1, G, 1), L.F32, gd, shift32(), 0.5, 1e-4, dev(bricks),
                  torch.tensor([len(bricks)], dtype=torch.int32, device="cuda"), m)
    ref = oracle.build_mask(D1, shift32(), 0.5, 1e-4)
    assert not np.array_equal(ref, oracle.build_mask(D0, shift32(), 0.5, 1e-4))
    assert np.array_equal(host(m), ref)
    # every brick (no list), on a grid whose side is not a multiple of 8
    Gs = [37, 29, 45]
    gds = L.GridDesc.make(-1.0, 1.0, Gs)
    Ds = rng.normal(-3, 4, (Gs[2], Gs[1], Gs[0])).astype(np.float32)
    ms = torch.zeros(Gs[2], Gs[1], Gs[0], dtype=torch.uint8, device="cuda")
    L.update_mask(_bricked(L, Ds, Gs, 1), L.F32, gds, shift32(), 0.5, 1e-4, None, None, ms)
    assert np.array_equal(host(ms), oracle.build_mask(Ds, shift32(), 0.5, 1e-4))


def test_trainer_mask_follows_training(L):
    """With the progressive update on, after every step the mask equals the
    mask built from the current density."""
    from paper_2206_05085_gb300 import train
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=2048, precision="f32tc", mask_update=True)
    changed = False
    m0 = host(tr.mask).copy()
    for it in range(3):
        o, d = synth.rays(cfg, seed=40 + it, n_rays=2048)
        t = synth.target_rgb(cfg, seed=40 + it, n_rays=2048)
        tr.step(dev(o), dev(d), dev(t))
        dens = host(tr.dense(tr.density, "p"))[..., 0]
        ref = oracle.build_mask(dens, shift32(), rp.interval, rp.mask_thres)
        assert np.array_equal(host(tr.mask), ref)
        changed |= not np.array_equal(ref, m0)
    assert changed     # the lr-0.1 Adam steps move grid points across the threshold


def test_live_samples_cull(L):
    rng = np.random.default_rng(91)
    counts = np.array([0, 1, 5, 31, 32, 33, 100, 300] + list(rng.integers(0, 260, 300)))
    R = len(counts)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    n_live = np.array([rng.integers(0, c + 1) for c in counts], np.int32)
    w = np.where(rng.uniform(size=S) < 0.4, 10.0 ** rng.uniform(-7, -1, S), 0.0).astype(np.float32)
    w_min = 1e-4
    live_idx = torch.full((S,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rgb = torch.full((S, 3), 5.0, device="cuda")
    gk = torch.full((S, 12), 5.0, device="cuda")
    ws = torch.empty(L.live_samples_workspace_size(R), dtype=torch.uint8, device="cuda")
    L.live_samples_cull(dev(off), dev(n_live), dev(w), w_min, R, live_idx, cnt, rgb, gk, ws)
    live = np.zeros(S, bool)
    for r in range(R):
        live[off[r]:off[r] + n_live[r]] = True
    keep = live & (w >= w_min)
    ref = np.nonzero(keep)[0]
    assert int(host(cnt)[0]) == len(ref)
    assert np.array_equal(host(live_idx)[:len(ref)], ref)
    culled = live & ~keep
    assert np.all(host(rgb)[culled] == 0) and np.all(host(gk)[culled] == 0)
    assert np.all(host(rgb)[~culled] == 5.0) and np.all(host(gk)[~culled] == 5.0)


# --------------------------------------------------------- zero-size calls
def test_zero_size_calls(L):
    """Every entry point over samples or rays accepts an empty batch (n_cap =
    0, R = 0, a device count of 0): it returns DVGO_OK, launches no work that
    faults, and leaves its outputs as they were, except the CSR offsets and
    counts that an empty batch defines (ray_off = [0], counts 0)."""
    f = lambda *s: torch.full(s or (4,), 7.0, device="cuda")                       # noqa: E731
    i32 = lambda *s: torch.full(s or (4,), 7, dtype=torch.int32, device="cuda")     # noqa: E731
    i64 = lambda *s: torch.full(s or (4,), 7, dtype=torch.int64, device="cuda")     # noqa: E731
    G = (16, 16, 16)
    gd = L.GridDesc.make((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), G)
    grid = torch.zeros(L.grid_bricked_elems(G, 12), device="cuda")
    touched = torch.zeros(L.grid_num_bricks(G), dtype=torch.uint8, device="cuda")
    params = dev(synth.mlp_params())
    zero_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    # samples: n_cap = 0, and n_cap > 0 with a device count of 0
    for n_cap, n_dev in ((0, None), (5, zero_dev)):
        out = f(5, 12)
        L.sample_grid_fwd(grid, L.F32, gd, 12, f(5, 3), None, n_cap, n_dev, out)
        assert torch.all(out == 7.0)
        gg = torch.zeros_like(grid)
        L.sample_grid_bwd(f(5, 12), gd, 12, f(5, 3), None, n_cap, n_dev, gg, touched)
        L.sample_grid_bwd2(f(5), 1, torch.zeros(L.grid_bricked_elems(G, 1), device="cuda"), touched,
                           f(5, 12), 12, gg, touched, gd, f(5, 3), None, n_cap, n_dev)
        assert not torch.any(gg) and not torch.any(touched)
        for prec in (L.F32, L.F32_TC, L.BF16):
            rgb = f(5, 3)
            act = torch.empty(max(L.rgbnet_act_bytes(5, prec), 16), dtype=torch.uint8, device="cuda")
            if prec == L.F32:
                act = torch.empty(5, 256, device="cuda")
            L.rgbnet_fwd(f(5, 12), f(2, 3), i32(5), None, n_cap, n_dev, params, prec, rgb, act)
            assert torch.all(rgb == 7.0)
            gp = torch.zeros_like(params)
            gk = f(5, 12)
            L.rgbnet_bwd(f(5, 3), None, None, f(5, 12), f(2, 3), i32(5), None, n_cap, n_dev, params,
                         prec, gp, gk, act, rgb)
            assert not torch.any(gp)
        logits = f(5)
        L.proposal_fwd(f(5, 3), None, n_cap, n_dev, dev(synth.proposal_params()), logits)
        assert torch.all(logits == 7.0)
    # rays: R = 0
    ray_off = i64(1)
    sd = L.SamplerDesc()
    sd.mode, sd.near, sd.far, sd.step, sd.max_steps = 0, 0.0, 4.0, 0.1, 64
    ws = torch.empty(max(L.sample_rays_workspace_size(0), 16), dtype=torch.uint8, device="cuda")
    L.sample_rays(f(1, 3), f(1, 3), 0, gd, sd, None, 0, ray_off, f(1, 3), i32(1), i32(1), f(1), f(1), ws)
    assert ray_off.tolist() == [0]
    live_idx, live_count = i32(1), i64(1)
    wsl = torch.empty(max(L.live_samples_workspace_size(0), 16), dtype=torch.uint8, device="cuda")
    L.live_samples(torch.zeros(1, dtype=torch.int64, device="cuda"), i32(1), 0, live_idx, live_count, wsl)
    assert int(live_count.item()) == 0
    color, L_r, n_live, T_end = f(1, 3), f(1), i32(1), f(1)
    off0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.alpha_weights_fwd(f(1), off0, 0, 0.0, 0.5, 1e-3, f(1), f(1), n_live, T_end)
    L.density_alpha_fwd(torch.zeros(L.grid_bricked_elems(G, 1), device="cuda"), L.F32, gd, f(1, 3), off0,
                        0, 0.0, 0.5, 1e-3, f(1), f(1), f(1), n_live, T_end)
    L.composite_rgb_fwd(f(1), f(1, 3), off0, n_live, T_end, 0, (0.0, 0.0, 0.0), color)
    L.composite_distortion_fwd(f(1), f(1, 3), f(1), f(1), off0, n_live, T_end, 0, (0.0, 0.0, 0.0),
                               color, L_r)
    L.distortion_fwd(f(1), f(1), f(1), off0, None, 0, L_r)
    L.distortion_bwd(f(1), 1.0, f(1), f(1), f(1), off0, None, 0, f(1))
    L.composite_bwd(f(1, 3), None, f(1), f(1), f(1, 3), off0, n_live, 0, 0.0, 0.5, (0.0, 0.0, 0.0), f(1))
    assert torch.all(color == 7.0) and torch.all(L_r == 7.0)
    assert L.device_status() == 0
