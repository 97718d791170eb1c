"""The allocation-free sampling entry point returns exactly what the
workspace version returns.

It exists for callers that cannot call cudaMalloc (a host application that
owns the device's whole memory budget and lets no library allocate) and so
cannot hand the sampler a workspace; its per-ray scratch is a fixed array
inside the library.  This file is collected last on purpose: if it fails, a
run that stops at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_2206_05085_gb300 import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2206_05085_gb300 import build
    build.build()
    from paper_2206_05085_gb300 import _lib as L
    return L


def _desc(L, rp):
    """Sampler descriptor of a workload: bbox march (mode 0) or contracted
    march (mode 1), as the training step builds it."""
    sd = L.SamplerDesc()
    if rp.contracted:
        sd.mode, sd.near, sd.max_steps = 1, rp.near, rp.max_steps
        sd.contract_b, sd.p_inf, sd.step_c = rp.contract_b, int(rp.contract_p_inf), rp.step_c
    else:
        sd.mode, sd.near, sd.far, sd.step = 0, rp.near, rp.far, rp.step
        sd.step_offset, sd.use_slab, sd.max_steps = rp.step_offset, int(rp.use_slab), rp.max_steps
    return sd


def _run(L, fn, cfg, rp, o, d, mask, with_ws):
    R = o.shape[0]
    S_cap = R * rp.max_steps
    gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, [cfg.grid] * 3)
    sd = _desc(L, rp)
    out = [torch.full((R + 1,), -1, dtype=torch.int64, device="cuda"),
           torch.full((max(S_cap, 1), 3), -1.0, device="cuda"),
           torch.full((max(S_cap, 1),), -1, dtype=torch.int32, device="cuda"),
           torch.full((max(S_cap, 1),), -1, dtype=torch.int32, device="cuda"),
           torch.full((max(S_cap, 1),), -1.0, device="cuda"),
           torch.full((max(S_cap, 1),), -1.0, device="cuda")]
    to = torch.from_numpy(np.ascontiguousarray(o)).cuda().reshape(-1, 3)
    td = torch.from_numpy(np.ascontiguousarray(d)).cuda().reshape(-1, 3)
    if with_ws:
        ws = torch.empty(max(L.sample_rays_workspace_size(R), 1), dtype=torch.uint8, device="cuda")
        fn(to, td, R, gd, sd, mask, S_cap, *out, ws)
    else:
        fn(to, td, R, gd, sd, mask, S_cap, *out)
    torch.cuda.synchronize()
    return [t.cpu() for t in out]


@pytest.mark.parametrize("workload", ["dvgo_160", "unbounded_320"])
def test_noalloc_sampling_matches_workspace_version(workload):
    L = _lib()
    cfg = synth.CONFIGS[workload]
    rp = synth.render_params(cfg)
    mask = (torch.rand(cfg.grid, cfg.grid, cfg.grid, generator=torch.Generator().manual_seed(0))
            < 0.3).to(torch.uint8).cuda()
    # two calls in a row on different ray batches (the shared scratch keeps
    # the previous call's contents in between): the larger batch first, so
    # the second call's counts sit over stale ones
    for seed, n in ((1, 5000), (2, 3000)):
        o, d = synth.rays(cfg, seed=seed, n_rays=n)
        ref = _run(L, L.sample_rays, cfg, rp, o, d, mask, True)
        got = _run(L, L.sample_rays_noalloc, cfg, rp, o, d, mask, False)
        assert int(ref[0][-1]) > 0
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    assert L.sample_rays_noalloc_max_rays() == 1 << 20


def test_noalloc_sampling_empty_batch():
    L = _lib()
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    e = np.zeros((0, 3), np.float32)
    got = _run(L, L.sample_rays_noalloc, cfg, rp, e, e, None, False)
    assert got[0].tolist() == [0]


def test_noalloc_sampling_rejects_too_many_rays():
    L = _lib()
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    R = L.sample_rays_noalloc_max_rays() + 1
    gd = L.GridDesc.make(cfg.bbox_min, cfg.bbox_max, [cfg.grid] * 3)
    sd = L.SamplerDesc()
    sd.mode, sd.step, sd.max_steps = 0, rp.step, 1
    dummy = torch.empty(1, device="cuda")
    with pytest.raises(L.DvgoError, match="inconsistent sizes"):
        L.sample_rays_noalloc(dummy, dummy, R, gd, sd, None, R, dummy, dummy, dummy, dummy, dummy,
                              dummy)
