"""GPU parity of a whole training iteration (forward, backward, TV, Adam)
against the same iteration composed from the FP64 oracle, on the seeded
synthetic workloads."""
import dataclasses

import numpy as np
import pytest
import torch

from conftest import rel_err
from oracle_step import forward_backward, optimizer
from paper_2206_05085_gb300 import synth

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
    tr = T.Trainer(cfg, rp, D, Fg, P, n_rays=len(o), precision=precision)
    to, td, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (o, d, tgt))
    tr.forward(to, td, tt)
    tr.backward(td)
    gpu = dict(loss=host(tr.loss), color=host(tr.color), n_live=host(tr.n_live),
               S=int(host(tr.ray_off)[-1]), g_mlp=host(tr.mlp_g),
               g_density=host(tr.dense(tr.density, "g"))[..., 0],
               g_feature=host(tr.dense(tr.feature, "g")))
    tr.regularize_and_step(tv_dense)
    gpu.update(density=host(tr.dense(tr.density, "p"))[..., 0], feature=host(tr.dense(tr.feature, "p")),
               params=host(tr.mlp))
    bf = precision == "bf16"
    Dr = synth.bf16_round(D) if bf else D
    Fr = synth.bf16_round(Fg) if bf else Fg
    Pr = synth.bf16_round(P) if bf else P
    fb = forward_backward(cfg, rp, Dr, Fr, Pr, o, d, tgt, bf16=bf)
    opt = optimizer(rp, 1, D, Fg, P, fb, tv_dense, Dr, Fr)
    return gpu, fb, opt


def _compare(gpu, fb, opt, tol):
    assert gpu["S"] == fb["smp"].S
    bad = np.nonzero(gpu["n_live"] != fb["n_live"])[0]
    assert len(bad) == 0, f"halting index differs on rays {bad[:10]}"
    assert rel_err(gpu["color"], fb["color"]) < tol
    assert rel_err(gpu["loss"], fb["loss"]) < tol
    assert rel_err(gpu["g_density"], fb["g_density"]) < tol
    assert rel_err(gpu["g_feature"], fb["g_feature"].reshape(gpu["g_feature"].shape)) < tol
    offs = np.cumsum([0, 128 * 39, 128, 128 * 128, 128, 3 * 128, 3])
    for a, b in zip(offs[:-1], offs[1:]):
        assert rel_err(gpu["g_mlp"][a:b], fb["g_params"][a:b]) < tol, (a, b)
    # parameters after TV + Adam (first step: the update is lr * sign-like)
    assert rel_err(gpu["density"], opt["density"]) < tol
    assert rel_err(gpu["feature"], opt["feature"].reshape(gpu["feature"].shape)) < tol
    assert rel_err(gpu["params"], opt["params"]) < tol


def test_step_small_fp32(T):
    gpu, fb, opt = _run(T, synth.CFG1, 512, "f32", tv_dense=False, ray_stride=4)
    assert fb["live"].sum() > 10000
    _compare(gpu, fb, opt, 1e-5)


def test_step_dvgo160_fp32_sparse_tv(T):
    gpu, fb, opt = _run(T, synth.CFG2, 1024, "f32", tv_dense=False, ray_stride=8)
    assert (fb["n_live"] < np.diff(fb["smp"].ray_off)).sum() > 50   # early stop is exercised
    _compare(gpu, fb, opt, 1e-5)


def test_step_dvgo160_fp32_dense_tv(T):
    gpu, fb, opt = _run(T, synth.CFG2, 256, "f32", tv_dense=True, ray_stride=32)
    _compare(gpu, fb, opt, 1e-5)


def test_step_dvgo160_bf16(T):
    gpu, fb, opt = _run(T, synth.CFG4, 1024, "bf16", tv_dense=False, ray_stride=16)
    _compare(gpu, fb, opt, 2e-3)


def test_step_unbounded_contracted(T):
    # the 320^3 grids of the workload are exercised by the benchmark; a 96^3
    # grid keeps the FP64 oracle's TV/Adam pass small here
    cfg = dataclasses.replace(synth.CFG3, grid=96)
    gpu, fb, opt = _run(T, cfg, 256, "f32", tv_dense=False, ray_stride=32)
    _compare(gpu, fb, opt, 1e-5)
