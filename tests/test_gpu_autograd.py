"""The autograd Functions of ``ops``: each backward (a hand-written adjoint
kernel) against the FP64 oracle's gradient and against central finite
differences of its own forward; the composed rendering loss against the
training step's explicit backward."""
import numpy as np
import pytest
import torch

import oracle
from conftest import rel_err
from paper_2206_05085_gb300 import synth

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def O():
    from paper_2206_05085_gb300 import build
    build.build()
    oracle.build()
    from paper_2206_05085_gb300 import _lib, ops
    return ops, _lib


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _fd(f, x, idx, eps):
    """Central difference of the scalar f at entries idx of tensor x (in place)."""
    out = []
    for i in idx:
        v = x.view(-1)[i].item()
        x.view(-1)[i] = v + eps
        fp = f()
        x.view(-1)[i] = v - eps
        fm = f()
        x.view(-1)[i] = v
        out.append((fp - fm) / (2 * eps))
    return np.array(out)


def _ragged(seed, R=60, scale=1.5, bias=0.0):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 70, R)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    raw = (rng.normal(size=S) * scale + bias).astype(np.float32)
    rgb = rng.uniform(0, 1, (S, 3)).astype(np.float32)
    m = np.zeros(S, np.float32)
    for r in range(R):
        m[off[r]:off[r + 1]] = np.sort(rng.uniform(0, 1, counts[r]))
    ds = rng.uniform(0.001, 0.01, S).astype(np.float32)
    return off, raw, rgb, m, ds


def test_sample_grid_function(O):
    ops, L = O
    rng = np.random.default_rng(1)
    G, C = (14, 11, 17), 12
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    dense = rng.normal(size=(G[2], G[1], G[0], C)).astype(np.float32)
    grid = torch.empty(L.grid_bricked_elems(G, C), device="cuda")
    L.grid_pack(dev(dense), grid, G, C, L.F32)
    grid.requires_grad_(True)
    xyz = dev(rng.uniform(-1, 1, (3000, 3)).astype(np.float32))
    gd = L.GridDesc.make(lo, hi, G)
    a = dev(rng.normal(size=(3000, C)).astype(np.float32))
    out = ops.sample_grid(grid, xyz, gd, C)
    assert rel_err(host(out), oracle.trilinear(dense, lo, hi, host(xyz))) < TOL32
    (out * a).sum().backward()
    gg = torch.empty(G[2], G[1], G[0], C, device="cuda")
    L.grid_unpack(grid.grad, gg, G, C, L.F32)
    ref = oracle.trilinear_adjoint(host(a), (G[2], G[1], G[0], C), lo, hi, host(xyz))
    assert rel_err(host(gg), ref) < TOL32
    # finite differences of the forward (linear in the grid: exact up to rounding)
    with torch.no_grad():
        f = lambda: float((ops.sample_grid(grid, xyz, gd, C).double() * a.double()).sum())
        idx = rng.choice(grid.numel(), 6, replace=False)
        fd = _fd(f, grid, idx, 0.25)
    assert np.allclose(fd, host(grid.grad)[idx], rtol=2e-3, atol=2e-3)


def test_composite_function(O):
    ops, L = O
    off, raw, rgb, m, ds = _ragged(2, scale=2.0, bias=1.0)
    R = len(off) - 1
    bg = np.array([0.3, 0.6, 0.9], np.float32)
    shift = float(np.float32(np.log(1 / (1 - 1e-4) - 1)))
    rng = np.random.default_rng(3)
    a = rng.normal(size=(R, 3)).astype(np.float32)
    b = rng.normal(size=raw.shape).astype(np.float32)
    traw = dev(raw).requires_grad_(True)
    trgb = dev(rgb).requires_grad_(True)
    color, w, n_live = ops.composite(traw, trgb, dev(off), shift, 0.5, 0.0, bg)
    ref = oracle.composite(raw, rgb, off, shift, 0.5, 0.0, bg)
    assert rel_err(host(color), ref["color"]) < TOL32
    assert rel_err(host(w), ref["w"]) < TOL32
    ((color * dev(a)).sum() + (w * dev(b)).sum()).backward()
    gr, gc = oracle.composite_bwd(raw, rgb, off, shift, 0.5, 0.0, bg, a, b)
    assert rel_err(host(traw.grad), gr) < TOL32
    assert rel_err(host(trgb.grad), gc) < TOL32
    with torch.no_grad():
        def f():
            c2, w2, _ = ops.composite(traw, trgb, dev(off), shift, 0.5, 0.0, bg)
            return float((c2.double() * dev(a).double()).sum() + (w2.double() * dev(b).double()).sum())
        idx = rng.choice(raw.size, 6, replace=False)
        fd = _fd(f, traw, idx, 1e-2)
    assert np.allclose(fd, host(traw.grad)[idx], rtol=3e-2, atol=3e-3)


def test_distortion_function(O):
    ops, L = O
    off, raw, rgb, m, ds = _ragged(4)
    rng = np.random.default_rng(5)
    w = rng.uniform(0, 0.05, raw.shape).astype(np.float32)
    tw = dev(w).requires_grad_(True)
    L_r = ops.distortion(tw, dev(m), dev(ds), dev(off))
    assert rel_err(host(L_r), oracle.distortion(w, m, ds, off, None)) < TOL32
    gL = rng.normal(size=len(off) - 1).astype(np.float32)
    (L_r * dev(gL)).sum().backward()
    assert rel_err(host(tw.grad), oracle.distortion_grad(gL, w, m, ds, off, None)) < TOL32
    with torch.no_grad():
        f = lambda: float((ops.distortion(tw, dev(m), dev(ds), dev(off)).double() * dev(gL).double()).sum())
        idx = rng.choice(w.size, 6, replace=False)
        fd = _fd(f, tw, idx, 1e-3)
    assert np.allclose(fd, host(tw.grad)[idx], rtol=2e-2, atol=1e-4)


@pytest.mark.parametrize("precision", ["f32tc", "f32", "bf16"])
def test_rgbnet_function(O, precision):
    ops, L = O
    from conftest import check_mlp_grads
    rng = np.random.default_rng(6)
    n, R = 700, 50
    k0 = rng.normal(0, 0.3, (n, 12)).astype(np.float32)
    d = rng.normal(size=(R, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    ray_id = rng.integers(0, R, n).astype(np.int32)
    params = (synth.mlp_params() * 2.0).astype(np.float32)
    bf = precision == "bf16"
    p_ref = synth.bf16_round(params) if bf else params
    tk0 = dev(k0).requires_grad_(True)
    tp = dev(params).requires_grad_(True)
    rgb = ops.rgbnet(tk0, tp, dev(d), dev(ray_id), precision)
    x = oracle.rgbnet_input(k0, d[ray_id])
    tol = 2e-3 if bf else TOL32
    assert rel_err(host(rgb), oracle.mlp_fwd(synth.RGBNET_DIMS, p_ref, x, True)) < tol
    g = rng.normal(size=(n, 3)).astype(np.float32)
    (rgb * dev(g)).sum().backward()
    check_mlp_grads(oracle, synth.RGBNET_DIMS, p_ref, x, g, host(tp.grad), host(tk0.grad), tol,
                    tau=2e-5 if bf else 1e-6)
    if not bf:
        with torch.no_grad():
            f = lambda: float((ops.rgbnet(tk0, tp, dev(d), dev(ray_id), precision).double()
                               * dev(g).double()).sum())
            idx = rng.choice(params.size, 6, replace=False)
            fd = _fd(f, tp, idx, 2e-2)
        assert np.allclose(fd, host(tp.grad)[idx], rtol=5e-2, atol=5e-2)


def test_composed_loss_matches_training_step(O):
    """loss.backward() through the Functions = the explicit backward of the
    training step (same batch, same parameters, before the optimizer)."""
    ops, L = O
    from paper_2206_05085_gb300 import train
    cfg = synth.CFG1
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    n = 512
    o, d = synth.rays(cfg, seed=7, n_rays=n)
    t = synth.target_rgb(cfg, seed=7, n_rays=n)
    to, td, tt = dev(o), dev(d), dev(t)
    tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=n, precision="f32tc")
    tr.forward(to, td, tt)
    tr.backward(td)
    torch.cuda.synchronize()
    S = int(tr.ray_off[-1].item())
    xyz = tr.xyz[:S]
    ray_off = tr.ray_off.clone()
    den = tr.density.p.clone().requires_grad_(True)
    fea = tr.feature.p.clone().requires_grad_(True)
    par = tr.mlp.clone().requires_grad_(True)
    raw = ops.sample_grid(den, xyz, tr.gd, 1).view(-1)
    k0 = ops.sample_grid(fea, xyz, tr.gd, 12)
    rgb = ops.rgbnet(k0, par, td, tr.ray_id[:S].contiguous(), "f32tc")
    color, w, n_live = ops.composite(raw, rgb, ray_off, tr.shift, rp.interval, rp.T_stop, rp.bg)
    L_r = ops.distortion(w, tr.s_mid[:S].contiguous(), tr.s_len[:S].contiguous(), ray_off, n_live)
    loss = ((color - tt) ** 2).mean() + rp.lambda_dist * L_r.mean()
    loss.backward()
    assert abs(float(loss.detach()) - float(tr.loss[2])) <= 1e-5 * abs(float(tr.loss[2]))
    for got, ref in ((par.grad, tr.mlp_g), (den.grad, tr.density.g), (fea.grad, tr.feature.g)):
        g, r = host(got).astype(np.float64), host(ref).astype(np.float64)
        assert np.max(np.abs(g - r)) <= 1e-4 * max(np.max(np.abs(r)), 1e-30)
