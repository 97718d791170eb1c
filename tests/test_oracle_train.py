"""Pins of the oracle's colour MLP, frequency encoding, TV gradient, Adam and
proposal pieces against torch library routines, identities and finite
differences."""
import numpy as np
import pytest
import torch

from conftest import rel_err
from paper_2206_05085_gb300 import synth


def _torch_mlp(dims, params, x, out_sigmoid):
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    h = xt
    off = 0
    L = len(dims) - 1
    for l in range(L):
        nW = dims[l + 1] * dims[l]
        W = p[off:off + nW].view(dims[l + 1], dims[l])
        b = p[off + nW:off + nW + dims[l + 1]]
        off += nW + dims[l + 1]
        h = torch.nn.functional.linear(h, W, b)
        if l < L - 1:
            h = torch.relu(h)
        elif out_sigmoid:
            h = torch.sigmoid(h)
    return p, xt, h


@pytest.mark.parametrize("dims,sig", [(synth.RGBNET_DIMS, True), (synth.PROPOSAL_DIMS, False)])
def test_mlp_against_torch_autograd(orc, dims, sig):
    rng = np.random.default_rng(0)
    params = synth.mlp_params(dims).astype(np.float64)
    x = rng.normal(size=(37, dims[0]))
    g_out = rng.normal(size=(37, dims[-1]))
    out = orc.mlp_fwd(dims, params, x, sig)
    gp, gx = orc.mlp_bwd(dims, params, x, g_out, sig)
    p, xt, h = _torch_mlp(dims, params, x, sig)
    (h * torch.tensor(g_out)).sum().backward()
    assert rel_err(out, h.detach().numpy()) < 1e-13
    assert rel_err(gp, p.grad.numpy()) < 1e-12
    assert rel_err(gx, xt.grad.numpy()) < 1e-12


def test_frequency_encoding_identities(orc):
    rng = np.random.default_rng(1)
    v = rng.normal(size=(50, 3)).astype(np.float32)
    F = 4
    e = orc.freq_encode(v, F)
    assert e.shape == (50, 27)
    assert np.array_equal(e[:, :3], v.astype(np.float64))
    s = e[:, 3:3 + 3 * F].reshape(50, 3, F)
    c = e[:, 3 + 3 * F:].reshape(50, 3, F)
    assert np.allclose(s ** 2 + c ** 2, 1.0, atol=1e-14)
    # doubling between consecutive frequencies: sin 2x = 2 sin x cos x
    assert np.allclose(s[:, :, 1:], 2 * s[:, :, :-1] * c[:, :, :-1], atol=1e-12)
    assert np.allclose(s[:, :, 0], np.sin(v.astype(np.float64)), atol=1e-15)


def test_tv_loss_against_huber_loss(orc):
    rng = np.random.default_rng(2)
    g = rng.normal(0, 1.5, (5, 6, 7, 3))
    t = torch.tensor(g)
    acc = 0.0
    for ax in range(3):
        a = t.narrow(ax, 1, t.shape[ax] - 1)
        b = t.narrow(ax, 0, t.shape[ax] - 1)
        acc += 2 * torch.nn.functional.huber_loss(a, b, reduction="sum", delta=1.0).item()
    expect = acc / (5 * 6 * 7 * 3)
    assert orc.tv_loss(g, 1.0) == pytest.approx(expect, rel=1e-12)


def test_tv_gradient_fd_and_sparse_mode(orc):
    rng = np.random.default_rng(3)
    g = rng.normal(0, 1.5, (4, 5, 6, 2))
    grad_in = np.zeros_like(g)
    out = orc.tv_add_grad(g, grad_in, 3.0, 1.0, dense_mode=True)
    h = 1e-6
    for _ in range(30):
        i = tuple(rng.integers(0, s) for s in g.shape)
        gp, gm = g.copy(), g.copy()
        gp[i] += h
        gm[i] -= h
        fd = 3.0 * (orc.tv_loss(gp, 1.0) - orc.tv_loss(gm, 1.0)) / (2 * h)
        assert out[i] == pytest.approx(fd, rel=1e-6, abs=1e-8)   # FD round-off ~1e-9
    grad_in = np.where(rng.uniform(size=g.shape) < 0.3, rng.normal(size=g.shape), 0.0)
    sp = orc.tv_add_grad(g, grad_in, 3.0, 1.0, dense_mode=False)
    dense = orc.tv_add_grad(g, grad_in, 3.0, 1.0, dense_mode=True)
    nz = grad_in != 0
    assert np.array_equal(sp[~nz], grad_in[~nz])
    assert np.array_equal(sp[nz], dense[nz])


def test_adam_against_torch(orc):
    rng = np.random.default_rng(4)
    n = 200
    p0 = rng.normal(size=n)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.1, betas=(0.9, 0.99), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 4):
        g = rng.normal(size=n)
        p, m, v = orc.adam(p, g, m, v, 0.1, 0.9, 0.99, 1e-15, t)
        tp.grad = torch.tensor(g)
        opt.step()
    assert rel_err(p, tp.detach().numpy()) < 1e-13


def test_adam_skips_zero_gradient_entries(orc):
    rng = np.random.default_rng(5)
    n = 100
    p0, m0, v0 = rng.normal(size=n), rng.normal(size=n), rng.uniform(0, 1, n)
    g = np.where(rng.uniform(size=n) < 0.5, rng.normal(size=n), 0.0)
    p, m, v = orc.adam(p0, g, m0, v0, 0.1, 0.9, 0.99, 1e-15, 7)
    z = g == 0
    assert np.array_equal(p[z], p0[z]) and np.array_equal(m[z], m0[z]) and np.array_equal(v[z], v0[z])
    assert np.all(p[~z] != p0[~z])
    # the non-skipped entries follow torch's Adam from the same state
    tp = torch.tensor(p0[~z].copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.1, betas=(0.9, 0.99), eps=1e-15)
    opt.state[tp] = {"step": torch.tensor(6.0), "exp_avg": torch.tensor(m0[~z].copy()),
                     "exp_avg_sq": torch.tensor(v0[~z].copy())}
    tp.grad = torch.tensor(g[~z])
    opt.step()
    assert rel_err(p[~z], tp.detach().numpy()) < 1e-13


def test_softmax_xent_against_torch(orc):
    rng = np.random.default_rng(6)
    z = rng.normal(0, 3, (7, 33))
    p = rng.uniform(0, 1, (7, 33))
    p /= p.sum(1, keepdims=True)
    loss, g, q = orc.softmax_xent(z, p)
    zt = torch.tensor(z, requires_grad=True)
    lt = torch.nn.functional.cross_entropy(zt, torch.tensor(p), reduction="none")
    lt.sum().backward()
    assert rel_err(loss, lt.detach().numpy()) < 1e-13
    assert rel_err(g, zt.grad.numpy()) < 1e-12
    assert np.allclose(q.sum(1), 1.0)


def test_inverse_cdf_select_against_searchsorted(orc):
    rng = np.random.default_rng(7)
    R, K, n = 20, 512, 64
    q = rng.gamma(0.3, size=(R, K))
    q = (q / q.sum(1, keepdims=True)).astype(np.float32)
    sel, n_sel = orc.inverse_cdf_select(q, n)
    u = ((np.arange(n, dtype=np.float32) + np.float32(0.5)) / np.float32(n)).astype(np.float32)
    for r in range(R):
        cdf = np.cumsum(q[r], dtype=np.float32)   # sequential FP32 sums
        j = np.minimum(np.searchsorted(cdf, u, side="right"), K - 1)
        uj = np.unique(j)
        assert n_sel[r] == uj.size
        assert np.array_equal(sel[r, :n_sel[r]], uj)
        assert np.all(sel[r, n_sel[r]:] == -1)


def test_min_abs_preact_against_torch(orc):
    rng = np.random.default_rng(12)
    dims = synth.RGBNET_DIMS
    params = synth.mlp_params(dims).astype(np.float64)
    x = rng.normal(size=(20, dims[0]))
    got = orc.mlp_min_abs_preact(dims, params, x)
    p = torch.tensor(params)
    W1 = p[:128 * 39].view(128, 39)
    b1 = p[128 * 39:128 * 40]
    W2 = p[128 * 40:128 * 40 + 128 * 128].view(128, 128)
    b2 = p[128 * 40 + 128 * 128:128 * 40 + 128 * 129]
    z1 = torch.nn.functional.linear(torch.tensor(x), W1, b1)
    z2 = torch.nn.functional.linear(torch.relu(z1), W2, b2)
    ref = torch.minimum(z1.abs().min(1).values, z2.abs().min(1).values).numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)


def test_ragged_proposal_pieces_match_per_ray_dense(orc):
    rng = np.random.default_rng(14)
    counts = [0, 1, 7, 64, 300]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    z = rng.normal(0, 2, S)
    w = np.where(rng.uniform(size=S) < 0.3, rng.uniform(0, 1, S), 0.0)
    loss, g, q = orc.proposal_xent_ragged(z, w, off, 1e-3)
    for r, n in enumerate(counts):
        sl = slice(off[r], off[r + 1])
        if n == 0:
            assert loss[r] == 0
            continue
        W = w[sl].sum()
        p = (w[sl] / W + 1e-3) / (1 + n * 1e-3) if W > 0 else np.full(n, 1.0 / n)
        assert abs(p.sum() - 1) < 1e-12
        l1, g1, q1 = orc.softmax_xent(z[sl][None], p[None])
        assert loss[r] == pytest.approx(l1[0], rel=1e-12)
        assert np.allclose(g[sl], g1[0], atol=1e-14) and np.allclose(q[sl], q1[0], atol=1e-15)
        qq = q[sl].astype(np.float32)
        s1, n1 = orc.inverse_cdf_select(qq[None], 64)
        s_all, n_all = orc.inverse_cdf_select_ragged(q.astype(np.float32), off, 64)
        assert n_all[r] == n1[0] and np.array_equal(s_all[r], s1[0])
