"""Pins of the oracle's raw->alpha, compositing, trilinear interpolation and
occupancy mask (Sec. 1, Sec. 3 "Re-implement rendering utils") against
closed forms, invariants, finite differences and torch library routines."""
import numpy as np
import pytest
import torch

from conftest import rel_err

SHIFT_INIT = 1e-4


def test_raw_zero_closed_form(orc):
    shift = orc.alpha_shift(SHIFT_INIT)
    for interval in (0.25, 0.5, 1.0, 2.0):
        a, _ = orc.raw2alpha(np.zeros(1), shift, interval)
        assert a[0] == pytest.approx(1 - (1 - SHIFT_INIT) ** interval, rel=1e-12)


def test_alpha_against_torch_and_fd(orc):
    shift = orc.alpha_shift(SHIFT_INIT)
    raw = np.linspace(-30, 30, 601)
    a, da = orc.raw2alpha(raw, shift, 0.5)
    t = torch.tensor(raw, dtype=torch.float64, requires_grad=True)
    ta = 1 - torch.exp(-0.5 * torch.nn.functional.softplus(t + shift))
    ta.sum().backward()
    assert rel_err(a, ta.detach().numpy()) < 1e-12
    assert rel_err(da, t.grad.numpy()) < 1e-12
    h = 1e-6
    fd = (orc.raw2alpha(raw + h, shift, 0.5)[0] - orc.raw2alpha(raw - h, shift, 0.5)[0]) / (2 * h)
    assert rel_err(da, fd) < 1e-7


def test_mask_threshold_is_inverse_of_alpha(orc):
    # alpha(raw) >= thr  <=>  raw >= softplus^{-1}(-log(1 - thr)/interval) - shift
    shift = orc.alpha_shift(SHIFT_INIT)
    rng = np.random.default_rng(0)
    D = rng.uniform(-5, 5, (8, 9, 10)).astype(np.float32)
    m = orc.build_mask(D, shift, 0.5, 1e-4)
    raw_thr = np.log(np.expm1(-np.log1p(-1e-4) / 0.5)) - shift
    assert np.array_equal(m.astype(bool), D.astype(np.float64) >= raw_thr)


def _rays_samples(rng, counts):
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    return off, rng.normal(0, 3, S), rng.uniform(0, 1, (S, 3))


def test_weights_sum_to_one_minus_T(orc):
    rng = np.random.default_rng(1)
    off, raw, rgb = _rays_samples(rng, [0, 1, 5, 40, 128])
    for T_stop in (0.0, 1e-3):
        c = orc.composite(raw, rgb, off, orc.alpha_shift(SHIFT_INIT), 0.5, T_stop, 1.0)
        for r in range(len(off) - 1):
            sw = c["w"][off[r]:off[r + 1]].sum()
            assert sw == pytest.approx(1 - c["T_end"][r], abs=1e-14)
        assert c["T_end"][0] == 1.0
        assert np.allclose(c["color"][0], 1.0)


def test_transparent_gives_background_and_opaque_gives_colour(orc):
    off = np.array([0, 3, 4])
    rgb = np.array([[0.2, 0.4, 0.6], [0.9, 0.1, 0.3], [0.5, 0.5, 0.5], [0.7, 0.8, 0.9]])
    raw = np.array([-500.0, -500.0, -500.0, 500.0])
    bg = np.array([0.3, 0.6, 0.9])
    c = orc.composite(raw, rgb, off, orc.alpha_shift(SHIFT_INIT), 0.5, 1e-3, bg)
    assert np.allclose(c["color"][0], bg, atol=1e-15)
    assert np.allclose(c["color"][1], rgb[3], atol=1e-15)


def test_two_sample_closed_form(orc):
    shift = orc.alpha_shift(SHIFT_INIT)
    raw = np.array([8.5, 10.2])
    rgb = np.array([[0.1, 0.2, 0.3], [0.6, 0.5, 0.4]])
    bg = np.array([1.0, 0.5, 0.25])
    c = orc.composite(raw, rgb, np.array([0, 2]), shift, 0.5, 0.0, bg)
    a = orc.raw2alpha(raw, shift, 0.5)[0]
    expect = a[0] * rgb[0] + (1 - a[0]) * a[1] * rgb[1] + (1 - a[0]) * (1 - a[1]) * bg
    assert np.allclose(c["color"][0], expect, rtol=1e-14)


def test_halting_index(orc):
    # constant alpha per sample: T_i = (1 - a)^i, the ray halts at the first
    # i with T_i < 1e-3 and that sample is not composited.
    shift = orc.alpha_shift(SHIFT_INIT)
    raw = np.full(64, 9.0)
    a = orc.raw2alpha(raw[:1], shift, 0.5)[0][0]
    expect = int(np.ceil(np.log(1e-3) / np.log(1 - a)))
    c = orc.composite(raw, np.zeros((64, 3)), np.array([0, 64]), shift, 0.5, 1e-3, 0.0)
    assert c["n_live"][0] == expect
    assert np.all(c["w"][expect:] == 0)
    assert c["T_end"][0] == pytest.approx((1 - a) ** expect, rel=1e-12)


def test_composite_backward_fd(orc):
    shift = orc.alpha_shift(SHIFT_INIT)
    rng = np.random.default_rng(5)
    off, raw, rgb = _rays_samples(rng, [1, 6, 20])
    raw = raw + 9.0
    R = len(off) - 1
    bg = np.array([0.3, 0.2, 0.9])
    u = rng.normal(size=(R, 3))
    v = rng.normal(size=raw.size)

    def L(raw_, rgb_):
        c = orc.composite(raw_, rgb_, off, shift, 0.5, 0.0, bg)
        return np.sum(c["color"] * u) + np.dot(c["w"], v)

    g_raw, g_rgb = orc.composite_bwd(raw, rgb, off, shift, 0.5, 0.0, bg, u, v)
    h = 1e-6
    fd = np.zeros_like(raw)
    for k in range(raw.size):
        rp, rm = raw.copy(), raw.copy()
        rp[k] += h
        rm[k] -= h
        fd[k] = (L(rp, rgb) - L(rm, rgb)) / (2 * h)
    assert rel_err(g_raw, fd) < 1e-7
    fdc = np.zeros_like(rgb)
    for k in range(rgb.shape[0]):
        for ch in range(3):
            cp, cm = rgb.copy(), rgb.copy()
            cp[k, ch] += h
            cm[k, ch] -= h
            fdc[k, ch] = (L(raw, cp) - L(raw, cm)) / (2 * h)
    assert rel_err(g_rgb, fdc) < 1e-7


def test_composite_backward_dead_samples_zero(orc):
    shift = orc.alpha_shift(SHIFT_INIT)
    raw = np.full(40, 11.0)
    rgb = np.full((40, 3), 0.5)
    c = orc.composite(raw, rgb, np.array([0, 40]), shift, 0.5, 1e-3, 1.0)
    n = c["n_live"][0]
    assert 0 < n < 40
    g_raw, g_rgb = orc.composite_bwd(raw, rgb, np.array([0, 40]), shift, 0.5, 1e-3, 1.0,
                                     np.ones((1, 3)))
    assert np.all(g_raw[n:] == 0) and np.all(g_rgb[n:] == 0)
    assert np.all(g_raw[:n] != 0)


# ----------------------------- trilinear -----------------------------------
def _grid(rng, G, C):
    return rng.normal(size=(G[2], G[1], G[0], C)).astype(np.float32)


def test_trilinear_exact_at_corners(orc):
    rng = np.random.default_rng(0)
    G = (5, 6, 7)
    g = _grid(rng, G, 3)
    lo, hi = np.array([-1.0, -2.0, 0.5]), np.array([1.0, 1.0, 2.5])
    idx = np.stack(np.meshgrid(np.arange(G[0]), np.arange(G[1]), np.arange(G[2]),
                               indexing="ij"), -1).reshape(-1, 3)
    # grid points with an exactly representable world position: use lo/hi
    # where (hi - lo)/(G - 1) is exact in binary
    lo2, hi2 = np.array([0.0, 0.0, 0.0]), np.array([4.0, 5.0, 6.0])
    xyz = (idx * (hi2 - lo2) / (np.array(G) - 1)).astype(np.float32)
    out = orc.trilinear(g, lo2, hi2, xyz)
    ref = g[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert np.array_equal(out, ref.astype(np.float64))
    del lo, hi


def test_trilinear_exact_on_affine_field(orc):
    rng = np.random.default_rng(1)
    G = (9, 8, 7)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    ax = [np.linspace(lo[a], hi[a], G[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    g = (0.5 * X - 0.25 * Y + 0.125 * Z + 1.0).astype(np.float32)
    xyz = rng.uniform(-1, 1, (1000, 3)).astype(np.float32)
    out = orc.trilinear(g, lo, hi, xyz)[:, 0]
    gt = g.astype(np.float64)
    # compare with the affine function evaluated through the same stored
    # values: trilinear reproduces the affine interpolant of the stored grid.
    x = xyz.astype(np.float64)
    expect = 0.5 * x[:, 0] - 0.25 * x[:, 1] + 0.125 * x[:, 2] + 1.0
    assert np.max(np.abs(out - expect)) < 1e-6   # float32 grid storage
    del gt


def test_trilinear_adjoint_identity(orc):
    rng = np.random.default_rng(2)
    G = (6, 7, 8)
    C = 4
    g = _grid(rng, G, C)
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    xyz = rng.uniform(-1.1, 1.1, (500, 3)).astype(np.float32)
    y = rng.normal(size=(500, C))
    lhs = np.sum(orc.trilinear(g, lo, hi, xyz) * y)
    adj = orc.trilinear_adjoint(y, g.shape, lo, hi, xyz)
    rhs = np.sum(adj * g.astype(np.float64))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_trilinear_against_grid_sample(orc):
    rng = np.random.default_rng(3)
    G = (10, 11, 12)
    C = 5
    g = _grid(rng, G, C)
    lo, hi = np.array([-1.0, -2.0, -0.5]), np.array([1.0, 0.0, 1.5])
    xyz = (lo + (hi - lo) * rng.uniform(0, 1, (300, 3))).astype(np.float32)
    out = orc.trilinear(g, lo, hi, xyz)
    inp = torch.tensor(g, dtype=torch.float64).permute(3, 0, 1, 2)[None]
    nrm = 2 * (xyz.astype(np.float64) - lo) / (hi - lo) - 1
    grid = torch.tensor(nrm, dtype=torch.float64).view(1, 1, 1, -1, 3)
    ref = torch.nn.functional.grid_sample(inp, grid, mode="bilinear", align_corners=True)
    ref = ref.view(C, -1).T.numpy()
    assert rel_err(out, ref) < 1e-12


def test_per_sample_interval_equals_repeated_samples(orc):
    """A sample whose interval is k voxel steps absorbs exactly as k equal
    samples of one step each (1 - (1 - a)^k = 1 - exp(-k delta sigma)), so a
    ray of merged spans renders the colour of the ray of repeated samples."""
    shift = orc.alpha_shift(SHIFT_INIT)
    rng = np.random.default_rng(11)
    ks = np.array([1, 3, 1, 7, 2, 5])
    raw = rng.normal(8.0, 2.0, ks.size)
    rgb = rng.uniform(0, 1, (ks.size, 3))
    bg = np.array([0.2, 0.7, 0.4])
    merged = orc.composite(raw, rgb, np.array([0, ks.size]), shift, 0.5, 0.0, bg, delta=0.5 * ks)
    rep = orc.composite(np.repeat(raw, ks), np.repeat(rgb, ks, axis=0), np.array([0, ks.sum()]),
                        shift, 0.5, 0.0, bg)
    assert np.allclose(merged["color"], rep["color"], rtol=1e-13, atol=1e-15)
    assert merged["T_end"][0] == pytest.approx(rep["T_end"][0], rel=1e-12)
    # the weight of a merged span is the summed weight of its copies
    ends = np.cumsum(ks)
    assert np.allclose(merged["w"], np.add.reduceat(rep["w"], ends - ks), rtol=1e-12)
    # a uniform per-sample interval is the scalar interval
    same = orc.composite(raw, rgb, np.array([0, ks.size]), shift, 0.5, 0.0, bg,
                         delta=np.full(ks.size, 0.5))
    plain = orc.composite(raw, rgb, np.array([0, ks.size]), shift, 0.5, 0.0, bg)
    assert np.array_equal(same["color"], plain["color"])


def test_composite_backward_per_sample_interval_fd(orc):
    shift = orc.alpha_shift(SHIFT_INIT)
    rng = np.random.default_rng(12)
    off, raw, rgb = _rays_samples(rng, [1, 6, 20])
    raw = raw + 8.0
    R = len(off) - 1
    delta = rng.uniform(0.2, 4.0, raw.size)
    bg = np.array([0.3, 0.2, 0.9])
    u = rng.normal(size=(R, 3))
    v = rng.normal(size=raw.size)

    def L(raw_):
        c = orc.composite(raw_, rgb, off, shift, 0.5, 0.0, bg, delta=delta)
        return np.sum(c["color"] * u) + np.dot(c["w"], v)

    g_raw, _ = orc.composite_bwd(raw, rgb, off, shift, 0.5, 0.0, bg, u, v, delta=delta)
    h = 1e-6
    fd = np.zeros_like(raw)
    for k in range(raw.size):
        rp, rm = raw.copy(), raw.copy()
        rp[k] += h
        rm[k] -= h
        fd[k] = (L(rp) - L(rm)) / (2 * h)
    assert rel_err(g_raw, fd) < 1e-7
