"""Pins of the oracle's ray samplers: bbox-limited sampling (Sec. 3
"Re-implement rendering utils") with occupancy culling (Sec. 1), and the
contracted-space sampling of unbounded scenes (Sec. 5.4, Eq. ub), and
the depth-layer sampling of forward-facing scenes (Sec. 5.3)."""
import numpy as np
import pytest

from paper_2206_05085_gb300 import synth


def test_axis_aligned_slab_closed_form(orc):
    # rays along +x / -x through the box [-1,1]^3 from |x| = 4: t_in = 3,
    # t_out = 5, n = ceil(2 / step).
    step = np.float32(0.5 * 2 / 159)
    o = np.array([[-4, 0.1, -0.2], [4, 0.3, 0.7], [-4, 1.5, 0.0], [0.2, -0.3, 0.9]], np.float32)
    d = np.array([[1, 0, 0], [-1, 0, 0], [1, 0, 0], [0, 0, -1]], np.float32)
    s = orc.sample_rays_bbox(o, d, -1, 1, 160, 0.0, 1e4, step, 0.0, True, 1024)
    # the count is an FP32 decision: ceil(fl32(fl32(t_out - t_in) / step))
    n = int(np.ceil(np.float32(2.0) / step))
    cnt = np.diff(s.ray_off)
    assert cnt[0] == n and cnt[1] == n
    assert cnt[2] == 0                      # misses the box
    # origin inside the box going -z: t from 0 to 1.9
    assert cnt[3] == int(np.ceil((np.float32(-1.0) - np.float32(0.9)) / np.float32(-1.0) / step))
    k = s.step_k[:n]
    assert np.array_equal(k, np.arange(n))
    assert np.allclose(s.xyz[:n, 0], -1 + k * float(step), atol=1e-6)
    assert np.allclose(s.s_mid[:n], k * float(step) / 2.0, rtol=1e-6)


def test_fixed_near_far_midpoints(orc):
    cfg = synth.CFG1
    o, d = synth.rays(cfg, n_rays=64)
    rp = synth.render_params(cfg)
    s = orc.sample_rays_bbox(o, d, cfg.bbox_min, cfg.bbox_max, cfg.grid, rp.near, rp.far,
                             rp.step, rp.step_offset, False, rp.max_steps)
    # brute force in FP64: t_k = 2 + (k + 0.5)/32, kept iff inside the box.
    # Points within 1e-5 of a face may go either way between FP32 and FP64.
    for r in range(64):
        got = set(s.step_k[s.ray_off[r]:s.ray_off[r + 1]].tolist())
        for k in range(128):
            t = 2.0 + (k + 0.5) * 4.0 / 128
            x = o[r].astype(np.float64) + t * d[r].astype(np.float64)
            margin = np.min(np.minimum(x - cfg.bbox_min, cfg.bbox_max - x))
            if abs(margin) < 1e-5:
                continue
            assert (k in got) == (margin > 0)
    ks = s.s_mid
    assert np.allclose(ks, (s.step_k + 0.5) / 128, rtol=1e-12)
    assert np.allclose(s.s_len, 1 / 128)


def test_mask_culling_nearest_voxel(orc):
    rng = np.random.default_rng(0)
    G = 24
    mask = (rng.uniform(size=(G, G, G)) < 0.4).astype(np.uint8)
    cfg = synth.CFG2
    o, d = synth.rays(cfg, n_rays=200)
    step = np.float32(0.5 * 2 / (G - 1))
    full = orc.sample_rays_bbox(o, d, -1, 1, G, 0.0, 1e4, step, 0.0, True, 200)
    cull = orc.sample_rays_bbox(o, d, -1, 1, G, 0.0, 1e4, step, 0.0, True, 200, mask)
    assert cull.S < full.S
    kept = set(zip(cull.ray_id.tolist(), cull.step_k.tolist()))
    amb = 0
    for i in range(full.S):
        u = (full.xyz[i].astype(np.float64) + 1.0) / 2.0 * (G - 1)
        frac = u - np.floor(u)
        if np.any(np.abs(frac - 0.5) < 1e-4):
            amb += 1
            continue
        n = np.clip(np.floor(u + 0.5).astype(int), 0, G - 1)
        on = mask[n[2], n[1], n[0]] != 0
        assert ((int(full.ray_id[i]), int(full.step_k[i])) in kept) == on
    assert amb < full.S // 100
    # every ray's surviving step indices are increasing, distances increasing
    for r in range(200):
        sl = slice(cull.ray_off[r], cull.ray_off[r + 1])
        assert np.all(np.diff(cull.step_k[sl]) > 0)
        assert np.all(np.diff(cull.s_mid[sl]) > 0)


def test_contraction_properties(orc):
    rng = np.random.default_rng(1)
    for p_inf in (0, 1):
        x = rng.uniform(-1, 1, (200, 3))
        nrm = np.max(np.abs(x), 1) if p_inf else np.linalg.norm(x, axis=1)
        x = x[nrm <= 1]
        assert np.array_equal(orc.contract(x, 1.0, p_inf), x)       # identity inside
        far = rng.normal(size=(50, 3)) * 1e9
        c = orc.contract(far, 1.0, p_inf)
        cn = np.max(np.abs(c), 1) if p_inf else np.linalg.norm(c, axis=1)
        assert np.allclose(cn, 2.0, atol=1e-8)                       # limit 1 + b
        u = rng.normal(size=(50, 3))
        un = np.max(np.abs(u), 1, keepdims=True) if p_inf else np.linalg.norm(u, axis=1, keepdims=True)
        u = u / un
        a = orc.contract(u * (1 + 1e-9), 1.0, p_inf)
        assert np.allclose(a, u, atol=1e-8)                          # continuous at 1
        ts = np.linspace(1.0, 50.0, 200)
        for v in u[:5]:
            cc = orc.contract(ts[:, None] * v[None], 1.0, p_inf)
            ccn = np.max(np.abs(cc), 1) if p_inf else np.linalg.norm(cc, axis=1)
            assert np.all(np.diff(ccn) > 0)                          # monotone


@pytest.mark.parametrize("p_inf", [0, 1])
def test_contracted_step_is_constant_in_contracted_space(orc, p_inf):
    # consecutive contracted samples are step_c apart to first order
    cfg = synth.CFG3
    o, d = synth.rays(cfg, n_rays=32)
    step_c = np.float32(0.5 * 4 / 319)
    s = orc.sample_rays_contracted(o, d, 1.0, p_inf, 0.0, step_c, 512, -2, 2, 320)
    for r in range(32):
        sl = slice(s.ray_off[r], s.ray_off[r + 1])
        x = s.xyz[sl].astype(np.float64)
        assert x.shape[0] > 100
        gaps = np.linalg.norm(np.diff(x, axis=0), axis=1)
        cn = np.max(np.abs(x), 1)
        pn = cn if p_inf else np.linalg.norm(x, axis=1)
        # first order: exact inside the unit ball, within a few percent while
        # the world step stays small against the radius (contracted radius
        # below 1.7); near 1 + b the march's chords shorten (curvature).
        inner = pn[1:] < 1.0
        assert np.all(np.abs(gaps[inner] / float(step_c) - 1) < 1e-4)
        mid = pn[:-1] < 1.7
        off = np.abs(gaps[mid] / float(step_c) - 1) >= 0.05
        # p = inf: the contraction has a kink where the largest axis changes;
        # the one step across it is not first-order accurate.
        assert off.sum() <= (2 if p_inf else 0), (r, gaps[mid].min())
        assert np.all(gaps > 0.5 * float(step_c))
        assert np.all(pn < 2.0 - float(step_c) + 1e-6)
        assert np.array_equal(s.step_k[sl], np.arange(x.shape[0]))
        # the march follows the contraction of a straight world ray
        if p_inf:
            assert np.all(cn <= 2.0)


# ------------------------------------------------ forward-facing (NDC) sampling
def _ndc_cfg():
    import dataclasses
    cfg = dataclasses.replace(synth.CFG6, dims=(48, 40, 32), grid=48)
    return cfg, synth.render_params(cfg)


def _ndc_sample(orc, cfg, rp, o, d, mask=None):
    return orc.sample_rays_ndc(o, d, cfg.bbox_min, cfg.bbox_max, synth.grid_dims(cfg), rp.ndc_fx,
                               rp.ndc_fy, rp.ndc_near, rp.step, rp.max_steps, mask)


def test_ndc_samples_lie_on_the_world_ray(orc):
    """Mapping every sample back to world space (the inverse of the NDC warp,
    written from the pinhole projection: world depth z = 2 near/(z' - 1),
    x = -x' z / fx, y = -y' z / fy) gives points on the original ray, at
    increasing depth."""
    cfg, rp = _ndc_cfg()
    o, d = synth.rays(cfg, n_rays=300)
    s = _ndc_sample(orc, cfg, rp, o, d)
    assert s.S > 1000
    for r in range(300):
        a, b = s.ray_off[r], s.ray_off[r + 1]
        if b == a:
            continue
        p = s.xyz[a:b].astype(np.float64)
        inf = p[:, 2] == 1.0          # the last layer is the plane at infinity: the vanishing point
        if inf.any():
            van = [-rp.ndc_fx * d[r, 0] / d[r, 2], -rp.ndc_fy * d[r, 1] / d[r, 2]]
            assert np.allclose(p[inf, :2], van, atol=1e-5)
            p = p[~inf]
        zw = 2.0 * rp.ndc_near / (p[:, 2] - 1.0)
        xw = -p[:, 0] * zw / rp.ndc_fx
        yw = -p[:, 1] * zw / rp.ndc_fy
        w = np.stack([xw, yw, zw], 1)
        ro, rd = o[r].astype(np.float64), d[r].astype(np.float64)
        v = w - ro
        off_line = np.linalg.norm(v - (v @ rd)[:, None] * rd, axis=1)
        assert np.all(off_line <= 1e-4 * np.abs(zw)), (r, off_line.max())
        assert np.all(np.diff(zw) < 0)            # further down -z, layer after layer
        assert np.all(np.diff(s.step_k[a:b]) > 0)
    assert s.S > 0


def test_ndc_central_ray_crosses_every_layer(orc):
    cfg, rp = _ndc_cfg()
    Gz = synth.grid_dims(cfg)[2]
    o = np.zeros((2, 3), np.float32)
    d = np.array([[0, 0, -1], [0, 0, 1]], np.float32)      # the second looks away: no samples
    s = _ndc_sample(orc, cfg, rp, o, d)
    assert np.diff(s.ray_off).tolist() == [Gz, 0]
    assert np.array_equal(s.step_k, np.arange(Gz))
    assert np.all(s.xyz[:, :2] == 0)
    dz = np.float32(np.float32(2.0) / np.float32(Gz - 1))
    z = (np.float32(-1.0) + (np.arange(Gz).astype(np.float32) * np.float32(rp.step)) * dz).astype(np.float32)
    assert np.array_equal(s.xyz[:, 2], z)
    assert s.xyz[0, 2] == -1.0                      # the near plane maps to z' = -1
    assert np.allclose(s.s_mid, (np.arange(Gz) + 0.5) / Gz) and np.allclose(s.s_len, 1.0 / Gz)


def test_ndc_box_and_mask_culling(orc):
    """Crossings outside the box are dropped; with a mask, exactly those whose
    nearest grid point (FP64, ties excluded) has the mask on are kept."""
    cfg, rp = _ndc_cfg()
    G = synth.grid_dims(cfg)
    o, d = synth.rays(cfg, n_rays=200)
    # widen the field of view beyond the image so that some crossings leave the box
    d = d.copy()
    d[:, :2] *= 1.6
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d.astype(np.float32)
    full = _ndc_sample(orc, cfg, rp, o, d)
    assert np.all(np.abs(full.xyz) <= 1.0)
    assert np.sum(np.diff(full.ray_off) < G[2]) > 20
    rng = np.random.default_rng(5)
    mask = (rng.uniform(size=(G[2], G[1], G[0])) < 0.5).astype(np.uint8)
    cut = _ndc_sample(orc, cfg, rp, o, d, mask)
    u = (full.xyz.astype(np.float64) + 1.0) / 2.0 * (np.array(G) - 1)
    near = np.floor(u + 0.5).astype(int)
    tie = np.any(np.abs(u - np.round(u) - 0.5 * np.sign(u - np.round(u))) < 1e-4, axis=1) & \
        np.any(np.abs(np.abs(u - np.floor(u)) - 0.5) < 1e-4, axis=1)
    on = mask[near[:, 2], near[:, 1], near[:, 0]] == 1
    keep_full = set()
    for r in range(200):
        for i in range(full.ray_off[r], full.ray_off[r + 1]):
            if on[i] and not tie[i]:
                keep_full.add((r, int(full.step_k[i])))
    got = set()
    for r in range(200):
        for i in range(cut.ray_off[r], cut.ray_off[r + 1]):
            got.add((r, int(cut.step_k[i])))
    amb = {(r, int(full.step_k[i])) for r in range(200) for i in range(full.ray_off[r], full.ray_off[r + 1])
           if tie[i]}
    assert keep_full <= got and got - keep_full <= amb
