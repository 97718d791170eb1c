"""GPU parity of the learned-proposal kernels against the FP64 oracle, and
what the trained proposal gains over drawing the same number of samples
without it."""
import numpy as np
import pytest
import torch

import oracle
from conftest import check_mlp_grads, rel_err
from paper_2206_05085_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2206_05085_gb300 import build
    build.build()
    from paper_2206_05085_gb300 import _lib
    _lib.lib()
    return _lib


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("n", [1, 200, 6000])
def test_proposal_network_fwd_bwd(L, n):
    rng = np.random.default_rng(20)
    xyz = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    params = (synth.proposal_params() * 1.5).astype(np.float32)
    p_ref = synth.bf16_round(params)
    idx = np.arange(0, n, 3 if n > 3 else 1).astype(np.int32)
    logits = torch.full((n,), -5.0, device="cuda")
    L.proposal_fwd(dev(xyz), dev(idx), len(idx), None, dev(params), logits)
    x = oracle.freq_encode(xyz[idx], 6)
    ref = oracle.mlp_fwd(synth.PROPOSAL_DIMS, p_ref, x, False)[:, 0]
    got = host(logits)
    assert rel_err(got[idx], ref) < 2e-3
    assert np.all(np.delete(got, idx) == -5.0)
    g = rng.normal(size=n).astype(np.float32)
    gp = torch.zeros(params.size, device="cuda")
    L.proposal_bwd(dev(g), dev(xyz), dev(idx), len(idx), None, dev(params), gp)
    check_mlp_grads(oracle, synth.PROPOSAL_DIMS, p_ref, x, g[idx][:, None], host(gp), None, 2e-3,
                    out_sigmoid=False, tau=2e-5)


def _ragged(seed, counts):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    z = rng.normal(0, 2.5, S).astype(np.float32)
    w = np.where(rng.uniform(size=S) < 0.2, rng.uniform(0, 1, S), 0.0).astype(np.float32)
    return off, z, w


COUNTS = [0, 1, 5, 31, 32, 33, 300, 512] + list(np.random.default_rng(21).integers(0, 513, 300))


def test_proposal_xent(L):
    off, z, w = _ragged(22, COUNTS)
    R = len(COUNTS)
    S = int(off[-1])
    loss = torch.empty(R, device="cuda")
    g = torch.empty(S, device="cuda")
    q = torch.empty(S, device="cuda")
    L.proposal_xent(dev(z), dev(w), dev(off), R, 1e-3, 0.5, loss, g, q)
    rl, rg, rq = oracle.proposal_xent_ragged(z, w, off, 1e-3)
    assert rel_err(host(loss), rl) < 1e-5
    assert rel_err(host(g), 0.5 * rg) < 1e-5
    assert rel_err(host(q), rq) < 1e-5
    q2 = torch.empty(S, device="cuda")
    L.proposal_xent(dev(z), None, dev(off), R, 0.0, 0.0, None, None, q2)
    assert rel_err(host(q2), rq) < 1e-5


def test_proposal_select_and_compact_bit_exact(L):
    off, z, w = _ragged(23, COUNTS)
    R = len(COUNTS)
    _, _, q = oracle.proposal_xent_ragged(z, w, off, 1e-3)
    q32 = q.astype(np.float32)
    sel = torch.empty(R * 64, dtype=torch.int32, device="cuda")
    n_sel = torch.empty(R, dtype=torch.int32, device="cuda")
    L.proposal_select(dev(q32), dev(off), R, 64, sel, n_sel)
    rs, rn = oracle.inverse_cdf_select_ragged(q32, off, 64)
    assert np.array_equal(host(n_sel), rn)
    assert np.array_equal(host(sel).reshape(R, 64), rs)
    # compaction of the picked samples
    S = int(off[-1])
    rng = np.random.default_rng(24)
    xyz = rng.normal(size=(S, 3)).astype(np.float32)
    rid = np.repeat(np.arange(R), COUNTS).astype(np.int32)
    sk = rng.integers(0, 1000, S).astype(np.int32)
    sm = rng.uniform(size=S).astype(np.float32)
    sl = rng.uniform(size=S).astype(np.float32)
    n_out = int(rn.sum())
    outs = dict(off=torch.zeros(R + 1, dtype=torch.int64, device="cuda"),
                xyz=torch.empty(n_out, 3, device="cuda"),
                rid=torch.empty(n_out, dtype=torch.int32, device="cuda"),
                sk=torch.empty(n_out, dtype=torch.int32, device="cuda"),
                sm=torch.empty(n_out, device="cuda"), sl=torch.empty(n_out, device="cuda"),
                src=torch.empty(n_out, dtype=torch.int32, device="cuda"))
    L.compact_samples(sel, n_sel, 64, dev(off), R, dev(xyz), dev(rid), dev(sk), dev(sm), dev(sl),
                      outs["off"], outs["xyz"], outs["rid"], outs["sk"], outs["sm"], outs["sl"],
                      outs["src"])
    src = np.concatenate([off[r] + rs[r, :rn[r]] for r in range(R)]).astype(np.int64)
    assert np.array_equal(host(outs["off"]), np.concatenate([[0], np.cumsum(rn)]))
    assert np.array_equal(host(outs["src"]), src)
    assert np.array_equal(host(outs["xyz"]), xyz[src])
    assert np.array_equal(host(outs["rid"]), rid[src])
    assert np.array_equal(host(outs["sk"]), sk[src])
    assert np.array_equal(host(outs["sm"]), sm[src]) and np.array_equal(host(outs["sl"]), sl[src])


def test_trained_proposal_beats_uniform_draws():
    """After training on the plain renderer's weights, 64 proposal-drawn
    samples per ray (each standing for the candidates up to the next pick)
    reproduce the dense (<= 512 samples) render better than 64 evenly spaced
    picks, far better than the same picks without their spans, and score
    within 0.1 dB of the dense render's PSNR against the held-out truth
    scene."""
    from paper_2206_05085_gb300 import build, proposal, train
    build.build()
    cfg = synth.CFG5
    rp = synth.render_params(cfg)
    R = 4096
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    dense, prop_tr, prop = proposal.make_forms(cfg, rp, D, Fg, P, synth.proposal_params(), R)
    losses = []
    for it in range(600):
        o, d = synth.rays(cfg, seed=100 + it, n_rays=R)
        lr = prop.train_step(dev(o), dev(d))
        if it == 0 or it == 599:
            losses.append(host(lr))
    # the smallest reachable cross-entropy is the entropy of the target itself
    w, off = host(prop.w), host(prop.ray_off)
    ent = np.zeros(R)
    for r in range(R):
        ww = w[off[r]:off[r + 1]].astype(np.float64)
        N = len(ww)
        if N == 0:
            continue
        W = ww.sum()
        p = (ww / W + 1e-3) / (1 + N * 1e-3) if W > 0 else np.full(N, 1.0 / N)
        ent[r] = -np.sum(p * np.log(p))
    L0, L1, H = float(losses[0].mean()), float(losses[1].mean()), float(ent.mean())
    print(f"cross-entropy first {L0:.3f} last {L1:.3f} target entropy {H:.3f}")
    assert L1 - H < 0.6 * (L0 - H)
    o, d = synth.rays(cfg, seed=7, n_rays=R)
    t = synth.target_rgb(cfg, seed=7, n_rays=R)
    to, td, tt = dev(o), dev(d), dev(t)
    dense.forward(to, td, tt)
    c_dense = dense.color.clone()
    renders = {}
    for name, kw in (("prop", {}), ("uniform", dict(uniform=True)), ("no_spans", dict(spans=False))):
        prop.select_into(prop_tr, to, td, **kw)
        prop_tr.forward(to, td, tt, sample=False)
        renders[name] = prop_tr.color.clone()
    n_prop = int(prop_tr.ray_off[-1].item())
    vs_dense = {k: proposal.psnr(c, c_dense) for k, c in renders.items()}
    truth = train.heldout_truth_render(cfg, proposal.candidate_params(cfg, rp), D, Fg, P, to, td, tt)
    p_dense = proposal.psnr(c_dense, truth)
    gap = abs(proposal.psnr(renders["prop"], truth) - p_dense)
    print(f"vs dense: proposal {vs_dense['prop']:.2f} dB, uniform {vs_dense['uniform']:.2f} dB, "
          f"without spans {vs_dense['no_spans']:.2f} dB; dense vs truth {p_dense:.2f} dB, "
          f"proposal gap {gap:.4f} dB; samples {n_prop} vs {int(dense.ray_off[-1].item())}")
    assert vs_dense["prop"] > vs_dense["uniform"] + 1.0
    assert vs_dense["prop"] > vs_dense["no_spans"] + 15.0
    assert 30.0 < p_dense < 36.0
    assert gap <= 0.1


def test_compact_spans_cover_the_candidates(L):
    """With out_delta, each pick stands for the candidates from itself up to
    the next pick (the last pick: up to the ray's last candidate): its alpha
    interval is interval x the gap, its distortion span runs from its own
    start to the next pick's start, bit-exact in FP32; the spans of a ray
    tile [first pick start, last candidate end] without overlap."""
    off, z, w = _ragged(25, COUNTS)
    R = len(COUNTS)
    S = int(off[-1])
    _, _, q = oracle.proposal_xent_ragged(z, w, off, 1e-3)
    q32 = q.astype(np.float32)
    sel = torch.empty(R * 64, dtype=torch.int32, device="cuda")
    n_sel = torch.empty(R, dtype=torch.int32, device="cuda")
    L.proposal_select(dev(q32), dev(off), R, 64, sel, n_sel)
    rs, rn = oracle.inverse_cdf_select_ragged(q32, off, 64)
    # contiguous candidate spans of uneven length per ray
    rng = np.random.default_rng(26)
    sl = np.zeros(S, np.float32)
    sm = np.zeros(S, np.float32)
    for r in range(R):
        n = int(off[r + 1] - off[r])
        if n:
            step = np.float32(rng.uniform(0.001, 0.01))
            k = np.arange(n, dtype=np.float32)
            sm[off[r]:off[r + 1]] = (k + np.float32(0.5)) * step
            sl[off[r]:off[r + 1]] = step
    xyz = rng.normal(size=(S, 3)).astype(np.float32)
    rid = np.repeat(np.arange(R), COUNTS).astype(np.int32)
    sk = np.arange(S, dtype=np.int32)
    n_out = int(rn.sum())
    o_off = torch.zeros(R + 1, dtype=torch.int64, device="cuda")
    o_xyz = torch.empty(n_out, 3, device="cuda")
    o_rid, o_sk = (torch.empty(n_out, dtype=torch.int32, device="cuda") for _ in range(2))
    o_sm, o_sl, o_dl = (torch.empty(n_out, device="cuda") for _ in range(3))
    interval = np.float32(0.37)
    L.compact_samples(sel, n_sel, 64, dev(off), R, dev(xyz), dev(rid), dev(sk), dev(sm), dev(sl),
                      o_off, o_xyz, o_rid, o_sk, o_sm, o_sl, interval=float(interval), out_delta=o_dl)
    e_sm, e_sl, e_dl = [], [], []
    half = np.float32(0.5)
    for r in range(R):
        n_c = int(off[r + 1] - off[r])
        picks = rs[r, :rn[r]]
        for i, j in enumerate(picks):
            jn = picks[i + 1] if i + 1 < len(picks) else n_c
            a = off[r] + j
            start = np.float32(sm[a] - np.float32(half * sl[a]))
            if jn < n_c:
                b = off[r] + jn
                end = np.float32(sm[b] - np.float32(half * sl[b]))
            else:
                b = off[r] + n_c - 1
                end = np.float32(sm[b] + np.float32(half * sl[b]))
            e_sm.append(np.float32(half * np.float32(start + end)))
            e_sl.append(np.float32(end - start))
            e_dl.append(np.float32(interval * np.float32(jn - j)))
    assert np.array_equal(host(o_sm), np.array(e_sm, np.float32))
    assert np.array_equal(host(o_sl), np.array(e_sl, np.float32))
    assert np.array_equal(host(o_dl), np.array(e_dl, np.float32))
    # per ray the intervals add up to the candidates from the first pick to the end
    dl, ro = host(o_dl).astype(np.float64), host(o_off)
    for r in range(R):
        if rn[r]:
            gap = int(off[r + 1] - off[r]) - int(rs[r, 0])
            assert np.sum(dl[ro[r]:ro[r + 1]]) == pytest.approx(float(interval) * gap, rel=1e-6)
    src = np.concatenate([off[r] + rs[r, :rn[r]] for r in range(R)]).astype(np.int64)
    assert np.array_equal(host(o_xyz), xyz[src]) and np.array_equal(host(o_sk), sk[src])
