"""Pins of the oracle's distortion loss (Sec. 2, Eq. dist_loss and its O(N)
rewrite and derivative) against brute force, closed forms and finite
differences."""
import os

import numpy as np
import pytest

from conftest import rel_err

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "distortion_closed_forms.txt")


def _ragged(rng, counts):
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    w = rng.uniform(0, 1, S)
    m = np.zeros(S)
    ds = rng.uniform(0.001, 0.05, S)
    for r in range(len(counts)):
        b, e = off[r], off[r + 1]
        m[b:e] = np.sort(rng.uniform(0, 1, e - b))
    return off, w, m, ds


def test_linear_form_equals_double_sum(orc):
    rng = np.random.default_rng(1)
    counts = [0, 1, 2, 3, 7, 31, 32, 33, 64]
    off, w, m, ds = _ragged(rng, counts)
    a = orc.distortion(w, m, ds, off)
    b = orc.distortion_naive(w, m, ds, off)
    assert rel_err(a, b) < 1e-13
    assert a[0] == 0.0


def test_closed_forms(orc):
    # N = 1: L = w^2 ds / 3;  N = 2: L = 2 w0 w1 (m1 - m0) + (w0^2 ds0 + w1^2 ds1)/3
    w = np.array([0.7, 0.3, 0.9])
    m = np.array([0.5, 0.2, 0.6])
    ds = np.array([0.1, 0.05, 0.02])
    off = np.array([0, 1, 3])
    L = orc.distortion(w, m, ds, off)
    assert L[0] == pytest.approx(0.7 ** 2 * 0.1 / 3, rel=1e-14)
    assert L[1] == pytest.approx(2 * 0.3 * 0.9 * 0.4 + (0.09 * 0.05 + 0.81 * 0.02) / 3, rel=1e-14)


def test_golden_hand_values(orc):
    # Hand-evaluated instances of Eq. (dist_loss); see the fixture's header.
    from fractions import Fraction
    for ln in open(GOLDEN):
        if not ln.strip() or ln.startswith("#"):
            continue
        cols = [c.split() for c in ln.split("|")]
        n = int(cols[0][0])
        w, m, ds = (np.array([float(Fraction(v)) for v in c]) for c in cols[1:4])
        assert len(w) == len(m) == len(ds) == n
        expect = float(Fraction(cols[4][0]))
        L = orc.distortion(w, m, ds, np.array([0, n]))
        assert L[0] == pytest.approx(expect, rel=1e-12, abs=1e-15)


def test_gradient_matches_fd_and_direct(orc):
    rng = np.random.default_rng(2)
    off, w, m, ds = _ragged(rng, [5, 17, 40])
    gL = np.array([1.0, 0.5, 2.0])
    g = orc.distortion_grad(gL, w, m, ds, off)
    g2 = orc.distortion_grad_naive(gL, w, m, ds, off)
    assert rel_err(g, g2) < 1e-12
    h = 1e-6
    fd = np.zeros_like(w)
    for k in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd[k] = (np.dot(gL, orc.distortion_naive(wp, m, ds, off)) -
                 np.dot(gL, orc.distortion_naive(wm, m, ds, off))) / (2 * h)
    assert rel_err(g, fd) < 1e-7


def test_printed_third_term_reading(orc):
    # The paper's last derivative line prints the third term as
    # 2 sum_{i>k} w_i m_j.  Reading it as m_i (the line above it) agrees with
    # finite differences; reading m_j as m_k (the only free index) does not.
    rng = np.random.default_rng(3)
    off, w, m, ds = _ragged(rng, [12])
    g = orc.distortion_grad(1.0, w, m, ds, off)
    N = w.size
    alt = np.zeros(N)
    for k in range(N):
        Wl, WMl = w[:k].sum(), (w[:k] * m[:k]).sum()
        Wg = w[k + 1:].sum()
        alt[k] = 2 * (m[k] * Wl - WMl + m[k] * Wg - m[k] * Wg) + 2 / 3 * w[k] * ds[k]
    fd = orc.distortion_grad_naive(1.0, w, m, ds, off)
    assert rel_err(g, fd) < 1e-12
    assert rel_err(alt, fd) > 1e-2


def test_segment_length_truncates(orc):
    rng = np.random.default_rng(4)
    off, w, m, ds = _ragged(rng, [10, 0, 6])
    seg = np.array([4, 0, 6], np.int32)
    L = orc.distortion(w, m, ds, off, seg)
    w2 = w.copy()
    w2[4:10] = 0.0
    assert rel_err(L, orc.distortion(w2, m, ds, off)) < 1e-14
    g = orc.distortion_grad(1.0, w, m, ds, off, seg)
    assert np.all(g[4:10] == 0.0)
