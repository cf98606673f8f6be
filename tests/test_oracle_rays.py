"""Pins of the oracle's other ray families and two-pass sampling (Sec. 3.5.1,
3.5.2): the segment geometry of V2V, V2E and W2W rays (vertices, antipodes,
edge midpoints, opposing faces), the Philox streams they draw from, uniform
face points, and the likelihood-proportional refinement pass against the
inverse CDF of its piecewise-constant density and against the quantiles of a
Gaussian along the ray."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import ndtri

import oracle
from paper_2601_19957_gb300.instances import make_instance


def _box(d, seed=1):
    inst = make_instance(d, 1, seed, s_range=(1.0, 1.0))
    rng = np.random.default_rng(seed)
    inst.lo = -rng.uniform(1.0, 5.0, d)
    inst.hi = rng.uniform(1.0, 5.0, d)
    return inst


def _stream_bit(seed, r, tag, purpose, b):
    o = oracle.philox4x32_10([b // 128, r, tag, purpose], [seed & 0xFFFFFFFF, seed >> 32])
    return (o[(b // 32) % 4] >> (b % 32)) & 1


def test_v2v_rays_join_distinct_vertices_from_their_bit_streams():
    d = 7
    inst = _box(d)
    seed = 0xABCDEF0123
    for r in range(40):
        a, b = oracle.ray_segment(inst, oracle.RAY_V2V, seed, r)
        assert np.all((a == inst.lo) | (a == inst.hi)) and np.all((b == inst.lo) | (b == inst.hi))
        assert np.any(a != b)
        bits = [_stream_bit(seed, r, 0x56325620, 0, i) for i in range(d)]
        np.testing.assert_array_equal(a, np.where(bits, inst.hi, inst.lo))
    # d = 1: two vertices only; a coinciding end becomes the antipode
    one = _box(1)
    for r in range(20):
        a, b = oracle.ray_segment(one, oracle.RAY_V2V, 5, r)
        assert {a[0], b[0]} == {one.lo[0], one.hi[0]}


def test_v2v_vertex_bits_are_fair_over_many_rays_and_dimensions():
    d = 130  # spans two Philox blocks of bits
    inst = _box(d, 3)
    hits = np.zeros(d)
    for r in range(400):
        a, _ = oracle.ray_segment(inst, oracle.RAY_V2V, 11, r)
        hits += a == inst.hi
    p = hits / 400
    assert np.abs(p - 0.5).max() < 0.1
    assert abs(p.mean() - 0.5) < 0.01


def test_v2e_rays_end_at_an_edge_midpoint():
    d = 6
    inst = _box(d, 4)
    c = 0.5 * (inst.lo + inst.hi)
    free = []
    for r in range(300):
        a, b = oracle.ray_segment(inst, oracle.RAY_V2E, 7, r)
        assert np.all((a == inst.lo) | (a == inst.hi))
        mid = b == c
        assert mid.sum() == 1 and np.all((b[~mid] == inst.lo[~mid]) | (b[~mid] == inst.hi[~mid]))
        free.append(int(np.flatnonzero(mid)[0]))
    counts = np.bincount(free, minlength=d)
    assert stats.chisquare(counts).pvalue > 1e-3


def test_w2w_rays_join_opposing_faces_with_uniform_points():
    d = 5
    inst = _box(d, 6)
    axes, us = [], []
    for r in range(2000):
        a, b = oracle.ray_segment(inst, oracle.RAY_W2W, 13, r)
        ax = np.flatnonzero((a == inst.lo) & (b == inst.hi))
        assert len(ax) >= 1
        i = int(ax[0])
        axes.append(i)
        others = np.arange(d) != i
        us.extend(((a - inst.lo) / (inst.hi - inst.lo))[others])
        us.extend(((b - inst.lo) / (inst.hi - inst.lo))[others])
    assert stats.chisquare(np.bincount(axes, minlength=d)).pvalue > 1e-3
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    with pytest.raises(ValueError):
        oracle.ray_segment(inst, 9, 1, 0)


def _line_gaussian(sig=0.05, mu=0.3):
    """1-d Gaussian on [0, 1]: the segment from 0 to 1 has l(t) = l(x = t)."""
    inst = make_instance(1, 1, 1, s_range=(1.0, 1.0), prior=(0.0, 1.0))
    inst.L[0] = 1.0 / sig
    inst.mu[0] = mu
    return inst


def test_refinement_is_the_inverse_cdf_of_the_piecewise_density():
    inst = _line_gaussian()
    n, n_ref, delta = 41, 64, 6.0
    lc, t, lr = oracle.ray_two_pass(inst, [0.0], [1.0], n, delta, n_ref)
    tc = np.arange(n) / (n - 1)
    np.testing.assert_allclose(lc, [oracle.loglik(inst, [x]) for x in tc], rtol=0, atol=0)
    h = 1 / (n - 1)
    lo_c, hi_c = np.clip(tc - h / 2, 0, 1), np.clip(tc + h / 2, 0, 1)
    w = np.where(lc > lc.max() - delta, np.exp(lc - lc.max()) * (hi_c - lo_c), 0.0)
    cdf = np.concatenate([[0.0], np.cumsum(w)])
    for k in range(n_ref):
        u = (k + 0.5) / n_ref * cdf[-1]
        j = int(np.searchsorted(cdf, u, side="right") - 1)
        expect = lo_c[j] + (u - cdf[j]) / w[j] * (hi_c[j] - lo_c[j])
        assert t[k] == pytest.approx(expect, abs=1e-12)
        assert w[j] > 0  # inside the active region
    assert np.all(np.diff(t) > 0)
    np.testing.assert_allclose(lr, [oracle.loglik(inst, [x]) for x in t], rtol=1e-15)


def test_refinement_follows_the_gaussian_quantiles_on_a_fine_grid():
    sig, mu = 0.05, 0.3
    inst = _line_gaussian(sig, mu)
    _, t, _ = oracle.ray_two_pass(inst, [0.0], [1.0], 2001, 50.0, 100)
    q = mu + sig * ndtri((np.arange(100) + 0.5) / 100)
    assert np.abs(t - q).max() < 2e-3
    # a tiny delta keeps only the best cell
    _, t1, _ = oracle.ray_two_pass(inst, [0.0], [1.0], 11, 1e-9, 5)
    assert np.all(np.abs(t1 - 0.3) <= 0.05 + 1e-15)
    # one coarse sample: its cell is the whole segment
    _, t2, _ = oracle.ray_two_pass(inst, [0.0], [1.0], 1, 1.0, 4)
    np.testing.assert_allclose(t2, [0.125, 0.375, 0.625, 0.875])
