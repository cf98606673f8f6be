"""Pins of the oracle's preprocessing (Sec. 3.4): the sensitivity probe against
its closed form on a Gaussian and against scipy log-densities on a mixture, the
flat / soft-nuisance thresholds against a brute-force classification (including
the even-count median), and the marginal terms against the exact evidence of a
separable Gaussian whose flagged coordinates are integrated out in closed form."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import logsumexp, ndtr

import oracle
from paper_2601_19957_gb300.instances import SolveConfig, make_instance


def _diag_instance(sig, prior=(-10.0, 10.0), mu=None, log_w=0.0):
    d = len(sig)
    inst = make_instance(d, 1, 1, s_range=(1.0, 1.0), prior=prior)
    inst.L[0] = np.diag(1.0 / np.asarray(sig, dtype=float))
    inst.mu[0] = 0.5 * (inst.lo + inst.hi) if mu is None else mu
    inst.log_w[:] = log_w
    return inst


def test_sensitivity_closed_form_off_centre_gaussian():
    """l(c + t e_i) - l(c) = -t (P (c - mu))_i - t^2 P_ii / 2 for one Gaussian."""
    inst = make_instance(7, 1, 91, s_range=(0.5, 3.0), mean_box=(-4, 4))
    res = oracle.precheck(inst)
    c = 0.5 * (inst.lo + inst.hi)
    delta = 0.5 * (inst.hi - inst.lo)
    P = inst.L[0] @ inst.L[0].T
    lin = P @ (c - inst.mu[0])
    expect = np.abs(-delta * lin - 0.5 * delta**2 * np.diag(P)) + np.abs(delta * lin - 0.5 * delta**2 * np.diag(P))
    np.testing.assert_allclose(res.s, expect, rtol=1e-12, atol=1e-10)


def test_sensitivity_matches_scipy_mixture_densities():
    inst = make_instance(5, 3, 92, s_range=(0.5, 3.0), mean_box=(-5, 5), sep=2.0)
    res = oracle.precheck(inst)
    comps = [stats.multivariate_normal(inst.mu[k], np.linalg.inv(inst.L[k] @ inst.L[k].T)) for k in range(inst.K)]
    ell = lambda x: logsumexp([inst.log_w[k] + comps[k].logpdf(x) for k in range(inst.K)])
    c = 0.5 * (inst.lo + inst.hi)
    delta = 0.5 * (inst.hi - inst.lo)
    l0 = ell(c)
    for i in range(inst.d):
        e = np.zeros(inst.d)
        e[i] = delta[i]
        ref = abs(ell(c + e) - l0) + abs(ell(c - e) - l0)
        assert res.s[i] == pytest.approx(ref, rel=1e-9, abs=1e-9)


def _brute_classes(s, eps_flat, eps_soft):
    fin = np.isfinite(s)
    med, smax = np.median(s[fin]), np.max(s[fin])
    cls = np.zeros(len(s), dtype=np.int8)
    cls[fin & (s < eps_flat * med)] = oracle.FLAT
    cls[fin & (cls == 0) & (s < eps_soft * smax)] = oracle.SOFT
    return cls


def test_classes_follow_the_thresholds_and_the_even_median():
    # s_i = (Delta_i / sigma_i)^2 at the centre; Delta = 10: s = [1.5e-6, 1, 3, 4]
    sig = 10.0 / np.sqrt([1.5e-6, 1.0, 3.0, 4.0])
    res = oracle.precheck(_diag_instance(sig))
    np.testing.assert_allclose(res.s, [1.5e-6, 1.0, 3.0, 4.0], rtol=1e-9, atol=1e-13)  # l differences cancel
    # median of four is (1 + 3) / 2 = 2: 1.5e-6 < 1e-6 * 2 is flat (the lower middle, 1, would not make it)
    assert res.cls.tolist() == [oracle.FLAT, 0, 0, 0] == _brute_classes(res.s, 1e-6, 1e-3).tolist()
    assert res.n_active == 3
    # soft: below 1e-3 max(s) but above the flat cut; odd count
    sig = 10.0 / np.sqrt([1e6, 1e6, 1e6, 100.0, 2e-7])
    res = oracle.precheck(_diag_instance(sig))
    assert res.cls.tolist() == [0, 0, 0, oracle.SOFT, oracle.FLAT] == _brute_classes(res.s, 1e-6, 1e-3).tolist()
    # custom thresholds
    res2 = oracle.precheck(_diag_instance(sig), eps_flat=1e-14, eps_soft=1e-5)
    assert res2.cls.tolist() == _brute_classes(res2.s, 1e-14, 1e-5).tolist() == [0, 0, 0, 0, oracle.SOFT]
    # a single coordinate is always active
    assert oracle.precheck(_diag_instance([3.0])).cls.tolist() == [0]


def test_soft_term_is_the_gaussian_integral_at_the_centre():
    sig = np.array([1e-2, 1e-2, 0.7])
    res = oracle.precheck(_diag_instance(sig))
    assert res.cls.tolist() == [0, 0, oracle.SOFT]
    val, _ = integrate.quad(lambda t: math.exp(-0.5 * (t / sig[2]) ** 2), -np.inf, np.inf)
    assert res.log_int == pytest.approx(math.log(val), abs=1e-10)
    assert res.log_vol == pytest.approx(math.log(20.0), abs=1e-15)


def test_marginalised_evidence_matches_the_exact_separable_evidence():
    """A diagonal Gaussian at the box centre with narrow, soft and flat coordinates:
    log Z of the active problem (flagged coordinates held at c, their density
    there folded into log w) + log_int - log_vol equals the exact log Z (products
    of truncated 1-d masses) up to the Gaussian tails beyond 10 sigma of the soft
    coordinates and the O(s_i) curvature of the flat one."""
    sig = np.array([0.01, 0.02, 0.015, 1.0, 0.8, 1e5])
    inst = _diag_instance(sig)
    res = oracle.precheck(inst)
    assert res.cls.tolist() == [0, 0, 0, oracle.SOFT, oracle.SOFT, oracle.FLAT]
    delta = 10.0
    exact = float(np.sum(np.log(ndtr(delta / sig) - ndtr(-delta / sig)))) - inst.d * math.log(20.0)
    act = res.cls == 0
    flg = ~act
    red = _diag_instance(sig[act], log_w=float(np.sum(-0.5 * math.log(2 * math.pi) - np.log(sig[flg]))))
    lz_red = oracle.evidence(red, SolveConfig(n_rays=64, n_steps=32, n_starts=16)).logZ
    total = lz_red + res.log_int - res.log_vol
    assert total == pytest.approx(exact, abs=1e-8)
    # dropping the correction is off by the flagged coordinates' terms
    assert abs(lz_red - exact) > 1.0
