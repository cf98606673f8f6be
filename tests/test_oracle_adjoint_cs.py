"""Pins of the complex-step reference for the adjoint of log Z (oracle/laplace_cs.py):
its log Z equals the C oracle's Laplace log Z on the same modes; its derivatives
vanish where log Z cannot depend on mu and L (one Gaussian, well separated
components, where Laplace gives log w_k per mode), and agree with central
differences of the C oracle's log Z on overlapping mixtures, where the
gradient is O(1)."""
import copy

import numpy as np
import pytest

import oracle
from oracle import laplace_cs
from paper_2601_19957_gb300.instances import SolveConfig, make_instance, workload


def _overlapping(d, K, seed):
    return make_instance(d, K, seed, s_range=(0.6, 1.0), mean_box=(-1.5, 1.5), sep=2.5, prior=(-12.0, 12.0))


def _c_logz(inst, cfg, modes):
    ell = np.array([oracle.loglik(inst, m) for m in modes])
    return oracle.laplace(inst, cfg, modes, ell).logZ


@pytest.mark.parametrize("d,K,seed", [(2, 2, 2), (3, 2, 5), (3, 3, 8)])
def test_log_evidence_matches_the_c_oracle(d, K, seed):
    inst = _overlapping(d, K, seed)
    cfg = SolveConfig(n_rays=128, n_steps=64, n_starts=128, seed=11)
    ref = oracle.evidence(inst, cfg)
    lz = laplace_cs.log_evidence(inst.log_w, inst.mu, inst.L, inst.lo, inst.hi, ref.modes)
    assert abs(lz.real - ref.logZ) <= 1e-12 * abs(ref.logZ)
    assert lz.imag == 0.0


def test_derivatives_vanish_for_one_gaussian_and_separated_components():
    insts, cfg = workload(0)
    g = insts[0]
    _, gmu, gL = laplace_cs.dlogz(g, g.mu[:1])
    assert np.abs(gmu).max() < 1e-12 and np.abs(gL).max() < 1e-12
    sep = make_instance(3, 3, 17, s_range=(0.2, 0.5), mean_box=(-6, 6), sep=12.0)
    _, gmu, gL = laplace_cs.dlogz(sep, sep.mu)
    assert np.abs(gmu).max() < 1e-9 and np.abs(gL).max() < 1e-9


@pytest.mark.parametrize("d,K,seed", [(2, 2, 2), (3, 2, 5)])
def test_derivatives_match_central_differences_of_the_c_oracle(d, K, seed):
    inst = _overlapping(d, K, seed)
    cfg = SolveConfig(n_rays=128, n_steps=64, n_starts=128, seed=11)
    modes = oracle.evidence(inst, cfg).modes
    _, gmu, gL = laplace_cs.dlogz(inst, modes)
    h = 1e-6
    scale = 1.0 + max(np.abs(gmu).max(), np.abs(gL).max())
    assert np.abs(gmu).max() > 1e-3  # a case with a real gradient
    for k in range(K):
        for i in range(d):
            ip, im = copy.deepcopy(inst), copy.deepcopy(inst)
            ip.mu[k, i] += h
            im.mu[k, i] -= h
            fd = (_c_logz(ip, cfg, modes) - _c_logz(im, cfg, modes)) / (2 * h)
            assert abs(fd - gmu[k, i]) <= 1e-6 * scale
            for j in range(i + 1):
                ip, im = copy.deepcopy(inst), copy.deepcopy(inst)
                ip.L[k, i, j] += h
                im.L[k, i, j] -= h
                fd = (_c_logz(ip, cfg, modes) - _c_logz(im, cfg, modes)) / (2 * h)
                assert abs(fd - gL[k, i, j]) <= 1e-6 * scale
    assert np.all(np.triu(gL, 1) == 0)


def test_step_size_does_not_matter():
    inst = _overlapping(2, 2, 2)
    modes = oracle.evidence(inst, SolveConfig(n_rays=128, n_steps=64, n_starts=128, seed=11)).modes
    a = laplace_cs.dlogz(inst, modes)
    old = laplace_cs._H
    try:
        laplace_cs._H = 1e-20
        b = laplace_cs.dlogz(inst, modes)
    finally:
        laplace_cs._H = old
    np.testing.assert_allclose(a[1], b[1], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(a[2], b[2], rtol=1e-13, atol=1e-15)
