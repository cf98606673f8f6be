"""Pins of the oracle's black-box derivatives and rotation detection (App. A.4,
Sec. 3.7.2): central differences are exact on a quadratic (up to rounding), so
on one Gaussian they must return the closed forms -P (x - mu) and -P; on
mixtures they converge at second order to the analytic derivatives; the
uniform-correlation probe recovers the off-diagonal of an equicorrelated
precision in closed form and the mean off-diagonal entry in general; the
perpendicular step fraction is checked on constructed steps and on Newton steps,
which are exactly along the whitened gradient when the Hessian is diagonal."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_19957_gb300.instances import haar_orthogonal, make_instance


def _gaussian(Sigma, mu):
    d = len(mu)
    inst = make_instance(d, 1, 1, s_range=(1.0, 1.0))
    inst.L[0] = np.linalg.cholesky(np.linalg.inv(Sigma))
    inst.mu[0] = mu
    return inst


@pytest.mark.parametrize("d", [1, 4, 9])
def test_fd_derivatives_of_a_gaussian_are_the_closed_forms(d):
    inst = make_instance(d, 1, 200 + d, s_range=(0.3, 2.0), mean_box=(-3, 3))
    P = inst.L[0] @ inst.L[0].T
    x = inst.mu[0] + np.random.default_rng(d).normal(0, 1.0, d)
    l0 = abs(oracle.loglik(inst, x))
    g = oracle.fd_grad(inst, x, eps=1e-5)
    np.testing.assert_allclose(g, -P @ (x - inst.mu[0]), rtol=0, atol=1e-9 * (1 + l0) * np.abs(P).max())
    H = oracle.fd_hess_full(inst, x, eps=1e-3)
    np.testing.assert_allclose(H, -P, rtol=0, atol=1e-8 * (1 + l0) * np.abs(P).max())
    np.testing.assert_array_equal(oracle.fd_hess_diag(inst, x, eps=1e-3), np.diag(H))
    assert np.array_equal(H, H.T)


def test_fd_derivatives_of_a_mixture_converge_at_second_order():
    inst = make_instance(5, 3, 211, s_range=(0.5, 1.5), mean_box=(-2, 2), sep=1.0)
    x = inst.mu[0] + 0.7
    _, g, hneg = oracle.loglik(inst, x, want_grad=True, want_hess=True)
    e1 = np.abs(oracle.fd_grad(inst, x, eps=2e-2) - g).max()
    e2 = np.abs(oracle.fd_grad(inst, x, eps=1e-2) - g).max()
    assert 3.0 < e1 / e2 < 5.0
    h1 = np.abs(oracle.fd_hess_full(inst, x, eps=4e-2) + hneg).max()
    h2 = np.abs(oracle.fd_hess_full(inst, x, eps=2e-2) + hneg).max()
    assert 3.0 < h1 / h2 < 5.0
    assert np.abs(oracle.fd_hess_full(inst, x, eps=1e-4) + hneg).max() < 1e-5


def test_uniform_correlation_probe_closed_form():
    d, rho = 6, 0.3
    Sigma = (1 - rho) * np.eye(d) + rho * np.ones((d, d))
    inst = _gaussian(Sigma, np.zeros(d))
    x = np.full(d, 0.2)
    hd = oracle.fd_hess_diag(inst, x)
    b = oracle.uniform_corr_probe(inst, x, hd)
    # Sigma^-1 = (I - rho / (1 + (d-1) rho) 1 1^T) / (1 - rho); H = -Sigma^-1
    assert b == pytest.approx(rho / ((1 - rho) * (1 + (d - 1) * rho)), rel=1e-6)
    # in general it is the mean off-diagonal entry of H; zero without correlation
    rng = np.random.default_rng(5)
    Q = haar_orthogonal(d, rng)
    inst2 = _gaussian(Q @ np.diag(rng.uniform(0.5, 2.0, d) ** 2) @ Q.T, rng.normal(size=d))
    H = -(inst2.L[0] @ inst2.L[0].T)
    b2 = oracle.uniform_corr_probe(inst2, x, oracle.fd_hess_diag(inst2, x))
    assert b2 == pytest.approx((H.sum() - np.trace(H)) / (d * (d - 1)), rel=1e-5, abs=1e-8)
    inst3 = _gaussian(np.diag(rng.uniform(0.5, 2.0, d) ** 2), rng.normal(size=d))
    assert abs(oracle.uniform_corr_probe(inst3, x, oracle.fd_hess_diag(inst3, x))) < 1e-7
    assert oracle.uniform_corr_probe(_gaussian(np.eye(1), np.zeros(1)), np.zeros(1), np.array([-1.0])) == 0.0


def test_perp_fraction_on_constructed_steps():
    h = np.array([-4.0, -1.0, -9.0])  # whitening w = (2, 1, 3)
    g = np.array([2.0, 0.0, 0.0])  # whitened gradient (1, 0, 0)
    assert oracle.perp_fraction([1.0, 0.0, 0.0], g, h) == 0.0  # along it
    assert oracle.perp_fraction([0.0, 5.0, 0.0], g, h) == pytest.approx(1.0)  # orthogonal
    # whitened step (2, 0, 3): perpendicular part 3 of length sqrt(13)
    assert oracle.perp_fraction([1.0, 0.0, 1.0], g, h) == pytest.approx(3 / math.sqrt(13))
    assert oracle.perp_fraction([0.0, 0.0, 0.0], g, h) == 0.0
    assert math.isnan(oracle.perp_fraction([1.0, 0.0, 0.0], g, [-1.0, 0.0, -1.0]))


def test_newton_steps_are_along_the_whitened_gradient_only_without_rotation():
    d = 6
    rng = np.random.default_rng(8)
    s = rng.uniform(0.3, 2.0, d)
    for rotated in (False, True):
        Q = haar_orthogonal(d, rng) if rotated else np.eye(d)
        inst = _gaussian(Q @ np.diag(s**2) @ Q.T, np.zeros(d))
        P = inst.L[0] @ inst.L[0].T
        hd = -np.diag(P)
        fp = []
        for _ in range(10):
            x = rng.uniform(-3, 3, d)
            _, g = oracle.loglik(inst, x, want_grad=True)
            fp.append(oracle.perp_fraction(np.linalg.solve(P, g), g, hd))  # Newton step x* - x
        if rotated:
            assert min(fp) > 0.05
        else:
            assert max(fp) < 1e-12
