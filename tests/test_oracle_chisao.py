"""Pins of the oracle's ChiSao oscillation (Sec. 3.5.5, Algorithm 1): the
momentum anti-convergence against its linear recurrence, the Golden Rooster
directions against numpy's QR, the ray search against the analytic maximiser,
and the whole oscillation against plain L-BFGS, brute-force stick filters and
mixtures whose modes are known."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_19957_gb300.instances import SolveConfig, make_instance


def _isotropic_1d_pair(w=(0.6, 0.4), means=(-5.0, 5.0)):
    inst = make_instance(1, 2, 1, s_range=(1.0, 1.0), sep=0.0)
    inst.L[:] = 1.0
    inst.mu[:, 0] = means
    inst.log_w[:] = np.log(np.asarray(w))
    return inst


def _precision(inst, k=0):
    return inst.L[k] @ inst.L[k].T


# ------------------------------------------------------------ anti-convergence
@pytest.mark.parametrize("d,steps,alpha", [(1, 1, 0.3), (3, 10, 0.05), (5, 7, 0.2)])
def test_anticonverge_is_the_momentum_recurrence(d, steps, alpha):
    """For one Gaussian, grad l = -P e with e = x - mu, so the steps are linear:
    v' = m v + alpha P e, e' = (I + alpha P) e + m v: a power of a 2d x 2d matrix."""
    inst = make_instance(d, 1, 40 + d, s_range=(0.5, 1.0), prior=(-1e4, 1e4))
    m = 0.9
    rng = np.random.default_rng(d)
    x0 = inst.mu[0] + rng.normal(0, 0.5, (4, d))
    got = oracle.chisao_anticonverge(inst, x0, steps, m, alpha)
    P = _precision(inst)
    I = np.eye(d)
    M = np.block([[I + alpha * P, m * I], [alpha * P, m * I]])
    Mt = np.linalg.matrix_power(M, steps)
    for s in range(4):
        ev = Mt @ np.concatenate([x0[s] - inst.mu[0], np.zeros(d)])
        np.testing.assert_allclose(got[s] - inst.mu[0], ev[:d], rtol=1e-11, atol=1e-12)


def test_anticonverge_moves_downhill_freezes_at_the_mode_and_clamps():
    inst = _isotropic_1d_pair(w=(1.0, 1e-300))
    # one step from e = -1: v = alpha * P e, so x = -5 - 1 - alpha
    x = oracle.chisao_anticonverge(inst, np.array([[-6.0]]), 1, 0.9, 0.25)
    assert x[0, 0] == pytest.approx(-6.25, abs=1e-15)
    assert oracle.loglik(inst, x[0]) < oracle.loglik(inst, np.array([-6.0]))
    # zero gradient at the mode: nothing moves
    x = oracle.chisao_anticonverge(inst, np.array([[-5.0]]), 10, 0.9, 0.25)
    assert x[0, 0] == -5.0
    # pushed through the box face at -10 it stays on the face
    x = oracle.chisao_anticonverge(inst, np.array([[-9.0]]), 10, 0.9, 0.5)
    assert x[0, 0] == inst.lo[0]


# --------------------------------------------------------- Golden Rooster basis
def _philox_normals(d, seed, w1, w2, tag):
    """Standard normals from the Philox4x32-10 blocks (known-answer pinned) by
    Box-Muller on 52-bit uniforms in (0, 1)."""
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    z = np.empty(d)
    for q in range((d + 1) // 2):
        o = oracle.philox4x32_10([q, w1, w2, tag], key)
        u1 = (((o[0] << 32) | o[1]) >> 12) + 0.5
        u2 = (((o[2] << 32) | o[3]) >> 12) + 0.5
        u1 /= 2.0**52
        u2 /= 2.0**52
        rad = math.sqrt(-2.0 * math.log(u1))
        z[2 * q] = rad * math.cos(2 * math.pi * u2)
        if 2 * q + 1 < d:
            z[2 * q + 1] = rad * math.sin(2 * math.pi * u2)
    return z


@pytest.mark.parametrize("d,osc,peak,basis", [(1, 0, 0, 0), (6, 1, 3, 0), (9, 2, 0, 2), (100, 1, 2, 3)])
def test_directions_are_the_q_of_the_normals(d, osc, peak, basis):
    """Groups of G = min(d, 64) orthonormal directions: the Q of the QR of G normals."""
    seed = 0x1234_5678_9ABC
    G = min(d, 64)
    Q = oracle.chisao_directions(d, G, seed, osc, peak, basis)
    np.testing.assert_allclose(Q @ Q.T, np.eye(G), atol=1e-13)
    Z = np.stack([_philox_normals(d, seed, basis * G + j, (osc << 16) | peak, 0x47525354) for j in range(G)], 1)
    q, r = np.linalg.qr(Z)
    q = q * np.sign(np.diag(r))[None, :]  # Gram-Schmidt keeps diag(R) > 0
    np.testing.assert_allclose(Q, q.T, atol=1e-12)
    # the first r columns do not depend on the later ones
    np.testing.assert_array_equal(oracle.chisao_directions(d, max(1, G // 2), seed, osc, peak, basis),
                                  Q[: max(1, G // 2)])
    # asking for more than a group gives the group
    np.testing.assert_array_equal(oracle.chisao_directions(d, G + 5, seed, osc, peak, basis), Q)


def test_directions_differ_by_peak_oscillation_and_basis():
    a = oracle.chisao_directions(5, 5, 7, 0, 0, 0)
    for other in (oracle.chisao_directions(5, 5, 7, 1, 0, 0), oracle.chisao_directions(5, 5, 7, 0, 1, 0),
                  oracle.chisao_directions(5, 5, 7, 0, 0, 1), oracle.chisao_directions(5, 5, 8, 0, 0, 0)):
        assert np.abs(a - other).max() > 1e-3


# ------------------------------------------------------------------ ray search
def test_ray_best_is_the_sample_nearest_the_quadratic_maximiser():
    d = 4
    inst = make_instance(d, 1, 51, s_range=(0.3, 1.0), prior=(-10.0, 10.0))
    rng = np.random.default_rng(2)
    for trial in range(20):
        o = rng.uniform(-9, 9, d)
        u = rng.normal(size=d)
        u /= np.linalg.norm(u)
        n = 50
        j, x, ell = oracle.chisao_ray_best(inst, o, u, n)
        t_exit = min(((inst.hi - o) / u)[u > 0].min(initial=np.inf), ((inst.lo - o) / u)[u < 0].min(initial=np.inf))
        t = (np.arange(n) + 1) / n * t_exit
        # along the ray l is a concave quadratic a - (b/2)(t - t*)^2
        P = _precision(inst)
        tstar = u @ P @ (inst.mu[0] - o) / (u @ P @ u)
        jj = int(np.argmin(np.abs(t - tstar)))
        assert j == jj
        np.testing.assert_allclose(x, o + t[jj] * u, rtol=1e-14, atol=1e-14)
        assert ell == oracle.loglik(inst, x)


def test_ray_best_past_the_valley_and_to_the_exit():
    inst = _isotropic_1d_pair(w=(0.7, 0.3))
    # from the heavier left mode to the right: the far mode wins only past the valley
    j0, x0, _ = oracle.chisao_ray_best(inst, np.array([-5.0]), np.array([1.0]), 60)
    assert x0[0] == pytest.approx(-5.0 + 15.0 / 60)  # first sample, next to the origin's peak
    j1, x1, _ = oracle.chisao_ray_best(inst, np.array([-5.0]), np.array([1.0]), 60, past_valley=True)
    assert x1[0] == pytest.approx(5.0)  # t = 10 is sample 40 of 60
    # towards the near face l only falls: the exit sample, on the box face
    j2, x2, _ = oracle.chisao_ray_best(inst, np.array([-5.0]), np.array([-1.0]), 60, past_valley=True)
    assert j2 == 59 and x2[0] == inst.lo[0]
    # an origin outside the box is clamped onto it first
    j3, x3, _ = oracle.chisao_ray_best(inst, np.array([-30.0]), np.array([1.0]), 20)
    assert x3[0] == pytest.approx(-5.0)


# ------------------------------------------------------------- the oscillation
def _brute_stick(inst, cfg, x, ell):
    wmax = float((inst.hi - inst.lo).max())
    lmax = np.max(ell[np.isfinite(ell)])
    conv = []
    for s in range(len(x)):
        _, g = oracle.loglik(inst, x[s], want_grad=True)
        conv.append(np.isfinite(ell[s]) and np.abs(g).max() <= cfg.eps_grad * (1 + abs(ell[s])))
    cand = [s for s in range(len(x)) if conv[s] and ell[s] >= lmax + math.log(0.1)]
    cand.sort(key=lambda s: (-ell[s], s))
    reps = []
    for s in cand:
        if all(np.abs(x[s] - x[r]).max() > cfg.dedup_coarse * wmax for r in reps):
            reps.append(s)
    return sorted(reps)


def test_one_oscillation_is_lbfgs_and_the_stick_filter():
    inst = make_instance(3, 3, 61, s_range=(0.4, 1.0), mean_box=(-5, 5), sep=4.0)
    cfg = SolveConfig(max_iter=1000)
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-6, 6, (40, 3))
    ref = oracle.lbfgs(inst, cfg, x0)
    res = oracle.chisao(inst, cfg, oracle.ChisaoConfig(n_osc=1, conv_iters=1000), x0)
    np.testing.assert_array_equal(res.x, ref.x)
    np.testing.assert_array_equal(res.ell, ref.ell)
    reps = _brute_stick(inst, cfg, ref.x, ref.ell)
    assert np.flatnonzero(res.stuck).tolist() == reps and res.n_peaks == len(reps)


def test_bimodal_1d_finds_the_mode_plain_lbfgs_misses():
    inst = _isotropic_1d_pair()
    cfg = SolveConfig(n_steps=64, seed=3)
    x0 = -5 + np.random.default_rng(0).uniform(-2, 2, (16, 1))
    assert np.allclose(oracle.lbfgs(inst, cfg, x0).x, -5.0)
    res = oracle.chisao(inst, cfg, oracle.ChisaoConfig(), x0)
    assert res.n_peaks == 2
    np.testing.assert_allclose(np.sort(res.x[res.stuck][:, 0]), [-5.0, 5.0], atol=1e-7)


def test_low_peaks_do_not_stick():
    """A mode whose peak is below 10 % of the highest never sticks (the likelihood
    threshold of the stick test), however it is reached."""
    inst = _isotropic_1d_pair(w=(0.95, 0.05))
    cfg = SolveConfig(n_steps=64, seed=3)
    x0 = np.array([[-6.0], [-4.0], [4.5], [5.5]] * 2)
    res = oracle.chisao(inst, cfg, oracle.ChisaoConfig(n_osc=2), x0)
    assert res.n_peaks == 1
    np.testing.assert_allclose(res.x[res.stuck][:, 0], [-5.0], atol=1e-7)


@pytest.mark.parametrize("d,seed", [(2, 5), (4, 12), (4, 13)])
def test_mixture_modes_found_from_one_basin(d, seed):
    inst = make_instance(d, 3, seed, s_range=(0.5, 1.0), mean_box=(-6, 6), sep=6.0)
    cfg = SolveConfig(n_steps=64, seed=seed)
    x0 = inst.mu[0] + np.random.default_rng(seed).uniform(-0.5, 0.5, (64, d))
    ref = oracle.lbfgs(inst, cfg, x0)
    assert np.abs(ref.x - inst.mu[0]).max() < 1e-6  # plain refinement: one mode
    res = oracle.chisao(inst, cfg, oracle.ChisaoConfig(n_osc=4), x0)
    # every mode whose peak passes the stick test is found, each once
    peaks = np.array([oracle.loglik(inst, mu) for mu in inst.mu])
    expect = np.flatnonzero(peaks >= peaks.max() + math.log(0.1))
    found = res.x[res.stuck]
    assert res.n_peaks == len(expect) == len(found)
    dist = np.abs(found[:, None, :] - inst.mu[None, expect, :]).max(2)
    assert dist.min(0).max() < 1e-6 and dist.min(1).max() < 1e-6


def test_many_unconverged_samples_reseed_by_repulse_monkey():
    """With few convergence iterations most samples stay unconverged, so lost
    samples are reseeded along rays from them; the stuck output still holds only
    distinct converged peaks above the threshold."""
    inst = make_instance(3, 3, 71, s_range=(0.3, 1.0), mean_box=(-5, 5), sep=4.0)
    cfg = SolveConfig(n_steps=32, seed=1)
    x0 = np.random.default_rng(4).uniform(-9, 9, (48, 3))
    # four iterations per phase leave most samples unconverged; a small step keeps some near peaks
    res = oracle.chisao(inst, cfg, oracle.ChisaoConfig(n_osc=3, conv_iters=4, anti_alpha=0.01), x0)
    assert np.all(np.isfinite(res.x)) and np.all(res.x >= inst.lo) and np.all(res.x <= inst.hi)
    assert 0 < res.n_peaks == res.stuck.sum()
    wmax = float((inst.hi - inst.lo).max())
    found = res.x[res.stuck]
    for a in range(len(found)):
        _, g = oracle.loglik(inst, found[a], want_grad=True)
        assert np.abs(g).max() <= cfg.eps_grad * (1 + abs(res.ell[res.stuck][a]))
        for b in range(a):
            assert np.abs(found[a] - found[b]).max() > cfg.dedup_coarse * wmax


def test_status_reading_of_the_stick_test():
    """conv_from_status: one oscillation sticks the CONVERGED / STALLED samples above the
    threshold (a MAXITER sample does not stick even at a good l)."""
    inst = make_instance(3, 3, 61, s_range=(0.4, 1.0), mean_box=(-5, 5), sep=4.0)
    cfg = SolveConfig(max_iter=1000)
    x0 = np.random.default_rng(3).uniform(-6, 6, (40, 3))
    cc = oracle.ChisaoConfig(n_osc=1, conv_iters=6, conv_from_status=True)
    res = oracle.chisao(inst, cfg, cc, x0)
    ref = oracle.lbfgs(inst, SolveConfig(max_iter=6), x0)
    np.testing.assert_array_equal(res.x, ref.x)
    ok = np.isin(ref.status, [oracle.CONVERGED, oracle.STALLED]) & np.isfinite(ref.ell)
    lmax = ref.ell[np.isfinite(ref.ell)].max()
    cand = [s for s in range(40) if ok[s] and ref.ell[s] >= lmax + math.log(0.1)]
    cand.sort(key=lambda s: (-ref.ell[s], s))
    wmax = float((inst.hi - inst.lo).max())
    reps = []
    for s in cand:
        if all(np.abs(ref.x[s] - ref.x[r]).max() > cfg.dedup_coarse * wmax for r in reps):
            reps.append(s)
    assert np.flatnonzero(res.stuck).tolist() == sorted(reps)
    assert (ref.status == oracle.MAXITER).any()  # the case has samples the status reading leaves out


@pytest.mark.parametrize("d,seed,plain_at_most", [(16, 0, 2), (64, 0, 1)])
def test_laplace_on_all_final_samples_recovers_every_component(d, seed, plain_at_most):
    """Six separated components: sunburst starts refined by L-BFGS reach only a few basins;
    after ChiSao the stick rule keeps only peaks within log 10 of the highest, but the
    Laplace stage run on every final sample finds all six (seeded regression of the
    method as built)."""
    inst = make_instance(d, 6, 100 * d + seed, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    cfg = SolveConfig(n_rays=128, n_steps=64, n_starts=128, m=10, seed=seed)
    starts, _ = oracle.discover(inst, cfg, n_threads=4)
    ref = oracle.lbfgs(inst, cfg, starts, n_threads=4)
    plain = oracle.laplace(inst, cfg, ref.x, ref.ell, ref.status)
    cs = oracle.chisao(inst, cfg, oracle.ChisaoConfig(n_osc=3), starts, n_threads=4)
    lap = oracle.laplace(inst, cfg, cs.x, cs.ell)
    comp = lambda M: sorted({int(np.argmin(np.abs(inst.mu - m).max(1))) for m in M})
    assert len(comp(plain.modes)) <= plain_at_most
    assert comp(lap.modes) == list(range(6))
    logV = float(np.log(inst.hi - inst.lo).sum())
    assert lap.logZ == pytest.approx(float(np.log(np.exp(inst.log_w).sum())) - logV, abs=1e-9)


def test_step_size_of_the_anti_convergence_matters_for_recovery():
    """Eight components at d = 128 (shaped like the d = 1024 workload): with the Laplace stage
    over every final sample, a momentum step of 0.1 recovers all eight where 0.01 leaves
    samples in too few basins (seeded regression of reading 26's default)."""
    d = 128
    inst = make_instance(d, 8, 4000 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=10.0)
    cfg = SolveConfig(n_rays=256, n_steps=64, n_starts=256, m=20, seed=0)
    starts, _ = oracle.discover(inst, cfg, n_threads=4)
    found = {}
    for alpha in (0.01, 0.1):
        cs = oracle.chisao(inst, cfg, oracle.ChisaoConfig(n_osc=3, anti_alpha=alpha), starts, n_threads=4)
        lap = oracle.laplace(inst, cfg, cs.x, cs.ell)
        found[alpha] = {int(np.argmin(np.abs(inst.mu - m).max(1))) for m in lap.modes}
    assert found[0.1] == set(range(8)) and len(found[0.01]) < 8


def test_nonfinite_start_is_left_alone():
    """A NaN start ends NONFINITE: it never sticks, is neither reseeded nor anti-converged,
    and the other samples find the same peaks as without it."""
    inst = _isotropic_1d_pair()
    cfg = SolveConfig(n_steps=64, seed=3)
    x0 = -5 + np.random.default_rng(0).uniform(-2, 2, (16, 1))
    ref = oracle.chisao(inst, cfg, oracle.ChisaoConfig(), x0)
    x1 = np.concatenate([x0, [[np.nan]]])
    res = oracle.chisao(inst, cfg, oracle.ChisaoConfig(), x1)
    assert np.isnan(res.x[-1, 0]) and not res.stuck[-1]
    assert res.n_peaks == ref.n_peaks == 2
    np.testing.assert_allclose(np.sort(res.x[:-1][res.stuck[:-1]][:, 0]), np.sort(ref.x[ref.stuck][:, 0]), atol=1e-7)
