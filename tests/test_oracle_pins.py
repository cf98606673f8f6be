"""Pins of the FP64 CPU oracle against things other than itself: published
known-answer vectors, library routines that compute the same definition
(scipy/numpy), closed forms the paper states, brute-force quadrature,
brute-force selection/dedup, and invariants. No GPU needed."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

import oracle
from paper_2601_19957_gb300.instances import SolveConfig, make_instance, workload
from tests.conftest import read_golden


def golden_claims():
    return {row[0]: float(row[1]) for row in read_golden("paper_accuracy_claims.txt")}


def scipy_loglik(inst, X):
    """Independent log-likelihood: scipy multivariate normal log-pdfs + logsumexp."""
    X = np.atleast_2d(X)
    comps = []
    for k in range(inst.K):
        P = inst.L[k] @ inst.L[k].T
        cov = np.linalg.inv(P)
        cov = 0.5 * (cov + cov.T)
        comps.append(inst.log_w[k] + stats.multivariate_normal(inst.mu[k], cov).logpdf(X))
    return logsumexp(np.stack(comps, 0).reshape(inst.K, -1), axis=0)


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        words = [int(w, 16) for w in row]
        assert oracle.philox4x32_10(words[0:4], words[4:6]) == words[6:10]


def test_ray_directions_unit_and_isotropic():
    u = oracle.ray_directions(5, 4000, 7)
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-14)
    # uniform on the sphere: each coordinate has mean 0 and variance 1/d
    assert np.abs(u.mean(0)).max() < 0.05
    assert np.allclose((u * u).mean(0), 0.2, atol=0.02)


def test_ray_directions_uniform_on_circle_and_sphere():
    u2 = oracle.ray_directions(2, 20000, 11)
    ang = (np.arctan2(u2[:, 1], u2[:, 0]) + np.pi) / (2 * np.pi)
    assert stats.kstest(ang, "uniform").pvalue > 1e-3
    # Archimedes: on S^2 every coordinate is uniform on [-1, 1]
    u3 = oracle.ray_directions(3, 20000, 12)
    for i in range(3):
        assert stats.kstest((u3[:, i] + 1) / 2, "uniform").pvalue > 1e-3


def test_ray_directions_depend_on_seed_and_odd_d():
    a = oracle.ray_directions(7, 10, 1)
    b = oracle.ray_directions(7, 10, 2)
    assert not np.allclose(a, b)
    # the first 7 coordinates of d=8 rays share the Philox pairs with d=7 up to normalisation
    c = oracle.ray_directions(8, 10, 1)
    cos = np.einsum("ri,ri->r", a, c[:, :7] / np.linalg.norm(c[:, :7], axis=1, keepdims=True))
    assert np.allclose(cos, 1.0, atol=1e-13)


# --------------------------------------------------------------------- likelihood
@pytest.mark.parametrize("d,K", [(1, 1), (3, 2), (6, 3), (8, 1)])
def test_loglik_matches_scipy(d, K):
    inst = make_instance(d, K, 100 + d, s_range=(0.3, 1.0), mean_box=(-2, 2), sep=3.0)
    rng = np.random.default_rng(0)
    X = inst.mu[0] + rng.normal(0, 1.0, (20, d))
    ref = scipy_loglik(inst, X)
    got = np.array([oracle.loglik(inst, x) for x in X])
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("d,K", [(2, 1), (5, 3), (9, 2)])
def test_gradient_matches_central_differences(d, K):
    """App. A.4.1 stencil, h = 1e-6."""
    inst = make_instance(d, K, 200 + d, s_range=(0.3, 1.0), mean_box=(-1, 1), sep=1.0)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(5):
        x = inst.mu[0] + rng.normal(0, 0.5, d)
        _, g = oracle.loglik(inst, x, want_grad=True)
        fd = np.empty(d)
        for i in range(d):
            e = np.zeros(d)
            e[i] = h
            fd[i] = (oracle.loglik(inst, x + e) - oracle.loglik(inst, x - e)) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(g).max()))


@pytest.mark.parametrize("d,K", [(2, 2), (4, 3)])
def test_negative_hessian_matches_fd_stencil(d, K):
    """App. A.4.3 four-point stencil on l, and central differences of the gradient."""
    inst = make_instance(d, K, 300 + d, s_range=(0.4, 1.0), mean_box=(-1, 1), sep=1.0)
    rng = np.random.default_rng(2)
    x = inst.mu[0] + rng.normal(0, 0.4, d)
    _, g, H = oracle.loglik(inst, x, want_grad=True, want_hess=True)
    assert np.allclose(H, H.T, atol=1e-12)
    eps = 1e-4
    fdH = np.empty((d, d))
    for i in range(d):
        for j in range(d):
            ei = np.zeros(d)
            ej = np.zeros(d)
            ei[i] = eps
            ej[j] = eps
            fpp = oracle.loglik(inst, x + ei + ej)
            fpm = oracle.loglik(inst, x + ei - ej)
            fmp = oracle.loglik(inst, x - ei + ej)
            fmm = oracle.loglik(inst, x - ei - ej)
            fdH[i, j] = -(fpp - fpm - fmp + fmm) / (4 * eps * eps)
    assert np.allclose(H, fdH, rtol=1e-5, atol=1e-5 * np.abs(H).max())
    h = 1e-6
    for i in range(d):
        e = np.zeros(d)
        e[i] = h
        _, gp = oracle.loglik(inst, x + e, want_grad=True)
        _, gm = oracle.loglik(inst, x - e, want_grad=True)
        assert np.allclose(-(gp - gm) / (2 * h), H[:, i], rtol=1e-6, atol=1e-6 * np.abs(H).max())


def test_single_gaussian_hessian_is_precision_and_peak_value():
    inst = make_instance(6, 1, 77, s_range=(0.1, 1.0))
    ell, g, H = oracle.loglik(inst, inst.mu[0], want_grad=True, want_hess=True)
    P = inst.L[0] @ inst.L[0].T
    assert np.abs(g).max() == 0.0
    assert np.allclose(H, P, rtol=1e-13, atol=1e-12 * np.abs(P).max())
    # peak of a normalised Gaussian: -d/2 log 2pi + 1/2 log det P
    assert ell == pytest.approx(-3 * math.log(2 * math.pi) + 0.5 * np.linalg.slogdet(P)[1], rel=1e-14)


# ------------------------------------------------------------------- Cholesky
def test_cholesky_matches_numpy_and_logdet():
    rng = np.random.default_rng(3)
    for d in (1, 2, 7, 33):
        A = rng.normal(size=(d, d))
        P = A @ A.T + d * np.eye(d)
        C = oracle.cholesky(P)
        assert np.allclose(C, np.linalg.cholesky(P), rtol=1e-12, atol=1e-12)
        assert 2 * np.log(np.diag(C)).sum() == pytest.approx(np.linalg.slogdet(P)[1], rel=1e-12)


def test_cholesky_rejects_indefinite_and_brute_force_det():
    A = np.diag([1.0, -1.0, 2.0])
    assert oracle.cholesky(A) is None
    # brute-force determinant (Leibniz expansion) at d = 4
    rng = np.random.default_rng(4)
    B = rng.normal(size=(4, 4))
    P = B @ B.T + np.eye(4)
    import itertools

    det = 0.0
    for perm in itertools.permutations(range(4)):
        sgn = np.linalg.det(np.eye(4)[list(perm)])
        det += sgn * np.prod([P[i, perm[i]] for i in range(4)])
    C = oracle.cholesky(P)
    assert np.prod(np.diag(C)) ** 2 == pytest.approx(det, rel=1e-12)


# -------------------------------------------------------------- two-loop recursion
def _bfgs_matrix(S, Y, gamma):
    """Dense inverse-Hessian recursion H <- V^T H V + rho s s^T, V = I - rho y s^T."""
    d = S.shape[1]
    H = gamma * np.eye(d)
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        V = np.eye(d) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def _pairs(d, count, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(d, d))
    A = A @ A.T + d * np.eye(d)
    S = rng.normal(size=(count, d))
    Y = S @ A.T  # y = A s for a quadratic, so s^T y > 0
    return S, Y, 1.0 / np.einsum("ij,ij->i", S, Y)


@pytest.mark.parametrize("d,count", [(5, 1), (8, 3), (16, 10), (3, 6)])
def test_two_loop_equals_dense_bfgs_recursion(d, count):
    S, Y, rho = _pairs(d, count, d * 10 + count)
    q = np.random.default_rng(9).normal(size=d)
    gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    ref = _bfgs_matrix(S, Y, gamma) @ q
    got = oracle.two_loop(S, Y, rho, q)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_two_loop_secant_identity_and_empty_history():
    S, Y, rho = _pairs(12, 5, 42)
    r = oracle.two_loop(S, Y, rho, Y[-1])
    assert np.allclose(r, S[-1], rtol=1e-11, atol=1e-12)
    q = np.arange(1.0, 6.0)
    assert np.array_equal(oracle.two_loop(np.zeros((0, 5)), np.zeros((0, 5)), np.zeros(0), q), q)


# --------------------------------------------------------------------- discovery
def test_ray_samples_on_grid_and_box_surface():
    inst = make_instance(4, 2, 5, s_range=(0.3, 1.0), sep=2.0, prior=(-3.0, 5.0))
    cfg = SolveConfig(n_rays=16, n_steps=8, n_starts=8, seed=99)
    u, te, ell = oracle.ray_loglik(inst, cfg)
    c = 0.5 * (inst.lo + inst.hi)
    half = 0.5 * (inst.hi - inst.lo)
    for r in range(16):
        x_end = c + te[r] * u[r]
        assert np.abs((x_end - c) / half).max() == pytest.approx(1.0, abs=1e-14)
        X = np.stack([c + ((j + 1) / 8) * te[r] * u[r] for j in range(8)])
        assert np.allclose(ell[r], scipy_loglik(inst, X), rtol=1e-11, atol=1e-11)


def _brute_select(ell, n_starts):
    R, S = ell.shape
    keys = []
    for r in range(R):
        for j in range(S):
            left = ell[r, j - 1] if j > 0 else -np.inf
            right = ell[r, j + 1] if j + 1 < S else -np.inf
            tier = 0 if (ell[r, j] > left and ell[r, j] >= right) else 1
            rank = sum(1 for j2 in range(S) if ell[r, j2] > ell[r, j] or (ell[r, j2] == ell[r, j] and j2 < j))
            keys.append((tier, rank, -ell[r, j], r * S + j))
    keys.sort()
    return sorted(k[3] for k in keys[:n_starts])


def test_select_starts_matches_brute_force_with_ties():
    rng = np.random.default_rng(5)
    for R, S, n in [(7, 9, 5), (12, 16, 40), (3, 4, 12)]:
        ell = np.round(rng.normal(size=(R, S)), 1)  # many exact ties
        cfg = SolveConfig(n_rays=R, n_steps=S, n_starts=n)
        assert list(oracle.select_starts(cfg, ell)) == _brute_select(ell, n)


def test_discover_returns_selected_samples():
    inst = make_instance(3, 2, 8, s_range=(0.3, 1.0), sep=2.0)
    cfg = SolveConfig(n_rays=20, n_steps=10, n_starts=15, seed=4)
    u, te, ell = oracle.ray_loglik(inst, cfg)
    idx = oracle.select_starts(cfg, ell)
    starts, ls = oracle.discover(inst, cfg)
    c = 0.5 * (inst.lo + inst.hi)
    for s, f in enumerate(idx):
        r, j = divmod(int(f), 10)
        assert np.allclose(starts[s], c + ((j + 1) / 10) * te[r] * u[r], rtol=0, atol=1e-15)
        assert ls[s] == ell[r, j]


# ------------------------------------------------------------------------ L-BFGS
def test_lbfgs_reaches_gaussian_mode():
    inst = make_instance(10, 1, 21, s_range=(0.1, 1.0))
    cfg = SolveConfig(m=10)
    rng = np.random.default_rng(6)
    x0 = inst.mu[0] + rng.uniform(-3, 3, (16, 10))
    res = oracle.lbfgs(inst, cfg, x0)
    assert set(res.status.tolist()) <= {oracle.CONVERGED, oracle.STALLED}
    # Armijo needs a visible decrease of f ~ 10, so walkers stop where 1/2 dx^T P dx
    # reaches the rounding of f (~1e-15): |dx| ~ 1e-8 along the widest axis (s = 1).
    assert np.abs(res.x - inst.mu[0]).max() < 1e-7
    assert res.evals >= 16 and res.iters.min() > 0


def test_lbfgs_quadratic_small_d_reaches_gradient_floor():
    inst = make_instance(4, 1, 22, s_range=(0.5, 1.0))
    cfg = SolveConfig(m=10, gtol=1e-10)
    res = oracle.lbfgs(inst, cfg, inst.mu[0] + np.array([[1.0, -2.0, 0.5, 3.0]]))
    assert res.status[0] == oracle.CONVERGED
    _, g = oracle.loglik(inst, res.x[0], want_grad=True)
    assert np.abs(g).max() <= 1e-10 * (1 + abs(res.ell[0]))


def test_lbfgs_max_iter_and_nonfinite():
    inst = make_instance(6, 1, 23, s_range=(0.1, 1.0))
    cfg = SolveConfig(max_iter=1)
    res = oracle.lbfgs(inst, cfg, np.full((1, 6), 5.0))
    assert res.status[0] == oracle.MAXITER and res.iters[0] == 1
    res2 = oracle.lbfgs(inst, SolveConfig(), np.full((1, 6), np.nan))
    assert res2.status[0] == oracle.NONFINITE


# ----------------------------------------------------------------------- Laplace
def test_single_gaussian_evidence_closed_form():
    """Laplace is exact for a Gaussian (Sec. 4.2): log Z = -log V, rel. error < 1e-12."""
    bound = golden_claims()["gaussian_rel_error_bound"]
    insts, cfg = workload(0)
    inst = insts[0]
    res = oracle.evidence(inst, cfg)
    logV = np.log(inst.hi - inst.lo).sum()
    assert res.n_modes == 1
    assert abs(res.logZ + logV) <= bound * abs(logV)
    assert abs(math.expm1(res.logZ + logV)) <= bound  # |Z/Z_true - 1|
    assert np.abs(res.modes[0] - inst.mu[0]).max() < 1e-12


def test_separated_mixture_evidence_closed_form():
    insts, cfg = workload(1, scale=1.0)
    inst = insts[0]
    res = oracle.evidence(inst, cfg, n_threads=4)
    logV = np.log(inst.hi - inst.lo).sum()
    assert res.n_modes == inst.K
    assert res.logZ == pytest.approx(logsumexp(inst.log_w) - logV, rel=1e-12)
    assert np.allclose(np.sort(res.logZk), np.sort(inst.log_w), atol=1e-10)  # Laplace term, no prior
    for k in range(inst.K):
        assert np.abs(res.modes - inst.mu[k]).max(1).min() < 1e-10


def test_newton_polish_lands_on_mean():
    inst = make_instance(12, 1, 31, s_range=(0.1, 1.0))
    rng = np.random.default_rng(7)
    x = inst.mu[0] + rng.normal(0, 0.3, (5, 12))
    ell = np.array([oracle.loglik(inst, xx) for xx in x])
    res = oracle.laplace(inst, SolveConfig(newton_steps=1, dedup_coarse=0.1), x, ell)
    assert res.n_modes == 1
    assert np.abs(res.modes[0] - inst.mu[0]).max() <= 1e-14 * (1 + np.abs(inst.mu[0]).max()) * 10


def test_saddle_and_outside_box_are_filtered():
    # two equal isotropic unit Gaussians: the midpoint is a saddle of l
    d = 3
    inst = make_instance(d, 2, 1, s_range=(1.0, 1.0), sep=0.0)
    inst.L[:] = np.eye(d)
    inst.mu[0] = np.array([-3.0, 0, 0])
    inst.mu[1] = np.array([3.0, 0, 0])
    inst.log_w[:] = np.log(0.5)
    mid = np.zeros((1, d))
    res = oracle.laplace(inst, SolveConfig(), mid, np.array([oracle.loglik(inst, mid[0])]))
    assert res.n_modes == 0 and res.logZ == -np.inf
    # a single Gaussian centred outside the prior box: its mode is dropped
    out = make_instance(2, 1, 2, s_range=(0.5, 0.5), prior=(-1.0, 1.0))
    out.mu[0] = np.array([3.0, 0.0])
    res2 = oracle.laplace(out, SolveConfig(), out.mu[:1].copy(), np.array([oracle.loglik(out, out.mu[0])]))
    assert res2.n_modes == 0


def _brute_dedup(X, ell, tau):
    order = sorted(range(len(ell)), key=lambda i: (-ell[i], i))
    assigned = set()
    reps = []
    for a in order:
        if a in assigned:
            continue
        reps.append(a)
        assigned.add(a)
        for b in order:
            if b not in assigned and np.abs(X[a] - X[b]).max() <= tau:
                assigned.add(b)
    return reps


def test_dedup_collapses_duplicates_to_one_mode_per_component():
    insts, _ = workload(1, scale=0.05)
    inst = insts[0]
    rng = np.random.default_rng(8)
    X = np.concatenate([inst.mu[k] + rng.normal(0, 1e-4, (6, inst.d)) for k in range(inst.K)])
    ell = np.array([oracle.loglik(inst, x) for x in X])
    cfg = SolveConfig(dedup_coarse=1e-3)
    # brute force coarse dedup gives exactly one representative per component
    assert len(_brute_dedup(X, ell, 1e-3 * 20)) == inst.K
    res = oracle.laplace(inst, cfg, X, ell)
    assert res.n_modes == inst.K
    logV = np.log(inst.hi - inst.lo).sum()
    assert np.allclose(np.sort(res.logZk), np.sort(inst.log_w), atol=1e-10)  # Laplace term, no prior


# ----------------------------------------------------------- brute-force quadrature
def _gl_quadrature_logZ(inst, n_panels=400, order=16):
    """Tensor Gauss-Legendre on panels of the box, log-accumulated (d = 1 or 2)."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    axes, weights = [], []
    for i in range(inst.d):
        edges = np.linspace(inst.lo[i], inst.hi[i], n_panels + 1)
        a, b = edges[:-1, None], edges[1:, None]
        axes.append((0.5 * (b - a) * xg[None, :] + 0.5 * (a + b)).ravel())
        weights.append((0.5 * (b - a) * wg[None, :]).ravel())
    if inst.d == 1:
        X = axes[0][:, None]
        logw = np.log(weights[0])
    else:
        g0, g1 = np.meshgrid(axes[0], axes[1], indexing="ij")
        X = np.stack([g0.ravel(), g1.ravel()], 1)
        logw = (np.log(weights[0])[:, None] + np.log(weights[1])[None, :]).ravel()
    ell = scipy_loglik(inst, X)
    return logsumexp(ell + logw) - np.log(inst.hi - inst.lo).sum()


@pytest.mark.parametrize("d,K,sep", [(1, 1, 8.0), (1, 3, 8.0), (2, 1, 8.0), (2, 2, 8.0)])
def test_evidence_matches_quadrature_low_d(d, K, sep):
    # means at least 10 sigma inside the box, so truncation is far below the tolerance
    inst = make_instance(d, K, 40 + 10 * d + K, s_range=(0.15, 0.4), mean_box=(-6, 6), sep=sep,
                         prior=(-10.0, 10.0))
    cfg = SolveConfig(n_rays=64, n_steps=64, n_starts=128, seed=3)
    res = oracle.evidence(inst, cfg)
    q = _gl_quadrature_logZ(inst, n_panels=200 if d == 2 else 2000)
    assert res.n_modes == K
    assert res.logZ == pytest.approx(q, abs=1e-9)


def test_overlapping_modes_overestimate_2d_quadrature():
    """Sec. 5.6: overlapping modes make the sum of per-mode Laplace terms over-count."""
    sep = golden_claims()["overlap_4d_separation_sigma"]
    inst = make_instance(2, 2, 9, s_range=(1.0, 1.0), prior=(-10.0, 10.0), sep=0.0)
    inst.L[:] = np.eye(2)
    inst.mu[0] = np.array([-sep / 2, 0.0])
    inst.mu[1] = np.array([sep / 2, 0.0])
    inst.log_w[:] = np.log(0.5)
    res = oracle.laplace(inst, SolveConfig(), inst.mu.copy(), np.array([oracle.loglik(inst, m) for m in inst.mu]))
    q = _gl_quadrature_logZ(inst, n_panels=200)
    assert res.n_modes == 2
    assert res.logZ > q + 1e-3


def test_overlapping_modes_4d_sign_and_size():
    """4 unit Gaussians 3.5 sigma apart in 4D (Sec. 5.6): Z over-estimated by percent-level amounts.
    The true Z is the mixture's total weight (closed form), so no quadrature is needed."""
    claims = golden_claims()
    sep = claims["overlap_4d_separation_sigma"]
    d = 4
    inst = make_instance(d, 4, 10, s_range=(1.0, 1.0), prior=(-12.0, 12.0), sep=0.0)
    inst.L[:] = np.eye(d)
    corners = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float) * sep
    inst.mu[:] = 0.0
    inst.mu[:, :2] = corners - corners.mean(0)
    inst.log_w[:] = np.log(0.25)
    cfg = SolveConfig(n_rays=256, n_steps=64, n_starts=256, seed=5)
    res = oracle.evidence(inst, cfg)
    logV = np.log(inst.hi - inst.lo).sum()
    rel = math.expm1(res.logZ + logV)  # Z_comp / Z_true - 1 with Z_true = 1 / V
    assert res.n_modes == 4
    assert rel * claims["overlap_4d_error_sign"] > 0
    assert 1e-3 < rel < 0.2


def test_first_step_is_unit_length_and_backtracking_halves():
    """Readings 8-9 on a 1-d Gaussian (sigma = 0.1, mean 0): the first trial is a unit
    step against grad f; Armijo (c1 = 1e-4) rejects trials until f drops enough, each
    rejection multiplying alpha by the backtrack factor. Worked by hand:
    x0 = 0.3: alpha 1 -> -0.7 (f 24.5 > 4.5), alpha 1/2 -> -0.2 (f 2) accepted;
    x0 = 0.05: alphas 1, 1/2, 1/4, 1/8 give f 45, 10.1, 2, 0.28 > 0.125, 1/16 -> -0.0125;
    x0 = 2: alpha 1 -> 1 (f 50 < 200) accepted; factor 1/4 from 0.3: alpha 1/4 -> 0.05."""
    inst = make_instance(1, 1, 1, s_range=(1.0, 1.0))
    inst.L[0] = 10.0
    inst.mu[0] = 0.0
    for x0, x1, bt in [(0.3, -0.2, 0.5), (0.05, -0.0125, 0.5), (2.0, 1.0, 0.5), (0.3, 0.05, 0.25)]:
        r = oracle.lbfgs(inst, SolveConfig(max_iter=1, backtrack=bt), np.array([[x0]]))
        assert r.x[0, 0] == pytest.approx(x1, abs=1e-15)
        assert r.status[0] == oracle.MAXITER and r.iters[0] == 1
