"""GPU parity of the preprocessing probe (Sec. 3.4), the other ray families with
their two-pass sampling (Sec. 3.5.1-3.5.2), the black-box central differences
(App. A.4, Sec. 3.7.2) and the quadratic-in-t form of the sunburst coarse pass,
against the FP64 CPU oracle, through the C ABI.

Tolerances, from the arithmetic of each side:
 - Every l is an FP64 sum of d K products; the two sides sum in different
   orders (and the GPU forms the precheck and segment values from z at two
   points), so an l differs by at most a few ulps of the largest term it
   cancels: |dl| <= 1e-12 (1 + |terms|), |terms| bounded by the largest |l| of
   the points involved (every term a_k - |z_k|^2 / 2 is at most that large
   where it matters).
 - Classes, ray end points (the same Philox blocks and the same rounded
   operations on both sides) and the count of active coordinates are exact.
 - A central difference divides an l error delta by its step, so the
   black-box gradient is off by at most delta / eps_g, the Hessian diagonal
   by 4 delta / eps_h^2, an off-diagonal entry by delta / eps_h^2.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import tc_bound
import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import SolveConfig, make_instance, workload

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _diag_instance(sig, prior=(-10.0, 10.0)):
    d = len(sig)
    inst = make_instance(d, 1, 1, s_range=(1.0, 1.0), prior=prior)
    inst.L[0] = np.diag(1.0 / np.asarray(sig, dtype=float))
    inst.mu[0] = 0.5 * (inst.lo + inst.hi)
    return inst.contiguous()


# ------------------------------------------------------------------ preprocessing probe (Sec. 3.4)
def _precheck_cases():
    return [
        ("mixture d=64 K=4", make_instance(64, 4, 1000, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)),
        ("flat + soft coordinates", _diag_instance([0.01, 0.02, 0.015, 1.0, 0.8, 1e5])),
        ("even-count median", _diag_instance(10.0 / np.sqrt([1.5e-6, 1.0, 3.0, 4.0]))),
        ("d=1", _diag_instance([3.0])),
        ("ragged d=1000 K=3", make_instance(1000, 3, 77, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)),
    ]


@pytest.mark.parametrize("name,inst", _precheck_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_precheck_matches_oracle(name, inst):
    prob = sb.Problem(inst)
    out = sb.precheck(prob)
    ref = oracle.precheck(inst)
    s = out.s.cpu().numpy()
    c = 0.5 * (inst.lo + inst.hi)
    l0 = abs(oracle.loglik(inst, c))
    # the oracle subtracts l at c +- Delta e_i from l(c); both l are at most |l(c)| + s_i
    tol = 1e-12 * (1.0 + l0 + ref.s)
    assert np.all(np.abs(s - ref.s) <= tol), np.max(np.abs(s - ref.s) / tol)
    assert out.cls.cpu().numpy().tolist() == ref.cls.tolist()
    assert out.n_active == ref.n_active
    assert out.log_int == pytest.approx(ref.log_int, rel=1e-12, abs=1e-12)
    assert out.log_vol == pytest.approx(ref.log_vol, rel=1e-12, abs=1e-12)


def test_precheck_full_size_workload():
    """The d = 1024, K = 8 mixture: every s_i against the oracle, nothing flagged (every
    coordinate of a mixture with these widths is informative)."""
    inst = workload(4)[0][0]
    out = sb.precheck(sb.Problem(inst))
    ref = oracle.precheck(inst)
    s = out.s.cpu().numpy()
    l0 = abs(oracle.loglik(inst, 0.5 * (inst.lo + inst.hi)))
    assert np.all(np.abs(s - ref.s) <= 1e-12 * (1.0 + l0 + ref.s))
    assert out.cls.cpu().numpy().tolist() == ref.cls.tolist()
    assert out.n_active == ref.n_active == inst.d


# ------------------------------------------------------------------ ray families and two-pass sampling
@pytest.mark.parametrize("family", [sb.RAY_V2V, sb.RAY_V2E, sb.RAY_W2W])
@pytest.mark.parametrize("d,K,n_rays,n_steps,delta,n_ref", [
    (1, 1, 5, 1, math.inf, 3),
    (7, 2, 33, 17, 5.0, 20),
    (64, 4, 130, 64, 10.0, 64),
    (100, 3, 65, 128, math.inf, 0),
])
def test_segments_match_oracle(family, d, K, n_rays, n_steps, delta, n_ref):
    inst = make_instance(d, K, 300 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0 if K > 1 else 0.0)
    seed = 0x1234_5678_9ABC + d
    out = sb.segments(sb.Problem(inst), family, seed, n_rays, n_steps, delta, n_ref)
    A, B = out.start.cpu().numpy(), out.end.cpu().numpy()
    lc = out.ell_coarse.cpu().numpy()
    tr = out.t_ref.cpu().numpy()
    lr = out.ell_ref.cpu().numpy()
    for r in range(n_rays):
        a, b = oracle.ray_segment(inst, family, seed, r)
        assert np.array_equal(A[r], a) and np.array_equal(B[r], b), r
        rc, rt, rl = oracle.ray_two_pass(inst, a, b, n_steps, delta, n_ref)
        scale = 1.0 + np.abs(rc).max()
        assert np.abs(lc[r] - rc).max() <= 1e-12 * scale, (r, np.abs(lc[r] - rc).max())
        if n_ref:
            # t comes from the cumulative weights exp(l_j - max l): an l error of 1e-12 scale
            # moves it by ~1e-12 of a cell
            assert np.abs(tr[r] - rt).max() <= 1e-9, r
            assert np.abs(lr[r] - rl).max() <= 1e-12 * scale + 1e-9 * np.abs(rl).max(), r


# ------------------------------------------------------------------ black-box derivatives (App. A.4)
@pytest.mark.parametrize("d,K,full", [(1, 1, True), (2, 2, True), (9, 3, True), (64, 4, True), (200, 2, False)])
def test_fd_derivatives_match_oracle(d, K, full):
    inst = make_instance(d, K, 600 + d, s_range=(0.2, 1.0), mean_box=(-4, 4), sep=4.0 if K > 1 else 0.0)
    x = inst.mu[0] + np.random.default_rng(d).normal(0, 0.1, d)
    eps_g, eps_h = 1e-5, 1e-4
    out = sb.fd_derivatives(sb.Problem(inst), torch.as_tensor(x, device="cuda"), eps_g, eps_h, full=full)
    lx = abs(oracle.loglik(inst, x))
    # l at points eps away from x: |l| <= |l(x)| + 1; both sides round each l to a few ulps of
    # its largest term, d K of them summed: delta = 4 d K u (1 + |l|)
    delta = 4 * d * K * U * (2.0 + lx)
    g = oracle.fd_grad(inst, x, eps_g)
    hd = oracle.fd_hess_diag(inst, x, eps_h)
    assert np.abs(out.grad.cpu().numpy() - g).max() <= delta / eps_g
    assert np.abs(out.hdiag.cpu().numpy() - hd).max() <= 4 * delta / eps_h ** 2
    if full:
        H = oracle.fd_hess_full(inst, x, eps_h)
        assert np.abs(out.H.cpu().numpy() - H).max() <= 4 * delta / eps_h ** 2
        assert np.array_equal(out.H.cpu().numpy(), out.H.cpu().numpy().T)
    b = oracle.uniform_corr_probe(inst, x, hd, eps_h)
    assert abs(out.b - b) <= 8 * delta / eps_h ** 2


def test_fd_probe_recovers_an_equicorrelated_precision():
    """Uniform correlation: P = a I + b 1 1^T gives b back from two evaluations (the GPU
    reads its diagonal from the same batch)."""
    d, a, b = 12, 2.0, 0.3
    inst = make_instance(d, 1, 5, s_range=(1.0, 1.0))
    P = a * np.eye(d) + b * np.ones((d, d))
    inst.L[0] = np.linalg.cholesky(P)
    inst.mu[0] = 0.0
    inst = inst.contiguous()
    out = sb.fd_derivatives(sb.Problem(inst), torch.zeros(d, dtype=torch.float64, device="cuda"), full=False)
    # the Hessian of l is -P: the probe returns the off-diagonal value -b
    assert out.b == pytest.approx(-b, abs=1e-5)
    np.testing.assert_allclose(out.hdiag.cpu().numpy(), -(a + b), atol=1e-5)


# ------------------------------------------------------------------ coarse pass from three scalars per ray
@pytest.mark.parametrize("d,K,n_rays,n_steps", [(8, 1, 64, 16), (64, 4, 300, 64), (130, 3, 129, 33)])
def test_ray_loglik_quad_fp64_matches_oracle(d, K, n_rays, n_steps):
    inst = make_instance(d, K, 700 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0 if K > 1 else 0.0)
    cfg = SolveConfig(n_rays=n_rays, n_steps=n_steps, n_starts=1, seed=d)
    u, te, ref = oracle.ray_loglik(inst, cfg)
    ell = sb.ray_loglik_quad(sb.Problem(inst), torch.as_tensor(u, device="cuda"), n_steps, form=0).cpu().numpy()
    # |z(t)|^2 = q0 + 2 tau q1 + tau^2 q2 cancels terms as large as the largest |l| on the ray
    scale = 1.0 + np.abs(ref).max(1, keepdims=True)
    assert np.all(np.abs(ell - ref) <= 1e-12 * scale), np.max(np.abs(ell - ref) / scale)


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("d,K,n_rays,n_steps", [(8, 1, 64, 16), (64, 4, 300, 64), (130, 3, 129, 33), (1, 2, 5, 3)])
def test_ray_loglik_quad_mixed_forms_match_oracle(form, d, K, n_rays, n_steps):
    """The FP32 SIMT form (1) and the tensor-core split forms (2 BF16, 3 TF32) at every
    sample of the oracle's rays, within the quadratic ray pass's error model
    (tc_bound.check_ray_samples; FP32: operands rounded to FP32, no accumulation bias)."""
    inst = make_instance(d, K, 700 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0 if K > 1 else 0.0)
    cfg = SolveConfig(n_rays=n_rays, n_steps=n_steps, n_starts=1, seed=d)
    u, te, ref = oracle.ray_loglik(inst, cfg)
    ell = sb.ray_loglik_quad(sb.Problem(inst), torch.as_tensor(u, device="cuda"), n_steps, form=form).cpu().numpy()
    c = 0.5 * (inst.lo + inst.hi)
    tau = (np.arange(1, n_steps + 1) / n_steps)[None, :] * te[:, None]
    X = (c[None, None, :] + tau[:, :, None] * u[:, None, :]).reshape(-1, d)
    prec = {1: 0, 2: sb.PREC_BF16, 3: sb.PREC_TF32}[form]
    tc_bound.check_ray_samples(inst, X, (ell - ref).reshape(-1), prec)


@pytest.mark.parametrize("form", [2, 3])
@pytest.mark.parametrize("d,K,n_rays,n_steps", [(64, 4, 130, 16), (300, 3, 70, 24), (1024, 8, 64, 16), (7, 2, 40, 8),
                                                (1, 1, 9, 5)])
def test_ray_loglik_origins_matches_oracle(form, d, K, n_rays, n_steps):
    """Rays from per-ray origins (the reseeding rays of ChiSao): half the origins near a
    component mean (Golden Rooster rays start at peaks), half uniform in the box (Repulse
    Monkey rays start at unconverged samples). t_exit against its definition (bit for
    bit), l at every sample against the FP64 oracle within the quadratic ray pass's error
    model for an origin pass (tc_bound.check_ray_samples with the origins)."""
    if d == 1024:
        inst = workload(4)[0][0]
    else:
        inst = make_instance(d, K, 800 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0 if K > 1 else 0.0)
    rng = np.random.default_rng(900 + d)
    O = rng.uniform(inst.lo, inst.hi, (n_rays, d))
    near = np.arange(n_rays) % 2 == 0
    ks = rng.integers(0, inst.K, n_rays)
    O[near] = np.clip(inst.mu[ks[near]] + 0.01 * rng.standard_normal((near.sum(), d)), inst.lo, inst.hi)
    U = rng.standard_normal((n_rays, d))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    ell, te = sb.ray_loglik_origins(sb.Problem(inst), torch.as_tensor(O), torch.as_tensor(U), n_steps, form=form)
    ell, te = ell.cpu().numpy(), te.cpu().numpy()
    with np.errstate(divide="ignore", invalid="ignore"):
        cand = np.where(U > 0, (inst.hi - O) / U, np.where(U < 0, (inst.lo - O) / U, np.inf))
    np.testing.assert_array_equal(te, cand.min(1))
    tau = (np.arange(1, n_steps + 1) / n_steps)[None, :] * te[:, None]
    X = (O[:, None, :] + tau[:, :, None] * U[:, None, :]).reshape(-1, d)
    Orep = np.repeat(O, n_steps, axis=0)
    ref = np.array([oracle.loglik(inst, x) for x in X])
    prec = {2: sb.PREC_BF16, 3: sb.PREC_TF32}[form]
    tc_bound.check_ray_samples(inst, X, ell.reshape(-1) - ref, prec, O=Orep)


@pytest.mark.parametrize("form", [2, 3])
def test_ray_loglik_origins_edge_cases(form):
    """Origins on the box surface and at a corner, axis-aligned directions (every other
    coordinate of u zero), a ray leaving through the face it starts on (t_exit = 0, every
    sample at the origin), one step per ray, one ray and 129 rays (a ragged 128-row
    tile): t_exit against its definition bit for bit and l within the error model."""
    d, K = 48, 3
    inst = make_instance(d, K, 4848, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    rng = np.random.default_rng(4849)
    n = 129
    O = rng.uniform(inst.lo, inst.hi, (n, d))
    U = rng.standard_normal((n, d))
    O[0] = inst.hi                            # a corner
    O[1, 5] = inst.lo[5]                      # on a face, leaving through it
    U[1] = 0.0
    U[1, 5] = -1.0
    O[2, 7] = inst.hi[7]                      # on a face, entering the box
    U[2] = 0.0
    U[2, 7] = -1.0
    U[3] = 0.0
    U[3, 0] = 1.0                             # axis-aligned from inside
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    prec = {2: sb.PREC_BF16, 3: sb.PREC_TF32}[form]
    for rows, n_steps in ((n, 1), (1, 7), (n, 5)):
        Or, Ur = O[:rows], U[:rows]
        ell, te = sb.ray_loglik_origins(sb.Problem(inst), torch.as_tensor(Or), torch.as_tensor(Ur), n_steps,
                                        form=form)
        ell, te = ell.cpu().numpy(), te.cpu().numpy()
        with np.errstate(divide="ignore", invalid="ignore"):
            cand = np.where(Ur > 0, (inst.hi - Or) / Ur, np.where(Ur < 0, (inst.lo - Or) / Ur, np.inf))
        np.testing.assert_array_equal(te, cand.min(1))
        if rows > 1:
            assert te[1] == 0.0 and te[2] > 0.0
        tau = (np.arange(1, n_steps + 1) / n_steps)[None, :] * te[:, None]
        X = (Or[:, None, :] + tau[:, :, None] * Ur[:, None, :]).reshape(-1, d)
        ref = np.array([oracle.loglik(inst, x) for x in X])
        tc_bound.check_ray_samples(inst, X, ell.reshape(-1) - ref, prec, O=np.repeat(Or, n_steps, axis=0))
