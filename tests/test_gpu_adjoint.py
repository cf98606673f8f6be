"""Adjoint of log Z (d log Z / d mu_k, d log Z / d L_k) through the C ABI and
torch.autograd, against central finite differences (h = 1e-6, FP64) of the
ORACLE's log Z. The oracle's difference quotient re-runs its own Laplace stage
at the perturbed parameters, started from its own unperturbed modes, so the
check covers the implicit shift of each mode. FD error ~ h^2 + eps |log Z| / h
~ 1e-9; the bound below is 1e-6 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import SolveConfig, make_instance, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _overlapping(d, K, seed):
    """Components about 2.5 sigma apart: distinct modes, O(1) gradients."""
    inst = make_instance(d, K, seed, s_range=(0.6, 1.0), mean_box=(-1.5, 1.5), sep=2.5, prior=(-12.0, 12.0))
    return inst


def _fd_oracle(inst, cfg, modes0, h=1e-6):
    def logZ(i2):
        ell = np.array([oracle.loglik(i2, m) for m in modes0])
        return oracle.laplace(i2, cfg, modes0, ell).logZ

    d, K = inst.d, inst.K
    gmu = np.zeros((K, d))
    gL = np.zeros((K, d, d))
    for k in range(K):
        for i in range(d):
            ip = _copy(inst)
            im = _copy(inst)
            ip.mu[k, i] += h
            im.mu[k, i] -= h
            gmu[k, i] = (logZ(ip) - logZ(im)) / (2 * h)
            for j in range(i + 1):
                ip = _copy(inst)
                im = _copy(inst)
                ip.L[k, i, j] += h
                im.L[k, i, j] -= h
                gL[k, i, j] = (logZ(ip) - logZ(im)) / (2 * h)
    return gmu, gL


def _copy(inst):
    import copy

    c = copy.deepcopy(inst)
    return c


@pytest.mark.parametrize("d,K,seed", [(2, 2, 2), (3, 2, 5), (3, 3, 8)])
def test_adjoint_matches_oracle_finite_differences(d, K, seed):
    inst = _overlapping(d, K, seed)
    cfg = SolveConfig(n_rays=128, n_steps=64, n_starts=128, seed=11)
    ref = oracle.evidence(inst, cfg)
    assert ref.n_modes >= 2
    gmu_fd, gL_fd = _fd_oracle(inst, cfg, ref.modes)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)
    mu = t(inst.mu).requires_grad_(True)
    L = t(inst.L).requires_grad_(True)
    logZ = sb.evidence_autograd(mu, L, t(inst.log_w), t(inst.lo), t(inst.hi), sb.make_config(cfg))
    assert abs(float(logZ) - ref.logZ) <= 1e-10 * abs(ref.logZ)
    logZ.backward()
    gmu, gL = mu.grad.cpu().numpy(), L.grad.cpu().numpy()
    scale = 1.0 + max(np.abs(gmu_fd).max(), np.abs(gL_fd).max())
    assert np.abs(gmu - gmu_fd).max() <= 1e-6 * scale, (gmu, gmu_fd)
    assert np.abs(np.tril(gL) - gL_fd).max() <= 1e-6 * scale, (gL, gL_fd)
    assert np.abs(np.triu(gL, 1)).max() == 0.0
    assert np.abs(gmu_fd).max() > 1e-3  # the check is not vacuous


def test_adjoint_vanishes_for_separated_mixture_d1024():
    """Separated normalised mixture: log Z = log sum w - log V does not depend on mu or L."""
    insts, c = workload(4, scale=1.0 / 64)
    inst = insts[0]
    c.prec = sb.PREC_BF16
    c.cand_cap = 16
    prob = sb.Problem(inst)
    out = sb.evidence(prob, sb.make_config(c))
    assert out.n_modes >= 1
    dmu, dL = sb.evidence_backward(prob, out.modes, out.logZk, out.n_modes)
    assert float(dmu.abs().max()) < 1e-8
    assert float(dL.abs().max()) < 1e-8


@pytest.mark.parametrize("d,K,seed", [(2, 2, 2), (3, 3, 8), (5, 2, 13), (8, 3, 23)])
def test_adjoint_matches_complex_step_reference(d, K, seed):
    """Element-wise against the complex-step derivatives of the Laplace evidence
    (oracle/laplace_cs.py: no subtraction, exact to rounding), at the same modes:
    every d log Z / d mu_k,i and d log Z / d L_k,ij to 1e-9 (absolute, or relative to the
    largest entry when that exceeds 1)."""
    from oracle import laplace_cs

    inst = _overlapping(d, K, seed)
    cfg = SolveConfig(n_rays=128, n_steps=64, n_starts=128, seed=11)
    prob = sb.Problem(inst)
    out = sb.evidence(prob, sb.make_config(cfg))
    assert out.n_modes >= 2
    dmu, dL = sb.evidence_backward(prob, out.modes, out.logZk, out.n_modes)
    logZ_cs, gmu, gL = laplace_cs.dlogz(inst, out.modes.cpu().numpy())
    assert abs(out.logZ - logZ_cs) <= 1e-10 * abs(logZ_cs)
    scale = max(np.abs(gmu).max(), np.abs(gL).max())
    assert scale > 1e-3  # overlapping components: the check is not vacuous
    tol = 1e-9 * max(1.0, scale)
    assert np.abs(dmu.cpu().numpy() - gmu).max() <= tol
    assert np.abs(np.tril(dL.cpu().numpy()) - gL).max() <= tol
    assert np.abs(np.triu(dL.cpu().numpy(), 1)).max() == 0.0


def test_adjoint_overlapping_mixture_d1024_central_differences():
    """d = 1024, two overlapping components (2 units apart, standard deviations 0.6-1,
    so each mode carries the other's responsibility and the derivatives are O(0.1)): the
    adjoint's directional derivatives along 3 random unit directions (over the means,
    over the diagonals of the L_k, over the whole lower triangles) and along 16 single
    coordinates (8 of the means, 8 diagonal entries of the L_k) against h = 1e-6
    central differences of the oracle's Laplace stage, re-polished from the modes at the
    perturbed parameters (the implicit shift of the modes included). FD error: h^2 terms
    ~1e-12 and rounding eps |log Z| / h ~ 7e-7; the bound is 5e-6 + 1e-6 |value|."""
    import concurrent.futures as cf
    import copy

    d, K = 1024, 2
    inst = make_instance(d, K, 41, s_range=(0.6, 1.0), mean_box=(-3, 3), sep=0.0, prior=(-12.0, 12.0))
    rng = np.random.default_rng(3)
    e = rng.normal(size=d)
    inst.mu[1] = inst.mu[0] + 2.0 * e / np.linalg.norm(e)
    inst = inst.contiguous()
    cfg = SolveConfig(n_rays=256, n_steps=64, n_starts=256, m=20, seed=5, prec=sb.PREC_BF16, cand_cap=16)
    prob = sb.Problem(inst)
    out = sb.evidence(prob, sb.make_config(cfg))
    assert out.n_modes == 2
    dmu, dL = sb.evidence_backward(prob, out.modes, out.logZk, out.n_modes)
    dmu, dL = dmu.cpu().numpy(), np.tril(dL.cpu().numpy())
    modes0 = out.modes.cpu().numpy()
    c64 = SolveConfig(**{**cfg.__dict__, "prec": 0})

    def logZ_at(vmu, vL, h):
        i2 = copy.deepcopy(inst)
        i2.mu = inst.mu + h * vmu
        i2.L = inst.L + h * vL
        i2 = i2.contiguous()
        ell = np.array([oracle.loglik(i2, m) for m in modes0])
        return oracle.laplace(i2, c64, modes0, ell).logZ

    dirs = []
    vmu = rng.normal(size=(K, d))
    dirs.append((vmu / np.linalg.norm(vmu), np.zeros((K, d, d))))
    vL = np.zeros((K, d, d))
    vL[:, np.arange(d), np.arange(d)] = rng.normal(size=(K, d))
    dirs.append((np.zeros((K, d)), vL / np.linalg.norm(vL)))
    vL = np.tril(rng.normal(size=(K, d, d)))
    dirs.append((np.zeros((K, d)), vL / np.linalg.norm(vL)))
    for t in range(16):
        vmu, vL = np.zeros((K, d)), np.zeros((K, d, d))
        k, i = int(rng.integers(K)), int(rng.integers(d))
        if t < 8:
            vmu[k, i] = 1.0
        else:
            vL[k, i, i] = 1.0
        dirs.append((vmu, vL))
    h = 1e-6
    jobs = [(v, s) for v in dirs for s in (h, -h)]
    with cf.ThreadPoolExecutor(max_workers=min(16, len(jobs))) as ex:  # the oracle releases the GIL
        vals = list(ex.map(lambda j: logZ_at(j[0][0], j[0][1], j[1]), jobs))
    worst = 0.0
    biggest = 0.0
    for q, (vmu, vL) in enumerate(dirs):
        fd = (vals[2 * q] - vals[2 * q + 1]) / (2 * h)
        ad = float((dmu * vmu).sum() + (dL * vL).sum())
        worst = max(worst, abs(ad - fd) / (5e-6 + 1e-6 * abs(fd)))
        biggest = max(biggest, abs(fd))
    assert worst <= 1.0, worst
    assert biggest > 1e-2  # the responsibilities overlap: the check is not vacuous
