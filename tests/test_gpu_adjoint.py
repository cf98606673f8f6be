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
