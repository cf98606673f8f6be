"""GPU parity of the tensor-core (tcgen05) log-likelihood and gradient against
the FP64 oracle, through the C ABI.

Error model: the MMA operands are (x - mu_k) and L_k rounded to bf16 (8-bit
significand, unit roundoff u = 2^-9) or tf32 (11 bits, u = 2^-12) with FP32
accumulation, so z_k = L_k^T (x - mu_k) carries a relative error of a few u
per entry and |z|^2 about 2u sqrt(d)-scaled; l = LSE(a - |z|^2/2) therefore
errs by about c u |z|^2, and grad l by about c u |grad l|. The bounds below
are those estimates with a safety factor; the exact FP64 answer comes from the
FP64 Newton polish, which these tests do not exercise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import make_instance

pytestmark = pytest.mark.gpu

U = {sb.PREC_BF16: 2.0 ** -9, sb.PREC_TF32: 2.0 ** -12}


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _check(inst, X, prec):
    prob = sb.Problem(inst)
    ell, g = sb.loglik(prob, torch.as_tensor(X, device="cuda"), prec=prec)
    ell, g = ell.cpu().numpy(), g.cpu().numpy()
    u = U[prec]
    worst_l, worst_g = 0.0, 0.0
    for i in range(X.shape[0]):
        le, ge = oracle.loglik(inst, X[i], want_grad=True)
        # |z|^2 of the dominant component ~ 2 (a_max - l)
        a_max = np.max(inst.log_w - 0.5 * inst.d * np.log(2 * np.pi) + np.log(np.diagonal(inst.L, axis1=1, axis2=2)).sum(1))
        q = max(2.0 * (a_max - le), 1.0)
        err_l = abs(ell[i] - le) / (u * (q + inst.d))
        err_g = np.linalg.norm(g[i] - ge) / (u * (np.linalg.norm(ge) + 1.0) * np.sqrt(inst.d))
        worst_l, worst_g = max(worst_l, err_l), max(worst_g, err_g)
    return worst_l, worst_g


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
@pytest.mark.parametrize("d,K,n", [(64, 1, 128), (64, 4, 300), (128, 2, 129), (256, 1, 200), (200, 3, 77),
                                   (1024, 2, 130)])
def test_tc_loglik_matches_oracle(prec, d, K, n):
    inst = make_instance(d, K, 900 + d + K, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    rng = np.random.default_rng(d + K)
    X = inst.mu[rng.integers(0, K, n)] + rng.normal(0, 0.3, (n, d)) * rng.uniform(0, 1, (n, 1))
    wl, wg = _check(inst, X, prec)
    assert wl < 16.0, wl
    assert wg < 16.0, wg


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_tc_gradient_vanishes_at_the_mean(prec):
    """Centring in FP32 before rounding keeps the stationary point: at x = mu_k the
    A operand is exactly zero, so z and the gradient are exactly zero."""
    inst = make_instance(256, 1, 4, s_range=(0.01, 1.0), mean_box=(-2, 2))
    prob = sb.Problem(inst)
    x = torch.as_tensor(inst.mu[:1].astype(np.float32).astype(np.float64), device="cuda")
    _, g = sb.loglik(prob, x, prec=prec)
    assert float(g.abs().max()) == 0.0


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_tc_far_points_values(prec):
    inst = make_instance(64, 4, 12, s_range=(0.05, 0.5), mean_box=(-6, 6))
    X = np.random.default_rng(3).uniform(-10, 10, (200, 64))
    wl, _ = _check(inst, X, prec)
    assert wl < 16.0


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_tc_gradient_overlapping_and_mixed_blocks(prec):
    """Overlapping components put several non-zero responsibilities in one row,
    so the store pass and the gradient GEMM visit several components of a row
    block; rows near a single mode are interleaved with them, so one 128-row
    block mixes shared and exactly-zero responsibilities, and a block of rows
    near one mode only (rows 256..383) leaves the other components unvisited."""
    inst = make_instance(96, 3, 77, s_range=(0.4, 0.6), mean_box=(-0.5, 0.5), sep=0.5)
    rng = np.random.default_rng(5)
    n = 400
    between = (inst.mu[0] + inst.mu[1] + inst.mu[2]) / 3.0 + rng.normal(0, 0.2, (n, inst.d))
    near = inst.mu[rng.integers(0, 3, n)] + rng.normal(0, 0.05, (n, inst.d))
    X = np.where((np.arange(n) % 2 == 0)[:, None], between, near)
    X[256:384] = inst.mu[1] + rng.normal(0, 0.05, (128, inst.d))
    wl, wg = _check(inst, X, prec)
    assert wl < 16.0, wl
    assert wg < 16.0, wg
