"""GPU parity of the tensor-core (tcgen05) log-likelihood and gradient against
the FP64 oracle, through the C ABI, element by element.

Two error models built from the FP64 operands (tests/tc_bound.py) bound each
value of l and each gradient coordinate:
 - a worst case (every rounding of x - mu_k and L_k to bf16 / tf32, every FP32
   accumulation, the FP32 LSE and responsibilities, all at their extremes and of
   one sign): the measured error must lie inside it;
 - a standard deviation under independent roundings (first-order probabilistic
   error analysis, sqrt(d) growth): the measured error must stay within C_SIGMA of
   it, a few times the largest ratio measured on a GB300 over these cases (about
   4 sigma over ~10^5 entries, as independent roundings give).
A kernel that dropped one K chunk of c of the d terms, read a mis-swizzled tile or
added a component twice would move z_kj by a partial sum, about
sqrt(c / d) sqrt(sum_i a_i^2 L_k,ij^2), that is sqrt(c / d) / u_p standard
deviations (64 for bf16 and 362 for tf32 at d = 1024, c = 64 and 32 elements of one
128-byte chunk), and fail.
The gradient's direction is also checked: 1 - cos(grad, oracle grad) <= u_p.
Largest ratios measured on a GB300 over these cases (worst case; sigma):
bf16 0.33; 3.64 (the overlapping mixture) and tf32 0.28; 4.75 (d = 128, K = 2);
1 - cos at most 2.2e-4 (bf16) and 3.0e-6 (tf32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
import tc_bound
from paper_2601_19957_gb300.instances import make_instance

pytestmark = pytest.mark.gpu

# allowed error in standard deviations of the rounding model: about 3.8 times the largest
# ratio measured per precision
C_SIGMA = {sb.PREC_BF16: 14.0, sb.PREC_TF32: 18.0}


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def ratios(inst, X, prec):
    """Largest error over the points as a fraction of the worst case (l, grad), in standard
    deviations of the rounding model (l, grad), and the largest 1 - cos of the gradients."""
    prob = sb.Problem(inst)
    ell, g = sb.loglik(prob, torch.as_tensor(X, device="cuda"), prec=prec)
    ell, g = ell.cpu().numpy(), g.cpu().numpy()
    B_l, B_g, _, _ = tc_bound.bounds(inst, X, prec)
    s_l, s_g = tc_bound.sigmas(inst, X, prec)
    w = np.zeros(5)
    for i in range(X.shape[0]):
        le, ge = oracle.loglik(inst, X[i], want_grad=True)
        dl, dg = abs(ell[i] - le), np.abs(g[i] - ge)
        w[0] = max(w[0], dl / B_l[i])
        w[1] = max(w[1], float(np.max(dg / B_g[i])))
        w[2] = max(w[2], dl / s_l[i])
        w[3] = max(w[3], float(np.max(dg / np.maximum(s_g[i], 1e-300))))
        ng = np.linalg.norm(ge) * np.linalg.norm(g[i])
        if ng > 0:
            w[4] = max(w[4], 1.0 - float(g[i] @ ge) / ng)
    return tuple(float(v) for v in w)


def _check(inst, X, prec, grad=True):
    wl, wg, sl, sg, wc = ratios(inst, X, prec)
    assert wl <= 1.0 and sl <= C_SIGMA[prec], (wl, sl)
    if grad:
        assert wg <= 1.0 and sg <= C_SIGMA[prec], (wg, sg)
        assert wc <= tc_bound.U_P[prec], wc


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
@pytest.mark.parametrize("d,K,n", [(64, 1, 128), (64, 4, 300), (128, 2, 129), (256, 1, 200), (200, 3, 77),
                                   (1024, 2, 130)])
def test_tc_loglik_matches_oracle(prec, d, K, n):
    inst = make_instance(d, K, 900 + d + K, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    rng = np.random.default_rng(d + K)
    X = inst.mu[rng.integers(0, K, n)] + rng.normal(0, 0.3, (n, d)) * rng.uniform(0, 1, (n, 1))
    _check(inst, X, prec)


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
    _check(inst, X, prec, grad=False)


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
    _check(inst, X, prec)


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_tc_loglik_components_beyond_32(prec):
    """K = 40: the component masks of the tensor-core path hold one bit per component
    (up to 64), so points near components 32..39 get those components' terms in l and
    their chunks in the gradient GEMM (a 32-bit mask would drop them: l would miss its
    largest term and the gradient would be the other components' alone)."""
    inst = make_instance(16, 40, 4400, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    rng = np.random.default_rng(40)
    ks = np.concatenate([np.arange(32, 40).repeat(24), rng.integers(0, 40, 64)])
    X = inst.mu[ks] + rng.normal(0, 0.1, (len(ks), inst.d))
    _check(inst, X, prec)
