"""sb_loglik_noalloc: the batched likelihood for callers that cannot allocate
device memory (code inside a host application that owns every device
allocation, or a plugin that may not call cudaMalloc). Its scratch is an array
inside the library, so the caller passes only inputs and outputs. Checked
against sb_loglik (caller-provided workspace) through the C ABI, on two calls in
a row with different inputs, within the tolerances of the other likelihood
tests: 1e-12 relative in FP64; for BF16 / TF32 the tensor-core rounding model of
tests/tc_bound.py, against sb_loglik and against the FP64 oracle. This file is
collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
import tc_bound
from paper_2601_19957_gb300.instances import make_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _noalloc(prob, x, want_grad=True, prec=sb.PREC_FP64):
    n = x.shape[0]
    ell = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(x) if want_grad else None
    code = sb.lib().sb_loglik_noalloc(C.byref(prob.s), C.c_int32(prec), sb._ptr(x), C.c_int32(n),
                                      sb._ptr(ell), sb._ptr(grad), sb._stream())
    return code, ell, grad


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    inst = make_instance(64, 4, 77, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    prob = sb.Problem(inst)
    rng = np.random.default_rng(5)
    for call, n in enumerate((300, 129)):
        X = inst.mu[rng.integers(0, inst.K, n)] + rng.normal(0, 0.3, (n, inst.d))
        x = torch.as_tensor(X, device="cuda")
        ref_ell, ref_grad = sb.loglik(prob, x)
        code, ell, grad = _noalloc(prob, x)
        assert code == sb.SB_OK, (call, sb.status_string(code))
        torch.cuda.synchronize()
        r_e, r_g = ref_ell.cpu().numpy(), ref_grad.cpu().numpy()
        e, g = ell.cpu().numpy(), grad.cpu().numpy()
        assert np.all(np.abs(e - r_e) <= 1e-12 * (1 + np.abs(r_e))), call
        assert np.all(np.abs(g - r_g) <= 1e-12 * (1 + np.abs(r_g).max())), call


def test_noalloc_rejects_requests_beyond_its_scratch():
    inst = make_instance(1024, 8, 3, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    prob = sb.Problem(inst)
    x = torch.zeros((4096, 1024), dtype=torch.float64, device="cuda")  # needs ~270 MB of scratch
    code, _, _ = _noalloc(prob, x)
    assert code == sb.SB_ERR_WORKSPACE


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_noalloc_tensor_core_path_on_two_calls(prec):
    """The tensor-core path through the library's array (its TMA maps point into it):
    two calls in a row, each within 14 (bf16) / 18 (tf32) standard deviations of the
    rounding model of sb_loglik's result and of the FP64 oracle's, and inside the
    worst-case bound."""
    c_sigma = {sb.PREC_BF16: 14.0, sb.PREC_TF32: 18.0}[prec]
    inst = make_instance(200, 3, 1203, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    prob = sb.Problem(inst)
    rng = np.random.default_rng(9)
    for call, n in enumerate((257, 100)):
        X = inst.mu[rng.integers(0, inst.K, n)] + rng.normal(0, 0.3, (n, inst.d)) * rng.uniform(0, 1, (n, 1))
        x = torch.as_tensor(X, device="cuda")
        code, ell, grad = _noalloc(prob, x, prec=prec)
        assert code == sb.SB_OK, (call, sb.status_string(code))
        ref_ell, ref_grad = sb.loglik(prob, x, prec=prec)
        e, g = ell.cpu().numpy(), grad.cpu().numpy()
        r_e, r_g = ref_ell.cpu().numpy(), ref_grad.cpu().numpy()
        s_l, s_g = tc_bound.sigmas(inst, X, prec)
        B_l, B_g, _, _ = tc_bound.bounds(inst, X, prec)
        assert np.all(np.abs(e - r_e) <= c_sigma * s_l), call
        assert np.all(np.abs(g - r_g) <= c_sigma * s_g), call
        for i in range(n):
            le, ge = oracle.loglik(inst, X[i], want_grad=True)
            assert abs(e[i] - le) <= min(c_sigma * s_l[i], B_l[i]), (call, i)
            assert np.all(np.abs(g[i] - ge) <= np.minimum(c_sigma * s_g[i], B_g[i])), (call, i)
    assert sb.lib().sb_loglik_noalloc_check(sb._stream()) == sb.SB_OK


def test_noalloc_status_word_reports_a_bad_cholesky_diagonal():
    """A device-side parameter error lands in the library array's status word, which
    sb_loglik_noalloc_check reads and clears."""
    inst = make_instance(16, 2, 5, s_range=(0.3, 0.5), mean_box=(-3, 3), sep=4.0)
    inst.L[1, 3, 3] = -abs(inst.L[1, 3, 3])
    prob = sb.Problem(inst)
    x = torch.as_tensor(inst.mu[:1], device="cuda")
    code, _, _ = _noalloc(prob, x)
    assert code == sb.SB_OK  # found only on the device
    assert sb.lib().sb_loglik_noalloc_check(sb._stream()) == sb.SB_ERR_INVALID_ARG
    assert sb.lib().sb_loglik_noalloc_check(sb._stream()) == sb.SB_OK  # cleared
