"""sb_loglik_noalloc: the batched likelihood for callers that cannot allocate
device memory. Its scratch is an array inside the library, so the caller
passes only inputs and outputs. Checked against sb_loglik (caller-provided
workspace) through the C ABI, on two calls in a row with different inputs,
within the FP64 tolerance of the other likelihood tests (1e-12 relative).
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import make_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()


def _noalloc(prob, x, want_grad=True):
    n = x.shape[0]
    ell = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(x) if want_grad else None
    code = sb.lib().sb_loglik_noalloc(C.byref(prob.s), C.c_int32(sb.PREC_FP64), sb._ptr(x), C.c_int32(n),
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
