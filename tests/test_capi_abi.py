"""The C-ABI library loads on a machine without a GPU and exports every
function include/sb.h declares; host-side argument checks need no device."""
import ctypes as C

import pytest

import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300 import build as sbbuild
from paper_2601_19957_gb300.instances import SolveConfig, workload


@pytest.fixture(scope="module", autouse=True)
def built():
    sbbuild.build()


def test_every_declared_symbol_is_exported():
    names = sb.declared_symbols()
    assert {"sb_discover", "sb_refine", "sb_laplace", "sb_evidence", "sb_loglik"} <= set(names)
    L = sb.lib()
    for n in names:
        assert hasattr(L, n), n


def test_status_strings():
    assert sb.status_string(0) == "SB_OK"
    assert sb.status_string(5) == "SB_ERR_NO_MODES"


def _fake_problem(d, K):
    # non-null dummy device pointers: the size query never dereferences them
    return sb._Problem(d, K, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000)


def test_workspace_query_grows_with_walkers_and_rejects_bad_args():
    _, cfg = workload(1, scale=0.125)
    p = _fake_problem(64, 4)
    small = sb.lib().sb_workspace_bytes(C.byref(p), C.byref(sb.make_config(cfg)))
    big = sb.lib().sb_workspace_bytes(C.byref(p), C.byref(sb.make_config(cfg, n_starts=cfg.n_starts * 2)))
    assert 0 < small < big
    assert sb.lib().sb_workspace_bytes(C.byref(p), C.byref(sb.make_config(cfg, m=0))) == 0
    assert sb.lib().sb_workspace_bytes(C.byref(_fake_problem(0, 1)), C.byref(sb.make_config(cfg))) == 0
    too_many = sb.make_config(cfg, n_starts=cfg.n_rays * cfg.n_steps + 1)
    assert sb.lib().sb_workspace_bytes(C.byref(p), C.byref(too_many)) == 0


def test_entry_points_reject_invalid_arguments_before_any_launch():
    cfg = sb.make_config(SolveConfig())
    p = _fake_problem(8, 1)
    L = sb.lib()
    # null outputs / null workspace are refused on the host
    assert L.sb_discover(C.byref(p), C.byref(cfg), None, None, None, C.c_size_t(0), None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_evidence(C.byref(p), C.byref(cfg), None, None, None, 1, None, None, C.c_size_t(0), None) == \
        sb.SB_ERR_INVALID_ARG
    d2000 = _fake_problem(2000, 1)
    assert L.sb_workspace_bytes(C.byref(d2000), C.byref(cfg)) == 0
    buf = (C.c_char * 16)()
    assert L.sb_evidence(C.byref(p), C.byref(cfg), buf, buf, buf, 1, buf, buf, C.c_size_t(16), None) == \
        sb.SB_ERR_WORKSPACE


def test_chisao_rejects_bad_config_and_mixed_precision_on_the_host():
    cfg = sb.make_config(SolveConfig(n_starts=16))
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    cc = sb.make_chisao_config()
    args = lambda cfg_, cc_: (C.byref(p), C.byref(cfg_), cc_, buf, 4, buf, buf, buf, buf, buf, C.c_size_t(16), None)
    assert L.sb_chisao(*args(cfg, None)) == sb.SB_ERR_INVALID_ARG
    assert L.sb_chisao(*args(cfg, C.byref(sb.make_chisao_config(min_unconverged=0)))) == sb.SB_ERR_INVALID_ARG
    assert L.sb_chisao(*args(cfg, C.byref(sb.make_chisao_config(n_osc=0)))) == sb.SB_ERR_INVALID_ARG
    assert L.sb_chisao(*args(cfg, C.byref(sb.make_chisao_config(momentum=float("nan"))))) == sb.SB_ERR_INVALID_ARG
    # the mixed path evaluates ray samples in chunks of n_starts rows: fewer starts than steps is refused
    bf16 = sb.make_config(SolveConfig(n_starts=16, n_steps=64, prec=sb.PREC_BF16))
    assert L.sb_chisao(*args(bf16, C.byref(cc))) == sb.SB_ERR_UNSUPPORTED
    too_many = (C.byref(p), C.byref(cfg), C.byref(cc), buf, 17, buf, buf, buf, buf, buf, C.c_size_t(16), None)
    assert L.sb_chisao(*too_many) == sb.SB_ERR_INVALID_ARG
    assert L.sb_chisao(*args(cfg, C.byref(cc))) == sb.SB_ERR_WORKSPACE
    base = L.sb_workspace_bytes(C.byref(p), C.byref(cfg))
    assert L.sb_chisao_workspace_bytes(C.byref(p), C.byref(cfg)) > base > 0


def test_precheck_rejects_bad_arguments_on_the_host():
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    ok = lambda ef, es, nbytes: L.sb_precheck(C.byref(p), ef, es, buf, buf, buf, buf, buf, buf, nbytes, None)
    assert ok(-1.0, 1e-3, 16) == sb.SB_ERR_INVALID_ARG
    assert ok(1e-6, float("nan"), 16) == sb.SB_ERR_INVALID_ARG
    assert ok(1e-6, 1e-3, 16) == sb.SB_ERR_WORKSPACE
    assert L.sb_precheck(C.byref(p), 1e-6, 1e-3, None, buf, buf, buf, buf, buf, 16, None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_precheck_workspace_bytes(C.byref(p)) > 0
    assert L.sb_precheck_workspace_bytes(C.byref(_fake_problem(2000, 1))) == 0


def test_segments_reject_bad_arguments_on_the_host():
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    call = lambda fam, nr, ns, delta, nref, tr, nbytes: L.sb_segments(C.byref(p), fam, 1, nr, ns, delta, nref, buf,
                                                                      buf, tr, tr, buf, nbytes, None)
    assert call(4, 8, 16, 1.0, 4, buf, 16) == sb.SB_ERR_INVALID_ARG  # unknown family
    assert call(sb.RAY_V2V, 0, 16, 1.0, 4, buf, 16) == sb.SB_ERR_INVALID_ARG
    assert call(sb.RAY_V2V, 8, 16, float("nan"), 4, buf, 16) == sb.SB_ERR_INVALID_ARG
    assert call(sb.RAY_V2V, 8, 16, 1.0, 4, None, 16) == sb.SB_ERR_INVALID_ARG  # refined outputs missing
    assert call(sb.RAY_W2W, 8, 16, float("inf"), 0, None, 16) == sb.SB_ERR_WORKSPACE
    small = L.sb_segments_workspace_bytes(C.byref(p), 8, 16)
    assert 0 < small < L.sb_segments_workspace_bytes(C.byref(p), 64, 16)
    assert L.sb_segments_workspace_bytes(C.byref(p), 0, 16) == 0


def test_fd_derivatives_reject_bad_arguments_on_the_host():
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    call = lambda eg, eh, full, H, nbytes: L.sb_fd_derivatives(C.byref(p), buf, eg, eh, full, buf, buf, H, buf, buf,
                                                               nbytes, None)
    assert call(0.0, 1e-4, 0, None, 16) == sb.SB_ERR_INVALID_ARG
    assert call(1e-5, float("inf"), 0, None, 16) == sb.SB_ERR_INVALID_ARG
    assert call(1e-5, 1e-4, 1, None, 16) == sb.SB_ERR_INVALID_ARG  # full Hessian needs H
    assert call(1e-5, 1e-4, 0, None, 16) == sb.SB_ERR_WORKSPACE
    assert 0 < L.sb_fd_workspace_bytes(C.byref(p), 0) < L.sb_fd_workspace_bytes(C.byref(_fake_problem(512, 1)), 1)


def test_evidence_chisao_rejects_bad_arguments_on_the_host():
    cfg = sb.make_config(SolveConfig(n_starts=16))
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    cc = sb.make_chisao_config()
    assert L.sb_evidence_chisao(C.byref(p), C.byref(cfg), None, buf, buf, buf, 4, buf, buf, C.c_size_t(16),
                                None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_evidence_chisao(C.byref(p), C.byref(cfg), C.byref(cc), buf, buf, buf, 0, buf, buf, C.c_size_t(16),
                                None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_evidence_chisao(C.byref(p), C.byref(cfg), C.byref(cc), buf, buf, buf, 4, buf, buf, C.c_size_t(16),
                                None) == sb.SB_ERR_WORKSPACE


def test_ray_loglik_quad_rejects_bad_arguments_on_the_host():
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    assert L.sb_ray_loglik_quad(C.byref(p), 4, buf, 4, 8, buf, buf, C.c_size_t(16), None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_ray_loglik_quad(C.byref(p), 1, buf, 0, 8, buf, buf, C.c_size_t(16), None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_ray_loglik_quad(C.byref(p), 1, buf, 4, 8, buf, buf, C.c_size_t(16), None) == sb.SB_ERR_WORKSPACE
    assert L.sb_ray_loglik_quad_workspace_bytes(C.byref(p), 0, 4) > 0
    assert L.sb_ray_loglik_quad_workspace_bytes(C.byref(p), 1, 4) > 0
    assert L.sb_ray_loglik_quad_workspace_bytes(C.byref(p), 2, 4) > 0
    assert L.sb_ray_loglik_quad_workspace_bytes(C.byref(p), 3, 4) > 0
    assert L.sb_ray_loglik_quad_workspace_bytes(C.byref(p), 4, 4) == 0


def test_ray_loglik_origins_rejects_bad_arguments_on_the_host():
    p = _fake_problem(8, 1)
    L = sb.lib()
    buf = (C.c_char * 16)()
    for form in (0, 1, 4):
        assert L.sb_ray_loglik_origins(C.byref(p), form, buf, buf, 4, 8, buf, None, buf, C.c_size_t(16),
                                       None) == sb.SB_ERR_INVALID_ARG
        assert L.sb_ray_loglik_origins_workspace_bytes(C.byref(p), form, 4) == 0
    assert L.sb_ray_loglik_origins(C.byref(p), 2, buf, buf, 0, 8, buf, None, buf, C.c_size_t(16),
                                   None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_ray_loglik_origins(C.byref(p), 2, buf, buf, 4, 0, buf, None, buf, C.c_size_t(16),
                                   None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_ray_loglik_origins(C.byref(p), 3, buf, buf, 4, 8, buf, None, buf, C.c_size_t(16),
                                   None) == sb.SB_ERR_WORKSPACE
    assert L.sb_ray_loglik_origins_workspace_bytes(C.byref(p), 2, 4) > 0
    assert L.sb_ray_loglik_origins_workspace_bytes(C.byref(p), 3, 4) > 0
