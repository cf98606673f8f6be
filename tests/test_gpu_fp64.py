"""GPU parity of the FP64 path against the FP64 CPU oracle, through the C ABI.

Tolerances: l and grad l agree to rounding (1e-12 relative, the sums are
reordered); start selection must match exactly; L-BFGS walkers stop within the
FP64 resolution floor of f of each other (1e-6 absolute in x); log Z agrees to
1e-10 relative (the target of the FP64 path)."""
import math

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


def _logV(inst):
    return float(np.log(inst.hi - inst.lo).sum())


# ------------------------------------------------------------------ likelihood
@pytest.mark.parametrize("d,K,n", [(1, 1, 7), (8, 1, 64), (33, 3, 200), (64, 4, 129), (130, 2, 65), (257, 5, 70)])
def test_loglik_fp64_matches_oracle(d, K, n):
    inst = make_instance(d, K, 500 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    prob = sb.Problem(inst)
    rng = np.random.default_rng(d)
    X = inst.mu[rng.integers(0, K, n)] + rng.normal(0, 0.2, (n, d))
    ell, g = sb.loglik(prob, torch.as_tensor(X, device="cuda"))
    ell, g = ell.cpu().numpy(), g.cpu().numpy()
    for i in range(n):
        le, ge = oracle.loglik(inst, X[i], want_grad=True)
        assert abs(ell[i] - le) <= 1e-12 * (1 + abs(le)), (i, ell[i], le)
        assert np.abs(g[i] - ge).max() <= 1e-11 * (1 + np.abs(ge).max()), i


def test_loglik_values_only_and_far_points():
    inst = make_instance(16, 3, 9, s_range=(0.05, 0.5), mean_box=(-6, 6))
    prob = sb.Problem(inst)
    X = np.random.default_rng(1).uniform(-10, 10, (100, 16))  # far from every mode: large |z|
    ell = sb.loglik(prob, torch.as_tensor(X, device="cuda"), want_grad=False).cpu().numpy()
    ref = np.array([oracle.loglik(inst, x) for x in X])
    assert np.allclose(ell, ref, rtol=1e-12, atol=0)


# ------------------------------------------------------------------ discover
@pytest.mark.parametrize("cfg_id,scale", [(0, None), (1, 0.125)])
def test_discover_matches_oracle(cfg_id, scale):
    insts, c = workload(cfg_id, scale=scale)
    inst = insts[0]
    prob = sb.Problem(inst)
    starts, ell = sb.discover(prob, sb.make_config(c))
    ref_s, ref_l = oracle.discover(inst, c)
    starts, ell = starts.cpu().numpy(), ell.cpu().numpy()
    assert starts.shape == ref_s.shape
    assert np.allclose(ell, ref_l, rtol=1e-12, atol=0)
    assert np.abs(starts - ref_s).max() <= 1e-13 * (1 + np.abs(ref_s).max())


def test_discover_ray_samples_span_box():
    inst = make_instance(5, 2, 3, s_range=(0.2, 0.5), sep=2.0, prior=(-4.0, 6.0))
    c = SolveConfig(n_rays=40, n_steps=3, n_starts=120, seed=17)  # every sample selected
    starts, _ = sb.discover(sb.Problem(inst), sb.make_config(c))
    s = starts.cpu().numpy()
    cen = 0.5 * (inst.lo + inst.hi)
    half = 0.5 * (inst.hi - inst.lo)
    rel = np.abs((s - cen) / half).max(1)
    # every third sample of a ray sits on the box surface (t = 1)
    assert np.isclose(rel, 1.0, atol=1e-13).sum() == 40


# ------------------------------------------------------------------ refine
@pytest.mark.parametrize("cfg_id,scale", [(0, None), (1, 0.0625)])
def test_refine_matches_oracle_from_same_starts(cfg_id, scale):
    insts, c = workload(cfg_id, scale=scale)
    inst = insts[0]
    x0, _ = oracle.discover(inst, c)
    ref = oracle.lbfgs(inst, c, x0, n_threads=8)
    prob = sb.Problem(inst)
    out = sb.refine(prob, sb.make_config(c), torch.as_tensor(x0, device="cuda"))
    x = out.x.cpu().numpy()
    st = out.status.cpu().numpy()
    assert set(st.tolist()) <= {sb.CONVERGED, sb.STALLED}
    assert set(ref.status.tolist()) <= {oracle.CONVERGED, oracle.STALLED}
    assert np.abs(x - ref.x).max() < 1e-6
    assert np.allclose(out.ell.cpu().numpy(), ref.ell, rtol=1e-12)
    assert out.n_evals > 0 and abs(out.n_evals - ref.evals) <= 0.1 * ref.evals


def test_refine_max_iter_and_single_walker():
    inst = make_instance(6, 1, 23, s_range=(0.1, 1.0))
    c = SolveConfig(n_rays=1, n_steps=1, n_starts=1, max_iter=1)
    out = sb.refine(sb.Problem(inst), sb.make_config(c), torch.full((1, 6), 5.0, device="cuda", dtype=torch.float64))
    ref = oracle.lbfgs(inst, c, np.full((1, 6), 5.0))
    assert out.status.item() == sb.MAXITER == ref.status[0]
    assert out.iters.item() == 1
    assert np.allclose(out.x.cpu().numpy(), ref.x, rtol=1e-13, atol=1e-13)


def test_refine_nonfinite_start():
    inst = make_instance(4, 1, 5)
    c = SolveConfig(n_rays=2, n_steps=1, n_starts=2)
    x0 = torch.tensor([[0.0, 0.0, 0.0, 0.0], [float("nan"), 0, 0, 0]], device="cuda", dtype=torch.float64)
    out = sb.refine(sb.Problem(inst), sb.make_config(c), x0)
    assert out.status.cpu().tolist()[1] == sb.NONFINITE


# ------------------------------------------------------------------ laplace
@pytest.mark.parametrize("cfg_id,scale", [(0, None), (1, 0.25)])
def test_laplace_matches_oracle_on_same_walkers(cfg_id, scale):
    insts, c = workload(cfg_id, scale=scale)
    inst = insts[0]
    x0, _ = oracle.discover(inst, c)
    ref = oracle.lbfgs(inst, c, x0, n_threads=8)
    lap = oracle.laplace(inst, c, ref.x, ref.ell, ref.status)
    prob = sb.Problem(inst)
    out = sb.laplace(prob, sb.make_config(c), torch.as_tensor(ref.x, device="cuda"),
                     torch.as_tensor(ref.ell, device="cuda"), torch.as_tensor(ref.status, device="cuda"))
    assert out.n_modes == lap.n_modes >= 1
    assert abs(out.logZ - lap.logZ) <= 1e-10 * abs(lap.logZ)
    assert np.allclose(out.logZk.cpu().numpy(), lap.logZk, rtol=0, atol=1e-10)
    assert np.abs(out.modes.cpu().numpy() - lap.modes).max() <= 1e-9


def test_laplace_zero_modes_and_saddle():
    d = 3
    inst = make_instance(d, 2, 1, s_range=(1.0, 1.0), sep=0.0)
    inst.L[:] = np.eye(d)
    inst.mu[0] = [-3.0, 0, 0]
    inst.mu[1] = [3.0, 0, 0]
    inst.log_w[:] = np.log(0.5)
    prob = sb.Problem(inst)
    mid = torch.zeros((1, d), dtype=torch.float64, device="cuda")
    ell = sb.loglik(prob, mid, want_grad=False)
    c = sb.make_config(SolveConfig(n_rays=1, n_steps=1, n_starts=1, cand_cap=4))
    out = sb.laplace(prob, c, mid, ell)
    assert out.n_modes == 0 and out.logZ == -math.inf
    with pytest.raises(sb.SbError) as e:
        sb.laplace(prob, c, mid, ell, raise_no_modes=True)
    assert e.value.code == sb.SB_ERR_NO_MODES


# ------------------------------------------------------------------ whole path
@pytest.mark.parametrize("cfg_id,scale", [(0, None), (1, 0.25), (1, None)])
def test_evidence_matches_oracle_and_closed_form(cfg_id, scale):
    insts, c = workload(cfg_id, scale=scale)
    inst = insts[0]
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    ref = oracle.evidence(inst, c, n_threads=8)
    assert out.n_modes == ref.n_modes
    assert abs(out.logZ - ref.logZ) <= 1e-10 * abs(ref.logZ)
    if ref.n_modes == inst.K:
        closed = float(np.log(np.exp(inst.log_w).sum())) - _logV(inst)
        assert abs(out.logZ - closed) <= 1e-10 * abs(closed)


@pytest.mark.parametrize("d,K", [(1, 1), (1, 3), (2, 2), (3, 1)])
def test_evidence_low_d(d, K):
    inst = make_instance(d, K, 70 + d * 10 + K, s_range=(0.15, 0.4), mean_box=(-6, 6), sep=8.0)
    c = SolveConfig(n_rays=64, n_steps=64, n_starts=128, seed=3)
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    ref = oracle.evidence(inst, c)
    assert out.n_modes == ref.n_modes == K
    assert abs(out.logZ - ref.logZ) <= 1e-10 * abs(ref.logZ)


@pytest.mark.parametrize("pinned", [False, True])
def test_evidence_host_buffers_closed_form(pinned):
    insts, c = workload(0)
    inst = insts[0]
    cfg = sb.make_config(c)
    ws = sb.evidence_host_workspace(inst, cfg)
    host = sb.PinnedHost(inst, cfg) if pinned else None
    logZ, modes, zk, nm = sb.evidence_host(inst, cfg, ws, host=host)
    assert nm == 1
    assert abs(math.expm1(logZ + _logV(inst))) < 1e-10
    assert np.abs(modes[0] - inst.mu[0]).max() < 1e-12


def _discover_then_check(inst, c):
    prob = sb.Problem(inst)
    ws = sb.workspace(prob, c)
    starts = torch.empty((c.n_starts, inst.d), device="cuda", dtype=torch.float64)
    ell = torch.empty(c.n_starts, device="cuda", dtype=torch.float64)
    code = sb.lib().sb_discover(sb.C.byref(prob.s), sb.C.byref(c), sb._ptr(starts), sb._ptr(ell), ws.ptr,
                                sb.C.c_size_t(ws.nbytes), sb._stream())
    assert code == sb.SB_OK
    return sb.lib().sb_check(ws.ptr, sb.C.c_size_t(ws.nbytes), sb._stream())


def test_device_status_reports_bad_parameters():
    c = sb.make_config(SolveConfig(n_rays=8, n_steps=4, n_starts=4))
    good = make_instance(4, 1, 2)
    assert _discover_then_check(good, c) == sb.SB_OK
    bad = make_instance(4, 1, 2)
    bad.mu[0, 1] = np.nan
    assert _discover_then_check(bad, c) == sb.SB_ERR_NONFINITE
    box = make_instance(4, 1, 2)
    box.lo[2] = box.hi[2]
    assert _discover_then_check(box, c) == sb.SB_ERR_INVALID_ARG
    neg = make_instance(4, 1, 2)
    neg.L[0, 1, 1] = -1.0
    assert _discover_then_check(neg, c) == sb.SB_ERR_INVALID_ARG
