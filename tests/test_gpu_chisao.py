"""GPU parity of the ChiSao oscillation (Sec. 3.5.5) against the FP64 CPU
oracle, through the C ABI.

Which sample of a cluster of duplicates becomes the stuck representative is
decided by rounding (their l agree to ~1e-15), so the tests compare what is
unique: the number of peaks and the peak positions as a set (1e-6 in x, the
FP64 resolution floor of the L-BFGS end points, as in the refinement's own
parity), and check that every peak is a valid, distinct converged maximum."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import SolveConfig, make_instance

pytestmark = pytest.mark.gpu

TOL_X = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _run(inst, cfg, x0, **cc):
    cc.setdefault("anti_alpha", 0.01)  # the step size these cases were first validated with
    prob = sb.Problem(inst)
    out = sb.chisao(prob, sb.make_config(cfg), sb.make_chisao_config(**cc), torch.as_tensor(x0, device="cuda"))
    ref = oracle.chisao(inst, cfg, oracle.ChisaoConfig(**cc), x0)
    return out, ref


def _peaks(x, stuck):
    p = np.asarray(x)[np.asarray(stuck)]
    return p[np.lexsort(p.T[::-1])] if len(p) else p


def _assert_same_peaks(out, ref):
    assert out.n_peaks == ref.n_peaks == int(out.stuck.sum().item())
    a = _peaks(out.x.cpu().numpy(), out.stuck.cpu().numpy())
    b = _peaks(ref.x, ref.stuck)
    dist = np.abs(a[:, None, :] - b[None, :, :]).max(2)
    assert dist.min(1).max() <= TOL_X and dist.min(0).max() <= TOL_X, dist


def _assert_valid_peaks(inst, cfg, out):
    x = out.x.cpu().numpy()
    ell = out.ell.cpu().numpy()
    st = out.stuck.cpu().numpy()
    assert np.all(np.isfinite(x)) and np.all(x >= inst.lo) and np.all(x <= inst.hi)
    pk = np.flatnonzero(st)
    lmax = ell[np.isfinite(ell)].max()
    wmax = float((inst.hi - inst.lo).max())
    for a, s in enumerate(pk):
        le, g = oracle.loglik(inst, x[s], want_grad=True)
        assert abs(ell[s] - le) <= 1e-12 * (1 + abs(le))
        assert np.abs(g).max() <= cfg.eps_grad * (1 + abs(le))
        assert ell[s] >= lmax + math.log(0.1)
        for b in pk[:a]:
            assert np.abs(x[s] - x[b]).max() > cfg.dedup_coarse * wmax


def test_one_oscillation_is_the_refinement_plus_the_stick_filter():
    inst = make_instance(3, 3, 61, s_range=(0.4, 1.0), mean_box=(-5, 5), sep=4.0)
    cfg = SolveConfig(n_starts=40)
    x0 = np.random.default_rng(3).uniform(-6, 6, (40, 3))
    out, ref = _run(inst, cfg, x0, n_osc=1)
    ref_lb = sb.refine(sb.Problem(inst), sb.make_config(cfg), torch.as_tensor(x0, device="cuda"))
    assert torch.equal(out.x, ref_lb.x) and torch.equal(out.ell, ref_lb.ell)
    assert np.abs(out.x.cpu().numpy() - ref.x).max() <= TOL_X
    _assert_same_peaks(out, ref)
    _assert_valid_peaks(inst, cfg, out)


def _bimodal_1d():
    inst = make_instance(1, 2, 1, s_range=(1.0, 1.0), sep=0.0)
    inst.L[:] = 1.0
    inst.mu[:, 0] = [-5.0, 5.0]
    inst.log_w[:] = np.log([0.6, 0.4])
    return inst


def test_bimodal_1d_golden_rooster_finds_the_second_mode():
    inst = _bimodal_1d()
    cfg = SolveConfig(n_steps=64, n_starts=16, seed=3)
    x0 = -5 + np.random.default_rng(0).uniform(-2, 2, (16, 1))
    out, ref = _run(inst, cfg, x0)
    _assert_same_peaks(out, ref)
    assert out.n_peaks == 2
    np.testing.assert_allclose(_peaks(out.x.cpu().numpy(), out.stuck.cpu().numpy())[:, 0], [-5.0, 5.0], atol=1e-7)


@pytest.mark.parametrize("d,seed", [(2, 5), (4, 12), (4, 13), (37, 14)])
def test_mixture_modes_from_one_basin_match_the_oracle(d, seed):
    inst = make_instance(d, 3, seed, s_range=(0.5, 1.0), mean_box=(-6, 6), sep=6.0)
    cfg = SolveConfig(n_steps=64, n_starts=64, seed=seed)
    x0 = inst.mu[0] + np.random.default_rng(seed).uniform(-0.5, 0.5, (64, d))
    out, ref = _run(inst, cfg, x0, n_osc=4)
    _assert_same_peaks(out, ref)
    _assert_valid_peaks(inst, cfg, out)


def test_repulse_monkey_path_gives_valid_distinct_peaks():
    inst = make_instance(3, 3, 71, s_range=(0.3, 1.0), mean_box=(-5, 5), sep=4.0)
    cfg = SolveConfig(n_steps=32, n_starts=48, seed=1)
    x0 = np.random.default_rng(4).uniform(-9, 9, (48, 3))
    out, ref = _run(inst, cfg, x0, n_osc=3, conv_iters=4)
    assert out.n_peaks > 0
    _assert_valid_peaks(inst, cfg, out)
    # every peak is a component mode, as the oracle's are
    for peaks in (_peaks(out.x.cpu().numpy(), out.stuck.cpu().numpy()), _peaks(ref.x, ref.stuck)):
        assert np.abs(peaks[:, None, :] - inst.mu[None]).max(2).min(1).max() < 1e-3


def test_small_and_degenerate_cases():
    inst = make_instance(5, 2, 81, s_range=(0.5, 1.0), mean_box=(-4, 4), sep=4.0)
    cfg = SolveConfig(n_starts=8)
    # one sample: it sticks at its mode, nothing is lost
    x0 = inst.mu[:1] + 0.3
    out, ref = _run(inst, cfg, x0)
    _assert_same_peaks(out, ref)
    assert out.n_peaks == 1
    # no anti-convergence steps, samples already at the two modes
    x0 = np.repeat(inst.mu, 4, axis=0)
    out, ref = _run(inst, cfg, x0, anti_steps=0)
    _assert_same_peaks(out, ref)
    # deterministic: a second run gives the same bits
    out2, _ = _run(inst, cfg, x0, anti_steps=0)
    assert torch.equal(out.x, out2.x) and torch.equal(out.stuck, out2.stuck)
