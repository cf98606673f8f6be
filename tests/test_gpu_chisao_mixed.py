"""GPU parity of the mixed-precision ChiSao oscillation (Sec. 3.5.5) and of the
evidence pipeline built on it (discovery, ChiSao, the FP64 Laplace stage over
every final sample), against the FP64 CPU oracle, through the C ABI.

The mixed path refines in FP32 with tensor-core gradients, so its samples do not
follow the oracle's FP64 trajectories point by point, and which samples get lost
and reseeded can differ. What is unique, and compared, is:
 - the set of components whose modes are found (a peak belongs to the component
   whose mean is nearest in max norm, and lies within the FP32 refinement's
   reach of that mode);
 - after the FP64 Newton polish, the modes themselves (1e-9 in x) and log Z
   (1e-10 relative to the oracle's, 1e-9 absolute to the closed form
   log sum_k w_k - log V of a separated mixture).
The stick test on the mixed path reads the refinement's CONVERGED / STALLED
state (the oracle's conv_from_status reading)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import SolveConfig, make_instance

pytestmark = pytest.mark.gpu

BF16, TF32 = 2, 1


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _comp(inst, pts):
    return sorted({int(np.argmin(np.abs(inst.mu - p).max(1))) for p in np.asarray(pts).reshape(-1, inst.d)})


def _closed(inst):
    return float(np.log(np.exp(inst.log_w).sum())) - float(np.log(inst.hi - inst.lo).sum())


@pytest.mark.parametrize("prec", [BF16, TF32])
@pytest.mark.parametrize("d,K,seed", [(16, 4, 1), (48, 3, 2)])
def test_mixed_chisao_peaks_match_oracle_status_reading(prec, d, K, seed):
    """Samples started in one basin: the peaks ChiSao keeps (stick test by the refinement's
    state) are the oracle's, component by component, each within the FP32 refinement's
    reach of the FP64 mode."""
    inst = make_instance(d, K, 900 + d, s_range=(0.3, 1.0), mean_box=(-6, 6), sep=6.0)
    cfg = SolveConfig(n_steps=64, n_starts=96, seed=seed, prec=prec)
    x0 = inst.mu[0] + np.random.default_rng(seed).uniform(-0.5, 0.5, (96, d))
    cc = dict(n_osc=4, anti_alpha=0.1)
    out = sb.chisao(sb.Problem(inst), sb.make_config(cfg), sb.make_chisao_config(**cc),
                    torch.as_tensor(x0, device="cuda"))
    ref = oracle.chisao(inst, cfg, oracle.ChisaoConfig(conv_from_status=True, **cc), x0, n_threads=8)
    gx = out.x.cpu().numpy()[out.stuck.cpu().numpy()]
    assert out.n_peaks == len(gx) > 0
    assert _comp(inst, gx) == _comp(inst, ref.x[ref.stuck])
    # every peak is near its component's mode (the oracle's FP64 peak of that component)
    rp = ref.x[ref.stuck]
    for p in gx:
        assert np.abs(rp - p).max(1).min() <= 2e-2


@pytest.mark.parametrize("prec", [BF16, TF32])
@pytest.mark.parametrize("d,K,n_starts,seed", [(16, 6, 128, 1601), (64, 6, 128, 6401), (128, 8, 256, 4128)])
def test_evidence_chisao_matches_oracle_pipeline(prec, d, K, n_starts, seed):
    """Separated mixtures where sunburst-only refinement reaches few basins: the GPU
    pipeline finds the components the oracle's pipeline finds, and after the FP64 polish
    its modes and log Z match the oracle's and the closed form."""
    sep = 10.0 if K == 8 else 8.0
    inst = make_instance(d, K, seed, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=sep)
    cfg = SolveConfig(n_rays=n_starts, n_steps=64, n_starts=n_starts, m=20 if K == 8 else 10, seed=0, prec=prec)
    cc = dict(n_osc=3, anti_alpha=0.1)
    out = sb.evidence_chisao(sb.Problem(inst), sb.make_config(cfg), sb.make_chisao_config(**cc))
    starts, _ = oracle.discover(inst, cfg, n_threads=8)
    cs = oracle.chisao(inst, cfg, oracle.ChisaoConfig(conv_from_status=True, **cc), starts, n_threads=8)
    lap = oracle.laplace(inst, cfg, cs.x, cs.ell, n_threads=8)
    gm = out.modes.cpu().numpy()
    assert _comp(inst, gm) == _comp(inst, lap.modes)
    assert out.n_modes == lap.n_modes
    dist = np.abs(gm[:, None, :] - lap.modes[None, :, :]).max(2)
    assert dist.min(1).max() <= 1e-9 and dist.min(0).max() <= 1e-9
    assert abs(out.logZ - lap.logZ) <= 1e-10 * abs(lap.logZ)
    if len(_comp(inst, gm)) == K:
        assert abs(out.logZ - _closed(inst)) <= 1e-9
