"""Whole evidence path with tensor-core discovery/refinement (BF16 or TF32,
FP32 L-BFGS) and the FP64 Laplace stage, through the C ABI.

After the FP64 Newton polish the modes and their Laplace terms are FP64
quantities again, so log Z must agree with the FP64 oracle (same mode set) to
1e-10 relative, and with the closed form log sum w - log V."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2601_19957_gb300 as sb
import tc_bound
from paper_2601_19957_gb300.instances import SolveConfig, make_instance, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    oracle.build()


def _closed(inst):
    return float(np.log(np.exp(inst.log_w).sum()) - np.log(inst.hi - inst.lo).sum())


def _check_modes_against_components(inst, out):
    """Each mode is a component mean (to 1e-9) with Laplace term log w_k (to 1e-9), no
    component twice; log Z = LSE of the found components' log w_k - log V (1e-10 rel)."""
    modes = out.modes.cpu().numpy()
    zk = out.logZk.cpu().numpy()
    seen = set()
    for t in range(out.n_modes):
        k = int(np.argmin(np.abs(inst.mu - modes[t]).max(1)))
        assert k not in seen
        seen.add(k)
        assert np.abs(inst.mu[k] - modes[t]).max() < 1e-9
        assert abs(zk[t] - inst.log_w[k]) < 1e-9
    found = np.array(sorted(seen))
    expect = float(np.log(np.exp(inst.log_w[found]).sum()) - np.log(inst.hi - inst.lo).sum())
    assert abs(out.logZ - expect) <= 1e-10 * abs(expect)
    return found


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_mixed_evidence_workload1(prec):
    """Mixed-precision discovery may pick other starts than the FP64 oracle (several
    start sets are correct), so the check is on the mode set: every mode found is a
    true component with its exact Laplace term, and the FP64 oracle's modes (same
    workload) are all found too."""
    insts, c = workload(1, scale=0.25)
    inst = insts[0]
    c.prec = prec
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    found = _check_modes_against_components(inst, out)
    c64 = type(c)(**{**c.__dict__, "prec": 0})
    ref = oracle.evidence(inst, c64, n_threads=8)
    ref_k = {int(np.argmin(np.abs(inst.mu - m).max(1))) for m in ref.modes}
    assert ref_k <= set(found.tolist())


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_mixed_evidence_ill_conditioned_gaussian_workload2(prec):
    """d=256, condition number up to 1e4: polish + Cholesky in FP64 recover log Z = -log V."""
    insts, c = workload(2, scale=1.0 / 16)
    inst = insts[0]
    c.prec = prec
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    assert out.n_modes == 1
    assert abs(out.logZ - _closed(inst)) <= 1e-10 * abs(_closed(inst))
    assert np.abs(out.modes[0].cpu().numpy() - inst.mu[0]).max() < 1e-9


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_mixed_evidence_d1024_k8_scaled(prec):
    """Sunburst-only discovery at d = 1024 reaches few of the eight basins (the rays pass
    far from most means); each mode it finds is exact. Completeness at this shape is
    the ChiSao pipeline's (test_full_size_workload_...)."""
    insts, c = workload(4, scale=1.0 / 32)
    inst = insts[0]
    c.prec = prec
    c.cand_cap = 64
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    assert out.n_modes >= 1
    _check_modes_against_components(inst, out)


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
@pytest.mark.parametrize("d,m", [(37, 7), (300, 20), (1000, 13)])
def test_mixed_evidence_ragged_dimension(prec, d, m):
    """Dimensions off the 8- and 16-coordinate grid (rows copied with zero padding,
    k-steps cut by d, warps with no coordinates) and history lengths off the
    4-pair groups: every mode found is a true component with its exact Laplace term,
    and where the FP64 oracle runs the same solve in seconds (d <= 300) the component
    set is the oracle's."""
    inst = make_instance(d, 3, 7000 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    c = SolveConfig(n_rays=256, n_steps=32, n_starts=256, m=m, seed=7000 + d, prec=prec)
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    assert out.n_modes >= 1
    found = _check_modes_against_components(inst, out)
    if d <= 300:
        ref = oracle.evidence(inst, SolveConfig(**{**c.__dict__, "prec": 0}), n_threads=16)
        ref_k = sorted({int(np.argmin(np.abs(inst.mu - m_).max(1))) for m_ in ref.modes})
        assert found.tolist() == ref_k


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
@pytest.mark.parametrize("d,m", [(64, 5), (300, 20), (1024, 20)])
def test_mixed_refine_reaches_gaussian_mean(prec, d, m):
    """The FP32 L-BFGS step on its own (bf16 pairs, tensor-core inner products, R^-1
    kept per walker; no FP64 polish to hide a poor direction): from uniform starts in
    the box every walker of a single Gaussian ends CONVERGED or STALLED within one
    standard deviation of the mean, |L^T (x - mu)|_2 <= 1, where FP32 f stops
    resolving progress (f ~ 1e3, so |z|^2 is resolved to ~1e-4)."""
    inst = make_instance(d, 1, 8100 + d, s_range=(0.05, 0.5), mean_box=(-6, 6))
    n = 64
    c = SolveConfig(n_rays=n, n_steps=1, n_starts=n, m=m, seed=8100 + d, prec=prec)
    x0 = np.random.default_rng(8100 + d).uniform(-10.0, 10.0, size=(n, d))
    out = sb.refine(sb.Problem(inst), sb.make_config(c), torch.as_tensor(x0, device="cuda"))
    st = out.status.cpu().numpy()
    assert set(st.tolist()) <= {sb.CONVERGED, sb.STALLED}
    x = out.x.cpu().numpy()
    z = (x - inst.mu[0]) @ inst.L[0]  # rows: (L^T (x - mu))^T
    assert np.sqrt((z * z).sum(1)).max() <= 1.0
    peak = oracle.loglik(inst, inst.mu[0])
    assert (peak - out.ell.cpu().numpy()).max() <= 0.5 + 1e-3 * abs(peak)


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_mixed_refine_walkers_independent_of_batch(prec):
    """A walker's refinement depends on its own start alone: its rows of a tensor-core
    round do not depend on the rows that share its 128-row block (the pairs a block
    skips contribute exact zeros to every row) and its L-BFGS step reads no other
    walker. So 40000 walkers refined in one call, where every thread of the active
    list's compaction holds several entries (40000 over 64 CTAs of 256 threads), end
    bit for bit where the same starts end in calls of at most 16000 walkers."""
    inst = make_instance(16, 3, 5150, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    n = 40000
    c = sb.make_config(SolveConfig(n_rays=1024, n_steps=64, n_starts=n, m=10, seed=17, prec=prec))
    prob = sb.Problem(inst)
    starts = torch.as_tensor(np.random.default_rng(9).uniform(-10.0, 10.0, (n, inst.d)), device="cuda")
    ws = sb.workspace(prob, c)
    whole = sb.refine(prob, c, starts, ws=ws)
    wx, wl, wst, wit = whole.x.clone(), whole.ell.clone(), whole.status.clone(), whole.iters.clone()
    parts = [sb.refine(prob, c, starts[i:i + 16000], ws=ws) for i in range(0, n, 16000)]
    assert torch.equal(wx, torch.cat([p.x for p in parts]))
    assert torch.equal(wl, torch.cat([p.ell for p in parts]))
    assert torch.equal(wst, torch.cat([p.status for p in parts]))
    assert torch.equal(wit, torch.cat([p.iters for p in parts]))
    assert whole.n_evals == sum(p.n_evals for p in parts)


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
def test_mixed_refine_components_beyond_32(prec):
    """K = 40: walkers started near components 32..39 keep those components in the
    walker rounds' component skip (one mask bit per component, up to 64) and end at
    their means, |L_k^T (x - mu_k)|_2 <= 1, as in the single-Gaussian test."""
    inst = make_instance(16, 40, 4400, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    rng = np.random.default_rng(41)
    ks = np.arange(32, 40).repeat(32)
    n = len(ks)
    x0 = inst.mu[ks] + rng.normal(0, 0.05, (n, inst.d))
    c = SolveConfig(n_rays=n, n_steps=1, n_starts=n, m=10, seed=41, prec=prec)
    out = sb.refine(sb.Problem(inst), sb.make_config(c), torch.as_tensor(x0, device="cuda"))
    assert set(out.status.cpu().numpy().tolist()) <= {sb.CONVERGED, sb.STALLED}
    x = out.x.cpu().numpy()
    for t, k in enumerate(ks):
        z = (x[t] - inst.mu[k]) @ inst.L[k]
        assert np.sqrt(z @ z) <= 1.0, (t, k)


def _check_ray_samples(inst, X, ell, prec):
    """Discovery's l at ray samples comes from the quadratic form of each ray (split
    tensor-core products): its error model is tc_bound.check_ray_samples."""
    ref = np.array([oracle.loglik(inst, x) for x in X])
    tc_bound.check_ray_samples(inst, X, ell - ref, prec)


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
@pytest.mark.parametrize("d,K,n_rays,n_steps", [(64, 4, 64, 16), (300, 3, 32, 32), (200, 2, 130, 8),
                                                (1024, 8, 32, 64), (7, 2, 16, 8), (1, 1, 4, 4), (5, 2, 1, 8)])
def test_discover_quadratic_ray_pass_against_oracle(prec, d, K, n_rays, n_steps):
    """Every ray sample (n_starts = n_rays x n_steps, so that discovery returns all of
    them) against the FP64 oracle's l at the returned point: ragged d (300, 200, 7, 1
    against 64-element bf16 and 32-element tf32 chunks), ragged ray blocks (130 rays
    over 128-row tiles), the bench's d = 1024, K = 8 instance."""
    if d == 1024:
        inst = workload(4)[0][0]
    else:
        inst = make_instance(d, K, 900 + d, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    c = SolveConfig(n_rays=n_rays, n_steps=n_steps, n_starts=n_rays * n_steps, m=10, seed=7, prec=prec)
    starts, ell = sb.discover(sb.Problem(inst), sb.make_config(c))
    X, ell = starts.cpu().numpy(), ell.cpu().numpy()
    assert X.shape == (n_rays * n_steps, d)
    # every sample, in flat order (ray r, step j): the oracle's rays, with directions
    # drawn in FP32 (the same Philox counters; Box-Muller in FP32), each ray's last sample
    # on the box surface and sample j at (j + 1) / n_steps of it
    ref_x, _ = oracle.discover(inst, c)
    cen, half = 0.5 * (inst.lo + inst.hi), 0.5 * (inst.hi - inst.lo)
    D = (X - cen).reshape(n_rays, n_steps, d)
    R = (ref_x - cen).reshape(n_rays, n_steps, d)
    cos = (D[:, -1] * R[:, -1]).sum(1) / np.linalg.norm(D[:, -1], axis=1) / np.linalg.norm(R[:, -1], axis=1)
    assert cos.min() >= 1 - 1e-6, cos.min()
    assert np.abs(np.abs(D[:, -1] / half).max(1) - 1).max() <= 1e-12
    frac = (np.arange(1, n_steps + 1) / n_steps)[None, :, None]
    assert np.abs(D - frac * D[:, -1:]).max() <= 1e-12 * np.abs(D).max()
    _check_ray_samples(inst, X, ell, prec)


def test_full_size_workload_sampled_against_oracle():
    """The configuration the bench times (d=1024, K=8, 16384 rays x 64 steps, 16384
    walkers, m=20, BF16, ChiSao), checked where the oracle can follow one output at a
    time: 64 sampled selected starts' l against the FP64 oracle within the quadratic
    ray pass's error model (tc_bound.check_ray_samples); then the whole
    pipeline on the same workspace: all eight components, every mode a component mean
    with its exact Laplace term, log Z the closed form to 1e-9."""
    insts, c = workload(4)
    inst = insts[0]
    cfg = sb.make_config(c)
    prob = sb.Problem(inst)
    ws = sb.chisao_workspace(prob, cfg)
    starts, ell = sb.discover(prob, cfg, ws=ws)
    starts, ell = starts.cpu().numpy(), ell.cpu().numpy()
    pick = np.random.default_rng(11).choice(c.n_starts, 64, replace=False)
    _check_ray_samples(inst, starts[pick], ell[pick], sb.PREC_BF16)
    out = sb.evidence_chisao(prob, cfg, sb.make_chisao_config(), ws=ws)
    found = _check_modes_against_components(inst, out)
    assert found.tolist() == list(range(inst.K))
    assert abs(out.logZ - _closed(inst)) <= 1e-9


@pytest.mark.parametrize("prec", [sb.PREC_BF16, sb.PREC_TF32])
@pytest.mark.parametrize("d,K,m,n_starts", [(1, 1, 1, 1), (2, 2, 1, 16), (3, 3, 2, 64), (7, 2, 10, 5)])
def test_mixed_evidence_small_and_degenerate(prec, d, K, m, n_starts):
    """Degenerate sizes on the tensor-core path: d below one K chunk, a one-pair
    history, a single walker: the modes found are true components with their
    exact Laplace terms (the FP64 polish), as at full size."""
    inst = make_instance(d, K, 7300 + 10 * d + K, s_range=(0.15, 0.4), mean_box=(-6, 6), sep=8.0)
    c = SolveConfig(n_rays=64, n_steps=16, n_starts=n_starts, m=m, seed=7300 + d, prec=prec)
    out = sb.evidence(sb.Problem(inst), sb.make_config(c))
    assert out.n_modes >= 1
    _check_modes_against_components(inst, out)
