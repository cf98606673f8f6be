"""The solve entry points read nothing back to the host, so a caller can capture
them into a CUDA graph of its own (here torch.cuda.graph, global capture mode):
the replayed graph must give the direct call's log Z and modes bit for bit,
again on a second replay and after the problem's contents change in place
(the graph reads its inputs when it runs). Graph mode (the library's own cached
graph, the default outside a capture) and eager mode (host reads, used while
per-launch profiling is on) run the same kernels in the same order: identical
results."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2601_19957_gb300 as sb
from paper_2601_19957_gb300.instances import SolveConfig, make_instance, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()


class _Out:
    def __init__(self, d, cap):
        self.modes = torch.zeros((cap, d), dtype=torch.float64, device="cuda")
        self.zk = torch.zeros(cap, dtype=torch.float64, device="cuda")
        self.nm = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.lz = torch.zeros(1, dtype=torch.float64, device="cuda")

    def values(self):
        k = int(self.nm.item())
        return float(self.lz.item()), k, self.modes[:k].cpu().numpy().copy(), self.zk[:k].cpu().numpy().copy()


def _call_evidence(prob, c, ws, out, stream, chisao=None):
    if chisao is None:
        return sb.lib().sb_evidence(C.byref(prob.s), C.byref(c), sb._ptr(out.lz), sb._ptr(out.modes), sb._ptr(out.zk),
                                    C.c_int32(c.cand_cap), sb._ptr(out.nm), ws.ptr, C.c_size_t(ws.nbytes),
                                    C.c_void_p(stream.cuda_stream))
    return sb.lib().sb_evidence_chisao(C.byref(prob.s), C.byref(c), C.byref(chisao), sb._ptr(out.lz),
                                       sb._ptr(out.modes), sb._ptr(out.zk), C.c_int32(c.cand_cap), sb._ptr(out.nm),
                                       ws.ptr, C.c_size_t(ws.nbytes), C.c_void_p(stream.cuda_stream))


def _same(a, b):
    assert a[0] == b[0] and a[1] == b[1]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


@pytest.mark.parametrize("prec,use_chisao", [(sb.PREC_FP64, False), (sb.PREC_BF16, False), (sb.PREC_BF16, True),
                                             (sb.PREC_TF32, True)])
def test_user_capture_replays_the_direct_call(prec, use_chisao):
    inst = make_instance(32, 4, 4100 + prec, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    cfg = SolveConfig(n_rays=128, n_steps=64, n_starts=128, m=10, cand_cap=32, seed=3, prec=prec)
    c = sb.make_config(cfg)
    cc = sb.make_chisao_config() if use_chisao else None
    prob = sb.Problem(inst)
    ws = sb.chisao_workspace(prob, c) if use_chisao else sb.workspace(prob, c)
    s = torch.cuda.Stream()
    direct = _Out(inst.d, c.cand_cap)
    with torch.cuda.stream(s):  # the first call (outside any capture) also tunes the tiles
        assert _call_evidence(prob, c, ws, direct, s, cc) == sb.SB_OK
    s.synchronize()
    ref = direct.values()
    assert ref[1] >= 1
    assert sb.lib().sb_check(ws.ptr, C.c_size_t(ws.nbytes), C.c_void_p(s.cuda_stream)) == sb.SB_OK
    g = torch.cuda.CUDAGraph()
    cap = _Out(inst.d, c.cand_cap)
    with torch.cuda.graph(g, stream=s):
        code = _call_evidence(prob, c, ws, cap, s, cc)
    assert code == sb.SB_OK
    for _ in range(2):
        cap.lz.zero_()
        cap.nm.zero_()
        g.replay()
        torch.cuda.synchronize()
        _same(cap.values(), ref)
    # new contents in the same arrays: the replay solves the new problem
    inst2 = make_instance(32, 4, 4200 + prec, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
    prob.mu.copy_(torch.as_tensor(inst2.mu))
    prob.L.copy_(torch.as_tensor(inst2.L))
    prob.log_w.copy_(torch.as_tensor(inst2.log_w))
    g.replay()
    torch.cuda.synchronize()
    replay2 = cap.values()
    with torch.cuda.stream(s):
        assert _call_evidence(prob, c, ws, direct, s, cc) == sb.SB_OK
    s.synchronize()
    _same(replay2, direct.values())
    # the modes moved with the means (log Z itself can stay at log sum w - log V)
    assert replay2[2].shape != ref[2].shape or not np.array_equal(replay2[2], ref[2])


@pytest.mark.parametrize("prec,use_chisao", [(sb.PREC_FP64, False), (sb.PREC_BF16, False), (sb.PREC_BF16, True)])
def test_graph_and_eager_modes_agree_bit_for_bit(prec, use_chisao):
    insts, cfg = workload(1, scale=1.0 / 16)
    inst = insts[0]
    cfg.prec = prec
    c = sb.make_config(cfg)
    prob = sb.Problem(inst)
    cc = sb.make_chisao_config()
    run = (lambda: sb.evidence_chisao(prob, c, cc)) if use_chisao else (lambda: sb.evidence(prob, c))
    g1 = run()
    g2 = run()  # the cached graph again
    sb.lib().sb_profile_enable(1)  # per-launch profiling runs the calls eagerly
    try:
        e = run()
    finally:
        sb.lib().sb_profile_enable(0)
        sb.lib().sb_profile_read(None, None)
    for o in (g2, e):
        assert o.logZ == g1.logZ and o.n_modes == g1.n_modes
        assert torch.equal(o.modes, g1.modes) and torch.equal(o.logZk, g1.logZk)


def test_batched_graph_replays_with_all_components():
    """Twelve problems of the batched workload's kind in one call (one graph launch in
    graph mode), twice: the same log Z both times, each the single solve's."""
    rng = np.random.default_rng(31)
    insts = [make_instance(int(d), int(k), 3100 + i, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
             for i, (d, k) in enumerate(zip(rng.choice([16, 48, 96, 160], 12), rng.integers(1, 5, 12)))]
    cfg = SolveConfig(n_rays=256, n_steps=64, n_starts=256, m=10, cand_cap=32, seed=3, prec=sb.PREC_TF32)
    c = sb.make_config(cfg)
    probs = [sb.Problem(i) for i in insts]
    a, na = sb.evidence_batched(probs, c, n_workers=4)
    b, nb = sb.evidence_batched(probs, c, n_workers=4)
    assert torch.equal(a, b) and torch.equal(na, nb)
    for i, p in enumerate(probs):
        one = sb.evidence(p, c)
        assert float(a[i]) == one.logZ and int(na[i]) == one.n_modes
