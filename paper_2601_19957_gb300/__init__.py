"""Python binding of libsb, the GB300 (sm_103a) evidence library.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels behind the C ABI of include/sb.h. PyTorch supplies device memory and
streams. The library must be built (``build.build()``); importing a function
that needs it fails loudly if ``_lib/libsb.so`` is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .instances import Instance, SolveConfig

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsb.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "sb.h")

SB_OK, SB_ERR_INVALID_ARG, SB_ERR_CUDA, SB_ERR_WORKSPACE, SB_ERR_NONFINITE, SB_ERR_NO_MODES, SB_ERR_TIMEOUT, \
    SB_ERR_UNSUPPORTED = range(8)
PREC_FP64, PREC_TF32, PREC_BF16 = 0, 1, 2
RUNNING, CONVERGED, STALLED, MAXITER, NONFINITE = range(5)


class SbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


class _Problem(C.Structure):
    _fields_ = [("d", C.c_int32), ("K", C.c_int32), ("log_w", C.c_void_p), ("mu", C.c_void_p),
                ("L", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("n_rays", C.c_int32), ("n_steps", C.c_int32), ("n_starts", C.c_int32), ("m", C.c_int32),
                ("max_iter", C.c_int32), ("max_backtracks", C.c_int32), ("newton_steps", C.c_int32),
                ("cand_cap", C.c_int32), ("gtol", C.c_double), ("armijo_c1", C.c_double),
                ("backtrack", C.c_double), ("dedup_coarse", C.c_double), ("dedup_tol", C.c_double),
                ("eps_grad", C.c_double), ("seed", C.c_uint64), ("prec", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def lib():
    """Load libsb.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsb.so not built ({LIB_PATH}); run paper_2601_19957_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.sb_status_string.restype = C.c_char_p
        L.sb_workspace_bytes.restype = C.c_size_t
        L.sb_loglik_workspace_bytes.restype = C.c_size_t
        L.sb_evidence_host_workspace_bytes.restype = C.c_size_t
        L.sb_evidence_backward_workspace_bytes.restype = C.c_size_t
        L.sb_evidence_batched_workspace_bytes.restype = C.c_size_t
        L.sb_evidence_chisao_batched_workspace_bytes.restype = C.c_size_t
        L.sb_evidence_chisao_batched.restype = C.c_int
        L.sb_evidence_batched.restype = C.c_int
        L.sb_profile_bytes.restype = C.c_double
        L.sb_profile_bytes.argtypes = [C.c_int32]
        L.sb_evidence_backward.restype = C.c_int
        L.sb_evidence_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.sb_chisao_workspace_bytes.restype = C.c_size_t
        L.sb_evidence_chisao_host_workspace_bytes.restype = C.c_size_t
        L.sb_profile_classes.argtypes = [C.c_uint32]
        L.sb_fp64_fma_peak.restype = C.c_double
        L.sb_fp64_fma_peak.argtypes = [C.c_void_p]
        L.sb_precheck_workspace_bytes.restype = C.c_size_t
        L.sb_segments_workspace_bytes.restype = C.c_size_t
        L.sb_fd_workspace_bytes.restype = C.c_size_t
        L.sb_ray_loglik_quad_workspace_bytes.restype = C.c_size_t
        L.sb_ray_loglik_quad.restype = C.c_int
        L.sb_ray_loglik_origins_workspace_bytes.restype = C.c_size_t
        L.sb_ray_loglik_origins.restype = C.c_int
        L.sb_fd_derivatives.restype = C.c_int
        L.sb_fd_derivatives.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.sb_segments.restype = C.c_int
        L.sb_segments.argtypes = [C.c_void_p, C.c_int32, C.c_uint64, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.c_void_p]
        L.sb_precheck.restype = C.c_int
        L.sb_precheck.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        for name in ("sb_loglik", "sb_loglik_noalloc", "sb_loglik_noalloc_check", "sb_discover", "sb_refine", "sb_laplace", "sb_evidence", "sb_evidence_host",
                     "sb_check", "sb_chisao", "sb_evidence_chisao", "sb_evidence_chisao_host", "sb_chisao_stats"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def declared_symbols():
    """Function names declared in include/sb.h."""
    with open(HEADER_PATH) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sb_[a-z0-9_]+)\s*\(", text)))


def status_string(code: int) -> str:
    try:
        return lib().sb_status_string(int(code)).decode()
    except Exception:
        return f"status {code}"


def _check(code: int, where: str):
    if code != SB_OK:
        raise SbError(code, where)


def _torch():
    import torch

    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Problem:
    """Device copy of one Instance plus the C struct that points at it."""

    def __init__(self, inst: Instance, device="cuda"):
        torch = _torch()
        self.inst = inst
        self.d, self.K = int(inst.d), int(inst.K)
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        self.log_w, self.mu, self.L, self.lo, self.hi = (f(inst.log_w), f(inst.mu), f(inst.L), f(inst.lo),
                                                         f(inst.hi))
        self.s = _Problem(self.d, self.K, self.log_w.data_ptr(), self.mu.data_ptr(), self.L.data_ptr(),
                          self.lo.data_ptr(), self.hi.data_ptr())


class TensorProblem:
    """C struct over caller-owned CUDA float64 tensors (log_w, mu, L, lo, hi)."""

    def __init__(self, log_w, mu, L, lo, hi):
        self.tensors = [t.contiguous() for t in (log_w, mu, L, lo, hi)]
        self.log_w, self.mu, self.L, self.lo, self.hi = self.tensors
        self.K, self.d = int(mu.shape[0]), int(mu.shape[1])
        self.s = _Problem(self.d, self.K, *[t.data_ptr() for t in self.tensors])


def host_problem(inst: Instance, pinned: bool = False):
    """C struct pointing at host arrays (for sb_evidence_host); keeps them alive.
    pinned=True places them in page-locked memory (torch pinned tensors)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (inst.log_w, inst.mu, inst.L, inst.lo, inst.hi)]
    if pinned:
        torch = _torch()
        arrs = [torch.from_numpy(a).pin_memory() for a in arrs]
        ptrs = [a.data_ptr() for a in arrs]
    else:
        ptrs = [a.ctypes.data for a in arrs]
    s = _Problem(int(inst.d), int(inst.K), *ptrs)
    return s, arrs


def make_config(cfg: SolveConfig, **over) -> _Config:
    v = dict(cfg.__dict__)
    v.update(over)
    return _Config(v["n_rays"], v["n_steps"], v["n_starts"], v["m"], v["max_iter"], v["max_backtracks"],
                   v["newton_steps"], v["cand_cap"], v["gtol"], v["armijo_c1"], v["backtrack"], v["dedup_coarse"],
                   v["dedup_tol"], v["eps_grad"], int(v["seed"]) & ((1 << 64) - 1), int(v["prec"]), 0)


def workspace_bytes(prob: Problem, cfg: _Config) -> int:
    return int(lib().sb_workspace_bytes(C.byref(prob.s), C.byref(cfg)))


class Workspace:
    """Caller-owned device scratch sized by the library's query."""

    def __init__(self, nbytes: int, device="cuda"):
        torch = _torch()
        if nbytes <= 0:
            raise SbError(SB_ERR_INVALID_ARG, "workspace query")
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        self.nbytes = int(nbytes)

    @property
    def ptr(self):
        return C.c_void_p(self.buf.data_ptr())


def workspace(prob: Problem, cfg: _Config) -> Workspace:
    return Workspace(workspace_bytes(prob, cfg))


def check(ws: Workspace, stream=None):
    """Synchronise and raise on the device status word (non-finite input, no modes, ...)."""
    _check(lib().sb_check(ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)), "sb_check")


def loglik(prob: Problem, x, prec: int = PREC_FP64, want_grad: bool = True, ws: Workspace = None, stream=None):
    torch = _torch()
    x = x.to(dtype=torch.float64).contiguous()
    n = x.shape[0]
    ell = torch.empty(n, dtype=torch.float64, device=x.device)
    grad = torch.empty_like(x) if want_grad else None
    if ws is None:
        ws = Workspace(lib().sb_loglik_workspace_bytes(C.byref(prob.s), int(prec), int(n)))
    _check(lib().sb_loglik(C.byref(prob.s), C.c_int32(prec), _ptr(x), C.c_int32(n), _ptr(ell), _ptr(grad), ws.ptr,
                           C.c_size_t(ws.nbytes), _stream(stream)), "sb_loglik")
    return (ell, grad) if want_grad else ell


def discover(prob: Problem, cfg: _Config, ws: Workspace = None, stream=None):
    torch = _torch()
    ws = ws or workspace(prob, cfg)
    starts = torch.empty((cfg.n_starts, prob.d), dtype=torch.float64, device="cuda")
    ell = torch.empty(cfg.n_starts, dtype=torch.float64, device="cuda")
    _check(lib().sb_discover(C.byref(prob.s), C.byref(cfg), _ptr(starts), _ptr(ell), ws.ptr, C.c_size_t(ws.nbytes),
                             _stream(stream)), "sb_discover")
    return starts, ell


@dataclass
class RefineOut:
    x: object
    ell: object
    status: object
    iters: object
    n_evals: int


def refine(prob: Problem, cfg: _Config, starts, ws: Workspace = None, stream=None) -> RefineOut:
    torch = _torch()
    ws = ws or workspace(prob, cfg)
    starts = starts.to(dtype=torch.float64).contiguous()
    n = starts.shape[0]
    x = torch.empty_like(starts)
    ell = torch.empty(n, dtype=torch.float64, device=starts.device)
    st = torch.empty(n, dtype=torch.int8, device=starts.device)
    it = torch.empty(n, dtype=torch.int32, device=starts.device)
    ev = torch.zeros(1, dtype=torch.int64, device=starts.device)
    _check(lib().sb_refine(C.byref(prob.s), C.byref(cfg), _ptr(starts), C.c_int32(n), _ptr(x), _ptr(ell), _ptr(st),
                           _ptr(it), _ptr(ev), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)), "sb_refine")
    return RefineOut(x, ell, st, it, int(ev.item()))


class _ChisaoConfig(C.Structure):
    _fields_ = [("n_osc", C.c_int32), ("conv_iters", C.c_int32), ("anti_steps", C.c_int32),
                ("min_unconverged", C.c_int32), ("momentum", C.c_double), ("anti_alpha", C.c_double)]


def make_chisao_config(n_osc=3, conv_iters=1000, anti_steps=10, min_unconverged=5, momentum=0.9,
                       anti_alpha=0.1) -> _ChisaoConfig:
    return _ChisaoConfig(int(n_osc), int(conv_iters), int(anti_steps), int(min_unconverged), float(momentum),
                         float(anti_alpha))


def chisao_workspace(prob: Problem, cfg: _Config) -> Workspace:
    return Workspace(int(lib().sb_chisao_workspace_bytes(C.byref(prob.s), C.byref(cfg))))


@dataclass
class ChisaoOut:
    x: object
    ell: object
    stuck: object
    n_peaks: int


def chisao(prob: Problem, cfg: _Config, cc: _ChisaoConfig, x0, ws: Workspace = None, stream=None) -> ChisaoOut:
    """ChiSao oscillation of the rows of x0 (FP64); the peaks are x[stuck]."""
    torch = _torch()
    ws = ws or chisao_workspace(prob, cfg)
    x0 = x0.to(dtype=torch.float64).contiguous()
    n = x0.shape[0]
    x = torch.empty_like(x0)
    ell = torch.empty(n, dtype=torch.float64, device=x0.device)
    stuck = torch.empty(n, dtype=torch.int8, device=x0.device)
    npk = torch.zeros(1, dtype=torch.int32, device=x0.device)
    _check(lib().sb_chisao(C.byref(prob.s), C.byref(cfg), C.byref(cc), _ptr(x0), C.c_int32(n), _ptr(x), _ptr(ell),
                           _ptr(stuck), _ptr(npk), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)), "sb_chisao")
    return ChisaoOut(x, ell, stuck.bool(), int(npk.item()))


def ray_loglik_quad(prob: Problem, u, n_steps: int, form: int = 1, stream=None):
    """l at the sunburst samples of directions u [n_rays][d] from the quadratic in t (form 0 FP64, 1 FP32)."""
    torch = _torch()
    u = u.to(dtype=torch.float64, device="cuda").contiguous()
    n_rays = u.shape[0]
    ws = Workspace(int(lib().sb_ray_loglik_quad_workspace_bytes(C.byref(prob.s), int(form), int(n_rays))))
    ell = torch.empty((n_rays, n_steps), dtype=torch.float64, device="cuda")
    _check(lib().sb_ray_loglik_quad(C.byref(prob.s), C.c_int32(form), _ptr(u), C.c_int32(n_rays), C.c_int32(n_steps),
                                    _ptr(ell), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)), "sb_ray_loglik_quad")
    return ell


def ray_loglik_origins(prob: Problem, o, u, n_steps: int, form: int = 2, stream=None):
    """l at the samples of rays from origins o [n_rays][d] along unit directions u (form 2
    BF16, 3 TF32 tensor-core split products); returns (ell [n_rays][n_steps], t_exit)."""
    torch = _torch()
    o = o.to(dtype=torch.float64, device="cuda").contiguous()
    u = u.to(dtype=torch.float64, device="cuda").contiguous()
    n_rays = u.shape[0]
    ws = Workspace(int(lib().sb_ray_loglik_origins_workspace_bytes(C.byref(prob.s), int(form), int(n_rays))))
    ell = torch.empty((n_rays, n_steps), dtype=torch.float64, device="cuda")
    te = torch.empty(n_rays, dtype=torch.float64, device="cuda")
    _check(lib().sb_ray_loglik_origins(C.byref(prob.s), C.c_int32(form), _ptr(o), _ptr(u), C.c_int32(n_rays),
                                       C.c_int32(n_steps), _ptr(ell), _ptr(te), ws.ptr, C.c_size_t(ws.nbytes),
                                       _stream(stream)), "sb_ray_loglik_origins")
    return ell, te


@dataclass
class FdOut:
    grad: object
    hdiag: object
    H: object
    b: float


def fd_derivatives(prob: Problem, x, eps_g: float = 1e-5, eps_h: float = 1e-4, full: bool = False,
                   stream=None) -> FdOut:
    """Central-difference gradient, Hessian diagonal (and full Hessian) of l at x, and the probe b."""
    torch = _torch()
    x = x.to(dtype=torch.float64, device="cuda").contiguous()
    ws = Workspace(int(lib().sb_fd_workspace_bytes(C.byref(prob.s), int(bool(full)))))
    g = torch.empty(prob.d, dtype=torch.float64, device="cuda")
    hd = torch.empty(prob.d, dtype=torch.float64, device="cuda")
    H = torch.empty((prob.d, prob.d), dtype=torch.float64, device="cuda") if full else None
    b = torch.zeros(1, dtype=torch.float64, device="cuda")
    _check(lib().sb_fd_derivatives(C.byref(prob.s), _ptr(x), float(eps_g), float(eps_h), int(bool(full)), _ptr(g),
                                   _ptr(hd), _ptr(H), _ptr(b), ws.ptr, ws.nbytes, _stream(stream)),
           "sb_fd_derivatives")
    return FdOut(g, hd, H, float(b.item()))


RAY_V2V, RAY_V2E, RAY_W2W = 1, 2, 3


@dataclass
class SegmentsOut:
    start: object
    end: object
    ell_coarse: object
    t_ref: object
    ell_ref: object


def segments(prob: Problem, family: int, seed: int, n_rays: int, n_steps: int, delta: float = float("inf"),
             n_ref: int = 0, stream=None) -> SegmentsOut:
    """V2V / V2E / W2W rays with their coarse and likelihood-proportional refined samples (FP64)."""
    torch = _torch()
    ws = Workspace(int(lib().sb_segments_workspace_bytes(C.byref(prob.s), int(n_rays), int(n_steps))))
    ends = torch.empty((2, n_rays, prob.d), dtype=torch.float64, device="cuda")
    lc = torch.empty((n_rays, n_steps), dtype=torch.float64, device="cuda")
    tr = torch.empty((n_rays, max(n_ref, 0)), dtype=torch.float64, device="cuda")
    lr = torch.empty((n_rays, max(n_ref, 0)), dtype=torch.float64, device="cuda")
    _check(lib().sb_segments(C.byref(prob.s), int(family), int(seed) & ((1 << 64) - 1), int(n_rays), int(n_steps),
                             float(delta), int(n_ref), _ptr(ends), _ptr(lc), _ptr(tr) if n_ref > 0 else None,
                             _ptr(lr) if n_ref > 0 else None, ws.ptr, ws.nbytes, _stream(stream)), "sb_segments")
    return SegmentsOut(ends[0], ends[1], lc, tr, lr)


def evidence_chisao(prob: Problem, cfg: _Config, cc: _ChisaoConfig, cap: Optional[int] = None, ws: Workspace = None,
                    stream=None, out: Optional["EvidenceBuffers"] = None, sync_check: bool = True) -> "LaplaceOut":
    """Discovery, the ChiSao oscillation, and the Laplace stage over every final sample
    (`out` as for evidence)."""
    ws = ws or chisao_workspace(prob, cfg)
    out = out or EvidenceBuffers(prob.d, cap or cfg.cand_cap)
    cap = out.cap
    modes, zk, nm, lz = out.modes, out.zk, out.nm, out.lz
    _check(lib().sb_evidence_chisao(C.byref(prob.s), C.byref(cfg), C.byref(cc), _ptr(lz), _ptr(modes), _ptr(zk),
                                    C.c_int32(cap), _ptr(nm), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)),
           "sb_evidence_chisao")
    if sync_check:
        code = lib().sb_check(ws.ptr, C.c_size_t(ws.nbytes), _stream(stream))
        if code not in (SB_OK, SB_ERR_NO_MODES):
            raise SbError(code, "sb_evidence_chisao")
    k = min(int(nm.item()), cap)
    return LaplaceOut(float(lz.item()), modes[:k], zk[:k], None, int(nm.item()))


@dataclass
class PrecheckOut:
    s: object
    cls: object
    log_int: float
    log_vol: float
    n_active: int


def precheck(prob: Problem, eps_flat: float = 1e-6, eps_soft: float = 1e-3, stream=None) -> PrecheckOut:
    """Sensitivity probe and flat / soft-nuisance classes (0 active, 1 flat, 2 soft)."""
    torch = _torch()
    ws = Workspace(int(lib().sb_precheck_workspace_bytes(C.byref(prob.s))))
    s = torch.empty(prob.d, dtype=torch.float64, device="cuda")
    cls = torch.empty(prob.d, dtype=torch.int8, device="cuda")
    sc = torch.zeros(2, dtype=torch.float64, device="cuda")
    na = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib().sb_precheck(C.byref(prob.s), float(eps_flat), float(eps_soft), _ptr(s), _ptr(cls),
                             C.c_void_p(sc.data_ptr()), C.c_void_p(sc.data_ptr() + 8), _ptr(na), ws.ptr,
                             ws.nbytes, _stream(stream)), "sb_precheck")
    v = sc.cpu().numpy()
    return PrecheckOut(s, cls, float(v[0]), float(v[1]), int(na.item()))


@dataclass
class LaplaceOut:
    logZ: float
    modes: object
    logZk: object
    ell: object
    n_modes: int


def laplace(prob: Problem, cfg: _Config, x, ell, status=None, cap: Optional[int] = None, ws: Workspace = None,
            stream=None, raise_no_modes: bool = False) -> LaplaceOut:
    torch = _torch()
    ws = ws or workspace(prob, cfg)
    x = x.to(dtype=torch.float64).contiguous()
    ell = ell.to(dtype=torch.float64).contiguous()
    n = x.shape[0]
    cap = cap or cfg.cand_cap
    modes = torch.empty((cap, prob.d), dtype=torch.float64, device=x.device)
    zk = torch.empty(cap, dtype=torch.float64, device=x.device)
    lm = torch.empty(cap, dtype=torch.float64, device=x.device)
    nm = torch.zeros(1, dtype=torch.int32, device=x.device)
    lz = torch.zeros(1, dtype=torch.float64, device=x.device)
    st = None if status is None else status.to(dtype=torch.int8).contiguous()
    _check(lib().sb_laplace(C.byref(prob.s), C.byref(cfg), _ptr(x), _ptr(ell), _ptr(st), C.c_int32(n), _ptr(modes),
                            _ptr(zk), _ptr(lm), C.c_int32(cap), _ptr(nm), _ptr(lz), ws.ptr, C.c_size_t(ws.nbytes),
                            _stream(stream)), "sb_laplace")
    code = lib().sb_check(ws.ptr, C.c_size_t(ws.nbytes), _stream(stream))
    if code != SB_OK and (code != SB_ERR_NO_MODES or raise_no_modes):
        raise SbError(code, "sb_laplace")
    k = min(int(nm.item()), cap)
    return LaplaceOut(float(lz.item()), modes[:k], zk[:k], lm[:k], int(nm.item()))


class EvidenceBuffers:
    """Device outputs of one evidence call (log Z, mode count, modes, log Z_k), kept
    across calls: a call with the same problem, knobs, workspace and buffers replays
    the library's cached graph instead of capturing a new one."""

    def __init__(self, d: int, cap: int):
        torch = _torch()
        self.cap = int(cap)
        self.modes = torch.zeros((cap, d), dtype=torch.float64, device="cuda")
        self.zk = torch.zeros(cap, dtype=torch.float64, device="cuda")
        self.nm = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.lz = torch.zeros(1, dtype=torch.float64, device="cuda")


def evidence(prob: Problem, cfg: _Config, cap: Optional[int] = None, ws: Workspace = None, stream=None,
             sync_check: bool = True, out: Optional[EvidenceBuffers] = None) -> LaplaceOut:
    """discover + refine + laplace. With `out`, the results are written into (and the
    returned modes / log Z_k are views of) those buffers."""
    ws = ws or workspace(prob, cfg)
    out = out or EvidenceBuffers(prob.d, cap or cfg.cand_cap)
    cap = out.cap
    modes, zk, nm, lz = out.modes, out.zk, out.nm, out.lz
    _check(lib().sb_evidence(C.byref(prob.s), C.byref(cfg), _ptr(lz), _ptr(modes), _ptr(zk), C.c_int32(cap),
                             _ptr(nm), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)), "sb_evidence")
    if sync_check:
        code = lib().sb_check(ws.ptr, C.c_size_t(ws.nbytes), _stream(stream))
        if code not in (SB_OK, SB_ERR_NO_MODES):
            raise SbError(code, "sb_evidence")
    k = min(int(nm.item()), cap)
    return LaplaceOut(float(lz.item()), modes[:k], zk[:k], None, int(nm.item()))


def evidence_host_workspace(inst: Instance, cfg: _Config) -> Workspace:
    s, _keep = host_problem(inst)
    return Workspace(lib().sb_evidence_host_workspace_bytes(C.byref(s), C.byref(cfg)))


class PinnedHost:
    """Page-locked host copies of one instance and of the outputs of
    sb_evidence_host, allocated once and reused across calls."""

    def __init__(self, inst: Instance, cfg: _Config):
        torch = _torch()
        self.inst = inst
        self.s, self.keep = host_problem(inst, pinned=True)
        cap = cfg.cand_cap
        pin = lambda *shape, dt=torch.float64: torch.zeros(*shape, dtype=dt).pin_memory()
        self.lz, self.nm = pin(1), pin(1, dt=torch.int32)
        self.modes, self.zk = pin(cap, inst.d), pin(cap)


def evidence_host(inst: Instance, cfg: _Config, ws: Workspace, stream=None, host: PinnedHost = None):
    """The whole path on HOST arrays: copies in, solves, copies log Z and the modes out.
    With `host` (a PinnedHost of this instance) the arrays are page-locked."""
    cap = cfg.cand_cap
    if host is not None:
        s, keep = host.s, None
        lz, nm, modes, zk = host.lz.numpy(), host.nm.numpy(), host.modes.numpy(), host.zk.numpy()
    else:
        s, keep = host_problem(inst)
        lz = np.zeros(1)
        nm = np.zeros(1, dtype=np.int32)
        modes = np.zeros((cap, inst.d))
        zk = np.zeros(cap)
    code = lib().sb_evidence_host(C.byref(s), C.byref(cfg), lz.ctypes.data_as(C.c_void_p),
                                  modes.ctypes.data_as(C.c_void_p), zk.ctypes.data_as(C.c_void_p), C.c_int32(cap),
                                  nm.ctypes.data_as(C.c_void_p), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream))
    if code not in (SB_OK, SB_ERR_NO_MODES):
        raise SbError(code, "sb_evidence_host")
    del keep
    k = min(int(nm[0]), cap)
    return float(lz[0]), modes[:k].copy(), zk[:k].copy(), int(nm[0])


def evidence_chisao_host_workspace(inst: Instance, cfg: _Config) -> Workspace:
    s, _keep = host_problem(inst)
    return Workspace(lib().sb_evidence_chisao_host_workspace_bytes(C.byref(s), C.byref(cfg)))


def evidence_chisao_host(inst: Instance, cfg: _Config, cc, ws: Workspace, stream=None, host: PinnedHost = None):
    """Discovery, ChiSao and the Laplace stage on HOST arrays (copies in, solves, copies
    log Z and the modes out). With `host` (a PinnedHost of this instance) the arrays are
    page-locked."""
    cap = cfg.cand_cap
    if host is not None:
        s, keep = host.s, None
        lz, nm, modes, zk = host.lz.numpy(), host.nm.numpy(), host.modes.numpy(), host.zk.numpy()
    else:
        s, keep = host_problem(inst)
        lz = np.zeros(1)
        nm = np.zeros(1, dtype=np.int32)
        modes = np.zeros((cap, inst.d))
        zk = np.zeros(cap)
    code = lib().sb_evidence_chisao_host(C.byref(s), C.byref(cfg), C.byref(cc), lz.ctypes.data_as(C.c_void_p),
                                         modes.ctypes.data_as(C.c_void_p), zk.ctypes.data_as(C.c_void_p),
                                         C.c_int32(cap), nm.ctypes.data_as(C.c_void_p), ws.ptr,
                                         C.c_size_t(ws.nbytes), _stream(stream))
    if code not in (SB_OK, SB_ERR_NO_MODES):
        raise SbError(code, "sb_evidence_chisao_host")
    del keep
    k = min(int(nm[0]), cap)
    return float(lz[0]), modes[:k].copy(), zk[:k].copy(), int(nm[0])


def chisao_stats(prob: Problem, cfg: _Config, ws: Workspace, stream=None):
    """(ray l evaluations, L-BFGS l+grad evaluations, anti-convergence l+grad evaluations,
    modes kept) of the last ChiSao solve on this workspace."""
    out = (C.c_int64 * 4)()
    _check(lib().sb_chisao_stats(C.byref(prob.s), C.byref(cfg), ws.ptr, C.c_size_t(ws.nbytes), out,
                                 _stream(stream)), "sb_chisao_stats")
    return tuple(int(v) for v in out)


def evidence_backward(prob, modes, logZk, n_modes: int, grad_logZ: float = 1.0, stream=None):
    """d log Z / d mu_k and d log Z / d L_k (lower) at the modes of a forward solve."""
    torch = _torch()
    dmu = torch.zeros((prob.K, prob.d), dtype=torch.float64, device="cuda")
    dL = torch.zeros((prob.K, prob.d, prob.d), dtype=torch.float64, device="cuda")
    ws = Workspace(lib().sb_evidence_backward_workspace_bytes(C.byref(prob.s)))
    modes = modes.contiguous()
    logZk = logZk.contiguous()
    _check(lib().sb_evidence_backward(C.byref(prob.s), _ptr(modes), _ptr(logZk), int(n_modes), float(grad_logZ),
                                      _ptr(dmu), _ptr(dL), ws.ptr, ws.nbytes, _stream(stream)),
           "sb_evidence_backward")
    return dmu, dL


def _autograd_function():
    torch = _torch()

    class EvidenceFunction(torch.autograd.Function):
        """log Z as a differentiable function of the component means and
        precision Cholesky factors (log_w and the box are treated as constants)."""

        @staticmethod
        def forward(ctx, mu, L, log_w, lo, hi, cfg):
            prob = TensorProblem(log_w.detach(), mu.detach(), L.detach(), lo.detach(), hi.detach())
            out = evidence(prob, cfg)
            ctx.prob = prob
            ctx.save_for_backward(out.modes.clone(), out.logZk.clone())
            ctx.n_modes = out.n_modes
            return torch.tensor(out.logZ, dtype=torch.float64, device=mu.device)

        @staticmethod
        def backward(ctx, grad):
            modes, logZk = ctx.saved_tensors
            if ctx.n_modes == 0:
                return None, None, None, None, None, None
            dmu, dL = evidence_backward(ctx.prob, modes, logZk, min(ctx.n_modes, modes.shape[0]),
                                        float(grad.item()))
            return dmu, dL, None, None, None, None

    return EvidenceFunction


def evidence_autograd(mu, L, log_w, lo, hi, cfg: _Config):
    """log Z with autograd support for mu and L (see EvidenceFunction)."""
    return _autograd_function().apply(mu, L, log_w, lo, hi, cfg)


def batched_workspace(problems, cfg: _Config, n_workers: int = 8, chisao: bool = False) -> Workspace:
    P = len(problems)
    arr = (_Problem * P)(*[p.s for p in problems])
    q = lib().sb_evidence_chisao_batched_workspace_bytes if chisao else lib().sb_evidence_batched_workspace_bytes
    return Workspace(q(arr, P, C.byref(cfg), int(n_workers)))


def evidence_batched(problems, cfg: _Config, n_workers: int = 8, stream=None, ws: Workspace = None, out=None,
                     cc: Optional[_ChisaoConfig] = None):
    """Solve many independent problems (list of Problem) in one library call (with the
    ChiSao oscillation when cc is given). Returns (logZ, n_modes) as CUDA tensors of
    length P (the tensors of `out`, a (logZ, n_modes) pair kept across calls, when
    given: with the same workspace the call then replays the library's cached graph)."""
    torch = _torch()
    P = len(problems)
    arr = (_Problem * P)(*[p.s for p in problems])
    ws = ws or batched_workspace(problems, cfg, n_workers, chisao=cc is not None)
    if out is None:
        out = (torch.empty(P, dtype=torch.float64, device="cuda"), torch.empty(P, dtype=torch.int32, device="cuda"))
    logZ, nm = out
    if cc is not None:
        _check(lib().sb_evidence_chisao_batched(arr, P, C.byref(cfg), C.byref(cc), _ptr(logZ), _ptr(nm),
                                                int(n_workers), ws.ptr, C.c_size_t(ws.nbytes), _stream(stream)),
               "sb_evidence_chisao_batched")
        return logZ, nm
    _check(lib().sb_evidence_batched(arr, P, C.byref(cfg), _ptr(logZ), _ptr(nm), int(n_workers), ws.ptr,
                                     C.c_size_t(ws.nbytes), _stream(stream)), "sb_evidence_batched")
    return logZ, nm
