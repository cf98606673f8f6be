"""ctypes binding of the plain FP64 CPU oracle (`sb_oracle.c`).

TEST INFRASTRUCTURE ONLY: imported by the tests, by `__graft_entry__.smoke()`
and by the benchmark's CPU-baseline leg; the product path never touches it.
It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libsb_oracle.so")
_SRC = os.path.join(_HERE, "sb_oracle.c")

RUNNING, CONVERGED, STALLED, MAXITER, NONFINITE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so x86 and Arm agree)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sb_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("d", C.c_int), ("K", C.c_int), ("log_w", C.c_void_p), ("mu", C.c_void_p),
                ("L", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("n_rays", C.c_int), ("n_steps", C.c_int), ("n_starts", C.c_int), ("m", C.c_int),
                ("max_iter", C.c_int), ("max_backtracks", C.c_int), ("newton_steps", C.c_int),
                ("cand_cap", C.c_int), ("gtol", C.c_double), ("armijo_c1", C.c_double),
                ("backtrack", C.c_double), ("dedup_coarse", C.c_double), ("dedup_tol", C.c_double),
                ("eps_grad", C.c_double), ("seed", C.c_uint64), ("n_threads", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_loglik.restype = C.c_double
        for name in ("orc_select_starts", "orc_discover", "orc_cholesky", "orc_laplace", "orc_evidence",
                     "orc_chisao_ray_best", "orc_chisao", "orc_precheck", "orc_ray_segment"):
            getattr(_lib, name).restype = C.c_int
        for name in ("orc_uniform_corr_probe", "orc_perp_fraction"):
            getattr(_lib, name).restype = C.c_double
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleProblem:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, inst):
        self.d, self.K = int(inst.d), int(inst.K)
        self.arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (inst.log_w, inst.mu, inst.L, inst.lo, inst.hi)]
        self.s = _Problem(self.d, self.K, *[_ptr(a) for a in self.arrs])


def _cfg(cfg, n_threads: int = 1) -> _Config:
    return _Config(cfg.n_rays, cfg.n_steps, cfg.n_starts, cfg.m, cfg.max_iter, cfg.max_backtracks,
                   cfg.newton_steps, cfg.cand_cap, cfg.gtol, cfg.armijo_c1, cfg.backtrack,
                   cfg.dedup_coarse, cfg.dedup_tol, cfg.eps_grad, int(cfg.seed) & ((1 << 64) - 1),
                   int(n_threads))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def ray_directions(d: int, n_rays: int, seed: int) -> np.ndarray:
    u = np.empty((n_rays, d))
    lib().orc_ray_directions(C.c_int(d), C.c_int(n_rays), C.c_uint64(seed), _ptr(u))
    return u


def loglik(inst, x, want_grad=False, want_hess=False):
    """l(x) for one point; optionally grad l and -hess l."""
    P = OracleProblem(inst)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.empty(P.d) if want_grad else None
    h = np.empty((P.d, P.d)) if want_hess else None
    val = lib().orc_loglik(C.byref(P.s), _ptr(x), _ptr(g) if g is not None else None,
                           _ptr(h) if h is not None else None)
    out = [val]
    if want_grad:
        out.append(g)
    if want_hess:
        out.append(h)
    return out[0] if len(out) == 1 else tuple(out)


def ray_loglik(inst, cfg, n_threads=1):
    P = OracleProblem(inst)
    c = _cfg(cfg, n_threads)
    u = np.empty((cfg.n_rays, P.d))
    te = np.empty(cfg.n_rays)
    ell = np.empty((cfg.n_rays, cfg.n_steps))
    lib().orc_ray_loglik(C.byref(P.s), C.byref(c), _ptr(u), _ptr(te), _ptr(ell))
    return u, te, ell


def select_starts(cfg, ell):
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    c = _cfg(cfg)
    idx = np.empty(max(cfg.n_starts, 1), dtype=np.int64)
    n = lib().orc_select_starts(C.byref(c), _ptr(ell), _ptr(idx))
    return idx[:n]


def discover(inst, cfg, n_threads=1):
    P = OracleProblem(inst)
    c = _cfg(cfg, n_threads)
    starts = np.empty((max(cfg.n_starts, 1), P.d))
    ls = np.empty(max(cfg.n_starts, 1))
    n = lib().orc_discover(C.byref(P.s), C.byref(c), _ptr(starts), _ptr(ls))
    return starts[:n], ls[:n]


def two_loop(S, Y, rho, q):
    S = np.ascontiguousarray(S, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    count, d = (S.shape[0], S.shape[1]) if S.ndim == 2 and S.shape[0] > 0 else (0, q.shape[0])
    r = np.empty(d)
    lib().orc_two_loop(C.c_int(d), C.c_int(count), _ptr(S), _ptr(Y), _ptr(rho), _ptr(q), _ptr(r))
    return r


@dataclass
class RefineResult:
    x: np.ndarray
    ell: np.ndarray
    status: np.ndarray
    iters: np.ndarray
    evals: int


def lbfgs(inst, cfg, x0, n_threads=1) -> RefineResult:
    P = OracleProblem(inst)
    c = _cfg(cfg, n_threads)
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, P.d)
    n = x0.shape[0]
    xo = np.empty_like(x0)
    lo = np.empty(n)
    st = np.empty(n, dtype=np.int8)
    it = np.empty(n, dtype=np.int32)
    ev = C.c_int64(0)
    lib().orc_lbfgs(C.byref(P.s), C.byref(c), _ptr(x0), C.c_int(n), _ptr(xo), _ptr(lo), _ptr(st), _ptr(it),
                    C.byref(ev))
    return RefineResult(xo, lo, st, it, int(ev.value))


def cholesky(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    d = A.shape[0]
    Cm = np.empty_like(A)
    rc = lib().orc_cholesky(C.c_int(d), _ptr(A), _ptr(Cm))
    return Cm if rc == 0 else None


@dataclass
class LaplaceResult:
    logZ: float
    modes: np.ndarray
    logZk: np.ndarray
    ell: np.ndarray
    n_modes: int


def laplace(inst, cfg, x, ell, status=None, cap=None, n_threads=1) -> LaplaceResult:
    P = OracleProblem(inst)
    c = _cfg(cfg, n_threads)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, P.d)
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    n = x.shape[0]
    cap = cap if cap is not None else max(cfg.cand_cap, 1)
    modes = np.empty((cap, P.d))
    zk = np.empty(cap)
    lm = np.empty(cap)
    nm = C.c_int(0)
    lz = C.c_double(0.0)
    st = None if status is None else np.ascontiguousarray(status, dtype=np.int8)
    lib().orc_laplace(C.byref(P.s), C.byref(c), _ptr(x), _ptr(ell), _ptr(st) if st is not None else None,
                      C.c_int(n), _ptr(modes), _ptr(zk), _ptr(lm), C.c_int(cap), C.byref(nm), C.byref(lz))
    k = min(nm.value, cap)
    return LaplaceResult(lz.value, modes[:k], zk[:k], lm[:k], nm.value)


def evidence(inst, cfg, n_threads=1) -> LaplaceResult:
    """discover + refine + laplace, exactly as the three functions above chain them."""
    starts, _ = discover(inst, cfg, n_threads)
    ref = lbfgs(inst, cfg, starts, n_threads)
    return laplace(inst, cfg, ref.x, ref.ell, ref.status, n_threads=n_threads)


# ------------------------------------------------------------------ ChiSao (Sec. 3.5.5)
class _ChisaoConfig(C.Structure):
    _fields_ = [("n_osc", C.c_int), ("conv_iters", C.c_int), ("anti_steps", C.c_int),
                ("min_unconverged", C.c_int), ("momentum", C.c_double), ("anti_alpha", C.c_double),
                ("conv_from_status", C.c_int)]


@dataclass
class ChisaoConfig:
    """Knobs of the ChiSao oscillation (defaults: the values the paper states where it states one)."""

    n_osc: int = 3
    conv_iters: int = 1000
    anti_steps: int = 10
    min_unconverged: int = 5
    momentum: float = 0.9
    anti_alpha: float = 0.1
    conv_from_status: bool = False


@dataclass
class ChisaoResult:
    x: np.ndarray
    ell: np.ndarray
    stuck: np.ndarray
    n_peaks: int


def chisao_anticonverge(inst, x, steps, momentum, alpha):
    """Momentum anti-convergence of the rows of x (returns a new array)."""
    P = OracleProblem(inst)
    x = np.array(x, dtype=np.float64).reshape(-1, P.d)
    lib().orc_chisao_anticonverge(C.byref(P.s), _ptr(x), C.c_int(x.shape[0]), C.c_int(steps),
                                  C.c_double(momentum), C.c_double(alpha))
    return x


def chisao_directions(d, r, seed, osc, peak, basis=0):
    """The first r (at most min(d, 64)) orthonormal directions of one group, one per row."""
    r = min(r, d, 64)
    Q = np.empty((r, d))
    lib().orc_chisao_directions(C.c_int(d), C.c_int(r), C.c_uint64(seed), C.c_int(osc), C.c_int(peak),
                                C.c_int(basis), _ptr(Q))
    return Q


def chisao_ray_best(inst, origin, direction, n_steps, past_valley=False):
    """(sample index, point, l) of the best sample on the ray to the box boundary."""
    P = OracleProblem(inst)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    u = np.ascontiguousarray(direction, dtype=np.float64)
    x = np.empty(P.d)
    ell = C.c_double(0.0)
    j = lib().orc_chisao_ray_best(C.byref(P.s), _ptr(o), _ptr(u), C.c_int(n_steps), C.c_int(int(past_valley)),
                                  _ptr(x), C.byref(ell))
    return j, x, ell.value


def chisao(inst, cfg, cc: ChisaoConfig, x0, n_threads=1) -> ChisaoResult:
    P = OracleProblem(inst)
    c = _cfg(cfg, n_threads)
    k = _ChisaoConfig(cc.n_osc, cc.conv_iters, cc.anti_steps, cc.min_unconverged, cc.momentum, cc.anti_alpha,
                      int(bool(cc.conv_from_status)))
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, P.d)
    n = x0.shape[0]
    xo = np.empty_like(x0)
    lo = np.empty(n)
    st = np.empty(n, dtype=np.int8)
    npk = lib().orc_chisao(C.byref(P.s), C.byref(c), C.byref(k), _ptr(x0), C.c_int(n), _ptr(xo), _ptr(lo),
                           _ptr(st))
    return ChisaoResult(xo, lo, st.astype(bool), int(npk))


# ------------------------------------------------------------- preprocessing (Sec. 3.4)
ACTIVE, FLAT, SOFT = 0, 1, 2


@dataclass
class PrecheckResult:
    s: np.ndarray
    cls: np.ndarray
    log_int: float
    log_vol: float
    n_active: int


def precheck(inst, eps_flat=1e-6, eps_soft=1e-3) -> PrecheckResult:
    """Sensitivity probe and flat / soft-nuisance classification with the marginal terms."""
    P = OracleProblem(inst)
    s = np.empty(P.d)
    cls = np.empty(P.d, dtype=np.int8)
    li = C.c_double(0.0)
    lv = C.c_double(0.0)
    na = lib().orc_precheck(C.byref(P.s), C.c_double(eps_flat), C.c_double(eps_soft), _ptr(s), _ptr(cls),
                            C.byref(li), C.byref(lv))
    return PrecheckResult(s, cls, li.value, lv.value, int(na))


# ------------------------------------------ black-box derivatives and rotation (App. A.4, Sec. 3.7.2)
def fd_grad(inst, x, eps=1e-5):
    P = OracleProblem(inst)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.empty(P.d)
    lib().orc_fd_grad(C.byref(P.s), _ptr(x), C.c_double(eps), _ptr(g))
    return g


def fd_hess_diag(inst, x, eps=1e-4):
    P = OracleProblem(inst)
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.empty(P.d)
    lib().orc_fd_hess_diag(C.byref(P.s), _ptr(x), C.c_double(eps), _ptr(h))
    return h


def fd_hess_full(inst, x, eps=1e-4):
    P = OracleProblem(inst)
    x = np.ascontiguousarray(x, dtype=np.float64)
    H = np.empty((P.d, P.d))
    lib().orc_fd_hess_full(C.byref(P.s), _ptr(x), C.c_double(eps), _ptr(H))
    return H


def uniform_corr_probe(inst, x, hdiag, eps=1e-4):
    P = OracleProblem(inst)
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.ascontiguousarray(hdiag, dtype=np.float64)
    return float(lib().orc_uniform_corr_probe(C.byref(P.s), _ptr(x), C.c_double(eps), _ptr(h)))


def perp_fraction(dtheta, grad, hdiag):
    dt = np.ascontiguousarray(dtheta, dtype=np.float64)
    g = np.ascontiguousarray(grad, dtype=np.float64)
    h = np.ascontiguousarray(hdiag, dtype=np.float64)
    return float(lib().orc_perp_fraction(C.c_int(len(dt)), _ptr(dt), _ptr(g), _ptr(h)))


# ------------------------------------------------ ray families and two-pass sampling (Sec. 3.5.1-3.5.2)
RAY_V2V, RAY_V2E, RAY_W2W = 1, 2, 3


def ray_segment(inst, family, seed, r):
    """(start, end) of ray r of a family."""
    P = OracleProblem(inst)
    a = np.empty(P.d)
    b = np.empty(P.d)
    rc = lib().orc_ray_segment(C.byref(P.s), C.c_int(family), C.c_uint64(seed), C.c_int(r), _ptr(a), _ptr(b))
    if rc != 0:
        raise ValueError(f"unknown ray family {family}")
    return a, b


def ray_two_pass(inst, start, end, n, delta, n_ref):
    """(coarse l [n], refined t [n_ref], refined l [n_ref]) along the segment."""
    P = OracleProblem(inst)
    a = np.ascontiguousarray(start, dtype=np.float64)
    b = np.ascontiguousarray(end, dtype=np.float64)
    lc = np.empty(n)
    tr = np.empty(n_ref)
    lr = np.empty(n_ref)
    lib().orc_ray_two_pass(C.byref(P.s), _ptr(a), _ptr(b), C.c_int(n), C.c_double(delta), C.c_int(n_ref), _ptr(lc),
                           _ptr(tr), _ptr(lr))
    return lc, tr, lr
