"""Seeded synthetic evidence problems: Gaussian and Gaussian-mixture
log-likelihoods under a uniform box prior.

This module only *builds inputs*. It holds none of the evidence method's
arithmetic (no log-likelihood, no rays, no optimiser, no Laplace step), so the
CPU oracle and the CUDA path can both consume it without sharing method code.

Parameterisation (the one the whole library uses):
    component k has log-weight log_w[k], mean mu[k] (d,), and the lower
    Cholesky factor L[k] (d, d) of its *precision* matrix, P_k = L_k L_k^T =
    Sigma_k^{-1}, with a positive diagonal. The mixture density is
    sum_k w_k N(x; mu_k, Sigma_k); the prior is uniform on prod_i [lo_i, hi_i].

Covariances follow the workloads of the paper's Gaussian / correlated /
mixture suites (Sec. 5): Sigma_k = Q diag(s^2) Q^T with Q Haar-random
orthogonal (QR of a Gaussian matrix with the sign fix of Mezzadri 2007) and s
log-uniform in [s_min, s_max]; mixture weights are Dirichlet(1) draws
(normalised Exp(1) variates); means are uniform in a box and, for mixtures,
redrawn until every pair is more than `sep` * sigma_max apart (Euclidean),
sigma_max being the largest s over all components and axes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Instance:
    """One evidence problem: mixture parameters plus the prior box (all float64)."""

    d: int
    K: int
    log_w: np.ndarray  # (K,)
    mu: np.ndarray  # (K, d)
    L: np.ndarray  # (K, d, d) lower-triangular precision Cholesky factors
    lo: np.ndarray  # (d,)
    hi: np.ndarray  # (d,)
    s: np.ndarray = field(default=None)  # (K, d) per-axis standard deviations used to build it
    seed: int = 0

    def contiguous(self) -> "Instance":
        for name in ("log_w", "mu", "L", "lo", "hi"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), dtype=np.float64))
        return self


@dataclass
class SolveConfig:
    """Knobs of one evidence solve (mirrors the C struct `sb_config`)."""

    n_rays: int = 256
    n_steps: int = 64
    n_starts: int = 64
    m: int = 10
    max_iter: int = 1000
    max_backtracks: int = 40
    newton_steps: int = 3
    cand_cap: int = 256
    gtol: float = 1e-12
    armijo_c1: float = 1e-4
    backtrack: float = 0.5
    dedup_coarse: float = 1e-3
    dedup_tol: float = 1e-6
    eps_grad: float = 1e-6
    seed: int = 0
    prec: int = 0  # 0 = FP64, 1 = TF32 tensor cores, 2 = BF16 tensor cores


def haar_orthogonal(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian matrix, signs fixed)."""
    z = rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    sgn = np.sign(np.diag(r))
    sgn[sgn == 0] = 1.0
    return q * sgn[None, :]


def precision_cholesky(q: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of P = Q diag(s^-2) Q^T (the instance's definition of L)."""
    p = (q * (1.0 / (s * s))[None, :]) @ q.T
    p = 0.5 * (p + p.T)
    return np.linalg.cholesky(p)


def make_instance(
    d: int,
    K: int,
    seed: int,
    s_range=(0.1, 1.0),
    mean_box=(-2.0, 2.0),
    prior=(-10.0, 10.0),
    sep: float = 8.0,
    max_attempts: int = 1_000_000,
) -> Instance:
    """Draw one seeded instance. Covariances first, then means (rejection on separation)."""
    rng = np.random.default_rng(seed)
    s_all = np.empty((K, d))
    L_all = np.empty((K, d, d))
    for k in range(K):
        q = haar_orthogonal(d, rng)
        s = np.exp(rng.uniform(np.log(s_range[0]), np.log(s_range[1]), size=d))
        s_all[k] = s
        L_all[k] = precision_cholesky(q, s)
    if K == 1:
        w = np.ones(1)
    else:
        e = rng.exponential(1.0, size=K)
        w = e / e.sum()
    sigma_max = float(s_all.max())
    mus: List[np.ndarray] = []
    attempts = 0
    while len(mus) < K:
        cand = rng.uniform(mean_box[0], mean_box[1], size=d)
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError(f"could not place {K} means {sep} sigma_max apart in d={d}")
        if all(np.linalg.norm(cand - m) > sep * sigma_max for m in mus):
            mus.append(cand)
    inst = Instance(
        d=d,
        K=K,
        log_w=np.log(w),
        mu=np.stack(mus),
        L=L_all,
        lo=np.full(d, prior[0], dtype=np.float64),
        hi=np.full(d, prior[1], dtype=np.float64),
        s=s_all,
        seed=seed,
    )
    return inst.contiguous()


# --------------------------------------------------------------------------
# The five seeded workloads (instance seed = 1000 * workload + rep).
# --------------------------------------------------------------------------

WORKLOADS = {
    0: "plain FP64, d=8, single correlated Gaussian, 256 rays x 64 steps, 64 starts, m=10",
    1: "FP64, d=64, Gaussian mixture K=4, 1024 rays x 128 steps, 4096 starts, m=10",
    2: "precision, d=256 single correlated Gaussian (s in [0.01,1]), 8192 starts, m=10",
    3: "batching, 512 problems, d in {16..512}, K in 1..8, 256 starts each, m=10",
    4: "d=1024, Gaussian mixture K=8 (>10 sigma_max apart), 16384 starts, m=20",
}


def workload(cfg_id: int, rep: int = 0, scale: Optional[float] = None):
    """Return (instances, SolveConfig) for one of the five workloads.

    `scale` (0 < scale <= 1) shrinks ray/start counts for small parity cases
    while keeping d, K and the value distributions.
    """
    seed = 1000 * cfg_id + rep
    if cfg_id == 0:
        insts = [make_instance(8, 1, seed, s_range=(0.1, 1.0), mean_box=(-2, 2))]
        cfg = SolveConfig(n_rays=256, n_steps=64, n_starts=64, m=10, gtol=1e-12, seed=seed)
    elif cfg_id == 1:
        insts = [make_instance(64, 4, seed, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)]
        cfg = SolveConfig(n_rays=1024, n_steps=128, n_starts=4096, m=10, seed=seed)
    elif cfg_id == 2:
        insts = [make_instance(256, 1, seed, s_range=(0.01, 1.0), mean_box=(-2, 2))]
        cfg = SolveConfig(n_rays=8192, n_steps=64, n_starts=8192, m=10, seed=seed)
    elif cfg_id == 3:
        rng = np.random.default_rng(seed)
        ds = rng.choice(np.arange(16, 513, 16), size=512)
        Ks = rng.integers(1, 9, size=512)
        insts = [
            make_instance(int(dd), int(kk), seed * 1000 + i, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=8.0)
            for i, (dd, kk) in enumerate(zip(ds, Ks))
        ]
        cfg = SolveConfig(n_rays=256, n_steps=64, n_starts=256, m=10, seed=seed, prec=1)
    elif cfg_id == 4:
        insts = [make_instance(1024, 8, seed, s_range=(0.05, 0.5), mean_box=(-6, 6), sep=10.0)]
        cfg = SolveConfig(n_rays=16384, n_steps=64, n_starts=16384, m=20, seed=seed, prec=2)
    else:
        raise ValueError(f"unknown workload {cfg_id}")
    if scale is not None:
        cfg.n_rays = max(1, int(round(cfg.n_rays * scale)))
        cfg.n_starts = max(1, min(cfg.n_rays * cfg.n_steps, int(round(cfg.n_starts * scale))))
    return insts, cfg
