"""Complex-step derivatives of the Laplace evidence with respect to the component
means and precision Cholesky factors.

TEST INFRASTRUCTURE ONLY: used by the tests as the reference for the adjoint
d log Z / d (mu_k, L_k); the product path never imports it. It shares no code
with the CUDA library, and none with the C oracle either: it is a second,
plain numpy statement of the Laplace evidence (Sec. 3.7.1, App. A.8), written
so that every step is analytic in the parameters and can run in complex
arithmetic:

    z_k = L_k^T (x - mu_k),  a_k = log w_k - (d/2) log 2 pi + sum_i log L_k,ii
    e_k = a_k - z_k^T z_k / 2,  l = LSE_k e_k,  r_k = exp(e_k - l)
    grad l = sum_k r_k g_k,  g_k = -L_k z_k
    H = -hess l = sum_k r_k L_k L_k^T - sum_k r_k g_k g_k^T + grad l grad l^T
    mode: Newton x <- x + H^-1 grad l from the given mode
    log Z_m = l(x*) + (d/2) log 2 pi - 1/2 log det H(x*),  log det by a
              Cholesky factorisation without conjugation
    log Z = LSE_m log Z_m - log V

(no conjugates anywhere, so the functions continue analytically off the real
axis). The derivative of log Z along a real parameter p is then
Im log Z(p + i h) / h with h = 1e-30: no subtraction, so it is exact to
rounding (complex-step differentiation, Squire & Trapp, SIAM Review 1998;
Martins, Sturdza & Alonso, ACM TOMS 2003). The Newton iterations carry the
imaginary part of each mode, so the implicit shift of the modes is included.
"""
from __future__ import annotations

import math

import numpy as np

_H = 1e-30
_LOG_2PI = math.log(2.0 * math.pi)


def _lse(v):
    m = np.max(v.real)
    return m + np.log(np.sum(np.exp(v - m)))


def _parts(log_w, mu, L, x):
    """l, grad l and H = -hess l at x (complex-safe)."""
    K, d = mu.shape
    diff = x[None, :] - mu  # (K, d)
    z = np.einsum("kij,ki->kj", L, diff)  # z_k = L_k^T (x - mu_k)
    a = log_w - 0.5 * d * _LOG_2PI + np.sum(np.log(np.diagonal(L, axis1=1, axis2=2)), axis=1)
    e = a - 0.5 * np.sum(z * z, axis=1)
    ell = _lse(e)
    r = np.exp(e - ell)
    g = -np.einsum("kij,kj->ki", L, z)  # g_k = -L_k z_k
    grad = np.sum(r[:, None] * g, axis=0)
    P = np.einsum("kij,klj->kil", L, L)  # L_k L_k^T
    H = np.einsum("k,kil->il", r, P) - np.einsum("k,ki,kl->il", r, g, g) + np.outer(grad, grad)
    return ell, grad, H


def _logdet_sym(H):
    """log det of a symmetric (complex) matrix by Cholesky without conjugation."""
    d = H.shape[0]
    C = np.zeros_like(H)
    for j in range(d):
        s = H[j, j] - np.sum(C[j, :j] * C[j, :j])
        C[j, j] = np.sqrt(s)
        for i in range(j + 1, d):
            C[i, j] = (H[i, j] - np.sum(C[i, :j] * C[j, :j])) / C[j, j]
    return 2.0 * np.sum(np.log(np.diagonal(C)))


def log_evidence(log_w, mu, L, lo, hi, modes, newton_steps=8):
    """Laplace log Z at the modes reached by Newton from `modes` (real or complex parameters)."""
    d = mu.shape[1]
    terms = []
    for m0 in np.asarray(modes, dtype=float):
        x = m0.astype(np.result_type(mu, L, complex))
        for _ in range(newton_steps):
            _, g, H = _parts(log_w, mu, L, x)
            x = x + np.linalg.solve(H, g)
        ell, _, H = _parts(log_w, mu, L, x)
        terms.append(ell + 0.5 * d * _LOG_2PI - 0.5 * _logdet_sym(H))
    logV = float(np.sum(np.log(np.asarray(hi) - np.asarray(lo))))
    return _lse(np.array(terms)) - logV


def dlogz(inst, modes, newton_steps=8):
    """(log Z, d log Z / d mu [K, d], d log Z / d L [K, d, d] on the lower triangle)."""
    log_w = np.asarray(inst.log_w, dtype=float)
    mu = np.asarray(inst.mu, dtype=float)
    L = np.asarray(inst.L, dtype=float)
    K, d = mu.shape
    base = log_evidence(log_w, mu, L, inst.lo, inst.hi, modes, newton_steps)
    gmu = np.zeros((K, d))
    gL = np.zeros((K, d, d))
    for k in range(K):
        for i in range(d):
            m2 = mu.astype(complex)
            m2[k, i] += 1j * _H
            gmu[k, i] = log_evidence(log_w, m2, L, inst.lo, inst.hi, modes, newton_steps).imag / _H
            for j in range(i + 1):
                L2 = L.astype(complex)
                L2[k, i, j] += 1j * _H
                gL[k, i, j] = log_evidence(log_w, mu, L2, inst.lo, inst.hi, modes, newton_steps).imag / _H
    return float(base.real), gmu, gL
