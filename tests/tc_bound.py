"""Element-wise error bounds of the tensor-core log-likelihood and gradient,
computed from the FP64 operands (test helper; no method arithmetic is checked
with it, only the size of the rounding the tensor-core path may add).

What the tensor-core path rounds, in order (p = bf16 or tf32, with unit
roundoff u_p = 2^-8 or 2^-11; u32 = 2^-24):
 1. x and mu_k to FP32, their difference a = x - mu_k in FP32, then a to p;
 2. L_k to p;
 3. z_kj = sum_{i >= j} a_i L_k,ij: exact products, FP32 accumulation
    (taken as at most 2^-22 per addition, i.e. truncating adds);
 4. |z_k|^2 in FP32 over tiles of at most 256 columns, tiles summed in FP64;
 5. l = LSE_k (a_k - |z_k|^2 / 2) with FP32 exponentials and logarithm;
    r_k = softmax_k in FP32;
 6. z_kj rounded to p when stored, then r_k z_kj in FP32 rounded to p again;
    grad_i = -sum_k sum_{j <= i} (r_k z_kj) L_k,ij with exact products and FP32
    accumulation over K d terms.
So per entry, with S_kj = sum_i |a_i| |L_k,ij| and T_kj = sum_i (|x_i| + |mu_k,i|) |L_k,ij|:
    |dz_kj| <= E_kj = (2 u_p + u_p^2 + u32 + g1 (1 + u_p)^2) S_kj + 2 u32 (1 + u_p)^2 T_kj,
    g1 = (d + 16) 2^-22;
    |d|z_k|^2| <= Eq_k = sum_j (2 |z_kj| E_kj + E_kj^2) + 512 u32 (|z_k|^2 + that);
then l lies between LSE(e - Eq/2) and LSE(e + Eq/2) (LSE is monotone and
shift-equivariant), r_k between exp(e_k -+ Eq_k/2 - LSE(e +- Eq/2)), and
    |dgrad_i| <= sum_k sum_j |L_k,ij| W_kj,
    W_kj = R_k E_kj + dr_k |z_kj| + (3 u_p + 2 u32 + g2) (1 + u_p)^3 R_k (|z_kj| + E_kj),
    R_k = r_k + dr_k, g2 = (K d + 16) 2^-22,
plus a floor of 2^-20 (1 + K) for the FP32 exponentials and logarithm of the LSE.
These are worst cases (every rounding at its extreme, all of one sign); the
tests assert the measured error is at most a calibrated fraction of them.
"""
from __future__ import annotations

import numpy as np

U_P = {2: 2.0 ** -8, 1: 2.0 ** -11}  # bf16 (8-bit significand), tf32 (11-bit significand)
U32 = 2.0 ** -24


def _lse(e):
    m = e.max(1, keepdims=True)
    with np.errstate(invalid="ignore"):
        return (m + np.log(np.exp(e - m).sum(1, keepdims=True)))[:, 0]


def bounds(inst, X, prec):
    """(B_l [n], B_g [n, d], l [n], z-free exact responsibilities [n, K]) for points X [n, d]."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    K = inst.K
    up = U_P[prec]
    g1 = (d + 16) * 2.0 ** -22
    g2 = (K * d + 16) * 2.0 ** -22
    a_k = inst.log_w - 0.5 * d * np.log(2 * np.pi) + np.log(np.diagonal(inst.L, axis1=1, axis2=2)).sum(1)
    Z, E, q, Eq = [], [], np.empty((n, K)), np.empty((n, K))
    for k in range(K):
        Lk = inst.L[k]
        aL = np.abs(Lk)
        A = X - inst.mu[k]
        z = A @ Lk
        S = np.abs(A) @ aL
        T = (np.abs(X) + np.abs(inst.mu[k])) @ aL
        e = (2 * up + up * up + U32 + g1 * (1 + up) ** 2) * S + 2 * U32 * (1 + up) ** 2 * T
        qk = (z * z).sum(1)
        eq = (2 * np.abs(z) * e + e * e).sum(1)
        eq += 512 * U32 * (qk + eq)
        Z.append(z)
        E.append(e)
        q[:, k] = qk
        Eq[:, k] = eq
    ee = a_k[None, :] - 0.5 * q
    ell = _lse(ee)
    hi = _lse(ee + 0.5 * Eq)
    lo = _lse(ee - 0.5 * Eq)
    floor = 2.0 ** -20 * (1 + K)
    B_l = np.maximum(hi - ell, ell - lo) + floor
    r = np.exp(ee - ell[:, None])
    with np.errstate(over="ignore"):
        r_hi = np.minimum(np.exp(ee + 0.5 * Eq - lo[:, None]), 1.0)
    r_lo = np.exp(ee - 0.5 * Eq - hi[:, None])
    dr = np.maximum(r_hi - r, r - r_lo) + 2.0 ** -20 * r + floor * r
    B_g = np.zeros((n, d))
    for k in range(K):
        R = (r[:, k] + dr[:, k])[:, None]
        az = np.abs(Z[k])
        W = R * E[k] + dr[:, k][:, None] * az + (3 * up + 2 * U32 + g2) * (1 + up) ** 3 * R * (az + E[k])
        B_g += W @ np.abs(inst.L[k]).T
    return B_l, B_g, ell, r


def sigmas(inst, X, prec):
    """(s_l [n], s_g [n, d]): standard deviations of the tensor-core errors of l and grad l
    under the first-order model of independent roundings (Higham and Mary's
    probabilistic error analysis): every rounding to p multiplies its value by
    (1 + delta), delta of mean 0 and variance v_p = u_p^2 / 3; FP32 roundings have
    v32 = u32^2 / 3. With a = x - mu_k, z = L^T a (row form a L), P = L L^T:
      dz_j   = sum_i a_i L_ij (da_i + dL_ij)
      dq     = 2 sum_j z_j dz_j,   Var = 4 v_p [sum_i a_i^2 (P a)_i^2 + sum_ij a_i^2 L_ij^2 z_j^2]
                                         + 4 d v32 sum_j z_j^2 s_j + 256 v32 q^2,  s_j = sum_i a_i^2 L_ij^2
      dl     = -1/2 sum_k r_k dq_k
      dgrad_i = -sum_k [r_k (sum_m a_m da_m P_im + sum_j L_ij (sum_m a_m L_mj dL_mj
                + z_j dL_ij + z_j dw_j)) + dr_k (P a)_i]
    where the same rounding dL of L_k feeds both contractions (its two terms are
    bounded by twice their squares), dw the two roundings of the stored z and of r z
    to p (variance 2 v_p), and
    dr_k = r_k (de_k - sum_m r_m de_m), de = -dq / 2. The FP32 exponentials of the
    LSE add a floor of 4 u32 to l. The FP32 roundings of x, mu_k and their difference
    (before the rounding to p) add v32 (x_i^2 + mu_k,i^2 + a_i^2) per coordinate to the
    variance of da_i."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    K = inst.K
    vp = U_P[prec] ** 2 / 3.0
    v32 = U32 ** 2 / 3.0
    a_k = inst.log_w - 0.5 * d * np.log(2 * np.pi) + np.log(np.diagonal(inst.L, axis1=1, axis2=2)).sum(1)
    q = np.empty((n, K))
    vq = np.empty((n, K))
    parts = []
    for k in range(K):
        Lk = inst.L[k]
        L2 = Lk * Lk
        Pk = Lk @ Lk.T
        A = X - inst.mu[k]
        A2 = A * A
        F2 = X * X + inst.mu[k] ** 2 + A2  # the FP32 roundings before the rounding to p
        Z = A @ Lk
        Z2 = Z * Z
        PA = A @ Pk  # (P a)_i as a row (P symmetric)
        S = A2 @ L2  # s_j = sum_i a_i^2 L_ij^2
        qk = Z2.sum(1)
        vq[:, k] = 4 * vp * ((A2 * PA * PA).sum(1) + (S * Z2).sum(1)) + 4 * d * v32 * (Z2 * S).sum(1) \
            + 256 * v32 * qk * qk + 4 * v32 * (F2 * PA * PA).sum(1)
        q[:, k] = qk
        parts.append((A2, Z2, PA, S, L2, Pk * Pk, F2))
    ee = a_k[None, :] - 0.5 * q
    ell = _lse(ee)
    r = np.exp(ee - ell[:, None])
    ve = vq / 4.0  # de = -dq / 2
    s_l = np.sqrt((r * r * ve).sum(1) + (4 * U32) ** 2)
    # dr_k = r_k ((1 - r_k) de_k - sum_{m != k} r_m de_m)
    tot = (r * r * ve).sum(1, keepdims=True)
    vr = r * r * ((1 - r) ** 2 * ve + (tot - r * r * ve))
    var_g = np.zeros((n, d))
    for k in range(K):
        A2, Z2, PA, S, L2, P2, F2 = parts[k]
        rk2 = (r[:, k] * r[:, k])[:, None]
        var_g += rk2 * vp * (A2 @ P2)                      # da through P a
        var_g += rk2 * v32 * (F2 @ P2)                     # FP32 x, mu_k and x - mu_k
        var_g += rk2 * 2 * vp * (S @ L2.T + Z2 @ L2.T)    # dL in both contractions
        var_g += rk2 * 2 * vp * (Z2 @ L2.T)                # dw: z, then r z, rounded to p
        var_g += rk2 * (K * d) * v32 * (Z2 @ L2.T)        # FP32 accumulation of the gradient
        var_g += rk2 * d * v32 * (S @ L2.T)                # FP32 accumulation of z
        var_g += vr[:, k][:, None] * PA * PA               # responsibilities
    return s_l, np.sqrt(var_g)
