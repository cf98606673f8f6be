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


def _quad_parts(inst, X, O=None):
    """Per sample x = o + tau u on a ray from its origin o (O [n, d], the box centre when
    None): tau = |x - o|, u = (x - o) / tau, the origins, and the components' a_k."""
    X = np.asarray(X, dtype=np.float64)
    O = np.broadcast_to(0.5 * (inst.lo + inst.hi), X.shape) if O is None else np.asarray(O, dtype=np.float64)
    D = X - O
    tau = np.sqrt((D * D).sum(1))
    U = D / np.where(tau > 0, tau, 1.0)[:, None]
    a_k = inst.log_w - 0.5 * inst.d * np.log(2 * np.pi) + np.log(np.diagonal(inst.L, axis1=1, axis2=2)).sum(1)
    return O, tau, U, a_k


def _quad_form(prec, d):
    """(worst-case and variance coefficients of one product u_i L_ij, accumulation steps
    of w_j, column tile of the |w|^2 and alpha . w partials) of a quadratic ray form:
    prec 2 / 1 the tensor-core split products at bf16 / tf32 (three split residuals of
    at most u_p^2 each, one of them the omitted u_lo L_lo; 3 d accumulation steps; tiles
    of 256 columns), prec 0 the FP32 SIMT form (u and L_k rounded to FP32; d
    accumulation steps; tiles of 128 columns)."""
    if prec == 0:
        return 2 * U32 + U32 * U32, 2 * U32 ** 2 / 3.0, d, 128
    up = U_P[prec]
    return 3 * up * up, up ** 4, 3 * d, 256


def _quad_terms(inst, X, prec, O):
    """Per component: alpha = z_k(o) (exact), the origins' product o L_k and -mu_k L_k
    (origin pass), w = L_k^T u, z(tau) = alpha + tau w, for every sample."""
    Og, tau, U, a_k = _quad_parts(inst, X, O)
    for k in range(inst.K):
        Lk = inst.L[k]
        oL = Og @ Lk
        mL = inst.mu[k] @ Lk
        al = oL - mL[None, :] if O is not None else np.broadcast_to((Og[0] - inst.mu[k]) @ Lk, oL.shape)
        W = U @ Lk
        yield k, Lk, Og, tau, U, a_k, oL, mL, al, W, al + tau[:, None] * W


def quad_bounds(inst, X, prec, O=None):
    """Worst case of a quadratic ray pass at ray samples X [n, d] (prec as _quad_form):
    w_j = sum_i u_i L_ij with the operand error of _quad_form and FP32 accumulation over
    n_acc terms; q1 = alpha . w and q2 = |w|^2 summed in FP32 over column tiles of
    n_tile, the tiles in FP64; |z|^2 = q0 + 2 tau q1 + tau^2 q2 in FP64. With
    E_j = (e_op + n_acc 2^-23)(1 + u_p)^2 sum_i |u_i| |L_ij|:
        d|z|^2 <= 2 tau sum_j |z_j| E_j + tau^2 sum_j E_j^2
                  + n_tile 2^-23 (tau^2 q2 + 2 tau sum_j |alpha_j w_j|) + 2^-24 2 tau sum_j |alpha_j w_j|
                  + 8 2^-53 (q0 + 2 tau |q1| + tau^2 q2).
    Rays from the box centre (O None) take alpha = z_k(c) in FP64 (q0 exact, alpha
    rounded to FP32 for q1). Rays from origins O (the origin pass): alpha = o L_k - mu_k L_k
    from the same split products plus the FP32 -mu_k L_k, kept in FP32, so alpha_j is off
    by Eo_j = (e_op + n_acc 2^-23)(1 + u_p)^2 sum_i |o_i| |L_ij| + 2^-23 (|(o L)_j| +
    |(mu L)_j| + |alpha_j|), which adds 2 sum_j |z_j| Eo_j + sum_j (Eo_j + tau E_j)^2 - ... (taken
    whole: (Eo_j + tau E_j) in place of tau E_j) and n_tile 2^-23 q0 for q0's tiles.
    l lies between LSE(e - d|z|^2 / 2) and LSE(e + d|z|^2 / 2), plus the FP32 LSE floor.
    Returns (B_l [n], l [n])."""
    d, K = inst.d, inst.K
    e_op, _, n_acc, n_tile = _quad_form(prec, d)
    up = U_P.get(prec, U32)
    cb = (e_op + n_acc * 2.0 ** -23) * (1 + up) ** 2
    n = np.asarray(X).shape[0]
    q = np.empty((n, K))
    dq = np.empty((n, K))
    for k, Lk, Og, tau, U, a_k, oL, mL, al, W, Z in _quad_terms(inst, X, prec, O):
        E = tau[:, None] * cb * (np.abs(U) @ np.abs(Lk))
        if O is not None:
            E = E + cb * (np.abs(Og) @ np.abs(Lk)) + 2.0 ** -23 * (np.abs(oL) + np.abs(mL)[None, :] + np.abs(al))
        aw = np.abs(al * W).sum(1)
        q2 = (W * W).sum(1)
        q1 = (al * W).sum(1)
        q0 = (al * al).sum(1)
        q[:, k] = (Z * Z).sum(1)
        dq[:, k] = (2 * (np.abs(Z) * E).sum(1) + (E * E).sum(1)
                    + n_tile * 2.0 ** -23 * (tau ** 2 * q2 + 2 * tau * aw) + 2.0 ** -24 * 2 * tau * aw
                    + 8 * 2.0 ** -53 * (q0 + 2 * tau * np.abs(q1) + tau ** 2 * q2))
        if O is not None:
            dq[:, k] += n_tile * 2.0 ** -23 * q0
    ee = a_k[None, :] - 0.5 * q
    ell = _lse(ee)
    hi = _lse(ee + 0.5 * dq)
    lo = _lse(ee - 0.5 * dq)
    return np.maximum(hi - ell, ell - lo) + 2.0 ** -20 * (1 + K), ell


def quad_sigmas(inst, X, prec, O=None):
    """Standard deviation of a quadratic ray pass's error at ray samples X (prec as
    _quad_form) under the first-order model of independent roundings: each product
    u_i L_ij carries the operand variance of _quad_form, an FP32 accumulation step
    v32 = u32^2 / 3 of the partial sum (n_acc steps for w_j, n_tile for the tile partials
    of q0, q1 and q2). To first order d|z|^2 = 2 z . (d alpha + tau dw) plus the tile
    partials' rounding:
        Var d|z_k|^2 = 4 sum_j z_j^2 (Var d alpha_j + tau^2 Var dw_j)
                       + n_tile v32 (tau^4 q2^2 + 4 tau^2 (sum_j |alpha_j w_j|)^2 [+ q0^2]) / n_tiles,
    Var dw_j = (v_op + n_acc v32) sum_i u_i^2 L_ij^2; from the box centre d alpha is the
    FP32 rounding of alpha in q1 alone (4 tau^2 v32 sum_j (alpha_j w_j)^2), from origins
    (the origin pass, q0 from FP32 tiles too) Var d alpha_j = (v_op + n_acc v32)
    sum_i o_i^2 L_ij^2 + v32 ((o L)_j^2 + (mu L)_j^2 + alpha_j^2). dl = -1/2 sum_k r_k d|z_k|^2
    (independent components) with the FP32 LSE floor 4 u32."""
    v32 = U32 ** 2 / 3.0
    d, K = inst.d, inst.K
    _, v_op, n_acc, n_tile = _quad_form(prec, d)
    n_tiles = max(1, -(-d // n_tile))
    n = np.asarray(X).shape[0]
    q = np.empty((n, K))
    vq = np.empty((n, K))
    for k, Lk, Og, tau, U, a_k, oL, mL, al, W, Z in _quad_terms(inst, X, prec, O):
        L2 = Lk * Lk
        Vw = (v_op + n_acc * v32) * ((U * U) @ L2)
        aw = np.abs(al * W).sum(1)
        q2 = (W * W).sum(1)
        q0 = (al * al).sum(1)
        q[:, k] = (Z * Z).sum(1)
        tiles = tau ** 4 * q2 ** 2 + 4 * tau ** 2 * aw ** 2
        if O is None:
            Va = 0.0
            extra = 4 * tau ** 2 * v32 * ((al * W) ** 2).sum(1)
        else:
            Va = (v_op + n_acc * v32) * ((Og * Og) @ L2) + v32 * (oL ** 2 + mL[None, :] ** 2 + al ** 2)
            extra = 0.0
            tiles = tiles + q0 ** 2
        vq[:, k] = (4 * (Z * Z * (Va + tau[:, None] ** 2 * Vw)).sum(1)
                    + n_tile * v32 * tiles / n_tiles + extra)
    ee = a_k[None, :] - 0.5 * q
    r = np.exp(ee - _lse(ee)[:, None])
    return np.sqrt(0.25 * (r * r * vq).sum(1) + (4 * U32) ** 2)


def quad_bias(inst, X, prec, O=None):
    """Signed first-order effect on l of tensor-core accumulation steps that each shrink
    an accumulator by 2^-24 of its magnitude (rounding toward zero). The split products
    run the small ones first, so only the last segment's n_j = ceil((d - j) / k) + 1 steps
    add to an accumulator of full magnitude (k the products one instruction sums: 16 for
    bf16, 8 for tf32): w_j becomes (1 - n_j 2^-24) w_j and, for the origin pass, (o L)_j
    becomes (1 - n_j 2^-24) (o L)_j, so that
        d|z_k|^2 = -2 sum_j n_j 2^-24 z_kj (tau w_kj [+ (o L_k)_j]),   dl = -1/2 sum_k r_k d|z_k|^2.
    Zero for the FP32 SIMT form (prec 0: round-to-nearest FMA chains)."""
    n = np.asarray(X).shape[0]
    if prec == 0:
        return np.zeros(n)
    d, K = inst.d, inst.K
    kin = 16 if prec == 2 else 8
    nj = np.ceil((d - np.arange(d)) / kin) + 1
    q = np.empty((n, K))
    dq = np.empty((n, K))
    for k, Lk, Og, tau, U, a_k, oL, mL, al, W, Z in _quad_terms(inst, X, prec, O):
        q[:, k] = (Z * Z).sum(1)
        acc = tau[:, None] * W + (oL if O is not None else 0.0)
        dq[:, k] = -2 * 2.0 ** -24 * (Z * acc * nj[None, :]).sum(1)
    ee = a_k[None, :] - 0.5 * q
    r = np.exp(ee - _lse(ee)[:, None])
    return -0.5 * (r * dq).sum(1)


# A quadratic ray pass's error at a sample is the accumulation bias, between 0 and
# quad_bias, plus independent roundings within C_Q of quad_sigmas, and never beyond
# quad_bounds. On a GB300 the largest distance outside [0, bias] over the parity cases
# was 1.05 standard deviations (BF16, d = 64) and the fitted bias fraction 0.35 - 0.42.
# A dropped K chunk moves w_j by a partial sum of its column, a swapped or repeated split
# segment by u_p |w_j| (2^8 or 2^11 times the split residual the model allows): either
# is thousands of standard deviations.
C_Q = 4.0


def check_ray_samples(inst, X, dl, prec, O=None):
    """Asserts the errors dl = l_gpu - l_oracle at ray samples X (rays from the box
    centre, or from the per-sample origins O) fit the model above."""
    s = quad_sigmas(inst, X, prec, O)
    B, _ = quad_bounds(inst, X, prec, O)
    bias = quad_bias(inst, X, prec, O)
    out = np.maximum(np.minimum(0.0, bias) - dl, dl - np.maximum(0.0, bias)) / s
    assert out.max() <= C_Q, (int(np.argmax(out)), float(out.max()))
    assert (np.abs(dl) <= B).all(), float((np.abs(dl) / B).max())
