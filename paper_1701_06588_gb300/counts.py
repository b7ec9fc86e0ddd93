"""Work-count model.

1. Contracted-element counts of Table II (Sec. IV A): for a family basis
   whose shells share one set of K exponents,
     SHG contracts the scalars (0_a|O|0_b)^{(k)}, k = 0..la_max+lb_max (plus
     one more order for gradients), for each of the K_a K_b primitive pairs;
     OS contracts every primitive spherical element: (sum over the distinct
     l present of (2l+1) K)^2 per side pair, four times with gradients.

2. Algorithmic FP64 operation counts of the two-center path as implemented
   (add/mul = 1 flop, fma = 2 flops, counted from the formulas the kernels
   evaluate; exp, rsqrt and the like counted separately as special ops).
   Used for the roofline fraction: algorithmic FLOP/s over the measured FP64
   FMA throughput.
"""
import numpy as np

OP_OVERLAP, OP_COULOMB, OP_ERFC, OP_ERF, OP_GAUSS, OP_GCOUL, OP_RA2N = 0, 1, 2, 3, 4, 5, 6


def shg_contracted_elements(l_a, l_b, k_a, k_b, gradients=False):
    """Scalars contracted by the SHG scheme for one pair of exponent sets
    (Table II convention: all orders 0..la_max+lb_max are contracted)."""
    return (max(l_a) + max(l_b) + 1 + (1 if gradients else 0)) * k_a * k_b


def os_contracted_elements(l_a, l_b, k_a, k_b, gradients=False):
    """Primitive spherical elements contracted by the Obara-Saika route."""
    na = sum(2 * l + 1 for l in sorted(set(l_a))) * k_a
    nb = sum(2 * l + 1 for l in sorted(set(l_b))) * k_b
    return na * nb * (4 if gradients else 1)


# --------------------------------------------------------------------------- #
# FP64 flop model of one shell pair                                           #
# --------------------------------------------------------------------------- #
_BOYS = 2 * 8 + 2 * 8 + 1          # Taylor of F_kmax (8 fma), exp Taylor (8 fma), scale by exp(-T_i)
_BOYS_F = 2 * 8                     # Taylor of F_kmax alone: J = 1 needs no exp(-T) (no recursion)
KBOYS_TMAX = 120.0                  # T = rho R^2 at and above which the fused 1/r sum takes the far field


def _boys(J):
    return _BOYS if J > 1 else _BOYS_F


def _radial_flops(op, J, kmin):
    """Per primitive pair: setup + operator part + contraction of J orders."""
    setup = 1 + 1 + 2 + 1 + 1       # c, 1/c from rsqrt^2, rho, T, w_a w_b
    powk = 2 * max(int(np.ceil(np.log2(kmin + 1))), 0)
    if op == OP_OVERLAP:
        return setup + 4 + powk + J * (1 + 1)
    if op == OP_GAUSS:
        return setup + 10 + powk + J * (1 + 1)
    if op == OP_RA2N:
        # algorithmic count of the FP64 formula (the kernel runs it in double-double):
        # coefficients of Q (n <= 5: 21 fma), kmax steps of the coefficient recursion
        # (6 x 3), J Horner evaluations (6 fma) and accumulations
        kmax = kmin + J - 1
        return setup + 10 + 2 * 21 + kmax * 18 + J * (12 + 2)
    if op == OP_GCOUL:
        # d, 1/d, p, q, prefactor, exp argument; Boys head and the full downward
        # recursion to F_0; kmax applications of v_i <- p v_i + q v_{i+1} over a
        # shrinking vector; J accumulations
        kmax = kmin + J - 1
        return setup + 12 + _BOYS + 3 * kmax + 3 * kmax * (kmax + 1) // 2 + J * (1 + 1)
    coul = 4 + _boys(J) + 3 * (J - 1) + powk + J * (2 + 1)
    att = 6 + _boys(J) + 3 * (J - 1) + powk + J * (2 + 1)
    if op == OP_COULOMB:
        return setup + coul
    if op == OP_ERF:
        return setup + 4 + att
    return setup + coul + att      # erfc


def _radial_special(op):
    """Special-function calls per primitive pair (rsqrt, exp)."""
    return {OP_OVERLAP: 2, OP_GAUSS: 3, OP_COULOMB: 1, OP_ERF: 2, OP_ERFC: 2, OP_GCOUL: 3, OP_RA2N: 3}[op]


def pair_flops(la, lb, ka, kb, op):
    """Algorithmic FP64 flops of one contracted shell pair (numpy-vectorised)."""
    la = np.asarray(la, dtype=np.int64)
    lb = np.asarray(lb, dtype=np.int64)
    kk = np.asarray(ka, dtype=np.int64) * np.asarray(kb, dtype=np.int64)
    J = np.minimum(la, lb) + 1
    kmin = np.maximum(la, lb)
    lmax = np.maximum(la, lb)
    na, nb = 2 * la + 1, 2 * lb + 1
    rad = np.zeros_like(kk, dtype=np.float64)
    for j in range(1, 8):
        for km in range(0, 7):
            m = (J == j) & (kmin == km)
            if m.any():
                rad[m] = _radial_flops(op, j, km)
    radial = kk * rad
    harmonics = 8.0 * (lmax + 1) * (lmax + 2) / 2            # R^c, R^s recursions
    w_rows = (na + nb) * J * J                              # one add per W entry
    scale = na * J * J + 2 * J * J                          # g_e and U_a scaling
    assembly = na * nb * (2 * J * J + 2)                    # J^2 fma + 2 mul per element
    return radial + harmonics + w_rows + scale + assembly


def _fused_radial_flops(ops, J, kmin, far=False):
    """Per primitive pair of the fused pass (shg_plan_2c_exec_fused), with the
    per-term counts of _radial_flops: shared setup and (-rho)^kmin, one Boys
    sum for 1/r and erfc, one attenuated sum per distinct omega of erf/erfc.
    far: the pair has T >= KBOYS_TMAX, where the 1/r sum is one multiply-add
    of the per-primitive far-field weights (the Boys head, (-rho)^kmin and
    the J orders are applied once per shell pair, fused_pair_flops)."""
    ops = dict(ops)                     # op id -> omega
    setup = 1 + 1 + 2 + 1 + 1
    powk = 2 * max(int(np.ceil(np.log2(kmin + 1))), 0)
    boys_sums = (OP_COULOMB in ops or OP_ERFC in ops)
    f = setup
    if OP_OVERLAP in ops or (boys_sums and not far):
        f += powk
    if OP_OVERLAP in ops:
        f += 4 + J * 2
    if OP_GAUSS in ops:
        f += 10 + powk + J * 2
    atts = {ops[o] for o in (OP_ERF, OP_ERFC) if o in ops}
    if boys_sums or atts:
        f += 2                          # 2 pi^{5/2} cw_a cw_b / sqrt(c)
    if boys_sums:
        f += 2 if far else _boys(max(J, 2 if OP_OVERLAP in ops else 1)) + 3 * (J - 1) + J * (2 + 1)
    f += len(atts) * (6 + _boys(J) + 3 * (J - 1) + powk + J * (2 + 1))
    return f


def far_primitive_pairs(shells, pair_a, pair_b, tmax=KBOYS_TMAX, chunk=1 << 16):
    """Per pair, the number of primitive pairs with rho R^2 >= tmax (FP64);
    pairs grouped by (Ka, Kb), one broadcast per group and chunk."""
    K = np.asarray(shells["nprim"]).astype(np.int64)
    off = np.zeros(len(K) + 1, dtype=np.int64)
    off[1:] = np.cumsum(K)
    ex = np.asarray(shells["exps"], dtype=np.float64)
    c = np.asarray(shells["centers"], dtype=np.float64).reshape(-1, 3)
    co = np.asarray(shells["center_of"])
    pa = np.asarray(pair_a)
    pb = np.asarray(pair_b)
    out = np.zeros(len(pa), dtype=np.int64)
    if not len(pa):
        return out
    R2 = ((c[co[pa]] - c[co[pb]]) ** 2).sum(axis=1)
    ka, kb = K[pa], K[pb]
    key = ka * 4096 + kb
    order = np.argsort(key, kind="stable")
    bounds = np.flatnonzero(np.diff(key[order])) + 1
    for grp in np.split(order, bounds):
        Ka, Kb = int(ka[grp[0]]), int(kb[grp[0]])
        for lo in range(0, len(grp), chunk):
            g = grp[lo:lo + chunk]
            A = ex[off[pa[g]][:, None] + np.arange(Ka)]
            B = ex[off[pb[g]][:, None] + np.arange(Kb)]
            rho = A[:, :, None] * B[:, None, :] / (A[:, :, None] + B[:, None, :])
            out[g] = np.count_nonzero(rho * R2[g, None, None] >= tmax, axis=(1, 2))
    return out


def fused_pair_flops(la, lb, ka, kb, ops, n_far=None):
    """Algorithmic FP64 flops of one contracted shell pair in the fused pass
    over `ops` ((op id, omega) pairs; numpy-vectorised over la, lb, ka, kb):
    radial sums as _fused_radial_flops, then per pair the harmonics, both W
    sides, the (2j-1)!! B weights on W_a, Q_j (J^2 fma per element) and per
    operator its J orders (fma) and the A_a A_b factor."""
    ops = list(ops)
    la = np.asarray(la, dtype=np.int64)
    lb = np.asarray(lb, dtype=np.int64)
    kk = np.asarray(ka, dtype=np.int64) * np.asarray(kb, dtype=np.int64)
    J = np.minimum(la, lb) + 1
    kmin = np.maximum(la, lb)
    lmax = np.maximum(la, lb)
    na, nb = 2 * la + 1, 2 * lb + 1
    nop = len(ops)
    shape = np.broadcast(la, lb, kk).shape
    rad = np.zeros(shape, dtype=np.float64)
    kkb = np.broadcast_to(kk, shape).astype(np.float64)
    nfar = np.zeros(shape) if n_far is None else np.broadcast_to(np.asarray(n_far, dtype=np.float64), shape)
    J = np.broadcast_to(J, shape)
    kmin = np.broadcast_to(kmin, shape)
    finish = np.zeros(shape)
    coul = any(o in (OP_COULOMB, OP_ERFC) for o, _ in ops)
    for j in range(1, 8):
        for km in range(0, 7):
            m = (J == j) & (kmin == km)
            if np.any(m):
                near_f = _fused_radial_flops(ops, j, km)
                far_f = _fused_radial_flops(ops, j, km, far=True)
                rad[m] = (kkb[m] - nfar[m]) * near_f + nfar[m] * far_f
                if coul:
                    # far-field order factors, once per pair that has far primitive pairs
                    finish[m] = (nfar[m] > 0) * (8 + 2 * max(int(np.ceil(np.log2(km + 1))), 0) + 4 * j)
    post = J * (nop + (1 if any(o == OP_ERFC for o, _ in ops) else 0))   # 2^{kmax-j} scaling, erfc = 1/r - erf
    harmonics = 8.0 * (lmax + 1) * (lmax + 2) / 2
    w_rows = (na + nb) * J * J
    scale = na * J * J                                                    # (2j-1)!! B weights on W_a
    assembly = na * nb * (2 * J * J + 1 + nop * (2 * J + 1))
    return rad + finish + post + harmonics + w_rows + scale + assembly


def workload_fused_flops(shells, pair_a, pair_b, ops, n_far=None):
    """Fused-pass flops of a pair list; n_far (far_primitive_pairs) per pair,
    else every primitive pair is counted as near."""
    l = np.asarray(shells["l"])
    k = np.asarray(shells["nprim"])
    return float(np.sum(fused_pair_flops(l[pair_a], l[pair_b], k[pair_a], k[pair_b], ops, n_far)))


def workload_flops(shells, pair_a, pair_b, op):
    l = np.asarray(shells["l"])
    k = np.asarray(shells["nprim"])
    return float(np.sum(pair_flops(l[pair_a], l[pair_b], k[pair_a], k[pair_b], op)))


def workload_elements(shells, pair_a, pair_b):
    l = np.asarray(shells["l"]).astype(np.int64)
    return int(np.sum((2 * l[pair_a] + 1) * (2 * l[pair_b] + 1)))


def triple_flops(la, lt, lb, ka, kt, kb):
    """Algorithmic FP64 flops of one contracted (a b a~) triple in the order the
    (aab) formula is evaluated (Eqs. Pa_aba, sra2ms, devsra2ms, I_jab; Sec. II D),
    numpy-vectorised.  Per (a, a~) primitive pair: alpha' = alpha + alpha~, its
    inverse square root and the powers alpha'^{-j}; per primitive triple: the
    setup, D_m^{(i)} by Horner times (beta^2/c)^i, (-rho)^n, the sums
    V[m][k] (one multiply-add per term, binom(k,i)(-rho)^{k-i} formed once per
    (k, i)) and P^{(k)} (binom(p,j)(L)_j alpha'^{-j} formed once per (L, j)).
    The Gaunt sum counts 2 nL terms per (m_a, m_a~), an upper estimate of the
    real Gaunt coefficients that are non-zero."""
    la, lt, lb = (np.asarray(v, dtype=np.int64) for v in (la, lt, lb))
    kat = np.asarray(ka, dtype=np.int64) * np.asarray(kt, dtype=np.int64)
    kk = kat * np.asarray(kb, dtype=np.int64)
    out = np.zeros(np.broadcast(la, lt, lb, kk).shape, dtype=np.float64)
    it = np.nditer([la, lt, lb, kk, np.broadcast_to(kat, kk.shape)], flags=["multi_index", "refs_ok"])
    for a, t, b, k, kp in it:
        a, t, b, k, kp = int(a), int(t), int(b), int(k), int(kp)
        Lmin, Lmax = abs(a - t), a + t
        nL = (Lmax - Lmin) // 2 + 1
        p = nL - 1
        kmaxA = Lmax + b
        kminA = max(Lmin, b)
        pair = 12 + p
        prim = 16 + 2 * p + p * (p + 1) * (p + 2) // 3 + (p + 1) * (p + 2) // 2 + kmaxA
        for kd in range(kminA, kmaxA + 1):
            prim += min(p, kd) + 1
            for m in range(p + 1):
                prim += 2 * (min(m, kd) + 1) + 1
        for iL in range(nL):
            L = Lmin + 2 * iL
            J = min(L, b) + 1
            prim += (p - iL + 1) + J * (2 * (p - iL + 1) + 2) + 1
        lmax = max(Lmax, b)
        nb = 2 * b + 1
        Jmax = min(Lmax, b) + 1
        ang = 8 * (lmax + 1) * (lmax + 2) // 2 + nb * Jmax * Jmax
        for iL in range(nL):
            L = Lmin + 2 * iL
            J = min(L, b) + 1
            ang += J * J + (2 * L + 1) * (2 * J * J + nb * (2 * J * J + 2))
        ang += (2 * a + 1) * (2 * t + 1) * 2 * nL * nb * 2
        out[it.multi_index] = k * prim + kp * pair + ang
    return out


def workload_triple_flops(shells, t_a, t_t, t_b):
    l = np.asarray(shells["l"])
    k = np.asarray(shells["nprim"])
    key = np.stack([l[t_a], l[t_t], l[t_b], k[t_a], k[t_t], k[t_b]], axis=1)
    uniq, cnt = np.unique(key, axis=0, return_counts=True)
    f = triple_flops(uniq[:, 0], uniq[:, 1], uniq[:, 2], uniq[:, 3], uniq[:, 4], uniq[:, 5])
    return float(np.sum(f * cnt))


def grad_pair_flops(la, lb, ka, kb, op):
    """Algorithmic FP64 flops of one pair's vector-Jacobian product (Eq. dev_ab,
    Eqs. cartesian_dev_x/y/z): the radial part with one more derivative order,
    harmonics and their gradients, W and dW rows, the two contractions with the
    upstream weights and the three gradient sums."""
    la = np.asarray(la, dtype=np.int64)
    lb = np.asarray(lb, dtype=np.int64)
    kk = np.asarray(ka, dtype=np.int64) * np.asarray(kb, dtype=np.int64)
    J = np.minimum(la, lb) + 1
    kmin = np.maximum(la, lb)
    lmax = np.maximum(la, lb)
    na, nb = 2 * la + 1, 2 * lb + 1
    rad = np.zeros(np.broadcast(la, lb, kk).shape, dtype=np.float64)
    for j in range(1, 8):
        for km in range(0, 7):
            m = (J == j) & (kmin == km)
            if np.any(m):
                rad[m] = _radial_flops(op, j + 1, km)
    nco = (lmax + 1) * (lmax + 2) / 2
    JJ = J * J
    ang = (3 * J * (J + 1) / 2 + 16 * nco + nb * JJ + na * 16 * JJ + na * nb * (4 * JJ + 3) + nb * 12 * JJ + 9)
    return kk * rad + ang


def workload_grad_flops(shells, pair_a, pair_b, op):
    l = np.asarray(shells["l"])
    k = np.asarray(shells["nprim"])
    return float(np.sum(grad_pair_flops(l[pair_a], l[pair_b], k[pair_a], k[pair_b], op)))
