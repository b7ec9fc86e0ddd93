"""Shared helpers for GPU-vs-oracle parity tests.

Element-wise bar, atomic units, normalised functions:

    |x_e - ref_e| <= rtol |ref_e| + atol + gamma C_e,      C_e = S_e + G_e

  FP64 integrals    rtol 1e-12, atol 1e-14, gamma 1e-15
  gradients         rtol 1e-10, atol 1e-12, gamma 1e-15
  mixed precision   rtol 1e-10, atol 1e-14, gamma 2e-13
  mixed gradients   rtol 1e-10, atol 1e-12, gamma 2e-13

Both conditioning terms belong to element e itself (no block maximum):

  S_e  the same element evaluated with |N c| in place of the normalised
       coefficients N c (for erfc the Coulomb and erf parts added).  For a
       fixed derivative order every primitive term of O^{(k)} (Eq.
       O_rab2_deriv) has one sign, so S_e is the sum of the magnitudes of
       the contraction: the scale of its forward error bound.  Random-sign
       coefficients cancel (sum |t| / |sum t| reaches ~1e5 on the synthetic
       sets), and there no FP64 evaluation reaches 1e-12 relative.

  G_e  sum_i |d ref_e / d v_i| |v_i|, v = R_a - R_b, from the oracle's
       analytic Jacobian: the first-order change of the element under a
       relative perturbation of each component of the separation.  Every
       implementation that starts from the two centers rounds v (the GPU's
       v_i = fl(A_i - B_i) is off by up to u |v_i|), and the angular part
       (harmonics and W of Sec. II E, the sum over j of Eq.
       final_r12int_ab) cancels exactly where the element is small against
       this sensitivity, near a node of the element as a function of v.
       At R = 0 it vanishes.

gamma C_e is a few units of rounding of these scales; where the element is
well conditioned (C_e within a small factor of |ref_e|) the rtol term is the
bar.  tests/test_gpu_plain_bar.py applies the bars with gamma = 0 to
same-sign coefficients on the elements with G_e <= 1e3 |ref_e|.
"""
import numpy as np

TOL_FP64 = (1e-12, 1e-14, 1e-15)
TOL_GRAD = (1e-10, 1e-12, 1e-15)
TOL_MIXED = (1e-10, 1e-14, 2e-13)
TOL_GRAD_MIXED = (1e-10, 1e-12, 2e-13)

# the bars with no conditioning term (the plain element-wise tolerances)
PLAIN_FP64 = (1e-12, 1e-14, 0.0)
PLAIN_GRAD = (1e-10, 1e-12, 0.0)
PLAIN_MIXED = (1e-10, 1e-14, 0.0)


def _bar(ref, tol, scale):
    rtol, atol = tol[0], tol[1]
    gamma = tol[2] if len(tol) > 2 else 0.0
    bar = rtol * np.abs(ref) + atol
    if scale is not None and gamma:
        bar = bar + gamma * np.asarray(scale, dtype=np.float64)
    return bar


def excess(got, ref, tol, scale=None):
    """max over elements of |got - ref| / bar; <= 1 passes."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape:
        raise AssertionError("shape %s != %s" % (got.shape, ref.shape))
    if got.size == 0:
        return 0.0
    if not np.all(np.isfinite(got)):
        return np.inf
    return float(np.max(np.abs(got - ref) / _bar(ref, tol, scale)))


def assert_parity(got, ref, tol, what="", scale=None):
    e = excess(got, ref, tol, scale)
    if not e <= 1.0:
        got = np.asarray(got)
        ref = np.asarray(ref)
        r = np.abs(got - ref) / _bar(ref, tol, scale)
        i = int(np.nanargmax(np.where(np.isfinite(r), r, np.inf)))
        raise AssertionError("%s: parity excess %.3g at element %d: got %.17g ref %.17g scale %s" % (
            what, e, i, got.flat[i], ref.flat[i], None if scale is None else np.asarray(scale).flat[i]))
    return e


def normalised(shells):
    """Shell set with coefficients N c (oracle normalisation) and its |N c| twin."""
    import oracle
    N = oracle.shell_norms(shells)
    prim_shell = np.repeat(np.arange(len(shells["l"])), shells["nprim"])
    cn = np.asarray(shells["coefs"], dtype=np.float64) * N[prim_shell]
    return dict(shells, coefs=cn), dict(shells, coefs=np.abs(cn))


def separations(shells, first, second):
    """v = R_first - R_second per entry (n, 3)."""
    c = np.asarray(shells["centers"], dtype=np.float64).reshape(-1, 3)
    co = np.asarray(shells["center_of"])
    return c[co[np.asarray(first)]] - c[co[np.asarray(second)]]


def geometric_scale(jac, off, sz, v):
    """G_e = sum_i |d e / d v_i| |v_i| from an oracle Jacobian laid out per
    entry p as [xyz][elements of p] at 3*off[p]."""
    n_el = int(np.sum(sz))
    g = np.zeros(n_el)
    if n_el == 0:
        return g
    # element index -> (entry, position); Jacobian rows at 3*off[p] + i*sz[p] + pos
    ent = np.repeat(np.arange(len(sz)), sz)
    pos = np.arange(n_el) - np.repeat(off, sz)
    av = np.abs(np.asarray(v, dtype=np.float64))
    for i in range(3):
        g += np.abs(jac[3 * off[ent] + i * sz[ent] + pos]) * av[ent, i]
    return g


def reference_2c_parts(shells, pair_a, pair_b, op, omega):
    """Oracle blocks (a|O|b), offsets, sizes and the two conditioning scales
    S (contraction) and G (separation), element by element."""
    import oracle
    shn, sha = normalised(shells)
    ref, off, sz = oracle.eval_2c(shn, pair_a, pair_b, op, omega, normalize=False)
    if op == oracle.OP_ERFC:
        s1, _, _ = oracle.eval_2c(sha, pair_a, pair_b, oracle.OP_COULOMB, 0.0, normalize=False)
        s2, _, _ = oracle.eval_2c(sha, pair_a, pair_b, oracle.OP_ERF, omega, normalize=False)
        S = np.abs(s1) + np.abs(s2)
    else:
        S, _, _ = oracle.eval_2c(sha, pair_a, pair_b, op, omega, normalize=False)
        S = np.abs(S)
    jac, _, _ = oracle.eval_2c_grad(shn, pair_a, pair_b, op, omega, center="A", normalize=False)
    G = geometric_scale(jac, off, sz, separations(shells, pair_a, pair_b))
    return dict(ref=ref, off=off, sz=sz, S=S, G=G)


def reference_2c(shells, pair_a, pair_b, op, omega):
    """Oracle blocks (a|O|b) and the element-wise conditioning scale C = S + G."""
    r = reference_2c_parts(shells, pair_a, pair_b, op, omega)
    return r["ref"], r["S"] + r["G"]


def reference_ra2n(shells, pair_a, pair_b, n):
    """Oracle blocks (a|r_a^{2n}|b) and the element-wise scale C = S + G."""
    import oracle
    shn, sha = normalised(shells)
    ref, off, sz = oracle.eval_2c_ra2n(shn, pair_a, pair_b, n, normalize=False)
    S, _, _ = oracle.eval_2c_ra2n(sha, pair_a, pair_b, n, normalize=False)
    jac, _, _ = oracle.eval_2c_ra2n_grad(shn, pair_a, pair_b, n, center="A", normalize=False)
    G = geometric_scale(jac, off, sz, separations(shells, pair_a, pair_b))
    return ref, np.abs(S) + G


def reference_3c(shells, t_a, t_atilde, t_b):
    """Oracle blocks (a b a~) and the element-wise scale C = S + G (v = R_a - R_b)."""
    import oracle
    shn, sha = normalised(shells)
    ref, off, sz = oracle.eval_3c_aab(shn, t_a, t_atilde, t_b, normalize=False)
    S, _, _ = oracle.eval_3c_aab(sha, t_a, t_atilde, t_b, normalize=False)
    jac, _, _ = oracle.eval_3c_aab_grad(shn, t_a, t_atilde, t_b, center="A", normalize=False)
    G = geometric_scale(jac, off, sz, separations(shells, t_a, t_b))
    return ref, np.abs(S) + G


def vjp_reference(jac, jac_abs, off, sz, w):
    """sum_e W_e dI_e/dR (per entry, 3 components) and its element-wise
    magnitude sum sum_e |W_e| |dI_e/dR| taken with the |N c| Jacobian (the
    forward-error scale of the dot product and of the contractions in it)."""
    n = len(off)
    g = np.zeros((n, 3))
    s = np.zeros((n, 3))
    aw = np.abs(w)
    for p in range(n):
        blk = jac[3 * off[p]: 3 * (off[p] + sz[p])].reshape(3, sz[p])
        ablk = np.abs(jac_abs[3 * off[p]: 3 * (off[p] + sz[p])]).reshape(3, sz[p])
        wp = w[off[p]: off[p] + sz[p]]
        g[p] = blk @ wp
        s[p] = np.maximum(ablk, np.abs(blk)) @ aw[off[p]: off[p] + sz[p]]
    return g, s
