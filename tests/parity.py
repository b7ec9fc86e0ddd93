"""Shared helpers for GPU-vs-oracle parity tests.

Element-wise bar, atomic units, normalised functions:

    |x - ref| <= rtol |ref| + atol + gamma S_p

  FP64 integrals    rtol 1e-12, atol 1e-14, gamma 1e-15
  gradients         rtol 1e-10, atol 1e-12, gamma 1e-15
  mixed precision   rtol 1e-10, atol 1e-14, gamma 2e-13

S_p is the conditioning scale of block p: the largest element magnitude of
the same block evaluated with |N c| in place of the normalised coefficients
N c (for erfc the Coulomb and erf scales added).  For fixed derivative order
every primitive term of O^{(k)} has the same sign, so with |N c| the
contraction sums the magnitudes of its terms: S_p is the sum-of-magnitudes
scale of the forward error bound of the contraction.  Where random-sign
coefficients cancel (sum |t| / |sum t| up to ~1e5 in the synthetic sets) no
FP64 evaluation can reach 1e-12 relative; there the gamma S_p term, a few
units of FP64 rounding of that scale, is the bar.  Where the contraction is
well conditioned, the rtol term dominates.
"""
import numpy as np

TOL_FP64 = (1e-12, 1e-14, 1e-15)
TOL_GRAD = (1e-10, 1e-12, 1e-15)
TOL_MIXED = (1e-10, 1e-14, 2e-13)


def _bar(ref, tol, scale):
    rtol, atol = tol[0], tol[1]
    gamma = tol[2] if len(tol) > 2 else 0.0
    bar = rtol * np.abs(ref) + atol
    if scale is not None:
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


def _block_max(values, offsets, sizes):
    """Each element replaced by the largest magnitude of its block."""
    out = np.empty_like(values)
    for o, z in zip(offsets, sizes):
        if z:
            out[o:o + z] = np.abs(values[o:o + z]).max()
    return out


def normalised(shells):
    """Shell set with coefficients N c (oracle normalisation) and its |N c| twin."""
    import oracle
    N = oracle.shell_norms(shells)
    prim_shell = np.repeat(np.arange(len(shells["l"])), shells["nprim"])
    cn = np.asarray(shells["coefs"], dtype=np.float64) * N[prim_shell]
    return dict(shells, coefs=cn), dict(shells, coefs=np.abs(cn))


def reference_2c(shells, pair_a, pair_b, op, omega):
    """Oracle blocks (a|O|b) and the per-element conditioning scale S_p."""
    import oracle
    shn, sha = normalised(shells)
    ref, off, sz = oracle.eval_2c(shn, pair_a, pair_b, op, omega, normalize=False)
    if op == oracle.OP_ERFC:
        s1, _, _ = oracle.eval_2c(sha, pair_a, pair_b, oracle.OP_COULOMB, 0.0, normalize=False)
        s2, _, _ = oracle.eval_2c(sha, pair_a, pair_b, oracle.OP_ERF, omega, normalize=False)
        sc = np.abs(s1) + np.abs(s2)
    else:
        sc, _, _ = oracle.eval_2c(sha, pair_a, pair_b, op, omega, normalize=False)
    return ref, _block_max(sc, off, sz)


def reference_ra2n(shells, pair_a, pair_b, n):
    """Oracle blocks (a|r_a^{2n}|b) and the per-element scale S_p (|N c| evaluation)."""
    import oracle
    shn, sha = normalised(shells)
    ref, off, sz = oracle.eval_2c_ra2n(shn, pair_a, pair_b, n, normalize=False)
    sc, _, _ = oracle.eval_2c_ra2n(sha, pair_a, pair_b, n, normalize=False)
    return ref, _block_max(sc, off, sz)


def reference_3c(shells, t_a, t_atilde, t_b):
    import oracle
    shn, sha = normalised(shells)
    ref, off, sz = oracle.eval_3c_aab(shn, t_a, t_atilde, t_b, normalize=False)
    sc, _, _ = oracle.eval_3c_aab(sha, t_a, t_atilde, t_b, normalize=False)
    return ref, _block_max(sc, off, sz)
