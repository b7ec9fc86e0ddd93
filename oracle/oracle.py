"""ctypes wrapper around the C oracle (test infrastructure only; see package doc)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

OP_OVERLAP, OP_COULOMB, OP_ERFC, OP_ERF, OP_GAUSS, OP_GCOUL = 0, 1, 2, 3, 4, 5

# The contracted integrals are taken from the long-double build by default:
# in FP64 the Cartesian recursion loses up to ~1e-13 absolute accuracy on the
# random-sign, wide-exponent shells of the synthetic workloads (cancellation
# in the recursion and in the Cartesian -> spherical transform), which is
# above the 1e-12 relative / 1e-14 absolute parity bar.
DEFAULT_LONG_DOUBLE = True

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs = {}


def lib_path(long_double=False):
    return os.path.join(_BUILD, "liboracle_ld.so" if long_double else "liboracle.so")


def build(long_double=False, force=False):
    """Compile the oracle with gcc (host only, any architecture)."""
    out = lib_path(long_double)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    if long_double:
        cmd.insert(1, "-DORACLE_LONG_DOUBLE")
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def _lib(long_double=False):
    if long_double is None:
        long_double = DEFAULT_LONG_DOUBLE
    long_double = bool(long_double)
    with _lock:
        if long_double not in _libs:
            lib = ctypes.CDLL(build(long_double))
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.oracle_boys.argtypes = [i32, f64, P]
            lib.oracle_ss.argtypes = [i32, f64, f64, f64, f64, i32, P]
            lib.oracle_sph_coef.argtypes = [i32, P]
            lib.oracle_cart_2c.argtypes = [i32, f64, i32, i32, f64, f64, P, P, P]
            lib.oracle_shell_norms.argtypes = [i32, P, P, P, P, P, P]
            lib.oracle_eval_2c.argtypes = [i32, P, P, P, P, P, P, P, i64, P, P, i32, f64, i32, i32, P, P, i32]
            lib.oracle_eval_3c_aab.argtypes = [i32, P, P, P, P, P, P, P, i64, P, P, P, i32, i32, P, P, i32]
            lib.oracle_eval_2c_ra2n.argtypes = [i32, P, P, P, P, P, P, P, i64, P, P, i32, i32, i32, P, P, i32]
            _libs[long_double] = lib
        return _libs[long_double]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def ncart(l):
    return (l + 1) * (l + 2) // 2


def boys(nmax, T, long_double=None):
    F = np.zeros(nmax + 1)
    if _lib(long_double).oracle_boys(int(nmax), float(T), _p(F)):
        raise ValueError("bad nmax")
    return F


def ss_deriv(op, alpha, beta, omega, R2, mmax, long_double=None):
    """(0_a|O|0_b)^{(m)} for m = 0..mmax (Table S1)."""
    G = np.zeros(mmax + 1)
    if _lib(long_double).oracle_ss(int(op), float(alpha), float(beta), float(omega), float(R2), int(mmax), _p(G)):
        raise ValueError("bad mmax")
    return G


def sph_coef(l, long_double=None):
    """Real solid harmonic coefficients: (2l+1) x ncart(l), rows m = -l..l."""
    T = np.zeros((2 * l + 1, ncart(l)))
    if _lib(long_double).oracle_sph_coef(int(l), _p(T)):
        raise ValueError("bad l")
    return T


def cart_2c(op, omega, la, lb, alpha, beta, A, B, long_double=None):
    out = np.zeros((ncart(la), ncart(lb)))
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if _lib(long_double).oracle_cart_2c(int(op), float(omega), la, lb, float(alpha), float(beta), _p(A), _p(B), _p(out)):
        raise ValueError("bad l")
    return out


class _Shells:
    def __init__(self, shells):
        self.l = np.ascontiguousarray(shells["l"], dtype=np.int32)
        self.nprim = np.ascontiguousarray(shells["nprim"], dtype=np.int32)
        self.off = np.zeros(len(self.l), dtype=np.int64)
        if len(self.l) > 1:
            self.off[1:] = np.cumsum(self.nprim[:-1])
        self.exps = np.ascontiguousarray(shells["exps"], dtype=np.float64)
        self.coefs = np.ascontiguousarray(shells["coefs"], dtype=np.float64)
        self.centers = np.ascontiguousarray(shells["centers"], dtype=np.float64).reshape(-1, 3)
        self.center_of = np.ascontiguousarray(shells["center_of"], dtype=np.int32)

    def args(self):
        return [len(self.l), _p(self.l), _p(self.nprim), _p(self.off), _p(self.exps), _p(self.coefs),
                _p(self.centers), _p(self.center_of)]


def shell_norms(shells, long_double=None):
    s = _Shells(shells)
    out = np.zeros(len(s.l))
    r = _lib(long_double).oracle_shell_norms(len(s.l), _p(s.l), _p(s.nprim), _p(s.off), _p(s.exps), _p(s.coefs), _p(out))
    if r:
        raise ValueError("bad shells")
    return out


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def _eval2c(shells, pair_a, pair_b, op, omega, deriv, nthreads, long_double, normalize=True, ra2n=None):
    s = _Shells(shells)
    pa = np.ascontiguousarray(pair_a, dtype=np.int32)
    pb = np.ascontiguousarray(pair_b, dtype=np.int32)
    sizes = (2 * s.l[pa].astype(np.int64) + 1) * (2 * s.l[pb].astype(np.int64) + 1)
    offsets = np.zeros(len(pa), dtype=np.int64)
    if len(pa) > 1:
        offsets[1:] = np.cumsum(sizes[:-1])
    total = int(sizes.sum())
    out = np.zeros(total * (3 if deriv else 1))
    if ra2n is None:
        r = _lib(long_double).oracle_eval_2c(*s.args(), len(pa), _p(pa), _p(pb), int(op), float(omega), int(deriv),
                                             int(bool(normalize)), _p(offsets), _p(out), _threads(nthreads))
    else:
        r = _lib(long_double).oracle_eval_2c_ra2n(*s.args(), len(pa), _p(pa), _p(pb), int(ra2n), int(deriv),
                                                  int(bool(normalize)), _p(offsets), _p(out), _threads(nthreads))
    if r:
        raise ValueError("oracle two-center evaluation failed: %d" % r)
    return out, offsets, sizes


def eval_2c(shells, pair_a, pair_b, op, omega=0.0, nthreads=None, long_double=None, normalize=True):
    """Contracted normalised blocks (a|O|b) of all pairs, concatenated.

    Returns (values, offsets, sizes); block p is values[offsets[p]:offsets[p]+sizes[p]]
    in row-major order [m_a = -la..la][m_b = -lb..lb].  normalize=False uses
    the coefficients as given.
    """
    return _eval2c(shells, pair_a, pair_b, op, omega, 0, nthreads, long_double, normalize)


def eval_2c_grad(shells, pair_a, pair_b, op, omega=0.0, center="A", nthreads=None, long_double=None,
                 normalize=True):
    """Jacobian of every block with respect to R_a (center='A') or R_b ('B').

    Returns (values, offsets, sizes): pair p owns values[3*offsets[p] : 3*(offsets[p]+sizes[p])]
    laid out [xyz][m_a][m_b].
    """
    return _eval2c(shells, pair_a, pair_b, op, omega, 1 if center == "A" else 2, nthreads, long_double, normalize)


def eval_2c_ra2n(shells, pair_a, pair_b, n, nthreads=None, long_double=None, normalize=True):
    """Contracted normalised blocks (a|r_a^{2n}|b) (Sec. II C), laid out as eval_2c."""
    return _eval2c(shells, pair_a, pair_b, 0, 0.0, 0, nthreads, long_double, normalize, ra2n=n)


def eval_2c_ra2n_grad(shells, pair_a, pair_b, n, center="A", nthreads=None, long_double=None, normalize=True):
    """Jacobian of the (a|r_a^{2n}|b) blocks with respect to R_a or R_b, laid out as eval_2c_grad."""
    return _eval2c(shells, pair_a, pair_b, 0, 0.0, 1 if center == "A" else 2, nthreads, long_double, normalize,
                   ra2n=n)


def _eval3c(shells, ta, tt, tb, deriv, nthreads, long_double, normalize=True):
    s = _Shells(shells)
    ta = np.ascontiguousarray(ta, dtype=np.int32)
    tt = np.ascontiguousarray(tt, dtype=np.int32)
    tb = np.ascontiguousarray(tb, dtype=np.int32)
    sizes = ((2 * s.l[ta].astype(np.int64) + 1) * (2 * s.l[tt].astype(np.int64) + 1)
             * (2 * s.l[tb].astype(np.int64) + 1))
    offsets = np.zeros(len(ta), dtype=np.int64)
    if len(ta) > 1:
        offsets[1:] = np.cumsum(sizes[:-1])
    out = np.zeros(int(sizes.sum()) * (3 if deriv else 1))
    r = _lib(long_double).oracle_eval_3c_aab(*s.args(), len(ta), _p(ta), _p(tt), _p(tb), int(deriv),
                                             int(bool(normalize)), _p(offsets), _p(out), _threads(nthreads))
    if r:
        raise ValueError("oracle_eval_3c_aab failed: %d" % r)
    return out, offsets, sizes


def eval_3c_aab(shells, t_a, t_atilde, t_b, nthreads=None, long_double=None, normalize=True):
    """Three-index overlaps (a b a~) with a, a~ on one center; blocks [m_a][m_a~][m_b]."""
    return _eval3c(shells, t_a, t_atilde, t_b, 0, nthreads, long_double, normalize)


def eval_3c_aab_grad(shells, t_a, t_atilde, t_b, center="A", nthreads=None, long_double=None, normalize=True):
    return _eval3c(shells, t_a, t_atilde, t_b, 1 if center == "A" else 2, nthreads, long_double, normalize)
