"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle function to the mathematics: a closed form, exact
quadrature through an independent route (tests/quadrature.py), a symmetry of
the integrals, or brute force.  A plausible slip anywhere in the oracle (sign,
index, dropped term, transposed operand) fails at least one of them.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import special

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests import quadrature as Q

OPS = [(0, 0.0), (1, 0.0), (2, 0.11), (3, 0.11), (4, 1.0), (5, 0.3)]


# --------------------------------------------------------------------------- #
# Boys function (SI Eq. 3): against the lower incomplete gamma function,      #
# F_n(T) = gamma(n+1/2, T) / (2 T^{n+1/2}), at 40 digits.                     #
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("long_double", [False, True])
def test_boys_against_incomplete_gamma(long_double):
    mpmath.mp.dps = 40
    for T in [0.0, 1e-8, 0.3, 2.5, 11.7, 29.9, 36.0, 49.99, 50.0, 51.3, 120.0, 700.0]:
        F = oracle.boys(18, T, long_double=long_double)
        for n in range(19):
            if T == 0.0:
                ref = mpmath.mpf(1) / (2 * n + 1)
            else:
                ref = mpmath.gammainc(n + 0.5, 0, T) / (2 * mpmath.mpf(T) ** (n + 0.5))
            assert abs(F[n] - float(ref)) <= 2e-15 * float(ref), (T, n, F[n], ref)


def test_boys_derivative_identity():
    # dF_n/dT = -F_{n+1}  (SI Eq. 4), central differences
    for T in [0.7, 8.0, 40.0, 60.0]:
        h = 1e-5 * max(1.0, T)
        Fp, Fm, F = oracle.boys(10, T + h), oracle.boys(10, T - h), oracle.boys(11, T)
        d = (Fp - Fm) / (2 * h)
        np.testing.assert_allclose(d, -F[1:12], rtol=1e-8)


# --------------------------------------------------------------------------- #
# Real solid harmonics                                                        #
# --------------------------------------------------------------------------- #
def _eval_sph(T, l, pts):
    carts = Q.cart_list(l)
    mon = np.stack([pts[:, 0] ** x * pts[:, 1] ** y * pts[:, 2] ** z for (x, y, z) in carts], axis=1)
    return mon @ T.T                     # (npts, 2l+1)


def test_sph_low_order_explicit():
    T1 = oracle.sph_coef(1)
    # rows m = -1, 0, 1 -> y, z, x ; columns x, y, z
    np.testing.assert_allclose(T1, [[0, 1, 0], [0, 0, 1], [1, 0, 0]], atol=1e-15)
    T2 = oracle.sph_coef(2)
    s3 = math.sqrt(3.0)
    # columns xx, xy, xz, yy, yz, zz
    ref = [[0, s3, 0, 0, 0, 0], [0, 0, 0, 0, s3, 0], [-0.5, 0, 0, -0.5, 0, 1], [0, 0, s3, 0, 0, 0],
           [s3 / 2, 0, 0, -s3 / 2, 0, 0]]
    np.testing.assert_allclose(T2, ref, atol=1e-15)


@pytest.mark.parametrize("l", range(0, 11))
def test_sph_against_scipy_spherical_harmonics(l):
    """S_lm = sqrt(4 pi/(2l+1)) r^l * real combination of Condon-Shortley Y_lm."""
    rng = np.random.default_rng(l)
    pts = rng.standard_normal((40, 3))
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(pts[:, 2] / r)
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    S = _eval_sph(oracle.sph_coef(l), l, pts)
    pref = np.sqrt(4 * np.pi / (2 * l + 1)) * r ** l
    for m in range(-l, l + 1):
        mu = abs(m)
        Y = special.sph_harm_y(l, mu, theta, phi)
        if m > 0:
            ref = np.sqrt(2) * (-1) ** mu * Y.real
        elif m < 0:
            ref = np.sqrt(2) * (-1) ** mu * Y.imag
        else:
            ref = Y.real
        np.testing.assert_allclose(S[:, m + l], pref * ref, rtol=1e-11, atol=1e-11 * pref.max())


@pytest.mark.parametrize("l", range(0, 9))
def test_sph_orthogonality_and_harmonicity(l):
    # angular quadrature: Gauss-Legendre in cos(theta) x trapezoid in phi (exact for these degrees)
    x, w = np.polynomial.legendre.leggauss(2 * l + 4)
    nphi = 4 * l + 6
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = np.stack([(st * np.cos(ph)).ravel(), (st * np.sin(ph)).ravel(), ct.ravel()], axis=1)
    wts = (np.repeat(w, nphi) * (2 * np.pi / nphi))
    S = _eval_sph(oracle.sph_coef(l), l, pts)
    G = (S * wts[:, None]).T @ S
    np.testing.assert_allclose(G, 4 * np.pi / (2 * l + 1) * np.eye(2 * l + 1), atol=1e-12)
    # Laplacian of each polynomial is zero
    T = oracle.sph_coef(l)
    carts = Q.cart_list(l)
    if l >= 2:
        lap = {}
        for k, (a, b, c) in enumerate(carts):
            for d, (e, f, g) in enumerate([(a - 2, b, c), (a, b - 2, c), (a, b, c - 2)]):
                p = (a, b, c)[d]
                if min(e, f, g) >= 0:
                    lap.setdefault((e, f, g), np.zeros(2 * l + 1))
                    lap[(e, f, g)] += p * (p - 1) * T[:, k]
        for v in lap.values():
            np.testing.assert_allclose(v, 0, atol=1e-12)


def test_sph_matches_paper_scaled_harmonic_recursion():
    """The real functions are A_{l,mu} R^{c/s}_{l,mu} of the recursion in
    Sec. II E, with A of Eq. (A): pins the output convention to the paper's."""
    rng = np.random.default_rng(7)
    pts = rng.standard_normal((25, 3))
    L = 8
    for p in pts:
        x, y, z = p
        r2 = p @ p
        Rc = np.zeros((L + 2, L + 2))
        Rs = np.zeros((L + 2, L + 2))
        Rc[0, 0] = 1
        for l in range(L):
            Rc[l + 1, l + 1] = -(x * Rc[l, l] - y * Rs[l, l]) / (2 * l + 2)
            Rs[l + 1, l + 1] = -(y * Rc[l, l] + x * Rs[l, l]) / (2 * l + 2)
            for m in range(l + 1):
                pc = Rc[l - 1, m] if l >= 1 else 0.0
                ps = Rs[l - 1, m] if l >= 1 else 0.0
                Rc[l + 1, m] = ((2 * l + 1) * z * Rc[l, m] - r2 * pc) / ((l + m + 1) * (l - m + 1))
                Rs[l + 1, m] = ((2 * l + 1) * z * Rs[l, m] - r2 * ps) / ((l + m + 1) * (l - m + 1))
        for l in range(L + 1):
            S = _eval_sph(oracle.sph_coef(l), l, p[None, :])[0]
            for m in range(-l, l + 1):
                mu = abs(m)
                A = (-1) ** mu * math.sqrt((2 - (mu == 0)) * math.factorial(l + mu) * math.factorial(l - mu))
                ref = A * (Rc[l, mu] if m >= 0 else Rs[l, mu])
                assert abs(S[m + l] - ref) <= 1e-11 * (1 + abs(ref)), (l, m)


# --------------------------------------------------------------------------- #
# Primitive Cartesian integrals against independent quadrature                #
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("op,omega", OPS)
def test_cartesian_primitives_against_quadrature(op, omega):
    rng = np.random.default_rng(100 + op)
    cases = [(0, 0), (1, 0), (0, 2), (1, 1), (2, 1), (2, 2)]
    if op in (0, 4):
        cases += [(3, 2), (4, 3)]
    for la, lb in cases:
        alpha, beta = np.exp(rng.uniform(np.log(0.2), np.log(8.0), 2))
        A = rng.uniform(-1, 1, 3)
        B = A + rng.uniform(0.3, 2.5) * W._unit_vectors(rng, 1)[0]
        I = oracle.cart_2c(op, omega, la, lb, alpha, beta, A, B)
        scale = np.abs(I).max()
        for ia, a in enumerate(Q.cart_list(la)):
            for ib, b in enumerate(Q.cart_list(lb)):
                ref = Q.cart_integral(op, a, b, alpha, beta, omega, A, B)
                assert abs(I[ia, ib] - ref) <= 1e-10 * scale, (op, la, lb, a, b, I[ia, ib], ref)


def test_ss_closed_form_limits():
    # erf + erfc = Coulomb; omega -> inf: erf -> Coulomb; (omega/pi)^{3/2} exp(-omega r^2) -> delta
    a, b, R2 = 0.7, 1.9, 1.3
    c = oracle.ss_deriv(1, a, b, 0, R2, 6)
    e1 = oracle.ss_deriv(3, a, b, 0.37, R2, 6)
    e2 = oracle.ss_deriv(2, a, b, 0.37, R2, 6)
    np.testing.assert_allclose(e1 + e2, c, rtol=1e-14)
    np.testing.assert_allclose(oracle.ss_deriv(3, a, b, 1e7, R2, 3), c[:4], rtol=1e-6)
    g = oracle.ss_deriv(4, a, b, 1e8, R2, 0)[0] * (1e8 / math.pi) ** 1.5
    s = oracle.ss_deriv(0, a, b, 0, R2, 0)[0]
    assert abs(g - s) < 1e-6 * s
    # exp(-omega r^2)/r: omega = 0 is the Coulomb operator, every derivative order
    np.testing.assert_allclose(oracle.ss_deriv(5, a, b, 0.0, R2, 6), c, rtol=1e-14)
    # omega -> inf: exp(-omega r^2)/r ~ (2 pi / omega) delta(r) on smooth densities
    w = 1e8
    gd = oracle.ss_deriv(5, a, b, w, R2, 0)[0] * w / (2 * math.pi)
    assert abs(gd - s) < 1e-6 * s


def test_ss_derivatives_by_finite_differences():
    a, b = 0.9, 2.3
    for op, om in OPS:
        for R2 in [0.4, 3.0, 20.0]:
            h = 1e-4
            G = oracle.ss_deriv(op, a, b, om, R2, 5)
            Gp = oracle.ss_deriv(op, a, b, om, R2 + h, 5)
            Gm = oracle.ss_deriv(op, a, b, om, R2 - h, 5)
            d = (Gp - Gm) / (2 * h)
            np.testing.assert_allclose(d[:5], G[1:6], rtol=1e-6, atol=1e-12 * abs(G[0]))


# --------------------------------------------------------------------------- #
# Contracted, normalised blocks                                               #
# --------------------------------------------------------------------------- #
def _small_two_center(seed, n=12, lmax=3, kmax=3):
    return W.two_center_workload(n, list(range(lmax + 1)), [1.0 / (lmax + 1)] * (lmax + 1),
                                 lambda r, m: r.integers(1, kmax + 1, size=m), (0.1, 20.0), (0.5, 3.0), seed)


def _blocks(vals, off, sz, shells, pa, pb):
    out = []
    for p in range(len(pa)):
        la, lb = shells["l"][pa[p]], shells["l"][pb[p]]
        out.append(vals[off[p]:off[p] + sz[p]].reshape(2 * la + 1, 2 * lb + 1))
    return out


def test_normalisation_closed_form_and_identity_self_overlap():
    sh, pa, pb = _small_two_center(1, n=20, lmax=6, kmax=5)
    N = oracle.shell_norms(sh)
    off = np.r_[0, np.cumsum(sh["nprim"])]
    for s in range(len(sh["l"])):
        l = int(sh["l"][s])
        e = sh["exps"][off[s]:off[s + 1]]
        c = sh["coefs"][off[s]:off[s + 1]]
        ssum = sum(math.sqrt(math.pi) * math.factorial(2 * l + 2) * ci * cj
                   / (2 ** (2 * l + 3) * math.factorial(l + 1) * (ai + aj) ** (l + 1.5))
                   for ai, ci in zip(e, c) for aj, cj in zip(e, c))
        Nl = math.sqrt((2 * l + 1) / (4 * math.pi)) / math.sqrt(ssum)
        assert abs(N[s] - Nl) <= 1e-12 * Nl
    # self overlap of each shell at one center is the identity
    sh2 = dict(sh)
    sh2["center_of"] = np.zeros_like(sh["center_of"])
    idx = np.arange(len(sh["l"]), dtype=np.int32)
    v, o, z = oracle.eval_2c(sh2, idx, idx, 0)
    for p, blk in enumerate(_blocks(v, o, z, sh2, idx, idx)):
        np.testing.assert_allclose(blk, np.eye(blk.shape[0]), atol=1e-13)


@pytest.mark.parametrize("op,omega", OPS)
def test_contracted_block_against_quadrature(op, omega):
    """Full chain (contract, transform, normalise) for a few small pairs:
    quadrature Cartesian integrals x explicit coefficients x closed-form N_l."""
    sh, pa, pb = _small_two_center(20 + op, n=3, lmax=2, kmax=2)
    v, o, z = oracle.eval_2c(sh, pa, pb, op, omega)
    N = oracle.shell_norms(sh)
    off = np.r_[0, np.cumsum(sh["nprim"])]
    for p, blk in enumerate(_blocks(v, o, z, sh, pa, pb)):
        a, b = pa[p], pb[p]
        la, lb = int(sh["l"][a]), int(sh["l"][b])
        A = sh["centers"][sh["center_of"][a]]
        B = sh["centers"][sh["center_of"][b]]
        C = np.zeros((len(Q.cart_list(la)), len(Q.cart_list(lb))))
        for i in range(off[a], off[a + 1]):
            for j in range(off[b], off[b + 1]):
                for ia, ca in enumerate(Q.cart_list(la)):
                    for ib, cb in enumerate(Q.cart_list(lb)):
                        C[ia, ib] += sh["coefs"][i] * sh["coefs"][j] * Q.cart_integral(
                            op, ca, cb, sh["exps"][i], sh["exps"][j], omega, A, B)
        ref = N[a] * N[b] * oracle.sph_coef(la) @ C @ oracle.sph_coef(lb).T
        np.testing.assert_allclose(blk, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _wigner_real(l, Rm):
    """Real rotation matrix D with S_l(R^T r) = D S_l(r), by angular quadrature."""
    x, w = np.polynomial.legendre.leggauss(2 * l + 4)
    nphi = 4 * l + 6
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = np.stack([(st * np.cos(ph)).ravel(), (st * np.sin(ph)).ravel(), ct.ravel()], axis=1)
    wts = np.repeat(w, nphi) * (2 * np.pi / nphi)
    T = oracle.sph_coef(l)
    S = _eval_sph(T, l, pts)
    Srot = _eval_sph(T, l, pts @ Rm)              # S(R^T r) for each row r
    return (Srot * wts[:, None]).T @ S * (2 * l + 1) / (4 * np.pi)


@pytest.mark.parametrize("op,omega", OPS)
def test_rotation_covariance(op, omega):
    """Rotating both centers by R: block' = D^{la} block D^{lb}^T."""
    sh, pa, pb = _small_two_center(40 + op, n=8, lmax=4, kmax=3)
    rng = np.random.default_rng(5)
    Rm = _rotation(rng)
    sh2 = dict(sh)
    sh2["centers"] = sh["centers"] @ Rm.T
    v1, o, z = oracle.eval_2c(sh, pa, pb, op, omega)
    v2, _, _ = oracle.eval_2c(sh2, pa, pb, op, omega)
    for b1, b2, a, b in zip(_blocks(v1, o, z, sh, pa, pb), _blocks(v2, o, z, sh, pa, pb), pa, pb):
        Da = _wigner_real(int(sh["l"][a]), Rm)
        Db = _wigner_real(int(sh["l"][b]), Rm)
        pred = Da.T @ b1 @ Db
        np.testing.assert_allclose(b2, pred, atol=1e-11 * max(1.0, np.abs(b1).max()))
        assert abs(np.linalg.norm(b1) - np.linalg.norm(b2)) <= 1e-11 * max(1.0, np.linalg.norm(b1))


@pytest.mark.parametrize("op,omega", OPS)
def test_swap_transpose_and_parity(op, omega):
    sh, pa, pb = _small_two_center(60 + op, n=10, lmax=4, kmax=3)
    v, o, z = oracle.eval_2c(sh, pa, pb, op, omega)
    vs, os_, zs = oracle.eval_2c(sh, pb, pa, op, omega)
    shi = dict(sh)
    shi["centers"] = -sh["centers"]
    vi, _, _ = oracle.eval_2c(shi, pa, pb, op, omega)
    B1 = _blocks(v, o, z, sh, pa, pb)
    B2 = _blocks(vs, os_, zs, sh, pb, pa)
    B3 = _blocks(vi, o, z, sh, pa, pb)
    for p in range(len(pa)):
        la, lb = int(sh["l"][pa[p]]), int(sh["l"][pb[p]])
        sc = max(1e-3, np.abs(B1[p]).max())
        np.testing.assert_allclose(B2[p], B1[p].T, atol=1e-12 * sc)
        np.testing.assert_allclose(B3[p], (-1) ** (la + lb) * B1[p], atol=1e-12 * sc)


@pytest.mark.parametrize("op,omega", OPS)
def test_one_center_limit_is_diagonal(op, omega):
    sh, pa, pb = _small_two_center(80 + op, n=12, lmax=4, kmax=3)
    sh2 = dict(sh)
    sh2["centers"] = np.zeros_like(sh["centers"])
    v, o, z = oracle.eval_2c(sh2, pa, pb, op, omega)
    for p, blk in enumerate(_blocks(v, o, z, sh2, pa, pb)):
        la, lb = int(sh["l"][pa[p]]), int(sh["l"][pb[p]])
        if la != lb:
            np.testing.assert_allclose(blk, 0, atol=1e-13)
        else:
            d = np.diag(blk)
            np.testing.assert_allclose(blk - np.diag(d), 0, atol=1e-13)
            np.testing.assert_allclose(d, d[0], rtol=1e-12, atol=1e-14)


def test_operator_limits_on_contracted_blocks():
    sh, pa, pb = _small_two_center(3, n=6, lmax=3, kmax=3)
    c, o, z = oracle.eval_2c(sh, pa, pb, 1)
    e1, _, _ = oracle.eval_2c(sh, pa, pb, 3, 0.6)
    e2, _, _ = oracle.eval_2c(sh, pa, pb, 2, 0.6)
    np.testing.assert_allclose(e1 + e2, c, atol=1e-13 * np.abs(c).max())
    big, _, _ = oracle.eval_2c(sh, pa, pb, 3, 1e6)
    np.testing.assert_allclose(big, c, atol=1e-5 * np.abs(c).max())
    s, _, _ = oracle.eval_2c(sh, pa, pb, 0)
    g, _, _ = oracle.eval_2c(sh, pa, pb, 4, 1e7)
    np.testing.assert_allclose(g * (1e7 / math.pi) ** 1.5, s, atol=1e-5 * np.abs(s).max())


# --------------------------------------------------------------------------- #
# (a|r_a^{2n}|b) (Sec. II C)                                                  #
# --------------------------------------------------------------------------- #
def test_ra2n_zero_is_the_overlap():
    """n = 0: the closed-form 1-D route equals the recursion-based overlap."""
    sh, pa, pb = _small_two_center(41, n=10, lmax=4, kmax=3)
    v, _, _ = oracle.eval_2c_ra2n(sh, pa, pb, 0)
    s, _, _ = oracle.eval_2c(sh, pa, pb, 0)
    np.testing.assert_allclose(v, s, rtol=0, atol=1e-13 * np.abs(s).max())


@pytest.mark.parametrize("n", [1, 2, 5])
def test_ra2n_contracted_blocks_against_3d_quadrature(n):
    """Contracted blocks vs 3-D quadrature of g_a |r - A|^{2n} g_b (no
    multinomial expansion, no 1-D closed form)."""
    sh, pa, pb = _small_two_center(50 + n, n=3, lmax=2, kmax=2)
    v, o, z = oracle.eval_2c_ra2n(sh, pa, pb, n)
    N = oracle.shell_norms(sh)
    off = np.r_[0, np.cumsum(sh["nprim"])]
    for p, blk in enumerate(_blocks(v, o, z, sh, pa, pb)):
        a, b = pa[p], pb[p]
        la, lb = int(sh["l"][a]), int(sh["l"][b])
        A = sh["centers"][sh["center_of"][a]]
        B = sh["centers"][sh["center_of"][b]]
        C = np.zeros((len(Q.cart_list(la)), len(Q.cart_list(lb))))
        for i in range(off[a], off[a + 1]):
            for j in range(off[b], off[b + 1]):
                for ia, ca in enumerate(Q.cart_list(la)):
                    for ib, cb in enumerate(Q.cart_list(lb)):
                        C[ia, ib] += sh["coefs"][i] * sh["coefs"][j] * Q.cart_ra2n(
                            ca, cb, sh["exps"][i], sh["exps"][j], A, B, n)
        ref = N[a] * N[b] * oracle.sph_coef(la) @ C @ oracle.sph_coef(lb).T
        np.testing.assert_allclose(blk, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_ra2n_s_functions_match_the_printed_closed_form():
    """(0_a|r_a^{2m}|0_b) = pi^{3/2} exp(-rho R^2) / (2^m c^{m+3/2}) sum_j I_j
    with I_j = 2^j (2m+1)!! C(m,j) / (2j+1)!! beta^{2j} R^{2j} / c^j (Eq. sra2ms, I_jab)."""
    def dfact(k):
        return math.prod(range(k, 0, -2)) if k > 0 else 1
    for (al, be, R) in [(0.7, 1.9, 1.3), (3.0, 0.2, 2.5), (0.05, 11.0, 0.4)]:
        c, rho = al + be, al * be / (al + be)
        sh = dict(l=np.array([0, 0], np.int32), nprim=np.array([1, 1], np.int32), exps=np.array([al, be]),
                  coefs=np.array([1.0, 1.0]), centers=np.array([[0.0, 0.0, 0.0], [0.3 * R, -0.4 * R, math.sqrt(0.75) * R]]),
                  center_of=np.array([0, 1], np.int32))
        for m in range(6):
            v, _, _ = oracle.eval_2c_ra2n(sh, [0], [1], m, normalize=False)
            I = sum(2 ** j * dfact(2 * m + 1) * math.comb(m, j) / dfact(2 * j + 1) * be ** (2 * j) * R ** (2 * j) / c ** j
                    for j in range(m + 1))
            ref = math.pi ** 1.5 * math.exp(-rho * R * R) / (2 ** m * c ** (m + 1.5)) * I
            assert abs(v[0] - ref) <= 1e-13 * ref, (al, be, R, m, v[0], ref)


@pytest.mark.parametrize("n", [1, 3])
def test_ra2n_gradient_against_finite_differences_and_translation(n):
    sh, pa, pb = _small_two_center(60 + n, n=4, lmax=3, kmax=2)
    ga, o, z = oracle.eval_2c_ra2n_grad(sh, pa, pb, n, center="A")
    gb, _, _ = oracle.eval_2c_ra2n_grad(sh, pa, pb, n, center="B")
    np.testing.assert_allclose(ga, -gb, rtol=0, atol=1e-12 * np.abs(ga).max())
    h = 1e-5
    for p in range(len(pa)):
        ca = sh["center_of"][pa[p]]
        for d in range(3):
            cp, cm = sh["centers"].copy(), sh["centers"].copy()
            cp[ca, d] += h
            cm[ca, d] -= h
            vp, _, _ = oracle.eval_2c_ra2n(dict(sh, centers=cp), pa[p:p + 1], pb[p:p + 1], n)
            vm, _, _ = oracle.eval_2c_ra2n(dict(sh, centers=cm), pa[p:p + 1], pb[p:p + 1], n)
            fd = (vp - vm) / (2 * h)
            an = ga[3 * o[p] + d * z[p]: 3 * o[p] + (d + 1) * z[p]]
            np.testing.assert_allclose(an, fd, rtol=0, atol=2e-7 * max(np.abs(fd).max(), 1e-3))


# --------------------------------------------------------------------------- #
# Three-index overlap                                                         #
# --------------------------------------------------------------------------- #
def test_aab_against_quadrature():
    sh, ta, tt, tb, _ = W.aab_workload(1, seed=11, n_clusters=1, n_atoms=2, n_orb=2, orb_l=(0, 2), orb_k=(1, 2),
                                       n_aux=2, aux_l=(0, 3), aux_k=(1, 2), exp_range=(0.2, 10.0))
    v, o, z = oracle.eval_3c_aab(sh, ta, tt, tb)
    N = oracle.shell_norms(sh)
    off = np.r_[0, np.cumsum(sh["nprim"])]
    for p in range(len(ta)):
        a, t, b = ta[p], tt[p], tb[p]
        la, lt, lb = (int(sh["l"][s]) for s in (a, t, b))
        A = sh["centers"][sh["center_of"][a]]
        B = sh["centers"][sh["center_of"][b]]
        ca_l, ct_l, cb_l = Q.cart_list(la), Q.cart_list(lt), Q.cart_list(lb)
        C = np.zeros((len(ca_l), len(ct_l), len(cb_l)))
        for i in range(off[a], off[a + 1]):
            for k in range(off[t], off[t + 1]):
                for j in range(off[b], off[b + 1]):
                    cc = sh["coefs"][i] * sh["coefs"][k] * sh["coefs"][j]
                    for ia, ca in enumerate(ca_l):
                        for it, ct in enumerate(ct_l):
                            for ib, cb in enumerate(cb_l):
                                C[ia, it, ib] += cc * Q.cart_triple_overlap(ca, ct, cb, sh["exps"][i], sh["exps"][k],
                                                                            sh["exps"][j], A, B)
        ref = np.einsum("ai,tk,bj,ikj->atb", oracle.sph_coef(la), oracle.sph_coef(lt), oracle.sph_coef(lb), C)
        ref *= N[a] * N[t] * N[b]
        blk = v[o[p]:o[p] + z[p]].reshape(ref.shape)
        np.testing.assert_allclose(blk, ref, atol=1e-11 * max(1e-3, np.abs(ref).max()))


def test_aab_with_s_function_reduces_to_two_center_overlap():
    """phi_s(alpha) * phi_a~(alpha~) on one center is a single (l~, alpha+alpha~)
    Gaussian, so (s b a~) equals a two-center overlap of that shell with b."""
    rng = np.random.default_rng(9)
    for lt in range(0, 5):
        for lb in range(0, 4):
            al, at, be = np.exp(rng.uniform(np.log(0.2), np.log(20), 3))
            A = rng.uniform(-2, 2, 3)
            B = A + rng.uniform(0.5, 3) * W._unit_vectors(rng, 1)[0]
            sh = dict(l=np.array([0, lt, lb], np.int32), nprim=np.ones(3, np.int32), exps=np.array([al, at, be]),
                      coefs=np.ones(3), centers=np.stack([A, B]), center_of=np.array([0, 0, 1], np.int32))
            v3, _, _ = oracle.eval_3c_aab(sh, [0], [1], [2])
            sh2 = dict(l=np.array([lt, lb], np.int32), nprim=np.ones(2, np.int32), exps=np.array([al + at, be]),
                       coefs=np.ones(2), centers=np.stack([A, B]), center_of=np.array([0, 1], np.int32))
            v2, _, _ = oracle.eval_2c(sh2, [0], [1], 0)
            N3 = oracle.shell_norms(sh)
            N2 = oracle.shell_norms(sh2)
            np.testing.assert_allclose(v3, v2 * N3[0] * N3[1] / N2[0], rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------- #
# Gradients                                                                   #
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("op,omega", OPS)
def test_gradient_against_finite_differences_and_translation(op, omega):
    sh, pa, pb = _small_two_center(200 + op, n=5, lmax=3, kmax=3)
    gA, o, z = oracle.eval_2c_grad(sh, pa, pb, op, omega, center="A")
    gB, _, _ = oracle.eval_2c_grad(sh, pa, pb, op, omega, center="B")
    np.testing.assert_allclose(gA, -gB, atol=1e-12 * np.abs(gA).max())
    h = 1e-5
    for p in range(len(pa)):
        ca = sh["center_of"][pa[p]]
        for d in range(3):
            shp = dict(sh); shp["centers"] = sh["centers"].copy(); shp["centers"][ca, d] += h
            shm = dict(sh); shm["centers"] = sh["centers"].copy(); shm["centers"][ca, d] -= h
            vp, _, _ = oracle.eval_2c(shp, pa[p:p + 1], pb[p:p + 1], op, omega)
            vm, _, _ = oracle.eval_2c(shm, pa[p:p + 1], pb[p:p + 1], op, omega)
            fd = (vp - vm) / (2 * h)
            an = gA[3 * o[p] + d * z[p]: 3 * o[p] + (d + 1) * z[p]]
            np.testing.assert_allclose(an, fd, atol=1e-8 * max(1.0, np.abs(an).max()))


def test_aab_gradient_against_finite_differences():
    sh, ta, tt, tb, _ = W.aab_workload(1, seed=12, n_clusters=1, n_atoms=2, n_orb=2, orb_l=(0, 3), orb_k=(1, 3),
                                       n_aux=2, aux_l=(0, 3), aux_k=(1, 2), exp_range=(0.2, 10.0))
    gA, o, z = oracle.eval_3c_aab_grad(sh, ta, tt, tb, center="A")
    gB, _, _ = oracle.eval_3c_aab_grad(sh, ta, tt, tb, center="B")
    np.testing.assert_allclose(gA, -gB, atol=1e-12 * np.abs(gA).max())
    h = 1e-5
    cb = sh["center_of"][tb[0]]
    for d in range(3):
        shp = dict(sh); shp["centers"] = sh["centers"].copy(); shp["centers"][cb, d] += h
        shm = dict(sh); shm["centers"] = sh["centers"].copy(); shm["centers"][cb, d] -= h
        vp, _, _ = oracle.eval_3c_aab(shp, ta, tt, tb)
        vm, _, _ = oracle.eval_3c_aab(shm, ta, tt, tb)
        fd = (vp - vm) / (2 * h)
        for p in range(len(ta)):
            an = gB[3 * o[p] + d * z[p]: 3 * o[p] + (d + 1) * z[p]]
            np.testing.assert_allclose(an, fd[o[p]:o[p] + z[p]], atol=1e-8 * max(1.0, np.abs(an).max()))


def test_fp64_and_extended_builds_agree_to_fp64_noise():
    sh, pa, pb = W.make("c2_200k_l4_k8", n=60)
    for op, om in OPS:
        v64, _, _ = oracle.eval_2c(sh, pa, pb, op, om, long_double=False)
        vld, _, _ = oracle.eval_2c(sh, pa, pb, op, om, long_double=True)
        np.testing.assert_allclose(v64, vld, rtol=0, atol=1e-11 * max(1.0, np.abs(vld).max()))
