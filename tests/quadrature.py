"""Independent numerical route to Cartesian Gaussian integrals (tests only).

Every integral here is a product over x, y, z of one- or two-variable Gaussian
integrals evaluated with Gauss-Hermite quadrature after diagonalising the
quadratic exponent; the rule is exact for the polynomial factors used here.
Coulomb-type kernels are reduced to the Gaussian kernel through
    1/r              = (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt,
    erf(w r)/r       = (2/sqrt(pi)) int_0^w   exp(-t^2 r^2) dt,
    exp(-w r^2)/r    = (2/sqrt(pi)) int_0^inf exp(-(w + t^2) r^2) dt,
with the t-integral done by adaptive quadrature.  None of this uses the Boys
function, Table S1 or any recursion, so it pins the oracle from outside.
"""
import math

import numpy as np
from scipy import integrate

_GH = {n: np.polynomial.hermite.hermgauss(n) for n in (24,)}


def _gauss_poly_integral(M, g, poly, const=0.0):
    """int p(z) exp(-(z^T M z + 2 g^T z + const)) dz over R^d (d = 1 or 2), p given as
    a callable on an (n, d) array of points.  Exact for polynomials of degree
    < 2*24 per variable."""
    M = np.atleast_2d(np.asarray(M, dtype=np.float64))
    g = np.atleast_1d(np.asarray(g, dtype=np.float64))
    d = len(g)
    mu = -np.linalg.solve(M, g)
    q0 = -g @ np.linalg.solve(M, g)               # value of the exponent at mu
    lam, V = np.linalg.eigh(M)
    x, w = _GH[24]
    if d == 1:
        Y = x[:, None]
        W = w
    else:
        X1, X2 = np.meshgrid(x, x, indexing="ij")
        Y = np.stack([X1.ravel(), X2.ravel()], axis=1)
        W = np.outer(w, w).ravel()
    Z = mu[None, :] + (Y / np.sqrt(lam)[None, :]) @ V.T
    val = np.sum(W * poly(Z))
    return math.exp(-(q0 + const)) * val / math.sqrt(np.prod(lam))


def overlap_1d(i, j, alpha, beta, A, B):
    """int (x-A)^i (x-B)^j exp(-alpha (x-A)^2 - beta (x-B)^2) dx."""
    # exponent alpha (x-A)^2 + beta (x-B)^2 = c x^2 - 2 (alpha A + beta B) x + const
    c = alpha + beta
    const = alpha * A * A + beta * B * B
    g = -(alpha * A + beta * B)
    return _gauss_poly_integral([[c]], [g], lambda Z: (Z[:, 0] - A) ** i * (Z[:, 0] - B) ** j, const)


def gauss_op_1d(i, j, alpha, beta, omega, A, B):
    """int int (x1-A)^i (x2-B)^j exp(-alpha (x1-A)^2 - omega (x1-x2)^2 - beta (x2-B)^2) dx1 dx2."""
    u0 = 0.0
    # work in u = x1 - A, v = x2 - B; x1 - x2 = u - v + X
    X = A - B
    M = [[alpha + omega, -omega], [-omega, beta + omega]]
    g = [omega * X, -omega * X]
    const = omega * X * X
    return _gauss_poly_integral(M, g, lambda Z: (Z[:, 0] + u0) ** i * Z[:, 1] ** j, const)


def cart_overlap(a, b, alpha, beta, A, B):
    return np.prod([overlap_1d(a[d], b[d], alpha, beta, A[d], B[d]) for d in range(3)])


def cart_gauss_op(a, b, alpha, beta, omega, A, B):
    return np.prod([gauss_op_1d(a[d], b[d], alpha, beta, omega, A[d], B[d]) for d in range(3)])


def cart_attenuated(a, b, alpha, beta, A, B, t_max, omega0=0.0):
    """(2/sqrt(pi)) int_0^t_max  (a| exp(-(omega0 + t^2) r12^2) |b) dt; t_max = inf gives
    exp(-omega0 r^2)/r (1/r for omega0 = 0)."""
    f = lambda t: cart_gauss_op(a, b, alpha, beta, omega0 + t * t, A, B)
    if math.isinf(t_max):
        # t = s / (1 - s) maps [0, 1) onto [0, inf)
        h = lambda s: f(s / (1.0 - s)) / (1.0 - s) ** 2 if s < 1.0 else 0.0
        val, _ = integrate.quad(h, 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=400)
    else:
        val, _ = integrate.quad(f, 0.0, t_max, epsabs=0.0, epsrel=1e-13, limit=400)
    return 2.0 / math.sqrt(math.pi) * val


def cart_list(l):
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


def cart_integral(op, a, b, alpha, beta, omega, A, B):
    if op == 0:
        return cart_overlap(a, b, alpha, beta, A, B)
    if op == 1:
        return cart_attenuated(a, b, alpha, beta, A, B, math.inf)
    if op == 3:
        return cart_attenuated(a, b, alpha, beta, A, B, omega)
    if op == 2:
        return (cart_attenuated(a, b, alpha, beta, A, B, math.inf)
                - cart_attenuated(a, b, alpha, beta, A, B, omega))
    if op == 4:
        return cart_gauss_op(a, b, alpha, beta, omega, A, B)
    if op == 5:
        return cart_attenuated(a, b, alpha, beta, A, B, math.inf, omega0=omega)
    raise ValueError(op)


def cart_triple_overlap(a, t, b, alpha, alpha_t, beta, A, B):
    """int g_a(alpha) g_t(alpha_t) g_b(beta), g_a and g_t on A."""
    return np.prod([overlap_1d(a[d] + t[d], b[d], alpha + alpha_t, beta, A[d], B[d]) for d in range(3)])


def cart_ra2n(a, b, alpha, beta, A, B, n):
    """int g_a(alpha) |r - A|^{2n} g_b(beta) over R^3 by a 3-D Gauss-Hermite
    product rule about the Gaussian product center (exact: the integrand is a
    polynomial of degree < 48 per variable times the product Gaussian)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    c = alpha + beta
    P = (alpha * A + beta * B) / c
    rho = alpha * beta / c
    x, w = _GH[24]
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    pts = P[None, :] + np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1) / math.sqrt(c)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    da, db = pts - A[None, :], pts - B[None, :]
    poly = np.prod(da ** np.asarray(a)[None, :], axis=1) * np.prod(db ** np.asarray(b)[None, :], axis=1)
    poly = poly * np.sum(da * da, axis=1) ** n
    return math.exp(-rho * float(np.dot(A - B, A - B))) * float(np.sum(W * poly)) / c ** 1.5
