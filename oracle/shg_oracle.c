/*
 * Plain, slow CPU oracle for contracted solid-harmonic Gaussian integrals.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or table with the
 * CUDA path.
 *
 * Route (deliberately different from the SHG scheme it checks):
 *   1. Cartesian primitive Gaussians x_A^i y_A^j z_A^k exp(-alpha r_A^2).
 *   2. A two-center Obara-Saika/Ahlrichs type recursion for any r12 kernel,
 *      seeded with the s-type integrals (0_a|O|0_b)^{(m)} of Table S1 and
 *      written out in the comment above cart_rec() below.
 *   3. Cartesian -> real solid harmonic transformation from the explicit
 *      closed-form coefficient formula for real solid harmonics (not from
 *      the translation-matrix recursion of the SHG scheme).
 *   4. Contraction, then normalisation to unit self-overlap computed with the
 *      oracle's own overlap integrals (not with the closed-form N_l of the
 *      paper, Sec. II A).
 *   5. (ab a~): the two Cartesian Gaussians on A are multiplied into one
 *      Cartesian Gaussian with exponent alpha+alpha~, then the overlap
 *      recursion is run (the Cartesian route described in Sec. III).
 *   6. Gradients: d/dA_x g_a = 2 alpha g_{a+1x} - a_x g_{a-1x} (Cartesian).
 *   7. Boys function: power series (T < 50), else F_0 = sqrt(pi/4T) erf(sqrt T)
 *      with upward recursion; SI Eqs. 3-4 define F_n and dF_n/dx = -F_{n+1}.
 *
 * Compile with -DORACLE_LONG_DOUBLE to run every step in long double (80-bit
 * on x86-64, binary128 on aarch64); used to settle disagreements.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef ORACLE_LONG_DOUBLE
typedef long double real;
#define R_EXP expl
#define R_SQRT sqrtl
#define R_ERF erfl
#define R_FABS fabsl
#define R_PI 3.141592653589793238462643383279502884L
#else
typedef double real;
#define R_EXP exp
#define R_SQRT sqrt
#define R_ERF erf
#define R_FABS fabs
#define R_PI 3.141592653589793238462643383279502884
#endif

enum { OP_OVERLAP = 0, OP_COULOMB = 1, OP_ERFC = 2, OP_ERF = 3, OP_GAUSS = 4, OP_GCOUL = 5 };

#define MAXLA 11  /* |a| on center A: la + la~ <= 10, plus one for gradients */
#define MAXLB 7   /* |b| on center B: lb <= 6, plus one for gradients        */
#define MAXM (MAXLA + MAXLB + 1)
#define NCA 364   /* number of Cartesian triples with |a| <= 11 = C(14,3) */
#define NCB 120   /* number of Cartesian triples with |b| <= 7  = C(10,3) */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Index of (x,y,z), x+y+z = L, among all triples of total <= L; within one L
 * the order is x descending, then y descending. */
static int cidx(int x, int y, int z)
{
    int L = x + y + z;
    return L * (L + 1) * (L + 2) / 6 + (L - x) * (L - x + 1) / 2 + z;
}

/* position of (x,y,z) within its own shell (0 .. ncart(L)-1) */
static int cpos(int x, int y, int z)
{
    int L = x + y + z;
    return (L - x) * (L - x + 1) / 2 + z;
}

/* ------------------------------------------------------------------------ */
/* Boys function F_n(T) = int_0^1 exp(-T t^2) t^{2n} dt,  n = 0..nmax.        */
/* For T < 50 each F_n is summed from the everywhere-convergent series        */
/*   F_n(T) = exp(-T) sum_i (2T)^i / ((2n+1)(2n+3)...(2n+2i+1)),              */
/* which has only positive terms.  For T >= 50, erf(sqrt T) = 1 to far below  */
/* rounding, F_0 = sqrt(pi/(4T)) erf(sqrt T) and the upward recursion         */
/*   F_{n+1} = ((2n+1) F_n - exp(-T)) / (2T)                                  */
/* (from integrating by parts) loses nothing because exp(-T) << (2n+1) F_n.   */
/* ------------------------------------------------------------------------ */
static void boys(int nmax, real T, real *F)
{
    if (T < 50) {
        real e = R_EXP(-T);
        for (int n = 0; n <= nmax; ++n) {
            real term = (real)1 / (real)(2 * n + 1);
            real sum = term;
            for (int i = 1; i < 2000; ++i) {
                term *= (2 * T) / (real)(2 * n + 2 * i + 1);
                sum += term;
                if (term < sum * (real)1e-22) break;
            }
            F[n] = e * sum;
        }
    } else {
        real e = R_EXP(-T);
        F[0] = R_SQRT(R_PI / (4 * T)) * R_ERF(R_SQRT(T));
        for (int n = 0; n < nmax; ++n)
            F[n + 1] = ((2 * n + 1) * F[n] - e) / (2 * T);
    }
}

/* ------------------------------------------------------------------------ */
/* (0_a|O|0_b)^{(m)}, the m-th derivative with respect to R_ab^2 of the       */
/* integral over two primitive s Gaussians, for m = 0..mmax (Table S1, with   */
/* rho = alpha beta/(alpha+beta) and T = rho R^2, SI Eqs. 1-2).               */
/* ------------------------------------------------------------------------ */
static void ss_deriv(int op, real a, real b, real omega, real R2, int mmax, real *G)
{
    real c = a + b;
    real rho = a * b / c;
    real T = rho * R2;
    real F[MAXM + 2], F2[MAXM + 2];
    switch (op) {
    case OP_OVERLAP: {
        real pre = R_SQRT(R_PI / c);
        pre = pre * pre * pre * R_EXP(-T);
        real f = 1;
        for (int m = 0; m <= mmax; ++m) { G[m] = f * pre; f *= -rho; }
        break;
    }
    case OP_COULOMB: {
        real pre = 2 * R_PI * R_PI * R_SQRT(R_PI) / (a * b * R_SQRT(c));
        boys(mmax, T, F);
        real f = 1;
        for (int m = 0; m <= mmax; ++m) { G[m] = pre * f * F[m]; f *= -rho; }
        break;
    }
    case OP_ERF:
    case OP_ERFC: {
        real pre = 2 * R_PI * R_PI * R_SQRT(R_PI) / (a * b * R_SQRT(c));
        real w2 = omega * omega;
        real s = w2 / (w2 + rho);            /* omega^2/(omega^2+rho)            */
        real sq = omega / R_SQRT(w2 + rho);  /* omega/sqrt(omega^2+rho)          */
        boys(mmax, s * T, F2);
        if (op == OP_ERFC) boys(mmax, T, F);
        real f = 1, f2 = 1;
        for (int m = 0; m <= mmax; ++m) {
            real lr = sq * f2 * F2[m];       /* long-range (erf) part            */
            G[m] = (op == OP_ERF) ? pre * lr : pre * (f * F[m] - lr);
            f *= -rho;
            f2 *= -rho * s;                  /* -(omega^2 rho)/(omega^2+rho)     */
        }
        break;
    }
    case OP_GAUSS: {
        real d = rho + omega;
        real base = R_PI * R_PI / (c * d);
        real pre = base * R_SQRT(base) * R_EXP(-omega * T / d);
        real f = 1;
        for (int m = 0; m <= mmax; ++m) { G[m] = f * pre; f *= -omega * rho / d; }
        break;
    }
    case OP_GCOUL: {
        /* exp(-omega r^2)/r (Table S1): (pi/c)^{3/2} 2 pi/d exp(-omega T/d) times, for
         * the n-th derivative, sum_j C(n,j) p^{n-j} q^j F_j(T rho/d) with d = rho + omega,
         * p = -omega rho/d, q = -rho^2/d                                           */
        real d = rho + omega;
        real pre = R_SQRT(R_PI / c);
        pre = pre * pre * pre * (2 * R_PI / d) * R_EXP(-omega * T / d);
        real p = -omega * rho / d, q = -rho * rho / d;
        real pp[MAXM + 2], qq[MAXM + 2];
        boys(mmax, T * rho / d, F);
        pp[0] = qq[0] = 1;
        for (int m = 1; m <= mmax; ++m) { pp[m] = pp[m - 1] * p; qq[m] = qq[m - 1] * q; }
        for (int m = 0; m <= mmax; ++m) {
            real sum = 0, binom = 1;             /* C(m, j) */
            for (int j = 0; j <= m; ++j) {
                sum += binom * pp[m - j] * qq[j] * F[j];
                binom = binom * (m - j) / (j + 1);
            }
            G[m] = pre * sum;
        }
        break;
    }
    default:
        for (int m = 0; m <= mmax; ++m) G[m] = 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Two-center recursion.                                                      */
/*                                                                            */
/* g_a(r) = x_A^ax y_A^ay z_A^az exp(-alpha r_A^2) equals D_a(d/dA) applied   */
/* to exp(-alpha r_A^2), where per direction D_0 = 1 and                      */
/*   D_{i+1}(xi) = (xi D_i(xi) + i D_{i-1}(xi)) / (2 alpha)                   */
/* because d/dA_x (x_A^i e) = -i x_A^{i-1} e + 2 alpha x_A^{i+1} e.  By       */
/* induction dD_i/dxi = i D_{i-1} / (2 alpha).  Hence the integral            */
/* I(a,b) = D_a(d/dA) D_b(d/dB) G(|A-B|^2), G = (0_a|O|0_b).  Define          */
/* I^{(m)}(a,b) the same way with G replaced by G^{(m)} = (d/dR^2)^m G.  With  */
/* X = A - B, d/dA_x G^{(m)} = 2 X_x G^{(m+1)}, and commuting D_a, D_b past   */
/* the factor X_x (commutator = formal derivative of D) gives                 */
/*                                                                            */
/* I^{(m)}(a+1x,b) = [ 2X_x I^{(m+1)}(a,b) + (a_x/alpha) I^{(m+1)}(a-1x,b)    */
/*                    - (b_x/beta) I^{(m+1)}(a,b-1x) + a_x I^{(m)}(a-1x,b) ]  */
/*                   / (2 alpha)                                              */
/* I^{(m)}(a,b+1x) = [ -2X_x I^{(m+1)}(a,b) - (a_x/alpha) I^{(m+1)}(a-1x,b)   */
/*                    + (b_x/beta) I^{(m+1)}(a,b-1x) + b_x I^{(m)}(a,b-1x) ]  */
/*                   / (2 beta)                                               */
/* and I^{(m)}(0,0) = G^{(m)}(R^2).                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    real alpha, beta;
    real X[3];
    real G[MAXM + 2];
    real *memo;       /* NCA * NCB * (MAXM+1) */
    uint32_t *stamp;  /* generation stamps, same size */
    uint32_t gen;
} rec_ctx;

static rec_ctx *ctx_new(void)
{
    rec_ctx *c = (rec_ctx *)calloc(1, sizeof(rec_ctx));
    size_t n = (size_t)NCA * NCB * (MAXM + 1);
    c->memo = (real *)malloc(n * sizeof(real));
    c->stamp = (uint32_t *)calloc(n, sizeof(uint32_t));
    c->gen = 0;
    return c;
}

static void ctx_free(rec_ctx *c)
{
    if (!c) return;
    free(c->memo);
    free(c->stamp);
    free(c);
}

static void ctx_begin(rec_ctx *c, int op, real a, real b, real omega, const real *A, const real *B, int mmax)
{
    c->alpha = a;
    c->beta = b;
    real R2 = 0;
    for (int i = 0; i < 3; ++i) { c->X[i] = A[i] - B[i]; R2 += c->X[i] * c->X[i]; }
    ss_deriv(op, a, b, omega, R2, mmax, c->G);
    c->gen++;
    if (c->gen == 0) {  /* wrapped: clear stamps */
        memset(c->stamp, 0, (size_t)NCA * NCB * (MAXM + 1) * sizeof(uint32_t));
        c->gen = 1;
    }
}

static real cart_rec(rec_ctx *c, const int *a, const int *b, int m)
{
    if (a[0] < 0 || a[1] < 0 || a[2] < 0 || b[0] < 0 || b[1] < 0 || b[2] < 0) return 0;
    size_t idx = ((size_t)cidx(a[0], a[1], a[2]) * NCB + (size_t)cidx(b[0], b[1], b[2])) * (MAXM + 1) + (size_t)m;
    if (c->stamp[idx] == c->gen) return c->memo[idx];
    int la = a[0] + a[1] + a[2], lb = b[0] + b[1] + b[2];
    real v;
    if (la == 0 && lb == 0) {
        v = c->G[m];
    } else if (la > 0) {
        int i = a[0] > 0 ? 0 : (a[1] > 0 ? 1 : 2);
        int ap[3] = {a[0], a[1], a[2]};
        ap[i] -= 1;                              /* a = ap + 1_i */
        int am[3] = {ap[0], ap[1], ap[2]};
        am[i] -= 1;                              /* ap - 1_i     */
        int bm[3] = {b[0], b[1], b[2]};
        bm[i] -= 1;                              /* b - 1_i      */
        v = 2 * c->X[i] * cart_rec(c, ap, b, m + 1);
        if (ap[i] > 0) v += (ap[i] / c->alpha) * cart_rec(c, am, b, m + 1) + ap[i] * cart_rec(c, am, b, m);
        if (b[i] > 0) v -= (b[i] / c->beta) * cart_rec(c, ap, bm, m + 1);
        v /= 2 * c->alpha;
    } else {
        int i = b[0] > 0 ? 0 : (b[1] > 0 ? 1 : 2);
        int bp[3] = {b[0], b[1], b[2]};
        bp[i] -= 1;                              /* b = bp + 1_i */
        int bm[3] = {bp[0], bp[1], bp[2]};
        bm[i] -= 1;
        v = -2 * c->X[i] * cart_rec(c, a, bp, m + 1);
        if (bp[i] > 0) v += (bp[i] / c->beta) * cart_rec(c, a, bm, m + 1) + bp[i] * cart_rec(c, a, bm, m);
        v /= 2 * c->beta;
    }
    c->memo[idx] = v;
    c->stamp[idx] = c->gen;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Real solid harmonics S_{l,m} (unit-normalised convention: S_{1,1} = x,     */
/* S_{1,-1} = y, S_{1,0} = z) as polynomials in Cartesian monomials, from the */
/* explicit closed form                                                       */
/*  S_lm = N_lm sum_t sum_u sum_v C^{lm}_{tuv} x^{2t+|m|-2(u+v)} y^{2(u+v)}   */
/*                                   z^{l-2t-|m|}                              */
/*  C^{lm}_{tuv} = (-1)^{t+v-v_m} (1/4)^t binom(l,t) binom(l-t,|m|+t)         */
/*                 binom(t,u) binom(|m|,2v)                                   */
/*  N_lm = sqrt(2 (l+|m|)! (l-|m|)! / 2^{delta_m0}) / (2^|m| l!)              */
/* with v_m = 0 (m >= 0) or 1/2 (m < 0); v runs over v_m, v_m+1, ... .        */
/* T has (2l+1) rows, m = -l..l, and ncart(l) columns in cpos() order.        */
/* ------------------------------------------------------------------------ */
static real fact(int n) { real f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }
static real binom(int n, int k) { if (k < 0 || k > n) return 0; return fact(n) / (fact(k) * fact(n - k)); }

static void sph_coef(int l, real *T)
{
    int nc = ncart(l);
    memset(T, 0, sizeof(real) * (size_t)(2 * l + 1) * (size_t)nc);
    for (int m = -l; m <= l; ++m) {
        int mu = m < 0 ? -m : m;
        int twovm = m < 0 ? 1 : 0;                      /* 2 v_m */
        real N = R_SQRT(2 * fact(l + mu) * fact(l - mu) / (m == 0 ? 2 : 1)) / (real)((1L << mu) * fact(l));
        real *row = T + (size_t)(m + l) * nc;
        for (int t = 0; t <= (l - mu) / 2; ++t)
            for (int u = 0; u <= t; ++u)
                for (int twov = twovm; twov <= mu; twov += 2) {
                    int sgn_exp = t + (twov - twovm) / 2;
                    real C = ((sgn_exp & 1) ? -1 : 1) * binom(l, t) * binom(l - t, mu + t) * binom(t, u) * binom(mu, twov);
                    for (int k = 0; k < t; ++k) C /= 4;
                    int px = 2 * t + mu - 2 * u - twov;
                    int py = 2 * u + twov;
                    int pz = l - 2 * t - mu;
                    if (px < 0 || pz < 0) continue;
                    row[cpos(px, py, pz)] += N * C;
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Exported helpers                                                           */
/* ------------------------------------------------------------------------ */
int oracle_boys(int nmax, double T, double *F)
{
    real Fr[64];
    if (nmax < 0 || nmax > 60) return -1;
    boys(nmax, (real)T, Fr);
    for (int n = 0; n <= nmax; ++n) F[n] = (double)Fr[n];
    return 0;
}

int oracle_ss(int op, double a, double b, double omega, double R2, int mmax, double *G)
{
    real Gr[MAXM + 2];
    if (mmax < 0 || mmax > MAXM) return -1;
    ss_deriv(op, a, b, omega, R2, mmax, Gr);
    for (int m = 0; m <= mmax; ++m) G[m] = (double)Gr[m];
    return 0;
}

int oracle_sph_coef(int l, double *T)
{
    if (l < 0 || l > MAXLA) return -1;
    int n = (2 * l + 1) * ncart(l);
    real *Tr = (real *)malloc(sizeof(real) * (size_t)n);
    sph_coef(l, Tr);
    for (int i = 0; i < n; ++i) T[i] = (double)Tr[i];
    free(Tr);
    return 0;
}

/* Primitive Cartesian block I^{(0)}(a,b), |a| = la, |b| = lb, rows in cpos order. */
int oracle_cart_2c(int op, double omega, int la, int lb, double alpha, double beta,
                   const double *A, const double *B, double *out)
{
    if (la < 0 || la > MAXLA || lb < 0 || lb > MAXLB) return -1;
    rec_ctx *c = ctx_new();
    real Ar[3] = {A[0], A[1], A[2]}, Br[3] = {B[0], B[1], B[2]};
    ctx_begin(c, op, alpha, beta, omega, Ar, Br, la + lb);
    int nb = ncart(lb);
    for (int ax = la; ax >= 0; --ax)
        for (int ay = la - ax; ay >= 0; --ay) {
            int a[3] = {ax, ay, la - ax - ay};
            for (int bx = lb; bx >= 0; --bx)
                for (int by = lb - bx; by >= 0; --by) {
                    int b[3] = {bx, by, lb - bx - by};
                    out[cpos(a[0], a[1], a[2]) * nb + cpos(b[0], b[1], b[2])] = (double)cart_rec(c, a, b, 0);
                }
        }
    ctx_free(c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Shell data                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n_shells;
    const int32_t *l, *nprim;
    const int64_t *prim_off;
    const double *exps, *coefs, *centers;
    const int32_t *center_of;
} shells_t;

/* Unit-self-overlap normalisation factor of a contracted shell, from the
 * oracle's own overlap integrals at R = 0 (component m = 0). */
static real shell_norm(rec_ctx *c, const shells_t *S, int s, const real *Tsph)
{
    int l = S->l[s], K = S->nprim[s];
    int nc = ncart(l);
    const real *row = Tsph + (size_t)l * nc;       /* m = 0 row */
    real zero[3] = {0, 0, 0};
    real sum = 0;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            real ai = S->exps[S->prim_off[s] + i], aj = S->exps[S->prim_off[s] + j];
            real ci = S->coefs[S->prim_off[s] + i], cj = S->coefs[S->prim_off[s] + j];
            ctx_begin(c, OP_OVERLAP, ai, aj, 0, zero, zero, 2 * l);
            real acc = 0;
            for (int ax = l; ax >= 0; --ax)
                for (int ay = l - ax; ay >= 0; --ay) {
                    int a[3] = {ax, ay, l - ax - ay};
                    real ta = row[cpos(a[0], a[1], a[2])];
                    if (ta == 0) continue;
                    for (int bx = l; bx >= 0; --bx)
                        for (int by = l - bx; by >= 0; --by) {
                            int b[3] = {bx, by, l - bx - by};
                            real tb = row[cpos(b[0], b[1], b[2])];
                            if (tb == 0) continue;
                            acc += ta * tb * cart_rec(c, a, b, 0);
                        }
                }
            sum += ci * cj * acc;
        }
    return 1 / R_SQRT(sum);
}

/* per-thread work space */
typedef struct {
    rec_ctx *c;
    real *tsph[MAXLA + 1];
} work_t;

static void work_init(work_t *w)
{
    w->c = ctx_new();
    for (int l = 0; l <= MAXLA; ++l) {
        w->tsph[l] = (real *)malloc(sizeof(real) * (size_t)(2 * l + 1) * (size_t)ncart(l));
        sph_coef(l, w->tsph[l]);
    }
}

static void work_free(work_t *w)
{
    ctx_free(w->c);
    for (int l = 0; l <= MAXLA; ++l) free(w->tsph[l]);
}

static void get_center(const shells_t *S, int s, real *P)
{
    const double *p = S->centers + 3 * (size_t)S->center_of[s];
    P[0] = p[0]; P[1] = p[1]; P[2] = p[2];
}

/*
 * Contracted, normalised two-center block of one pair.
 * deriv = 0: the integrals (a|O|b), out[(2la+1)(2lb+1)], rows m_a, columns m_b.
 * deriv = 1: d/dA_{x,y,z} of the block, out[3][(2la+1)(2lb+1)], via
 *            d/dA_x g_a = 2 alpha g_{a+1x} - a_x g_{a-1x}.
 * deriv = 2: d/dB_{x,y,z}, via the same identity on g_b.
 */
static void pair_2c(work_t *w, const shells_t *S, int sa, int sb, int op, real omega, int deriv, int normalize,
                    double *out)
{
    int la = S->l[sa], lb = S->l[sb];
    int nca = ncart(la), ncb = ncart(lb);
    int na = 2 * la + 1, nb = 2 * lb + 1;
    real A[3], B[3];
    get_center(S, sa, A);
    get_center(S, sb, B);
    real Na = normalize ? shell_norm(w->c, S, sa, w->tsph[la]) : 1;
    real Nb = normalize ? shell_norm(w->c, S, sb, w->tsph[lb]) : 1;
    int ncomp = deriv ? 3 : 1;
    real *C = (real *)calloc((size_t)ncomp * nca * ncb, sizeof(real));
    for (int i = 0; i < S->nprim[sa]; ++i)
        for (int j = 0; j < S->nprim[sb]; ++j) {
            real al = S->exps[S->prim_off[sa] + i], be = S->exps[S->prim_off[sb] + j];
            real cc = (real)S->coefs[S->prim_off[sa] + i] * (real)S->coefs[S->prim_off[sb] + j];
            ctx_begin(w->c, op, al, be, omega, A, B, la + lb + (deriv ? 1 : 0));
            for (int ax = la; ax >= 0; --ax)
                for (int ay = la - ax; ay >= 0; --ay) {
                    int a[3] = {ax, ay, la - ax - ay};
                    int pa = cpos(a[0], a[1], a[2]);
                    for (int bx = lb; bx >= 0; --bx)
                        for (int by = lb - bx; by >= 0; --by) {
                            int b[3] = {bx, by, lb - bx - by};
                            int pb = cpos(b[0], b[1], b[2]);
                            if (!deriv) {
                                C[pa * ncb + pb] += cc * cart_rec(w->c, a, b, 0);
                            } else {
                                for (int d = 0; d < 3; ++d) {
                                    int up[3], dn[3], base[3];
                                    const int *f = (deriv == 1) ? a : b;
                                    real ex = (deriv == 1) ? al : be;
                                    for (int k = 0; k < 3; ++k) { up[k] = f[k]; dn[k] = f[k]; base[k] = f[k]; }
                                    up[d] += 1;
                                    dn[d] -= 1;
                                    real v;
                                    if (deriv == 1)
                                        v = 2 * ex * cart_rec(w->c, up, b, 0) - (base[d] > 0 ? base[d] * cart_rec(w->c, dn, b, 0) : 0);
                                    else
                                        v = 2 * ex * cart_rec(w->c, a, up, 0) - (base[d] > 0 ? base[d] * cart_rec(w->c, a, dn, 0) : 0);
                                    C[((size_t)d * nca + pa) * ncb + pb] += cc * v;
                                }
                            }
                        }
                }
        }
    const real *Ta = w->tsph[la], *Tb = w->tsph[lb];
    for (int d = 0; d < ncomp; ++d)
        for (int ma = 0; ma < na; ++ma)
            for (int mb = 0; mb < nb; ++mb) {
                real acc = 0;
                for (int pa = 0; pa < nca; ++pa) {
                    real ta = Ta[ma * nca + pa];
                    if (ta == 0) continue;
                    for (int pb = 0; pb < ncb; ++pb) {
                        real tb = Tb[mb * ncb + pb];
                        if (tb == 0) continue;
                        acc += ta * tb * C[((size_t)d * nca + pa) * ncb + pb];
                    }
                }
                out[(size_t)d * na * nb + ma * nb + mb] = (double)(Na * Nb * acc);
            }
    free(C);
}

/* ------------------------------------------------------------------------ */
/* (a|r_a^{2n}|b) (Sec. II C) by a route independent of the SHG formula:     */
/* r_A^{2n} = (x_A^2 + y_A^2 + z_A^2)^n is expanded multinomially, each term  */
/* raising the Cartesian powers on A by (2p, 2q, 2s); the overlap of two      */
/* Cartesian Gaussians factorises over x, y, z and each 1-D factor has the    */
/* textbook closed form (Gaussian product theorem, binomial expansion about   */
/* P = (alpha A + beta B)/c, even moments of exp(-c t^2)):                     */
/*   int (x-A)^i (x-B)^j exp(-alpha (x-A)^2 - beta (x-B)^2) dx                */
/*     = exp(-rho X^2) sum_{k<=i, l<=j} C(i,k) C(j,l) (P-A)^{i-k} (P-B)^{j-l}  */
/*       M_{k+l},   M_t = sqrt(pi/c) (t-1)!! / (2c)^{t/2} (t even), 0 (t odd). */
/* ------------------------------------------------------------------------ */
static real ipow(real x, int n) { real r = 1; for (int i = 0; i < n; ++i) r *= x; return r; }

static real ov1d(int i, int j, real alpha, real beta, real A, real B)
{
    if (i < 0 || j < 0) return 0;
    real c = alpha + beta, rho = alpha * beta / c;
    real P = (alpha * A + beta * B) / c, X = A - B;
    real sum = 0;
    for (int k = 0; k <= i; ++k)
        for (int l = 0; l <= j; ++l) {
            int t = k + l;
            if (t & 1) continue;
            real m = R_SQRT(R_PI / c);
            for (int u = t - 1; u > 0; u -= 2) m *= u;
            for (int u = 0; u < t / 2; ++u) m /= 2 * c;
            sum += binom(i, k) * binom(j, l) * ipow(P - A, i - k) * ipow(P - B, j - l) * m;
        }
    return R_EXP(-rho * X * X) * sum;
}

/* Cartesian primitive integral of g_a r_A^{2n} against g_b; deriv = 1: d/dA_dir,
 * deriv = 2: d/dB_dir (d/dA_x of (x-A)^e exp(-alpha (x-A)^2) is
 * 2 alpha (x-A)^{e+1} exp(..) - e (x-A)^{e-1} exp(..), the same on B). */
static real cart_ra2n(const int *a, const int *b, int n, real al, real be, const real *A, const real *B, int deriv,
                      int dir)
{
    real tot = 0;
    for (int p = 0; p <= n; ++p)
        for (int q = 0; q <= n - p; ++q) {
            int r = n - p - q;
            real mult = fact(n) / (fact(p) * fact(q) * fact(r));
            int e[3] = {a[0] + 2 * p, a[1] + 2 * q, a[2] + 2 * r};
            real f = 1;
            for (int d = 0; d < 3; ++d) {
                real v;
                if (deriv == 1 && d == dir)
                    v = 2 * al * ov1d(e[d] + 1, b[d], al, be, A[d], B[d]) - e[d] * ov1d(e[d] - 1, b[d], al, be, A[d], B[d]);
                else if (deriv == 2 && d == dir)
                    v = 2 * be * ov1d(e[d], b[d] + 1, al, be, A[d], B[d]) - b[d] * ov1d(e[d], b[d] - 1, al, be, A[d], B[d]);
                else
                    v = ov1d(e[d], b[d], al, be, A[d], B[d]);
                f *= v;
            }
            tot += mult * f;
        }
    return tot;
}

/* Contracted, normalised block of (a|r_a^{2n}|b) (deriv as in pair_2c). */
static void pair_ra2n(work_t *w, const shells_t *S, int sa, int sb, int n, int deriv, int normalize, double *out)
{
    int la = S->l[sa], lb = S->l[sb];
    int nca = ncart(la), ncb = ncart(lb);
    int na = 2 * la + 1, nb = 2 * lb + 1;
    real A[3], B[3];
    get_center(S, sa, A);
    get_center(S, sb, B);
    real Na = normalize ? shell_norm(w->c, S, sa, w->tsph[la]) : 1;
    real Nb = normalize ? shell_norm(w->c, S, sb, w->tsph[lb]) : 1;
    int ncomp = deriv ? 3 : 1;
    real *C = (real *)calloc((size_t)ncomp * nca * ncb, sizeof(real));
    for (int i = 0; i < S->nprim[sa]; ++i)
        for (int j = 0; j < S->nprim[sb]; ++j) {
            real al = S->exps[S->prim_off[sa] + i], be = S->exps[S->prim_off[sb] + j];
            real cc = (real)S->coefs[S->prim_off[sa] + i] * (real)S->coefs[S->prim_off[sb] + j];
            for (int ax = la; ax >= 0; --ax)
                for (int ay = la - ax; ay >= 0; --ay) {
                    int a[3] = {ax, ay, la - ax - ay};
                    int pa = cpos(a[0], a[1], a[2]);
                    for (int bx = lb; bx >= 0; --bx)
                        for (int by = lb - bx; by >= 0; --by) {
                            int b[3] = {bx, by, lb - bx - by};
                            int pb = cpos(b[0], b[1], b[2]);
                            for (int d = 0; d < ncomp; ++d)
                                C[((size_t)d * nca + pa) * ncb + pb] += cc * cart_ra2n(a, b, n, al, be, A, B, deriv, d);
                        }
                }
        }
    const real *Ta = w->tsph[la], *Tb = w->tsph[lb];
    for (int d = 0; d < ncomp; ++d)
        for (int ma = 0; ma < na; ++ma)
            for (int mb = 0; mb < nb; ++mb) {
                real acc = 0;
                for (int pa = 0; pa < nca; ++pa) {
                    real ta = Ta[ma * nca + pa];
                    if (ta == 0) continue;
                    for (int pb = 0; pb < ncb; ++pb) {
                        real tb = Tb[mb * ncb + pb];
                        if (tb == 0) continue;
                        acc += ta * tb * C[((size_t)d * nca + pa) * ncb + pb];
                    }
                }
                out[(size_t)d * na * nb + ma * nb + mb] = (double)(Na * Nb * acc);
            }
    free(C);
}

/*
 * Contracted, normalised three-index overlap (a b a~) = int phi_a phi_a~ phi_b,
 * with a and a~ on the same center A.  Output block [m_a][m_a~][m_b].
 * deriv = 1: d/dA (both functions on A move), out[3][block], product rule.
 * deriv = 2: d/dB, out[3][block].
 */
static void triple_aab(work_t *w, const shells_t *S, int sa, int st, int sb, int deriv, int normalize, double *out)
{
    int la = S->l[sa], lt = S->l[st], lb = S->l[sb];
    int nca = ncart(la), nct = ncart(lt), ncb = ncart(lb);
    int na = 2 * la + 1, nt = 2 * lt + 1, nb = 2 * lb + 1;
    real A[3], B[3];
    get_center(S, sa, A);
    get_center(S, sb, B);
    real Na = normalize ? shell_norm(w->c, S, sa, w->tsph[la]) : 1;
    real Nt = normalize ? shell_norm(w->c, S, st, w->tsph[lt]) : 1;
    real Nb = normalize ? shell_norm(w->c, S, sb, w->tsph[lb]) : 1;
    int ncomp = deriv ? 3 : 1;
    size_t csz = (size_t)nca * nct * ncb;
    real *C = (real *)calloc((size_t)ncomp * csz, sizeof(real));
    for (int i = 0; i < S->nprim[sa]; ++i)
        for (int k = 0; k < S->nprim[st]; ++k)
            for (int j = 0; j < S->nprim[sb]; ++j) {
                real al = S->exps[S->prim_off[sa] + i] + S->exps[S->prim_off[st] + k];
                real be = S->exps[S->prim_off[sb] + j];
                real cc = (real)S->coefs[S->prim_off[sa] + i] * (real)S->coefs[S->prim_off[st] + k] *
                          (real)S->coefs[S->prim_off[sb] + j];
                ctx_begin(w->c, OP_OVERLAP, al, be, 0, A, B, la + lt + lb + (deriv ? 1 : 0));
                for (int ax = la; ax >= 0; --ax)
                    for (int ay = la - ax; ay >= 0; --ay) {
                        int a[3] = {ax, ay, la - ax - ay};
                        int pa = cpos(a[0], a[1], a[2]);
                        for (int tx = lt; tx >= 0; --tx)
                            for (int ty = lt - tx; ty >= 0; --ty) {
                                int t[3] = {tx, ty, lt - tx - ty};
                                int pt = cpos(t[0], t[1], t[2]);
                                int p[3] = {a[0] + t[0], a[1] + t[1], a[2] + t[2]};
                                for (int bx = lb; bx >= 0; --bx)
                                    for (int by = lb - bx; by >= 0; --by) {
                                        int b[3] = {bx, by, lb - bx - by};
                                        int pb = cpos(b[0], b[1], b[2]);
                                        size_t o = ((size_t)pa * nct + pt) * ncb + pb;
                                        if (!deriv) {
                                            C[o] += cc * cart_rec(w->c, p, b, 0);
                                            continue;
                                        }
                                        for (int d = 0; d < 3; ++d) {
                                            real v;
                                            if (deriv == 1) {
                                                int up[3] = {p[0], p[1], p[2]}, dn[3] = {p[0], p[1], p[2]};
                                                up[d] += 1;
                                                dn[d] -= 1;
                                                v = 2 * al * cart_rec(w->c, up, b, 0);
                                                if (p[d] > 0) v -= p[d] * cart_rec(w->c, dn, b, 0);
                                            } else {
                                                int up[3] = {b[0], b[1], b[2]}, dn[3] = {b[0], b[1], b[2]};
                                                up[d] += 1;
                                                dn[d] -= 1;
                                                v = 2 * be * cart_rec(w->c, p, up, 0);
                                                if (b[d] > 0) v -= b[d] * cart_rec(w->c, p, dn, 0);
                                            }
                                            C[(size_t)d * csz + o] += cc * v;
                                        }
                                    }
                            }
                    }
            }
    const real *Ta = w->tsph[la], *Tt = w->tsph[lt], *Tb = w->tsph[lb];
    for (int d = 0; d < ncomp; ++d)
        for (int ma = 0; ma < na; ++ma)
            for (int mt = 0; mt < nt; ++mt)
                for (int mb = 0; mb < nb; ++mb) {
                    real acc = 0;
                    for (int pa = 0; pa < nca; ++pa) {
                        real ta = Ta[ma * nca + pa];
                        if (ta == 0) continue;
                        for (int pt = 0; pt < nct; ++pt) {
                            real tt = Tt[mt * nct + pt];
                            if (tt == 0) continue;
                            for (int pb = 0; pb < ncb; ++pb) {
                                real tb = Tb[mb * ncb + pb];
                                if (tb == 0) continue;
                                acc += ta * tt * tb * C[(size_t)d * csz + ((size_t)pa * nct + pt) * ncb + pb];
                            }
                        }
                    }
                    out[(size_t)d * na * nt * nb + ((size_t)ma * nt + mt) * nb + mb] = (double)(Na * Nt * Nb * acc);
                }
    free(C);
}

static int check_shells(const shells_t *S, int maxl)
{
    for (int s = 0; s < S->n_shells; ++s) {
        if (S->l[s] < 0 || S->l[s] > maxl || S->nprim[s] < 1) return -1;
    }
    return 0;
}

/*
 * Normalisation factors of all shells (unit self-overlap, oracle's own route).
 */
int oracle_shell_norms(int n_shells, const int32_t *l, const int32_t *nprim, const int64_t *prim_off,
                       const double *exps, const double *coefs, double *norms)
{
    shells_t S = {n_shells, l, nprim, prim_off, exps, coefs, NULL, NULL};
    if (check_shells(&S, 6)) return -1;
    work_t w;
    work_init(&w);
    for (int s = 0; s < n_shells; ++s) norms[s] = (double)shell_norm(w.c, &S, s, w.tsph[l[s]]);
    work_free(&w);
    return 0;
}

/*
 * Batched two-center blocks.  deriv as in pair_2c; for deriv > 0 each pair
 * writes 3 consecutive blocks starting at out + 3*offsets[p].  normalize = 0
 * uses the coefficients as given (no unit-self-overlap factor).
 */
int oracle_eval_2c(int n_shells, const int32_t *l, const int32_t *nprim, const int64_t *prim_off,
                   const double *exps, const double *coefs, const double *centers, const int32_t *center_of,
                   int64_t n_pairs, const int32_t *pa, const int32_t *pb, int op, double omega, int deriv,
                   int normalize, const int64_t *offsets, double *out, int nthreads)
{
    shells_t S = {n_shells, l, nprim, prim_off, exps, coefs, centers, center_of};
    if (check_shells(&S, 6)) return -1;
    if (op < 0 || op > 5) return -2;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        work_t w;
        work_init(&w);
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < n_pairs; ++p)
            pair_2c(&w, &S, pa[p], pb[p], op, (real)omega, deriv, normalize, out + (deriv ? 3 : 1) * offsets[p]);
        work_free(&w);
    }
    return 0;
}

/*
 * (a|r_a^{2n}|b) blocks, 0 <= n <= 8 (n = 0 is the overlap); layout and
 * deriv/normalize as oracle_eval_2c.
 */
int oracle_eval_2c_ra2n(int n_shells, const int32_t *l, const int32_t *nprim, const int64_t *prim_off,
                        const double *exps, const double *coefs, const double *centers, const int32_t *center_of,
                        int64_t n_pairs, const int32_t *pa, const int32_t *pb, int n, int deriv, int normalize,
                        const int64_t *offsets, double *out, int nthreads)
{
    shells_t S = {n_shells, l, nprim, prim_off, exps, coefs, centers, center_of};
    if (check_shells(&S, 6)) return -1;
    if (n < 0 || n > 8) return -2;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        work_t w;
        work_init(&w);
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < n_pairs; ++p)
            pair_ra2n(&w, &S, pa[p], pb[p], n, deriv, normalize, out + (deriv ? 3 : 1) * offsets[p]);
        work_free(&w);
    }
    return 0;
}

int oracle_eval_3c_aab(int n_shells, const int32_t *l, const int32_t *nprim, const int64_t *prim_off,
                       const double *exps, const double *coefs, const double *centers, const int32_t *center_of,
                       int64_t n_triples, const int32_t *ta, const int32_t *tt, const int32_t *tb, int deriv,
                       int normalize, const int64_t *offsets, double *out, int nthreads)
{
    shells_t S = {n_shells, l, nprim, prim_off, exps, coefs, centers, center_of};
    if (check_shells(&S, 6)) return -1;
    for (int64_t p = 0; p < n_triples; ++p)
        if (center_of[ta[p]] != center_of[tt[p]]) return -3;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        work_t w;
        work_init(&w);
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < n_triples; ++p)
            triple_aab(&w, &S, ta[p], tt[p], tb[p], deriv, normalize, out + (deriv ? 3 : 1) * offsets[p]);
        work_free(&w);
    }
    return 0;
}
