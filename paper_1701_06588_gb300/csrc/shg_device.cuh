// Device helpers shared by the SHG kernels: Boys function, scaled solid
// harmonics R^{c/s}_{l,m}, rows of the real translation matrix W (Sec. II E).
#pragma once

#include "shg_internal.h"

namespace shg {
namespace dev {

constexpr double kPi32 = 5.568327996831707845284817982118835702;      // pi^{3/2}
constexpr double kTwoPi52 = 34.98683665524972569252564335974;         // 2 pi^{5/2}
constexpr double kPi3 = 31.00627668029982017547631506710139520;       // pi^3
constexpr double kSqrtPiHalf = 0.886226925452758013649083741670572591; // sqrt(pi)/2
constexpr double kPi = 3.141592653589793238462643383279502884;        // pi

enum { OP_OVERLAP = 0, OP_COULOMB = 1, OP_ERFC = 2, OP_ERF = 3, OP_GAUSS = 4, OP_GCOUL = 5, OP_RA2N = 6,
       OP_PRE = 7 /* contracted radial terms precomputed (family path) */ };

// ------------------------------------------------------------------------- //
// Boys function F_k(T), k = kmax-J+1 .. kmax, into F[j] = F_{kmax-j}.       //
// T < 120: Taylor expansion of F_kmax about the nearest grid point         //
//   F_n(T_i + d) = sum_t F_{n+t}(T_i) (-d)^t / t!  (dF_n/dT = -F_{n+1}, SI  //
//   Eq. 4) and exp(-T) = exp(-T_i) exp(-d);                                //
// T >= 120: the asymptotic F_kmax (terms with exp(-T) < 1e-52 dropped);    //
// then, for both, the stable downward recursion                            //
//   F_{k-1} = (2T F_k + exp(-T)) / (2k-1).                                 //
// The two branches differ only in how F_kmax and exp(-T) are obtained, so  //
// a warp whose lanes straddle T = 120 runs both short heads and one tail.  //
//                                                                          //
// Grid T_i = i/32, |d| <~ 1/64: seven terms leave a remainder below        //
// (1/64)^7/7! = 5e-17 of F (F_{n+t} <= F_n).  Terms 0..3 are summed in      //
// FP64; terms 4..6, together at most (1/64)^4/4! = 2.5e-9 of F, in FP32     //
// (relative error ~2e-7 there, so ~5e-16 of F), which moves three of the    //
// seven multiply-adds of each series off the FP64 pipe.  The float <->      //
// double conversions are done on the integer pipe (dbl_to_flt, flt_to_dbl). //
// ------------------------------------------------------------------------- //
__device__ __forceinline__ double powi(double x, int n);

// float with the sign, exponent and leading 23 significand bits of x
// (truncated); 0 when |x| is below the normal float range.  For |x| < 2^127.
__device__ __forceinline__ float dbl_to_flt(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;                     // float exponent field
    const unsigned b = (hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return e > 0 ? __uint_as_float(b) : 0.0f;
}

// the double equal to x (normal x or 0; denormal floats read as 0)
__device__ __forceinline__ double flt_to_dbl(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return e ? __hiloint2double((int)hi, (int)(b << 29)) : 0.0;
}

// One Taylor head: grid index i and y = T_i - T (exact) for 0 <= T < kBoysTmax.
// The index is rounded from the float of 32 T (dbl_to_flt truncates, 32 T
// < 3840 loses at most 5e-4), so |y| <= 1/64 + 2e-5; adding 1.5 * 2^23
// rounds to an integer held in the low bits of the float, and T_i = i / 32 is
// exact in FP32, so only y itself is an FP64 operation.
__device__ __forceinline__ int boys_grid(double T, double &y)
{
    constexpr float kRound = 12582912.0f;                     // 1.5 * 2^23
    const float t = fmaf(dbl_to_flt(T), 32.0f, kRound);
    y = flt_to_dbl((t - kRound) * 0.03125f) - T;
    return __float_as_int(t) - __float_as_int(kRound);
}

// F_n(T) from the entry of (i, n): c0..c3 in FP64, c4..c6 in FP32 (see above)
__device__ __forceinline__ double boys_series(const double *__restrict__ tab, int i, int n, double y)
{
    const double *c = tab + ((size_t)i * kBoysN + n) * kBoysStride;
    const double2 c01 = __ldg(reinterpret_cast<const double2 *>(c));
    const double2 c23 = __ldg(reinterpret_cast<const double2 *>(c) + 1);
    const float4 c46 = __ldg(reinterpret_cast<const float4 *>(c + 4));
    const float yf = dbl_to_flt(y);
    const float t = fmaf(fmaf(c46.z, yf, c46.y), yf, c46.x);
    double f = fma(flt_to_dbl(t), y, c23.y);
    f = fma(f, y, c23.x);
    f = fma(f, y, c01.y);
    return fma(f, y, c01.x);
}

// exp(-T) = exp(-T_i) exp(y), |y| <= 1/64: Taylor to degree 6 (remainder
// < 5e-17), terms 4..6 in FP32 as for F
__device__ __forceinline__ double boys_exp(const double *__restrict__ etab, int i, double y)
{
    const float yf = dbl_to_flt(y);
    const float t = fmaf(fmaf(1.0f / 720.0f, yf, 1.0f / 120.0f), yf, 1.0f / 24.0f);
    double x = fma(flt_to_dbl(t), y, 1.0 / 6.0);
    x = fma(x, y, 0.5);
    x = fma(x, y, 1.0);
    x = fma(x, y, 1.0);
    return x * __ldg(etab + i);
}

// F_kmax by the Taylor head of the table, T < kBoysTmax; with NeedE also
// exp(-T) (else e is left untouched).
template <bool NeedE>
__device__ __forceinline__ void boys_head_near(double T, int kmax, const double *__restrict__ tab,
                                               const double *__restrict__ etab, double &f, double &e)
{
    double y;
    const int i = boys_grid(T, y);
    f = boys_series(tab, i, kmax, y);
    if (NeedE) e = boys_exp(etab, i, y);
}

// F_kmax and exp(-T) (0 where it is below 1e-52).
__device__ __forceinline__ void boys_head(double T, int kmax, const double *__restrict__ tab,
                                          const double *__restrict__ etab, const Consts &k, double &f, double &e)
{
    if (T < kBoysTmax) {
        double y;
        const int i = boys_grid(T, y);
        f = boys_series(tab, i, kmax, y);
        e = boys_exp(etab, i, y);
    } else {
        // F_kmax = (2kmax-1)!! (2T)^-kmax sqrt(pi/(4T)); exp(-T) < 1e-52 is dropped
        const double rT = rsqrt(T);
        f = k.dfact[kmax] * powi(0.5 * rT * rT, kmax) * (kSqrtPiHalf * rT);
        e = 0.0;
    }
}

// e returns exp(-T) as the head computes it (0 for T >= kBoysTmax, where exp(-T) < 1e-52).
template <int J>
__device__ __forceinline__ void boys_top(double T, int kmax, const double *__restrict__ tab,
                                         const double *__restrict__ etab, const Consts &k, double (&F)[J], double &e)
{
    double f;
    boys_head(T, kmax, tab, etab, k, f, e);
    // downward recursion F_{k-1} = (2T F_k + exp(-T)) / (2k-1), shared by both branches
    F[0] = f;
    const double twoT = T + T;
#pragma unroll
    for (int j = 1; j < J; ++j) {
        const int kk = kmax - j + 1;
        F[j] = fma(twoT, F[j - 1], e) * k.inv_int[2 * kk - 1];
    }
}

template <int J>
__device__ __forceinline__ void boys_top(double T, int kmax, const double *__restrict__ tab,
                                         const double *__restrict__ etab, const Consts &k, double (&F)[J])
{
    double e;
    boys_top<J>(T, kmax, tab, etab, k, F, e);
}

// All of F_0 .. F_kmax (F[n] = F_n, runtime kmax <= kBoysN - 1): the same head
// and the same downward recursion, run to n = 0.
__device__ __forceinline__ void boys_all(double T, int kmax, const double *__restrict__ tab,
                                         const double *__restrict__ etab, const Consts &k, double *F)
{
    double f, e;
    boys_head(T, kmax, tab, etab, k, f, e);
    F[kmax] = f;
    const double twoT = T + T;
    for (int n = kmax; n > 0; --n) F[n - 1] = fma(twoT, F[n], e) * k.inv_int[2 * n - 1];
}

__device__ __forceinline__ double powi(double x, int n)
{
    double p = 1.0;
    while (n) {
        if (n & 1) p *= x;
        x *= x;
        n >>= 1;
    }
    return p;
}

// ------------------------------------------------------------------------- //
// Regular scaled solid harmonics R^{c/s}_{l,m}(v), 0 <= m <= l <= lmax      //
// (recursions of Sec. II E), stored at l(l+1)/2 + m.                       //
// ------------------------------------------------------------------------- //
__device__ __forceinline__ void scaled_harmonics(double x, double y, double z, int lmax, const Consts &k,
                                                 double *Rc, double *Rs)
{
    const double r2 = x * x + y * y + z * z;
    Rc[0] = 1.0;
    Rs[0] = 0.0;
    for (int l = 0; l < lmax; ++l) {
        const int d0 = l * (l + 1) / 2, d1 = (l + 1) * (l + 2) / 2, dm = (l - 1) * l / 2;
        const double cll = Rc[d0 + l], sll = Rs[d0 + l];
        const double inv = k.inv_int[2 * l + 2];
        Rc[d1 + l + 1] = -(x * cll - y * sll) * inv;
        Rs[d1 + l + 1] = -(y * cll + x * sll) * inv;
        const double zl = k.dint[2 * l + 1] * z;
        for (int m = 0; m <= l; ++m) {
            const double im = k.inv_int[(l + m + 1) * (l - m + 1)];
            const double pc = (m <= l - 1) ? Rc[dm + m] : 0.0;
            const double ps = (m <= l - 1) ? Rs[dm + m] : 0.0;
            Rc[d1 + m] = (zl * Rc[d0 + m] - r2 * pc) * im;
            Rs[d1 + m] = (m == 0) ? 0.0 : (zl * Rs[d0 + m] - r2 * ps) * im;
        }
    }
}

// R^c_{L,m} and R^s_{L,m} for any integer m, with R_{L,-m} from the symmetry
// relations R^c_{l,-m} = (-1)^m R^c_{l,m}, R^s_{l,-m} = -(-1)^m R^s_{l,m}
// and zero for |m| > L.
__device__ __forceinline__ double rc_get(const double *Rc, int L, int m)
{
    const int am = m < 0 ? -m : m;
    if (L < 0 || am > L) return 0.0;
    const double v = Rc[L * (L + 1) / 2 + am];
    return (m < 0 && (am & 1)) ? -v : v;
}
__device__ __forceinline__ double rs_get(const double *Rs, int L, int m)
{
    const int am = m < 0 ? -m : m;
    if (L < 0 || am > L) return 0.0;
    const double v = Rs[L * (L + 1) / 2 + am];
    return (m < 0 && !(am & 1)) ? -v : v;
}

// One row of the translation matrix W_{l,mu,j,kappa} (Sec. II E) for the
// real function m (cosine part for m >= 0, sine part for m < 0), flattened
// over e = (j, kappa, z): j^2 + (kappa == 0 ? 0 : 2 kappa - 1 + z).
// kappa = 0 keeps only the z = c column (the z = s column is exactly zero);
// the factor (1/2)^{delta_kappa0} cancels the doubled m +- 0 term.
template <int J>
__device__ __forceinline__ void w_row(const double *Rc, const double *Rs, int l, int m, double (&w)[J * J])
{
    const int mu = m < 0 ? -m : m;
    const bool sine = m < 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int L = l - j;
#pragma unroll
        for (int kp = 0; kp <= j; ++kp) {
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            if (kp == 0) {
                w[e0] = sine ? rs_get(Rs, L, mu) : rc_get(Rc, L, mu);
            } else {
                const double cm = rc_get(Rc, L, mu - kp), cp = rc_get(Rc, L, mu + kp);
                const double sm = rs_get(Rs, L, mu - kp), sp = rs_get(Rs, L, mu + kp);
                if (!sine) {
                    w[e0] = (kp & 1) ? cm - cp : cm + cp;       // W^{cc}
                    w[e0 + 1] = (kp & 1) ? -sm - sp : sp - sm;   // W^{cs}
                } else {
                    w[e0] = (kp & 1) ? sm - sp : sm + sp;        // W^{sc}
                    w[e0 + 1] = (kp & 1) ? cm + cp : cm - cp;    // W^{ss}
                }
            }
        }
    }
}


// ------------------------------------------------------------------------- //
// Double-double arithmetic (unevaluated sums h + l of two FP64 numbers) from //
// the error-free transformations TwoSum (Knuth), FastTwoSum (Dekker) and the //
// FMA TwoProd; about 2^-104 relative per operation.  Used where a formula    //
// cancels although the quantity it computes is well conditioned.            //
// ------------------------------------------------------------------------- //
struct ddv {
    double h, l;
};
__device__ __forceinline__ ddv dd_fast(double a, double b)
{
    const double s = a + b;
    return ddv{s, b - (s - a)};
}
__device__ __forceinline__ ddv dd_sum(double a, double b)
{
    const double s = a + b, bb = s - a;
    return ddv{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ddv dd_prod(double a, double b)
{
    const double p = a * b;
    return ddv{p, fma(a, b, -p)};
}
__device__ __forceinline__ ddv dd_add(ddv a, ddv b)
{
    ddv s = dd_sum(a.h, b.h);
    const ddv t = dd_sum(a.l, b.l);
    s = dd_fast(s.h, s.l + t.h);
    return dd_fast(s.h, s.l + t.l);
}
__device__ __forceinline__ ddv dd_mul(ddv a, ddv b)
{
    const double p = a.h * b.h;
    double e = fma(a.h, b.h, -p);
    e = fma(a.h, b.l, e);
    e = fma(a.l, b.h, e);
    return dd_fast(p, e);
}
__device__ __forceinline__ ddv dd_mul_d(ddv a, double b)
{
    const double p = a.h * b;
    const double e = fma(a.l, b, fma(a.h, b, -p));
    return dd_fast(p, e);
}
__device__ __forceinline__ ddv dd_neg(ddv a) { return ddv{-a.h, -a.l}; }
__device__ __forceinline__ ddv dd_sub(ddv a, ddv b) { return dd_add(a, dd_neg(b)); }
// a b + c
__device__ __forceinline__ ddv dd_fma(ddv a, ddv b, ddv c) { return dd_add(dd_mul(a, b), c); }

// 1/a: FP64 reciprocal and one Newton step r + r (1 - a r) carried in double-double
__device__ __forceinline__ ddv dd_inv(ddv a)
{
    const double r = 1.0 / a.h;
    const ddv ar = dd_mul_d(a, r);
    const ddv e = dd_add(ddv{1.0, 0.0}, ddv{-ar.h, -ar.l});
    return dd_add(ddv{r, 0.0}, dd_mul_d(e, r));
}

// ------------------------------------------------------------------------- //
// Radial terms of one primitive pair, accumulated into the contracted        //
// O[j] = O^{(kmax-j)}, j = 0..J-1 (Table S1 and Eq. O_rab2_deriv).          //
//   w = w_alpha w_beta = N_a N_b c_alpha c_beta / ((2alpha)^la (2beta)^lb)  //
// Coulomb-type operators (1/r, erfc, erf) accumulate only the top order     //
// O[0] and the exp(-T') terms E[j], j >= 1, of the downward recursion,      //
// which radial_finish_fp64 runs once on the contracted sums: for both the   //
// 1/r and the attenuated term, X_n = P q^n F_n(T') satisfies                //
//   X_n = (-2R^2 X_{n+1} + P q^n exp(-T')) / (2n+1)                        //
// (2T'/q = -2R^2), the same for every primitive pair of the shell pair,     //
// with the two terms of one sign for each primitive pair.                   //
// ------------------------------------------------------------------------- //
template <int OP>
__device__ __forceinline__ constexpr bool coulomb_type() { return OP == OP_COULOMB || OP == OP_ERFC || OP == OP_ERF; }

template <int OP, int J>
__device__ __forceinline__ void radial_finish_fp64(double R2, int kmax, const Consts &k, double (&O)[J],
                                                   const double (&E)[J])
{
    if (!coulomb_type<OP>()) return;
    const double m2R2 = -2.0 * R2;
#pragma unroll
    for (int j = 1; j < J; ++j) O[j] = fma(m2R2, O[j - 1], E[j]) * k.inv_int[2 * (kmax - j) + 1];
}

template <int OP, int J>
__device__ __forceinline__ void radial_acc_fp64(const PrimRec &pa, const PrimRec &pb, double R2, int kmax, int la,
                                                const Args2c &g, double (&O)[J], double (&E)[J])
{
    const int kmin = kmax - J + 1;
    const double w = pa.w2c * pb.w2c;
    const double c = pa.alpha + pb.alpha;
    const double rc = rsqrt(c);
    const double ic = rc * rc;
    const double rho = pa.alpha * pb.alpha * ic;
    const double T = rho * R2;
    if (OP == OP_OVERLAP) {
        // (pi/c)^{3/2} exp(-T) (-rho)^k
        double q = w * kPi32 * ic * rc * exp(-T) * powi(-rho, kmin);
#pragma unroll
        for (int j = J - 1; j >= 0; --j) {
            O[j] += q;
            q *= -rho;
        }
    } else if (OP == OP_GAUSS) {
        // (pi^2/(c (rho+w)))^{3/2} exp(-w T/(rho+w)) (-w rho/(rho+w))^k
        const double rd = rsqrt(rho + g.omega);
        const double id = rd * rd;
        const double f = -g.omega * rho * id;
        double q = w * kPi3 * ic * rc * id * rd * exp(-g.omega * T * id) * powi(f, kmin);
#pragma unroll
        for (int j = J - 1; j >= 0; --j) {
            O[j] += q;
            q *= f;
        }
    } else if (OP == OP_RA2N) {
        // (a|r_a^{2n}|b), Eq. T_rab2_deriv with Eqs. sra2ms and I_jab.  Per primitive
        // pair T(x) = w pi^{3/2} c^{-3/2} e^{-rho x} Q(x), x = R^2, with Q of degree n:
        //   Q(x) = sum_d (beta^2 x / c)^d sum_{m=d}^{n} C(n, n-m) (la)_{n-m} alpha^{m-n} c^{-m} k_{m,d},
        //   k_{m,d} = 2^{d-m} (2m+1)!! C(m,d) / (2d+1)!!  (an integer times a power of 2),
        // (la)_j the rising factorial ((0)_0 = 1, (0)_j = 0).  Derivatives:
        // T^{(k)} = w pi^{3/2} c^{-3/2} e^{-rho x} Q_k(x), Q_{k+1}[d] = (d+1) Q_k[d+1] - rho Q_k[d].
        // For beta >> alpha the terms of Q_k are all of order alpha^{k-n} with
        // alternating signs (T^{(k)} itself is well conditioned), so Q and its
        // recursion run in double-double; the common factor stays in FP64.
        const int n = __double2int_rn(g.omega);
        const ddv cc = dd_sum(pa.alpha, pb.alpha);
        const ddv icd = dd_inv(cc);
        const ddv rhod = dd_mul(dd_prod(pa.alpha, pb.alpha), icd);
        const ddv bcd = dd_mul(dd_prod(pb.alpha, pb.alpha), icd);
        const ddv iad = dd_inv(ddv{pa.alpha, 0.0});
        ddv tm[kRa2nMax + 1];
#pragma unroll
        for (int m = 0; m <= kRa2nMax; ++m) {
            tm[m] = ddv{0.0, 0.0};
            if (m <= n) {
                const int j = n - m;
                double rf = g.k.binom[n][j];                 // C(n, j) (la)_j: exact integer
                for (int i = 0; i < j; ++i) rf *= (double)(la + i);
                ddv t = ddv{rf, 0.0};
                for (int i = 0; i < j; ++i) t = dd_mul(t, iad);
                for (int i = 0; i < m; ++i) t = dd_mul(t, icd);
                tm[m] = t;
            }
        }
        ddv q[kRa2nMax + 2];
        ddv bd = ddv{1.0, 0.0};
#pragma unroll
        for (int d = 0; d <= kRa2nMax; ++d) {
            ddv sum = ddv{0.0, 0.0};
#pragma unroll
            for (int m = d; m <= kRa2nMax; ++m) sum = dd_add(sum, dd_mul_d(tm[m], g.k.ra2n_k[m][d]));
            q[d] = dd_mul(bd, sum);
            bd = dd_mul(bd, bcd);
        }
        q[kRa2nMax + 1] = ddv{0.0, 0.0};
        const ddv mrho = ddv{-rhod.h, -rhod.l};
        for (int k = 0; k < kmin; ++k) {
#pragma unroll
            for (int d = 0; d <= kRa2nMax; ++d) q[d] = dd_add(dd_mul_d(q[d + 1], (double)(d + 1)), dd_mul(mrho, q[d]));
        }
        const double we = w * kPi32 * ic * rc * exp(-T);
#pragma unroll
        for (int t = 0; t < J; ++t) {
            ddv val = q[kRa2nMax];
#pragma unroll
            for (int d = kRa2nMax - 1; d >= 0; --d) val = dd_add(dd_mul_d(val, R2), q[d]);
            O[J - 1 - t] += we * (val.h + val.l);
            if (t + 1 < J) {
#pragma unroll
                for (int d = 0; d <= kRa2nMax; ++d)
                    q[d] = dd_add(dd_mul_d(q[d + 1], (double)(d + 1)), dd_mul(mrho, q[d]));
            }
        }
    } else if (OP == OP_GCOUL) {
        // exp(-w r^2)/r: (pi/c)^{3/2} (2 pi/d) exp(-w T/d) sum_i C(k,i) p^{k-i} q^i F_i(T rho/d),
        // d = rho + w, p = -w rho/d, q = -rho^2/d.  Every order comes from one vector
        // F_0..F_kmax by k applications of v_i <- p v_i + q v_{i+1} (p, q < 0: no
        // cancellation); the first kmin run over the whole vector, the last J-1
        // over a J-wide register window.
        const double id = 1.0 / (rho + g.omega);
        const double p = -g.omega * rho * id, q = -rho * rho * id;
        const double pre = w * kPi32 * ic * rc * (2.0 * kPi) * id * exp(-g.omega * T * id);
        double F[kBoysN];
        boys_all(T * rho * id, kmax, g.boys, g.boys_e, g.k, F);
        for (int m = 1; m <= kmin; ++m)
            for (int i = 0; i <= kmax - m; ++i) F[i] = fma(p, F[i], q * F[i + 1]);
        double v[J];
#pragma unroll
        for (int i = 0; i < J; ++i) v[i] = F[i];
        O[J - 1] += pre * v[0];
#pragma unroll
        for (int t = 1; t < J; ++t) {
#pragma unroll
            for (int i = 0; i < J - t; ++i) v[i] = fma(p, v[i], q * v[i + 1]);
            O[J - 1 - t] += pre * v[0];
        }
    } else {
        // Coulomb-type: 2 pi^{5/2} / (alpha beta sqrt(c)) (-rho)^kmin * ...
        const double pk = w * kTwoPi52 * pa.inv_alpha * pb.inv_alpha * rc * powi(-rho, kmin);
        if (OP == OP_COULOMB || OP == OP_ERFC) {
            double F, e;
            boys_head(T, kmax, g.boys, g.boys_e, g.k, F, e);
            double q = pk;
#pragma unroll
            for (int j = J - 1; j >= 1; --j) {
                E[j] = fma(q, e, E[j]);
                q *= -rho;
            }
            O[0] = fma(q, F, O[0]);
        }
        if (OP == OP_ERF || OP == OP_ERFC) {
            // omega/sqrt(omega^2+rho) (-omega^2 rho/(omega^2+rho))^k F_k(omega^2 T/(omega^2+rho)):
            // with u = omega/sqrt(omega^2+rho), s = u^2 the order kmin factor is pk u s^kmin
            const double u = g.omega * rsqrt(g.omega * g.omega + rho);
            const double s = u * u;
            double F, e;
            boys_head(s * T, kmax, g.boys, g.boys_e, g.k, F, e);
            double q = pk * u * powi(s, kmin);
            if (OP == OP_ERFC) q = -q;
            const double f = -rho * s;
#pragma unroll
            for (int j = J - 1; j >= 1; --j) {
                E[j] = fma(q, e, E[j]);
                q *= f;
            }
            O[0] = fma(q, F, O[0]);
        }
    }
}

// Rigorous upper bound on every element magnitude of a contracted overlap
// (op 0) or Gaussian-operator (op 4) block, from |S_{l,m}(r)| <= sqrt(2) r^l,
// r^l exp(-a r^2) <= (l/(a e))^{l/2} exp(-a r^2/2) and the s-type integral at
// halved exponents, maximised over the primitives by the smallest exponents.
__device__ __forceinline__ double screen_bound(const ScreenRec &a, const ScreenRec &b, double R2, int op, double omega)
{
    const double ah = 0.5 * a.amin, bh = 0.5 * b.amin;
    const double c = ah + bh, rho = ah * bh / c;
    double s;
    if (op == OP_OVERLAP) {
        const double t = kPi32 / (c * sqrt(c));
        s = t * exp(-rho * R2);
    } else {
        const double d = rho + omega;
        const double base = 9.869604401089358 / (c * d);
        s = base * sqrt(base) * exp(-omega * rho * R2 / d);
    }
    return 2.0 * a.lfac * b.lfac * a.sabs * b.sabs * s;
}

// Runtime-J variant of w_row (used where J varies inside one thread).
__device__ __forceinline__ void w_row_rt(const double *Rc, const double *Rs, int l, int m, int J, double *w)
{
    const int mu = m < 0 ? -m : m;
    const bool sine = m < 0;
    for (int j = 0; j < J; ++j) {
        const int L = l - j;
        for (int kp = 0; kp <= j; ++kp) {
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            if (kp == 0) {
                w[e0] = sine ? rs_get(Rs, L, mu) : rc_get(Rc, L, mu);
            } else {
                const double cm = rc_get(Rc, L, mu - kp), cp = rc_get(Rc, L, mu + kp);
                const double sm = rs_get(Rs, L, mu - kp), sp = rs_get(Rs, L, mu + kp);
                const bool odd = kp & 1;
                if (!sine) {
                    w[e0] = odd ? cm - cp : cm + cp;
                    w[e0 + 1] = odd ? -sm - sp : sp - sm;
                } else {
                    w[e0] = odd ? sm - sp : sm + sp;
                    w[e0 + 1] = odd ? cm + cp : cm - cp;
                }
            }
        }
    }
}

}  // namespace dev
}  // namespace shg
