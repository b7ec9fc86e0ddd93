// Mixed-precision two-center SHG kernel: the same formula as the FP64 path
// (Sec. II B and Table S1 of arXiv:1701.06588) evaluated in double-float
// arithmetic on the FP32 pipes (GB300 issues FP32 at 74x its FP64 rate), with
// FP64 used only to write the result.
//
// Range: the FP64 path forms w_a w_b (-rho)^k with w = N c (2 alpha)^-l, whose
// factors leave the FP32 exponent range (rho^k reaches 1e44 for alpha, beta
// ~ 5000).  Here every primitive term enters the assembly already multiplied
// by the 2^{la+lb-j} of Eq. final_r12int_ab, and
//   2^k (-rho)^k (2 alpha)^-la (2 beta)^-lb = (-1)^k (beta/c)^la (alpha/c)^lb (2 rho)^-j,
// k = la+lb-j, whose factors are all bounded: (beta/c), (alpha/c) <= 1 and
// (2 rho)^-j <= 4e9 on the synthetic sets.  So the accumulated quantity is
//   S_j = sum (-1)^k N_a c_a N_b c_b (beta/c)^la (alpha/c)^lb (2 rho)^-j X_k
// with X_k the operator part of (0_a|O|0_b)^{(k)} without its (-rho)^k.
//
// Precision: double-float (about 2^-44); Taylor tails of the Boys function and
// of exp whose size is below 1e-7 of the leading term are summed in plain
// FP32 (their rounding is below 1e-14 of the result).
#include "shg_device.cuh"
#include "shg_df.cuh"
#include "shg_mix_angular.cuh"
#include "shg_grad_angular.cuh"

namespace shg {
namespace {
using namespace dev;
using namespace dfm;
using namespace mixa;


__device__ __forceinline__ df powi_df(df x, int n)
{
    df p = df_f(1.0f);
    while (n) {
        if (n & 1) p = mul(p, x);
        x = mul(x, x);
        n >>= 1;
    }
    return p;
}

// exp(-x), x >= 0, in double-float: x = n ln2 + r, |r| <= ln2/2, Taylor of
// exp(-r) (degree 13; terms 7..13 in FP32), times 2^-n.  Below FP32 range for
// x > 87 the result is flushed to zero (terms that small are far below the
// absolute parity floor for the weights of the synthetic sets).
__device__ __noinline__ df exp_neg_df(df x, const ConstsMix &k)
{
    if (x.hi > 87.0f) return df_f(0.0f);
    const float n = rintf(x.hi * 1.44269504088896341f);
    const float ln2_hi = 0.693147182464599609375f;        // float(ln 2)
    const float ln2_lo = -1.904654299957768e-09f;          // ln 2 - ln2_hi
    const float ph = n * ln2_hi;
    const df p = df{ph, fmaf(n, ln2_hi, -ph)};             // exact n ln2_hi
    df r = sub(x, p);
    r = add_f(r, -n * ln2_lo);
    const df y = neg(r);                                   // exp(y), |y| <= 0.35
    float t = k.inv_fact_f[13];
    for (int i = 12; i >= 7; --i) t = fmaf(t, y.hi, k.inv_fact_f[i]);
    df e = add(mul_f(y, t), ldf(k.inv_fact[6]));
    for (int i = 5; i >= 0; --i) e = add(mul(y, e), ldf(k.inv_fact[i]));
    const float s = exp2f(-n);                              // exact power of two (or 0 below range)
    return df{e.hi * s, e.lo * s};
}

// Taylor head in double-float on the grid T_i = i/32 (|y| <= 1/64, y = T_i - T):
// F_n(T) = sum_{t<=6} c_t y^t with c0..c2 in double-float and the terms 3..6,
// together at most (1/64)^3/3! = 6.4e-7 of F, in FP32 (relative error ~1e-7
// there, so ~6e-14 of F); exp(-T) = exp(-T_i) exp(y) the same way.  The
// index is rounded by adding 1.5 * 2^23 (no float-to-int conversion);
// T.hi - T_i is exact (Sterbenz), so y is exact in double-float.
__device__ __forceinline__ void boys_taylor_mix(df T, int kmax, const float4 *__restrict__ tab,
                                                const float2 *__restrict__ etab, df &f, df *e)
{
    constexpr float kRound = 12582912.0f;                          // 1.5 * 2^23
    const float t32 = fmaf(T.hi, 32.0f, kRound);
    const int i = __float_as_int(t32) - __float_as_int(kRound);
    const float d0 = T.hi - (t32 - kRound) * 0.03125f;             // exact
    const df y = two_sum(-d0, -T.lo);                              // T_i - T
    const float4 *c = tab + ((size_t)i * kBoysN + kmax) * 3;
    const float4 q0 = __ldg(c), q1 = __ldg(c + 1), q2 = __ldg(c + 2);
    float t = fmaf(q2.y, y.hi, q2.x);                              // c6 y + c5
    t = fmaf(t, y.hi, q1.w);                                       // + c4
    t = fmaf(t, y.hi, q1.z);                                       // + c3
    f = add(mul_f(y, t), df{q1.x, q1.y});
    f = add(mul(y, f), df{q0.z, q0.w});
    f = add(mul(y, f), df{q0.x, q0.y});
    if (e) {
        const float te = fmaf(fmaf(fmaf(1.0f / 720.0f, y.hi, 1.0f / 120.0f), y.hi, 1.0f / 24.0f), y.hi,
                              1.0f / 6.0f);
        df x = add(mul_f(y, te), df_f(0.5f));
        x = add(mul(y, x), df_f(1.0f));
        x = add(mul(y, x), df_f(1.0f));
        *e = mul(x, ldf(__ldg(etab + i)));
    }
}

// Boys head in double-float: F_kmax and exp(-T) (0 above the table range),
// the same scheme as the FP64 path: Taylor head from the table below T = 120,
// asymptotic head above.
__device__ __forceinline__ void boys_head_mix(df T, int kmax, const float4 *__restrict__ tab,
                                              const float2 *__restrict__ etab, const ConstsMix &k, df &f, df &e)
{
    if (T.hi < (float)kBoysTmax) {
        boys_taylor_mix(T, kmax, tab, etab, f, &e);
    } else {
        // (2kmax-1)!! (2T)^-kmax sqrt(pi/(4T)); exp(-T) is below FP32 range here
        const df rT = rsqrt_df(T);
        f = mul(mul(ldf(k.dfact[kmax]), powi_df(scale2(mul(rT, rT), 0.5f), kmax)), mul(rT, ldf(k.sqrt_pi_half)));
        e = df_f(0.0f);
    }
}

// F_kmax (and exp(-T)) for T < kBoysTmax only: the Taylor head of boys_head_mix.
__device__ __forceinline__ void boys_head_mix_near(df T, int kmax, const float4 *__restrict__ tab,
                                                   const float2 *__restrict__ etab, const ConstsMix &k, df &f, df &e)
{
    (void)k;
    boys_taylor_mix(T, kmax, tab, etab, f, &e);
}

// Boys F_k(T), k = kmax-J+1..kmax, F[j] = F_{kmax-j}: head, then one shared
// downward recursion.
template <int J>
__device__ __forceinline__ void boys_top_mix(df T, int kmax, const float4 *__restrict__ tab,
                                             const float2 *__restrict__ etab, const ConstsMix &k, df (&F)[J])
{
    df f, e;
    boys_head_mix(T, kmax, tab, etab, k, f, e);
    F[0] = f;
    const df twoT = scale2(T, 2.0f);
#pragma unroll
    for (int j = 1; j < J; ++j) {
        const int kk = kmax - j + 1;
        F[j] = mul(add(mul(twoT, F[j - 1]), e), ldf(k.inv_int[2 * kk - 1]));
    }
}

// All of F_0 .. F_kmax (F[n] = F_n, runtime kmax <= kBoysN - 1).
__device__ __forceinline__ void boys_all_mix(df T, int kmax, const float4 *__restrict__ tab,
                                             const float2 *__restrict__ etab, const ConstsMix &k, df *F)
{
    df f, e;
    boys_head_mix(T, kmax, tab, etab, k, f, e);
    F[kmax] = f;
    const df twoT = scale2(T, 2.0f);
    for (int n = kmax; n > 0; --n) F[n - 1] = mul(add(mul(twoT, F[n]), e), ldf(k.inv_int[2 * n - 1]));
}

// Common part of one primitive pair: c, 1/sqrt(c), 1/c, rho, T and the
// order factors hp[j] = base (2 rho)^-j (-1)^{kmax-j}.
struct MixPair {
    df c, rc, ic, rho, T;
};

template <int J>
__device__ __forceinline__ MixPair mix_setup(const MixPrim &pa, const MixPrim &pb, df R2, int la, int lb, df (&hp)[J])
{
    const int kmax = la + lb;
    MixPair m;
    const df a = ldf(pa.alpha), b = ldf(pb.alpha);
    m.c = add(a, b);
    m.rc = rsqrt_df(m.c);
    m.ic = mul(m.rc, m.rc);
    m.rho = mul(mul(a, b), m.ic);
    m.T = mul(m.rho, R2);
    df base = mul(ldf(pa.wN), powi_df(mul(b, m.ic), la));
    base = mul(base, mul(ldf(pb.wN), powi_df(mul(a, m.ic), lb)));
    const df h = scale2(mul(mul(m.c, ldf(pa.inv_alpha)), ldf(pb.inv_alpha)), 0.5f);   // 1/(2 rho)
    hp[0] = (kmax & 1) ? neg(base) : base;
#pragma unroll
    for (int j = 1; j < J; ++j) hp[j] = neg(mul(hp[j - 1], h));
    return m;
}

// the operator parts: S_j += hp[j] X_k
template <int J>
__device__ __forceinline__ void mix_overlap(const MixPair &m, const df (&hp)[J], const ConstsMix &km, df (&S)[J])
{
    const df X = mul(mul(ldf(km.pi32), mul(m.ic, m.rc)), exp_neg_df(m.T, km));
#pragma unroll
    for (int j = 0; j < J; ++j) S[j] = add(S[j], mul(hp[j], X));
}

template <int J>
__device__ __forceinline__ void mix_gauss(const MixPair &m, const df (&hp)[J], df omega, int kmax, const ConstsMix &km,
                                          df (&S)[J])
{
    const df d = add(m.rho, omega);
    const df rd = rsqrt_df(d);
    const df id = mul(rd, rd);
    const df wd = mul(omega, id);                                            // omega / (rho + omega)
    df X = mul(mul(ldf(km.pi3), mul(mul(m.ic, m.rc), mul(id, rd))), exp_neg_df(mul(m.T, wd), km));
    X = mul(X, powi_df(wd, kmax - J + 1));                                  // X_k at k = kmax - J + 1
#pragma unroll
    for (int j = J - 1; j >= 0; --j) {
        S[j] = add(S[j], mul(hp[j], X));
        X = mul(X, wd);
    }
}

// the 1/r part for T < kBoysTmax (the fused pass sums the far field separately)
template <int J>
__device__ __forceinline__ void mix_coulomb_near(const MixPair &m, const df (&hp)[J], df pre, int kmax,
                                                 const float4 *boys, const float2 *boys_e, const ConstsMix &km,
                                                 df (&S)[J])
{
    df F[J], e;
    boys_head_mix_near(m.T, kmax, boys, boys_e, km, F[0], e);
    const df twoT = scale2(m.T, 2.0f);
#pragma unroll
    for (int j = 1; j < J; ++j) F[j] = mul(add(mul(twoT, F[j - 1]), e), ldf(km.inv_int[2 * (kmax - j + 1) - 1]));
#pragma unroll
    for (int j = 0; j < J; ++j) S[j] = add(S[j], mul(mul(hp[j], pre), F[j]));
}

template <int J>
__device__ __forceinline__ void mix_coulomb(const MixPair &m, const df (&hp)[J], df pre, int kmax, const float4 *boys,
                                            const float2 *boys_e, const ConstsMix &km, df (&S)[J])
{
    df F[J];
    boys_top_mix<J>(m.T, kmax, boys, boys_e, km, F);
#pragma unroll
    for (int j = 0; j < J; ++j) S[j] = add(S[j], mul(mul(hp[j], pre), F[j]));
}

// attenuated part omega/sqrt(omega^2+rho) (-omega^2 rho/(omega^2+rho))^k F_k(omega^2 T/(omega^2+rho)),
// subtracted when negate (the erfc share of a single-operator pass)
template <int J>
__device__ __forceinline__ void mix_attenuated(const MixPair &m, const df (&hp)[J], df pre, df omega, df omega2,
                                               bool negate, int kmax, const float4 *boys, const float2 *boys_e,
                                               const ConstsMix &km, df (&S)[J])
{
    const df rw = rsqrt_df(add(omega2, m.rho));
    const df s = mul(omega2, mul(rw, rw));                                   // omega^2 / (omega^2 + rho)
    df F[J];
    boys_top_mix<J>(mul(s, m.T), kmax, boys, boys_e, km, F);
    df X = mul(mul(pre, mul(omega, rw)), powi_df(s, kmax - J + 1));
    if (negate) X = neg(X);
#pragma unroll
    for (int j = J - 1; j >= 0; --j) {
        S[j] = add(S[j], mul(mul(hp[j], X), F[j]));
        X = mul(X, s);
    }
}

__device__ __forceinline__ df mix_boys_prefactor(const MixPair &m, const MixPrim &pa, const MixPrim &pb,
                                                 const ConstsMix &km)
{
    return mul(mul(ldf(km.two_pi52), m.rc), mul(ldf(pa.inv_alpha), ldf(pb.inv_alpha)));
}

// Top order and recursion terms of the fused pass (contracted downward
// recursion, as in the FP64 fused kernel): with the order factors hp[j] of
// this path (they carry (-2 rho)^k), a Coulomb-type term Y_n = hp(n) X_n
// obeys Y_n = (-R^2 Y_{n+1} + hp(n) P q^n exp(-T')) / (2n+1) for the 1/r
// (P = pre, q = 1, T' = T) and the attenuated (P = pre omega / sqrt(omega^2 +
// rho), q = s, T' = s T) sums alike; -R^2 is the same for every primitive pair,
// so only the top order S[0] and the terms E[j], j >= 1, are summed here.
template <int J>
__device__ __forceinline__ void mix_coulomb_near_top(const MixPair &m, const df (&hp)[J], df pre, int kmax,
                                                     const float4 *boys, const float2 *boys_e, const ConstsMix &km,
                                                     df (&S)[J], df (&E)[J])
{
    df F, e;
    boys_head_mix_near(m.T, kmax, boys, boys_e, km, F, e);
    S[0] = add(S[0], mul(mul(hp[0], pre), F));
    if (J > 1) {
        const df pe = mul(pre, e);
#pragma unroll
        for (int j = 1; j < J; ++j) E[j] = add(E[j], mul(hp[j], pe));
    }
}

template <int J>
__device__ __forceinline__ void mix_attenuated_top(const MixPair &m, const df (&hp)[J], df pre, df omega, df omega2,
                                                   int kmax, const float4 *boys, const float2 *boys_e,
                                                   const ConstsMix &km, df (&S)[J], df (&E)[J])
{
    const df rw = rsqrt_df(add(omega2, m.rho));
    const df s = mul(omega2, mul(rw, rw));                                   // omega^2 / (omega^2 + rho)
    df F, e;
    boys_head_mix(mul(s, m.T), kmax, boys, boys_e, km, F, e);
    df X = mul(mul(pre, mul(omega, rw)), powi_df(s, kmax - J + 1));          // order kmin
    if (J > 1) {
        df Xe = mul(X, e);
#pragma unroll
        for (int j = J - 1; j >= 1; --j) {
            E[j] = add(E[j], mul(hp[j], Xe));
            Xe = mul(Xe, s);
            X = mul(X, s);
        }
    }
    S[0] = add(S[0], mul(mul(hp[0], X), F));
}

// S_j += hp[j] X_k for one primitive pair, k = kmax-j, j = 0..J-1: the
// operator parts X_k of Table S1 without their (-rho)^k, which hp carries
// (with the weights and the 2^k of the assembly).
template <int OP, int J>
__device__ __forceinline__ void radial_mix_orders(const MixPair &m, const df (&hp)[J], int kmax, const MixPrim &pa,
                                                  const MixPrim &pb, const ArgsMix &g, df (&S)[J])
{
    if (OP == OP_OVERLAP) {
        mix_overlap<J>(m, hp, g.km, S);
    } else if (OP == OP_GAUSS) {
        mix_gauss<J>(m, hp, ldf(g.omega), kmax, g.km, S);
    } else if (OP == OP_GCOUL) {
        // exp(-w r^2)/r without the (-rho)^k carried by hp:
        //   X_k = (pi/c)^{3/2} (2 pi/d) exp(-w T/d) sum_i C(k,i) (w/d)^{k-i} (rho/d)^i F_i(T rho/d),
        // d = rho + w: binomial weights of a convex combination, applied as
        // v_i <- (w/d) v_i + (rho/d) v_{i+1} (kmin times over F_0..F_kmax, then
        // over a J-wide register window)
        const int kmin = kmax - J + 1;
        const df rd = rsqrt_df(add(m.rho, ldf(g.omega)));
        const df id = mul(rd, rd);
        const df sw = mul(ldf(g.omega), id), sr = mul(m.rho, id);
        const df pre = mul(mul(ldf(g.km.pi32), mul(m.ic, m.rc)),
                           mul(mul(ldf(g.km.two_pi), id), exp_neg_df(mul(m.T, sw), g.km)));
        df F[kBoysN];
        boys_all_mix(mul(m.T, sr), kmax, g.boys, g.boys_e, g.km, F);
        for (int mm = 1; mm <= kmin; ++mm)
            for (int i = 0; i <= kmax - mm; ++i) F[i] = add(mul(sw, F[i]), mul(sr, F[i + 1]));
        df v[J];
#pragma unroll
        for (int i = 0; i < J; ++i) v[i] = F[i];
        S[J - 1] = add(S[J - 1], mul(hp[J - 1], mul(pre, v[0])));
#pragma unroll
        for (int t = 1; t < J; ++t) {
#pragma unroll
            for (int i = 0; i < J - t; ++i) v[i] = add(mul(sw, v[i]), mul(sr, v[i + 1]));
            S[J - 1 - t] = add(S[J - 1 - t], mul(hp[J - 1 - t], mul(pre, v[0])));
        }
    } else {
        const df pre = mix_boys_prefactor(m, pa, pb, g.km);
        if (OP == OP_COULOMB || OP == OP_ERFC) mix_coulomb<J>(m, hp, pre, kmax, g.boys, g.boys_e, g.km, S);
        if (OP == OP_ERF || OP == OP_ERFC)
            mix_attenuated<J>(m, hp, pre, ldf(g.omega), ldf(g.omega2), OP == OP_ERFC, kmax, g.boys, g.boys_e, g.km, S);
    }
}

// S_j += (-1)^k base (2 rho)^-j X_k for one primitive pair, k = la+lb-j.
template <int OP, int J>
__device__ __forceinline__ void radial_acc_mix(const MixPrim &pa, const MixPrim &pb, df R2, int la, int lb,
                                               const ArgsMix &g, df (&S)[J])
{
    df hp[J];                       // base (2 rho)^-j (-1)^{kmax-j}
    const MixPair m = mix_setup<J>(pa, pb, R2, la, lb, hp);
    radial_mix_orders<OP, J>(m, hp, la + lb, pa, pb, g, S);
}

// ------------------------------------------------------------------------- //
// Vector-Jacobian product of the two-center blocks (Eq. dev_ab) with the     //
// radial orders O^{(k)}, k = la+lb+1-J .. la+lb+1, in double-float and the   //
// angular part (harmonics, their gradients, W and the contractions with the  //
// upstream weights) in FP64 (gradang::grad_from_orders).  The orders carry   //
// this path's scaling S_j = 2^k O^{(k)}: for k = la+lb+1-j,                  //
//   2^k (-rho)^k (2 alpha)^-la (2 beta)^-lb = (-1)^k (beta/c)^la (alpha/c)^lb (2 rho)^{1-j},
// so the weights are those of the integrals shifted by one order, with
// (-1)^{kmax+1} base 2 rho in front.                                         //
// ------------------------------------------------------------------------- //
template <int OP, int J>
__device__ void pair_grad_mix(const ArgsGradMix &a, int p)
{
    const ArgsMix &g = a.m;
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l, kmax = la + lb;
    const MixCenter A = g.centers[sa.center];
    const MixCenter B = g.centers[sb.center];
    const df vx = sub(ldf(A.x), ldf(B.x)), vy = sub(ldf(A.y), ldf(B.y)), vz = sub(ldf(A.z), ldf(B.z));
    const df R2 = add(add(mul(vx, vx), mul(vy, vy)), mul(vz, vz));
    df S[J + 1];
#pragma unroll
    for (int j = 0; j <= J; ++j) S[j] = df_f(0.0f);
    const int Kb = sb.nprim, npp = sa.nprim * Kb;
    for (int q = 0; q < npp; ++q) {
        const int ia = q / Kb, ib = q - ia * Kb;
        const MixPrim pa = g.prims[sa.prim_off + ia], pb = g.prims[sb.prim_off + ib];
        df hp[J];
        const MixPair m = mix_setup<J>(pa, pb, R2, la, lb, hp);
        df hq[J + 1];
        hq[0] = neg(mul(scale2(m.rho, 2.0f), hp[0]));
#pragma unroll
        for (int j = 0; j < J; ++j) hq[j + 1] = hp[j];
        radial_mix_orders<OP, J + 1>(m, hq, kmax + 1, pa, pb, g, S);
    }
    // f0[e] = 2^{kmax-j} (2j-1)!! B O^{(kmax-j)} = jB S_{j+1},
    // f1[e] = 2^{kmax-j} (2j-1)!! B O^{(kmax-j+1)} = jB S_j / 2
    const Args2c &f = a.g;
    double f0[J * J], f1[J * J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const double s0 = to_double(S[j + 1]), s1 = 0.5 * to_double(S[j]);
#pragma unroll
        for (int kp = 0; kp <= j; ++kp) {
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            f0[e0] = f.k.jB[j][kp] * s0;
            f1[e0] = f.k.jB[j][kp] * s1;
            if (kp) {
                f0[e0 + 1] = f0[e0];
                f1[e0 + 1] = f1[e0];
            }
        }
    }
    const Vec4 Ad = f.centers[sa.center];
    const Vec4 Bd = f.centers[sb.center];
    const double v[3] = {Ad.x - Bd.x, Ad.y - Bd.y, Ad.z - Bd.z};
    gradang::grad_from_orders<J>(f, p, la, lb, v, f0, f1);
}

template <int OP>
__global__ void __launch_bounds__(128) k_2c_grad_mixed_persistent(const ArgsGradMix a)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.m.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + a.m.tile_begin;
        if (t >= a.m.tile_end) break;
        const Tile tl = a.m.tiles[t];
        if (lane < tl.count) {
            const int la = tl.cls / (kLmax2c + 1), lb = tl.cls % (kLmax2c + 1);
            const int p = a.m.perm[tl.start + lane];
            // J <= 4: the classes with both l >= kMixedFp64MinL run in FP64
            switch ((la < lb ? la : lb) + 1) {
            case 1: pair_grad_mix<OP, 1>(a, p); break;
            case 2: pair_grad_mix<OP, 2>(a, p); break;
            case 3: pair_grad_mix<OP, 3>(a, p); break;
            case 4: pair_grad_mix<OP, 4>(a, p); break;
            default: break;
            }
        }
        __syncwarp();
    }
}

template <int OP>
static int grid_grad_mix()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_grad_mixed_persistent<OP>, 128, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    return (sms > 0 ? sms : 1) * per;
}

// Angular part and store of one pair from its contracted S_j (runtime J).
__device__ __noinline__ void assemble_mix(const ArgsMix &g, int p, int la, int lb, df vx, df vy, df vz, const df *S,
                                          int J)
{
    const int JJ = J * J;
    df ge[kJmax * kJmax];
    for (int j = 0; j < J; ++j)
        for (int kp = 0; kp <= j; ++kp) {
            const df v = mul(S[j], ldf(g.km.jB[j][kp]));
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            ge[e0] = v;
            if (kp) ge[e0 + 1] = v;
        }
    df Rc[(kLmax2c + 1) * (kLmax2c + 2) / 2], Rs[(kLmax2c + 1) * (kLmax2c + 2) / 2];
    scaled_harmonics_mix(vx, vy, vz, la > lb ? la : lb, g.km, Rc, Rs);
    const int nb = 2 * lb + 1;
    df Ub[2 * kLmax2c + 1][kJmax * kJmax];
    for (int mb = -lb; mb <= lb; ++mb) w_row_mix_rt(Rc, Rs, lb, mb, J, Ub[mb + lb]);
    double *out = g.out + g.out_off[p];
    for (int ma = -la; ma <= la; ++ma) {
        df ua[kJmax * kJmax];
        w_row_mix_rt(Rc, Rs, la, ma, J, ua);
        for (int e = 0; e < JJ; ++e) ua[e] = mul(ua[e], ge[e]);
        df Aa = ldf(g.km.A[la][ma < 0 ? -ma : ma]);
        if (lb & 1) Aa = neg(Aa);
        for (int mb = -lb; mb <= lb; ++mb) {
            const df *ub = Ub[mb + lb];
            // compensated dot product (Ogita, Rump and Oishi, "Dot2"): exact
            // products of the high parts by FMA, their running sum by TwoSum,
            // every rounding error and the cross terms summed in one FP32
            // accumulator; as accurate as double-float accumulation
            float sh = 0.0f, sl = 0.0f;
            for (int e = 0; e < JJ; ++e) {
                const float p = ua[e].hi * ub[e].hi;
                float ep = fmaf(ua[e].hi, ub[e].hi, -p);
                ep = fmaf(ua[e].hi, ub[e].lo, ep);
                ep = fmaf(ua[e].lo, ub[e].hi, ep);
                const df t = two_sum(sh, p);
                sh = t.hi;
                sl += t.lo + ep;
            }
            const df s = fast_two_sum(sh, sl);
            out[(ma + la) * nb + (mb + lb)] = to_double(mul(Aa, mul(ldf(g.km.A[lb][mb < 0 ? -mb : mb]), s)));
        }
    }
}

template <int OP, int J>
__device__ void pair_2c_mix(const ArgsMix &g, int p)
{
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l;
    const MixCenter A = g.centers[sa.center];
    const MixCenter B = g.centers[sb.center];
    const df vx = sub(ldf(A.x), ldf(B.x)), vy = sub(ldf(A.y), ldf(B.y)), vz = sub(ldf(A.z), ldf(B.z));
    const df R2 = add(add(mul(vx, vx), mul(vy, vy)), mul(vz, vz));
    if ((OP == OP_OVERLAP || OP == OP_GAUSS) && g.screen_thresh > 0.0 &&
        screen_bound(g.screen[g.pair_a[p]], g.screen[g.pair_b[p]], to_double(R2), OP, g.omega_d) < g.screen_thresh) {
        double *o = g.out + g.out_off[p];
        for (int i = 0; i < (2 * la + 1) * (2 * lb + 1); ++i) o[i] = 0.0;
        return;
    }

    df S[J];
#pragma unroll
    for (int j = 0; j < J; ++j) S[j] = df_f(0.0f);
    const int Kb = sb.nprim, npp = sa.nprim * Kb;
    for (int q = 0; q < npp; ++q) {
        const int ia = q / Kb, ib = q - ia * Kb;
        radial_acc_mix<OP, J>(g.prims[sa.prim_off + ia], g.prims[sb.prim_off + ib], R2, la, lb, g, S);
    }
    df Sr[kJmax];
#pragma unroll
    for (int j = 0; j < J; ++j) Sr[j] = S[j];
    assemble_mix(g, p, la, lb, vx, vy, vz, Sr, J);
}

// ------------------------------------------------------------------------- //
// Fused multi-operator pass in double-float (the FP64 fused pass of          //
// shg_fused.cu with this file's arithmetic): per primitive pair the common   //
// setup once and one sum per requested operator (erfc = 1/r - attenuated),   //
// then Q_j = sum_{e in block j} A_a (2j-1)!! B_{j,kappa} W_a[e] A_b W_b[e]    //
// by a compensated dot product per block, read once for all operators.      //
// ------------------------------------------------------------------------- //
__device__ __noinline__ void assemble_mix_fused(const ArgsMixFused &g, int p, int la, int lb, df vx, df vy, df vz,
                                                const df (*S)[kJmax], int J)
{
    df Rc[(kLmax2c + 1) * (kLmax2c + 2) / 2], Rs[(kLmax2c + 1) * (kLmax2c + 2) / 2];
    scaled_harmonics_mix(vx, vy, vz, la > lb ? la : lb, g.km, Rc, Rs);
    const int nb = 2 * lb + 1;
    const int JJ = J * J;
    df Ub[2 * kLmax2c + 1][kJmax * kJmax];
    for (int mb = -lb; mb <= lb; ++mb) {
        df *ub = Ub[mb + lb];
        w_row_mix_rt(Rc, Rs, lb, mb, J, ub);
        const df Ab = ldf(g.km.A[lb][mb < 0 ? -mb : mb]);
        for (int e = 0; e < JJ; ++e) ub[e] = mul(ub[e], Ab);
    }
    const long long o = g.out_off[p];
    for (int ma = -la; ma <= la; ++ma) {
        df ua[kJmax * kJmax];
        w_row_mix_rt(Rc, Rs, la, ma, J, ua);
        df Aa = ldf(g.km.A[la][ma < 0 ? -ma : ma]);
        if (lb & 1) Aa = neg(Aa);
        for (int j = 0; j < J; ++j)
            for (int kp = 0; kp <= j; ++kp) {
                const df gv = mul(Aa, ldf(g.km.jB[j][kp]));
                const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
                ua[e0] = mul(ua[e0], gv);
                if (kp) ua[e0 + 1] = mul(ua[e0 + 1], gv);
            }
        for (int mb = -lb; mb <= lb; ++mb) {
            const df *ub = Ub[mb + lb];
            df Q[kJmax];
            for (int j = 0; j < J; ++j) {
                // compensated dot product over block j (Dot2 of Ogita, Rump and Oishi)
                float sh = 0.0f, sl = 0.0f;
                for (int e = j * j; e < (j + 1) * (j + 1); ++e) {
                    const float pr = ua[e].hi * ub[e].hi;
                    float ep = fmaf(ua[e].hi, ub[e].hi, -pr);
                    ep = fmaf(ua[e].hi, ub[e].lo, ep);
                    ep = fmaf(ua[e].lo, ub[e].hi, ep);
                    const df t = two_sum(sh, pr);
                    sh = t.hi;
                    sl += t.lo + ep;
                }
                Q[j] = fast_two_sum(sh, sl);
            }
            const long long idx = o + (ma + la) * nb + (mb + lb);
            for (int op = 0; op < 5; ++op) {
                if (!g.out[op]) continue;
                df s = mul(S[op][0], Q[0]);
                for (int j = 1; j < J; ++j) s = add(s, mul(S[op][j], Q[j]));
                g.out[op][idx] = to_double(s);
            }
        }
    }
}

template <int J>
__device__ void pair_2c_mix_fused(const ArgsMixFused &g, int p)
{
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l, kmax = la + lb;
    const MixCenter A = g.centers[sa.center];
    const MixCenter B = g.centers[sb.center];
    const df vx = sub(ldf(A.x), ldf(B.x)), vy = sub(ldf(A.y), ldf(B.y)), vz = sub(ldf(A.z), ldf(B.z));
    const df R2 = add(add(mul(vx, vx), mul(vy, vy)), mul(vz, vz));
    const bool f_ov = g.out[OP_OVERLAP] != nullptr;
    const bool f_ga = g.out[OP_GAUSS] != nullptr;
    const bool f_co = g.out[OP_COULOMB] != nullptr || g.out[OP_ERFC] != nullptr;
    const bool f_er = g.out[OP_ERF] != nullptr;
    const bool f_x = g.out[OP_ERFC] != nullptr && !(f_er && g.share_att);

    // S*[j]: order kmax - j; E*[j], j >= 1: the exp(-T') terms of the contracted recursion
    df Sov[J], Sco[J], Sx[J], Ser[J], Sga[J], Eco[J], Ex[J], Eer[J];
#pragma unroll
    for (int j = 0; j < J; ++j) Sov[j] = Sco[j] = Sx[j] = Ser[j] = Sga[j] = Eco[j] = Ex[j] = Eer[j] = df_f(0.0f);
    // far field of the 1/r sum, T >= kBoysTmax: sum of the FP64 weights fw_a fw_b
    // (on the FP64 pipe), times the per-pair order factors after the loop
    double far = 0.0;
    const int Kb = sb.nprim, npp = sa.nprim * Kb;
    for (int q = 0; q < npp; ++q) {
        const int ia = q / Kb, ib = q - ia * Kb;
        const MixPrim pa = g.prims[sa.prim_off + ia], pb = g.prims[sb.prim_off + ib];
        df hp[J];
        const MixPair m = mix_setup<J>(pa, pb, R2, la, lb, hp);
        if (f_ov) mix_overlap<J>(m, hp, g.km, Sov);
        if (f_ga) mix_gauss<J>(m, hp, ldf(g.w_gauss), kmax, g.km, Sga);
        if (f_co || f_er || f_x) {
            const df pre = mix_boys_prefactor(m, pa, pb, g.km);
            if (f_co) {
                if (m.T.hi < (float)kBoysTmax)
                    mix_coulomb_near_top<J>(m, hp, pre, kmax, g.boys, g.boys_e, g.km, Sco, Eco);
                else far = fma(pa.fw, pb.fw, far);
            }
            if (f_er)
                mix_attenuated_top<J>(m, hp, pre, ldf(g.w_erf), ldf(g.w_erf2), kmax, g.boys, g.boys_e, g.km, Ser, Eer);
            if (f_x)
                mix_attenuated_top<J>(m, hp, pre, ldf(g.w_erfc), ldf(g.w_erfc2), kmax, g.boys, g.boys_e, g.km, Sx, Ex);
        }
    }
    // contracted downward recursion, orders kmax-1 .. kmin (far field added afterwards)
    if (J > 1) {
        const df mR2 = neg(R2);
#pragma unroll
        for (int j = 1; j < J; ++j) {
            const df inv = ldf(g.km.inv_int[2 * (kmax - j) + 1]);
            Sco[j] = mul(add(mul(mR2, Sco[j - 1]), Eco[j]), inv);
            Ser[j] = mul(add(mul(mR2, Ser[j - 1]), Eer[j]), inv);
            Sx[j] = mul(add(mul(mR2, Sx[j - 1]), Ex[j]), inv);
        }
    }
    if (far != 0.0) {
        // pi^3 (-1)^n (2n-1)!! R^{-2n-1}, n = kmax - j: the far-field orders with the
        // 2^n of this path's scaling (R > 0: T >= kBoysTmax)
        const int kmin = kmax - J + 1;
        const double ir2 = 1.0 / to_double(R2);
        double dfk = 1.0;                                       // (2 kmin - 1)!!
        for (int i = 2 * kmin - 1; i > 1; i -= 2) dfk *= (double)i;
        double t = far * kPi3 * sqrt(ir2) * dfk * powi(-ir2, kmin);
#pragma unroll
        for (int j = J - 1; j >= 0; --j) {
            const float th = __double2float_rn(t);
            Sco[j] = add(Sco[j], df{th, __double2float_rn(t - (double)th)});
            t *= -ir2 * (double)(2 * (kmax - j) + 1);
        }
    }
    df Sr[5][kJmax];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        Sr[OP_OVERLAP][j] = Sov[j];
        Sr[OP_COULOMB][j] = Sco[j];
        Sr[OP_ERFC][j] = sub(Sco[j], f_x ? Sx[j] : Ser[j]);
        Sr[OP_ERF][j] = Ser[j];
        Sr[OP_GAUSS][j] = Sga[j];
    }
    assemble_mix_fused(g, p, la, lb, vx, vy, vz, Sr, J);
}

__device__ __forceinline__ void run_tile_mix_fused(const ArgsMixFused &g, const Tile &tl, int lane)
{
    if (lane >= tl.count) return;
    const int p = g.perm[tl.start + lane];
    const int la = tl.cls / (kLmax2c + 1), lb = tl.cls % (kLmax2c + 1);
    // J = min(la, lb) + 1 <= 4: the host runs the classes with both l >=
    // kMixedFp64MinL (J >= 5) in FP64, so they never reach this kernel
    switch ((la < lb ? la : lb) + 1) {
    case 1: pair_2c_mix_fused<1>(g, p); break;
    case 2: pair_2c_mix_fused<2>(g, p); break;
    case 3: pair_2c_mix_fused<3>(g, p); break;
    case 4: pair_2c_mix_fused<4>(g, p); break;
    default: break;
    }
}

// MinB = 0: registers as the compiler sees fit (about 124, four 128-thread
// CTAs per SM); MinB = 5: at most 96 per thread, five CTAs per SM; MinB = 6:
// at most 85, six CTAs (more warps to hide load and instruction-fetch
// latency, more spilled values).  The autotuner picks (shg_plan_2c_set_variant).
template <int MinB>
__global__ void __launch_bounds__(128, MinB) k_2c_mixed_fused_persistent(const ArgsMixFused g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        run_tile_mix_fused(g, g.tiles[t], lane);
        __syncwarp();
    }
}

template <int MinB>
__global__ void __launch_bounds__(128, MinB) k_2c_mixed_fused_static(const ArgsMixFused g)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int t = g.tile_begin + warp;
    if (t >= g.tile_end) return;
    run_tile_mix_fused(g, g.tiles[t], lane);
}

template <int OP>
__device__ __forceinline__ void mix_dispatch(const ArgsMix &g, int p, int J)
{
    // J <= 4 only: the classes with J >= 5 run in FP64 (see run_tile_mix_fused)
    switch (J) {
    case 1: pair_2c_mix<OP, 1>(g, p); break;
    case 2: pair_2c_mix<OP, 2>(g, p); break;
    case 3: pair_2c_mix<OP, 3>(g, p); break;
    case 4: pair_2c_mix<OP, 4>(g, p); break;
    default: break;
    }
}

template <int OP>
__global__ void __launch_bounds__(128) k_2c_mixed_persistent(const ArgsMix g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        const Tile tl = g.tiles[t];
        if (lane < tl.count) {
            const int la = tl.cls / (kLmax2c + 1), lb = tl.cls % (kLmax2c + 1);
            mix_dispatch<OP>(g, g.perm[tl.start + lane], (la < lb ? la : lb) + 1);
        }
        __syncwarp();
    }
}

template <int OP>
__global__ void __launch_bounds__(128) k_2c_mixed_static(const ArgsMix g)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int t = g.tile_begin + warp;
    if (t >= g.tile_end) return;
    const Tile tl = g.tiles[t];
    if (lane < tl.count) {
        const int la = tl.cls / (kLmax2c + 1), lb = tl.cls % (kLmax2c + 1);
        mix_dispatch<OP>(g, g.perm[tl.start + lane], (la < lb ? la : lb) + 1);
    }
}

template <int OP>
static int grid_mix(int threads, int ctas_per_sm)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_mixed_persistent<OP>, threads, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    return (sms > 0 ? sms : 1) * per;
}

template <int OP>
static cudaError_t launch_mix_op(const ArgsMix &a, int grid, int threads, bool persistent, cudaStream_t s)
{
    if (persistent) {
        k_2c_mixed_persistent<OP><<<grid, threads, 0, s>>>(a);
    } else {
        const int tiles = a.tile_end - a.tile_begin;
        if (tiles <= 0) return cudaSuccess;
        const int wpb = threads / 32;
        k_2c_mixed_static<OP><<<(tiles + wpb - 1) / wpb, threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_2c_grad_mixed(const ArgsGradMix &a, int op, cudaStream_t s)
{
    switch (op) {
    case OP_OVERLAP: k_2c_grad_mixed_persistent<OP_OVERLAP><<<grid_grad_mix<OP_OVERLAP>(), 128, 0, s>>>(a); break;
    case OP_COULOMB: k_2c_grad_mixed_persistent<OP_COULOMB><<<grid_grad_mix<OP_COULOMB>(), 128, 0, s>>>(a); break;
    case OP_ERFC: k_2c_grad_mixed_persistent<OP_ERFC><<<grid_grad_mix<OP_ERFC>(), 128, 0, s>>>(a); break;
    case OP_ERF: k_2c_grad_mixed_persistent<OP_ERF><<<grid_grad_mix<OP_ERF>(), 128, 0, s>>>(a); break;
    case OP_GAUSS: k_2c_grad_mixed_persistent<OP_GAUSS><<<grid_grad_mix<OP_GAUSS>(), 128, 0, s>>>(a); break;
    case OP_GCOUL: k_2c_grad_mixed_persistent<OP_GCOUL><<<grid_grad_mix<OP_GCOUL>(), 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_2c_mixed(const ArgsMix &a, int op, int grid, bool persistent, cudaStream_t s, int threads)
{
    switch (op) {
    case OP_OVERLAP: return launch_mix_op<OP_OVERLAP>(a, grid, threads, persistent, s);
    case OP_COULOMB: return launch_mix_op<OP_COULOMB>(a, grid, threads, persistent, s);
    case OP_ERFC: return launch_mix_op<OP_ERFC>(a, grid, threads, persistent, s);
    case OP_ERF: return launch_mix_op<OP_ERF>(a, grid, threads, persistent, s);
    case OP_GAUSS: return launch_mix_op<OP_GAUSS>(a, grid, threads, persistent, s);
    case OP_GCOUL: return launch_mix_op<OP_GCOUL>(a, grid, threads, persistent, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_2c_mixed_fused(const ArgsMixFused &a, int grid, bool persistent, cudaStream_t s, int threads,
                                  int variant)
{
    if (persistent) {
        switch (variant) {
        case 1: k_2c_mixed_fused_persistent<5><<<grid, threads, 0, s>>>(a); break;
        case 2: k_2c_mixed_fused_persistent<6><<<grid, threads, 0, s>>>(a); break;
        default: k_2c_mixed_fused_persistent<0><<<grid, threads, 0, s>>>(a); break;
        }
    } else {
        const int tiles = a.tile_end - a.tile_begin;
        if (tiles <= 0) return cudaSuccess;
        const int wpb = threads / 32;
        if (variant) k_2c_mixed_fused_static<5><<<(tiles + wpb - 1) / wpb, threads, 0, s>>>(a);
        else k_2c_mixed_fused_static<0><<<(tiles + wpb - 1) / wpb, threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int persistent_grid_2c_mixed_fused(int threads, int ctas_per_sm, int variant)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *kern = variant == 1   ? (const void *)k_2c_mixed_fused_persistent<5>
                       : variant == 2 ? (const void *)k_2c_mixed_fused_persistent<6>
                                      : (const void *)k_2c_mixed_fused_persistent<0>;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
    if (e != cudaSuccess || per < 1)
        per = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    return (sms > 0 ? sms : 1) * per;
}

int persistent_grid_2c_mixed(int op, int threads, int ctas_per_sm)
{
    switch (op) {
    case OP_OVERLAP: return grid_mix<OP_OVERLAP>(threads, ctas_per_sm);
    case OP_COULOMB: return grid_mix<OP_COULOMB>(threads, ctas_per_sm);
    case OP_ERFC: return grid_mix<OP_ERFC>(threads, ctas_per_sm);
    case OP_ERF: return grid_mix<OP_ERF>(threads, ctas_per_sm);
    case OP_GAUSS: return grid_mix<OP_GAUSS>(threads, ctas_per_sm);
    default: return grid_mix<OP_GCOUL>(threads, ctas_per_sm);
    }
}

}  // namespace shg
