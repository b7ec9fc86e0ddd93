// Three-index overlap (a b a~), a and a~ on center A, b on center B, by the
// SHG scheme of Sec. II D (arXiv:1701.06588), FP64.
//
// The product of the two functions on A is expanded with real Gaunt
// coefficients into solid harmonics L_a = |la-la~|..la+la~ (step 2) times
// r_a^{2p}, p = (la+la~-L_a)/2 (Eq. product_SHG_STGO); each term is a
// two-center block of shell (L_a, exponent alpha' = alpha+alpha~) with b,
// whose monopole P^{(k)} (Eq. Pa_aba) contracts
//   binom(p,j) (L_a)_j alpha'^{-j} (0_a'|r_a^{2(p-j)}|0_b)^{(k)}
// over primitive triples, with (0_a'|r_a^{2m}|0_b)^{(k)} from Eqs. sra2ms and
// devsra2ms.  The angular part is the real translation matrix of Sec. II E.
//
// One thread per triple; a warp owns a class-pure tile (la, la~, lb).
#include "shg_device.cuh"
#include "shg_mix_angular.cuh"

namespace shg {
namespace {
using namespace dev;
using namespace dfm;
using namespace mixa;

constexpr int kPmax = 5;          // min(la, la~) <= 5 when la + la~ <= 10
constexpr int kNL = kPmax + 1;    // number of L_a terms
constexpr int kKmax3 = kLmaxAabA + kLmax2c;  // highest derivative order, 16
constexpr int kLR = kLmaxAabA;    // scaled harmonics up to l = 10

// Geometry of one triple and the L_a range of its product expansion.
struct TripleGeom {
    int la, lt, lb, Lmin, Lmax, nL;
    double vx, vy, vz;
};

// Radial sums P[iL][j] = P_{L_a}^{(L_a+lb-j)} of one triple in FP64 (also in
// the mixed form: the sum over i below alternates in sign).
__device__ __forceinline__ TripleGeom aab_radial(const Args3c &g, int p, double (&P)[kNL][kJmax])
{
    const ShellRec sa = g.orb_shells[g.t_a[p]];
    const ShellRec st = g.orb_shells[g.t_t[p]];
    const ShellRec sb = g.aux_shells[g.t_b[p]];
    const int la = sa.l, lt = st.l, lb = sb.l;
    const Vec4 A = g.orb_centers[sa.center];
    const Vec4 B = g.aux_centers[sb.center];
    const double vx = A.x - B.x, vy = A.y - B.y, vz = A.z - B.z;
    const double R2 = vx * vx + vy * vy + vz * vz;
    const int Lmin = la > lt ? la - lt : lt - la;
    const int Lmax = la + lt;
    const int nL = (Lmax - Lmin) / 2 + 1;
    const int pmax = nL - 1;
    const int kmaxA = Lmax + lb;
    const int kminA = Lmin > lb ? Lmin : lb;

    for (int i = 0; i < kNL; ++i)
        for (int j = 0; j < kJmax; ++j) P[i][j] = 0.0;

    const int Ka = sa.nprim, Kt = st.nprim, Kb = sb.nprim;
    const int ntrip = Ka * Kt * Kb;
    // per (a, a~) primitive pair (ib == 0): alpha' = alpha + alpha~ and its powers
    double ap = 0.0, wat = 0.0, wL0 = 0.0, i2ap2 = 0.0;
    double ia_p[kPmax + 1];
    for (int q = 0; q < ntrip; ++q) {
        const int ib = q % Kb;
        if (ib == 0) {
            const int it = (q / Kb) % Kt;
            const int ia = q / (Kb * Kt);
            const PrimRec pa = g.orb_prims[sa.prim_off + ia];
            const PrimRec pt = g.orb_prims[st.prim_off + it];
            ap = pa.alpha + pt.alpha;
            const double rap = rsqrt(ap);
            const double iap = rap * rap;                   // 1 / alpha'
            wat = pa.wN * pt.wN * kPi32;
            ia_p[0] = 1.0;
            for (int m = 1; m <= pmax; ++m) ia_p[m] = ia_p[m - 1] * iap;
            const double i2ap = 0.5 * iap;
            wL0 = powi(i2ap, Lmin);                          // (2 alpha')^{-L_min}
            i2ap2 = i2ap * i2ap;
        }
        const PrimRec pb = g.aux_prims[sb.prim_off + ib];
        const double be = pb.alpha;
        const double c = ap + be;
        const double rc = rsqrt(c);
        const double ic = rc * rc;
        const double rho = ap * be * ic;
        const double gg = be * be * ic;                 // beta^2 / c
        const double x = gg * R2;
        const double h = 0.5 * ic;                      // 1 / (2c)
        // pi^{3/2} c^{-3/2} exp(-rho R^2) and the weights N c of a, a~ and N c / (2beta)^lb of b
        const double w0 = wat * pb.w2c * ic * rc * exp(-rho * R2);

        double gp[kPmax + 1], hm[kPmax + 1];
        gp[0] = hm[0] = 1.0;
        for (int m = 1; m <= pmax; ++m) {
            gp[m] = gp[m - 1] * gg;
            hm[m] = hm[m - 1] * h;
        }
        // GD[m][i] = (beta^2/c)^i D_m^{(i)}(x),  D_m^{(i)}(x) = sum_{j=i..m} d_{m,j} j!/(j-i)! x^{j-i}
        double GD[kPmax + 1][kPmax + 1];
        for (int m = 0; m <= pmax; ++m)
            for (int i = 0; i <= m; ++i) {
                double s = g.k3.dd[m][i][m];
                for (int jj = m - 1; jj >= i; --jj) s = fma(s, x, g.k3.dd[m][i][jj]);
                GD[m][i] = gp[i] * s;
            }
        double nr[kKmax3 + 1];                          // (-rho)^n
        nr[0] = 1.0;
        for (int n = 1; n <= kmaxA; ++n) nr[n] = nr[n - 1] * -rho;
        // V[m][k] = (2c)^{-m} sum_{i<=min(m,k)} binom(k,i) (-rho)^{k-i} GD[m][i]
        double V[kPmax + 1][kKmax3 + 1];
        for (int k = kminA; k <= kmaxA; ++k) {
            double bn[kPmax + 1];
            const int imax = pmax < k ? pmax : k;
            for (int i = 0; i <= imax; ++i) bn[i] = g.k3.binom[k][i] * nr[k - i];
            for (int m = 0; m <= pmax; ++m) {
                double v = 0.0;
                const int im = m < k ? m : k;
                for (int i = 0; i <= im; ++i) v = fma(bn[i], GD[m][i], v);
                V[m][k] = hm[m] * v;
            }
        }
        // P_L^{(k)} += w0 (2 alpha')^{-L} sum_j binom(p,j) (L)_j alpha'^{-j} V[p-j][k]
        double wL = w0 * wL0;
        for (int iL = 0; iL < nL; ++iL) {
            const int L = Lmin + 2 * iL;
            const int pL = pmax - iL;
            const int J = (L < lb ? L : lb) + 1;
            const int kmaxL = L + lb;
            double bj[kPmax + 1];
            for (int jj = 0; jj <= pL; ++jj) bj[jj] = g.k3.bj[L][pL][jj] * ia_p[jj];
            for (int j = 0; j < J; ++j) {
                const int k = kmaxL - j;
                double s = 0.0;
                for (int jj = 0; jj <= pL; ++jj) s = fma(bj[jj], V[pL - jj][k], s);
                P[iL][j] = fma(wL, s, P[iL][j]);
            }
            wL *= i2ap2;
        }
    }
    return TripleGeom{la, lt, lb, Lmin, Lmax, nL, vx, vy, vz};
}

// Screening of one triple: |phi_a phi_a~| <= 2 sabs_a sabs_a~ lfac_a lfac_a~
// exp(-(amin_a + amin_a~) r^2 / 2) (the single-shell bound of the two-center
// screen, multiplied), so the two-center overlap bound of the combined record
// and b bounds every element of the block.  Writes zeros and returns true
// when that bound is below the threshold.
__device__ __forceinline__ bool aab_screened(const Args3c &g, int p)
{
    if (!(g.screen_thresh > 0.0)) return false;
    const ScreenRec ra = g.orb_screen[g.t_a[p]], rt = g.orb_screen[g.t_t[p]], rb = g.aux_screen[g.t_b[p]];
    const ScreenRec at{ra.amin + rt.amin, ra.sabs * rt.sabs, 1.4142135623730950488 * ra.lfac * rt.lfac, 0.0};
    const ShellRec sa = g.orb_shells[g.t_a[p]], st = g.orb_shells[g.t_t[p]], sb = g.aux_shells[g.t_b[p]];
    const Vec4 A = g.orb_centers[sa.center], B = g.aux_centers[sb.center];
    const double vx = A.x - B.x, vy = A.y - B.y, vz = A.z - B.z;
    if (screen_bound(at, rb, vx * vx + vy * vy + vz * vz, OP_OVERLAP, 0.0) >= g.screen_thresh) return false;
    double *o = g.out + g.out_off[p];
    const int n = (2 * sa.l + 1) * (2 * st.l + 1) * (2 * sb.l + 1);
    for (int i = 0; i < n; ++i) o[i] = 0.0;
    return true;
}

__device__ void triple_aab_fp64(const Args3c &g, int p)
{
    if (aab_screened(g, p)) return;
    double P[kNL][kJmax];
    const TripleGeom tg = aab_radial(g, p, P);
    const int la = tg.la, lt = tg.lt, lb = tg.lb, Lmin = tg.Lmin, Lmax = tg.Lmax, nL = tg.nL;
    const double vx = tg.vx, vy = tg.vy, vz = tg.vz;

    // angular part: R^{c/s}_{l,m}(R_a - R_b) up to max(L_a max, lb)
    double Rc[(kLR + 1) * (kLR + 2) / 2], Rs[(kLR + 1) * (kLR + 2) / 2];
    scaled_harmonics(vx, vy, vz, Lmax > lb ? Lmax : lb, g.k, Rc, Rs);
    const int nb = 2 * lb + 1;
    const int Jmax = (Lmax < lb ? Lmax : lb) + 1;
    double Wb[2 * kLmax2c + 1][kJmax * kJmax];
    for (int mb = -lb; mb <= lb; ++mb) w_row_rt(Rc, Rs, lb, mb, Jmax, Wb[mb + lb]);

    // blocks B_L[M][mb] of every L_a term, each a two-center formula with P
    double Bst[(1 + 5 + 9 + 13 + 17 + 21) * (2 * kLmax2c + 1)];
    const double sgn_b = (lb & 1) ? -1.0 : 1.0;
    // lambda K_L = sqrt(4 pi (2L+1) / ((2la+1)(2la~+1)))
    const double lam0 = 3.5449077018110320545963349666822903 / (g.k3.sqrt_int[2 * la + 1] * g.k3.sqrt_int[2 * lt + 1]);
    int boff = 0;
    for (int iL = 0; iL < nL; ++iL) {
        const int L = Lmin + 2 * iL;
        const int J = (L < lb ? L : lb) + 1;
        const double lamK = lam0 * g.k3.sqrt_int[2 * L + 1];
        double ge[kJmax * kJmax];
        for (int j = 0; j < J; ++j) {
            const double oj = P[iL][j] * lamK * g.k.pow2[L + lb - j];
            for (int kp = 0; kp <= j; ++kp) {
                const double v = oj * g.k.jB[j][kp];
                const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
                ge[e0] = v;
                if (kp) ge[e0 + 1] = v;
            }
        }
        for (int M = -L; M <= L; ++M) {
            double wa[kJmax * kJmax];
            w_row_rt(Rc, Rs, L, M, J, wa);
            const double Aa = g.k.A[L][M < 0 ? -M : M] * sgn_b;
            for (int e = 0; e < J * J; ++e) wa[e] *= ge[e];
            for (int mb = -lb; mb <= lb; ++mb) {
                double s = 0.0;
                for (int e = 0; e < J * J; ++e) s = fma(wa[e], Wb[mb + lb][e], s);
                Bst[boff + (M + L) * nb + (mb + lb)] = Aa * (g.k.A[lb][mb < 0 ? -mb : mb] * s);
            }
        }
        boff += (2 * L + 1) * nb;
    }

    // Gaunt sum over (L_a, M_a) for each (m_a, m_a~)
    const int nt = 2 * lt + 1;
    const int rbase = g.gaunt_base[la * 7 + lt];
    double *out = g.out + g.out_off[p];
    for (int ma = 0; ma < 2 * la + 1; ++ma)
        for (int mt = 0; mt < nt; ++mt) {
            const int r = rbase + ma * nt + mt;
            double acc[2 * kLmax2c + 1];
            for (int mb = 0; mb < nb; ++mb) acc[mb] = 0.0;
            for (int q = g.gaunt_row[r]; q < g.gaunt_row[r + 1]; ++q) {
                const GauntEnt ge = g.gaunt[q];
                const int iL = (ge.L - Lmin) / 2;
                // offset of block L = sum_{L' < L} (2L'+1) nb over the L' of this triple
                const int off_L = iL * (2 * Lmin + 1 + 2 * (iL - 1)) * nb;
                const double *bl = Bst + off_L + (ge.M + ge.L) * nb;
                for (int mb = 0; mb < nb; ++mb) acc[mb] = fma(ge.g, bl[mb], acc[mb]);
            }
            double *o = out + (ma * nt + mt) * nb;
            for (int mb = 0; mb < nb; ++mb) o[mb] = acc[mb];
        }
}

// Mixed form: the radial sums in FP64 (aab_radial), the angular part and the
// Gaunt sum in double-float on the FP32 pipes.  Per L_a the radial factors
// are scaled by a power of two 2^e into FP32 range; the block is scaled back
// by 2^e (in two exact steps) before the Gaunt sum.
__device__ __forceinline__ df split_d(double v)
{
    const float hi = __double2float_rn(v);
    return df{hi, __double2float_rn(v - (double)hi)};
}

__device__ void triple_aab_mixed(const Args3c &g, int p)
{
    if (aab_screened(g, p)) return;
    double P[kNL][kJmax];
    const TripleGeom tg = aab_radial(g, p, P);
    const int la = tg.la, lt = tg.lt, lb = tg.lb, Lmin = tg.Lmin, Lmax = tg.Lmax, nL = tg.nL;

    df Rc[(kLR + 1) * (kLR + 2) / 2], Rs[(kLR + 1) * (kLR + 2) / 2];
    scaled_harmonics_mix(split_d(tg.vx), split_d(tg.vy), split_d(tg.vz), Lmax > lb ? Lmax : lb, g.km, Rc, Rs);
    const int nb = 2 * lb + 1;
    const int Jmax = (Lmax < lb ? Lmax : lb) + 1;
    df Wb[2 * kLmax2c + 1][kJmax * kJmax];
    for (int mb = -lb; mb <= lb; ++mb) w_row_mix_rt(Rc, Rs, lb, mb, Jmax, Wb[mb + lb]);

    df Bst[(1 + 5 + 9 + 13 + 17 + 21) * (2 * kLmax2c + 1)];
    const double lam0 = 3.5449077018110320545963349666822903 / (g.k3.sqrt_int[2 * la + 1] * g.k3.sqrt_int[2 * lt + 1]);
    int boff = 0;
    for (int iL = 0; iL < nL; ++iL) {
        const int L = Lmin + 2 * iL;
        const int J = (L < lb ? L : lb) + 1;
        const double lamK = lam0 * g.k3.sqrt_int[2 * L + 1];
        double oj[kJmax];
        double omax = 0.0;
        for (int j = 0; j < J; ++j) {
            oj[j] = P[iL][j] * lamK * g.k.pow2[L + lb - j];
            omax = fmax(omax, fabs(oj[j]));
        }
        int ex = 0;
        if (omax > 0.0) frexp(omax, &ex);
        ex = ex > 250 ? 250 : (ex < -250 ? -250 : ex);
        df ge[kJmax * kJmax];
        for (int j = 0; j < J; ++j) {
            const df oe = split_d(ldexp(oj[j], -ex));
            for (int kp = 0; kp <= j; ++kp) {
                const df v = mul(oe, ldf(g.km.jB[j][kp]));
                const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
                ge[e0] = v;
                if (kp) ge[e0 + 1] = v;
            }
        }
        const float s1 = ldexpf(1.0f, ex / 2), s2 = ldexpf(1.0f, ex - ex / 2);
        for (int M = -L; M <= L; ++M) {
            df wa[kJmax * kJmax];
            w_row_mix_rt(Rc, Rs, L, M, J, wa);
            df Aa = ldf(g.km.A[L][M < 0 ? -M : M]);
            if (lb & 1) Aa = neg(Aa);
            for (int e = 0; e < J * J; ++e) wa[e] = mul(wa[e], ge[e]);
            for (int mb = -lb; mb <= lb; ++mb) {
                const df *wb = Wb[mb + lb];
                df sum = mul(wa[0], wb[0]);
                for (int e = 1; e < J * J; ++e) sum = add(sum, mul(wa[e], wb[e]));
                const df blk = mul(Aa, mul(ldf(g.km.A[lb][mb < 0 ? -mb : mb]), sum));
                Bst[boff + (M + L) * nb + (mb + lb)] = scale2(scale2(blk, s1), s2);
            }
        }
        boff += (2 * L + 1) * nb;
    }

    const int nt = 2 * lt + 1;
    const int rbase = g.gaunt_base[la * 7 + lt];
    double *out = g.out + g.out_off[p];
    for (int ma = 0; ma < 2 * la + 1; ++ma)
        for (int mt = 0; mt < nt; ++mt) {
            const int r = rbase + ma * nt + mt;
            df acc[2 * kLmax2c + 1];
            for (int mb = 0; mb < nb; ++mb) acc[mb] = df_f(0.0f);
            for (int q = g.gaunt_row[r]; q < g.gaunt_row[r + 1]; ++q) {
                const GauntEnt ge = g.gaunt[q];
                const int iL = (ge.L - Lmin) / 2;
                const int off_L = iL * (2 * Lmin + 1 + 2 * (iL - 1)) * nb;
                const df *bl = Bst + off_L + (ge.M + ge.L) * nb;
                const df gd = split_d(ge.g);
                for (int mb = 0; mb < nb; ++mb) acc[mb] = add(acc[mb], mul(gd, bl[mb]));
            }
            double *o = out + (ma * nt + mt) * nb;
            for (int mb = 0; mb < nb; ++mb) o[mb] = to_double(acc[mb]);
        }
}

// d R^{c/s}_{l,m} / dv_d (d = x, y, z) for 0 <= m <= l <= lmax from the (l-1)
// harmonics (lowering rules of the regular scaled solid harmonics).
__device__ __forceinline__ void harmonic_gradients3(const double *Rc, const double *Rs, int lmax, double (*dRc)[66],
                                                    double (*dRs)[66])
{
    for (int l = 0; l <= lmax; ++l)
        for (int m = 0; m <= l; ++m) {
            const int i = l * (l + 1) / 2 + m;
            if (l == 0) {
                for (int d = 0; d < 3; ++d) dRc[d][i] = dRs[d][i] = 0.0;
                continue;
            }
            const double cp = rc_get(Rc, l - 1, m + 1), cm = rc_get(Rc, l - 1, m - 1);
            const double sp = rs_get(Rs, l - 1, m + 1), sm = rs_get(Rs, l - 1, m - 1);
            dRc[0][i] = 0.5 * (cp - cm);
            dRs[0][i] = 0.5 * (sp - sm);
            dRc[1][i] = 0.5 * (sp + sm);
            dRs[1][i] = -0.5 * (cp + cm);
            dRc[2][i] = rc_get(Rc, l - 1, m);
            dRs[2][i] = rs_get(Rs, l - 1, m);
        }
}

// Vector-Jacobian product of one (a b a~) block with respect to the common
// center R_a of a and a~: the upstream block U is projected through the real
// Gaunt coefficients onto each L_a term, U_L[M][mb] = sum G U[ma][ma~][mb],
// and each term contributes the two-center VJP of Eq. dev_ab with P_L:
//   2 (R_a - R_b) sum_j P_L^{(L+lb-j+1)} <U_L, Q~_j> + sum_j P_L^{(L+lb-j)} <U_L, dQ~_j>.
__device__ void triple_aab_grad_fp64(const Args3c &g, int p)
{
    const ShellRec sa = g.orb_shells[g.t_a[p]];
    const ShellRec st = g.orb_shells[g.t_t[p]];
    const ShellRec sb = g.aux_shells[g.t_b[p]];
    const int la = sa.l, lt = st.l, lb = sb.l;
    const Vec4 A = g.orb_centers[sa.center];
    const Vec4 B = g.aux_centers[sb.center];
    const double v[3] = {A.x - B.x, A.y - B.y, A.z - B.z};
    const double R2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const int Lmin = la > lt ? la - lt : lt - la;
    const int Lmax = la + lt;
    const int nL = (Lmax - Lmin) / 2 + 1;
    const int pmax = nL - 1;
    const int kmaxA = Lmax + lb + 1;
    const int kminA = Lmin > lb ? Lmin : lb;

    // P[iL][j] = P_L^{(L+lb+1-j)}, j = 0..J_L
    double P[kNL][kJmax + 1];
    for (int i = 0; i < kNL; ++i)
        for (int j = 0; j <= kJmax; ++j) P[i][j] = 0.0;
    const int Ka = sa.nprim, Kt = st.nprim, Kb = sb.nprim;
    const int ntrip = Ka * Kt * Kb;
    // per (a, a~) primitive pair (ib == 0), as in aab_radial
    double ap = 0.0, wat = 0.0, wL0 = 0.0, i2ap2 = 0.0;
    double ia_p[kPmax + 1];
    for (int q = 0; q < ntrip; ++q) {
        const int ib = q % Kb;
        if (ib == 0) {
            const int it = (q / Kb) % Kt;
            const int ia = q / (Kb * Kt);
            const PrimRec pa = g.orb_prims[sa.prim_off + ia];
            const PrimRec pt = g.orb_prims[st.prim_off + it];
            ap = pa.alpha + pt.alpha;
            const double rap = rsqrt(ap);
            const double iap = rap * rap;
            wat = pa.wN * pt.wN * kPi32;
            ia_p[0] = 1.0;
            for (int m = 1; m <= pmax; ++m) ia_p[m] = ia_p[m - 1] * iap;
            const double i2ap = 0.5 * iap;
            wL0 = powi(i2ap, Lmin);
            i2ap2 = i2ap * i2ap;
        }
        const PrimRec pb = g.aux_prims[sb.prim_off + ib];
        const double be = pb.alpha;
        const double c = ap + be;
        const double rc = rsqrt(c);
        const double ic = rc * rc;
        const double rho = ap * be * ic;
        const double gg = be * be * ic;
        const double x = gg * R2;
        const double h = 0.5 * ic;
        const double w0 = wat * pb.w2c * ic * rc * exp(-rho * R2);
        double gp[kPmax + 1], hm[kPmax + 1];
        gp[0] = hm[0] = 1.0;
        for (int m = 1; m <= pmax; ++m) {
            gp[m] = gp[m - 1] * gg;
            hm[m] = hm[m - 1] * h;
        }
        double GD[kPmax + 1][kPmax + 1];
        for (int m = 0; m <= pmax; ++m)
            for (int i = 0; i <= m; ++i) {
                double s = g.k3.dd[m][i][m];
                for (int jj = m - 1; jj >= i; --jj) s = fma(s, x, g.k3.dd[m][i][jj]);
                GD[m][i] = gp[i] * s;
            }
        double nr[kKmax3 + 2];
        nr[0] = 1.0;
        for (int n = 1; n <= kmaxA; ++n) nr[n] = nr[n - 1] * -rho;
        double V[kPmax + 1][kKmax3 + 2];
        for (int k = kminA; k <= kmaxA; ++k) {
            double bn[kPmax + 1];
            const int imax = pmax < k ? pmax : k;
            for (int i = 0; i <= imax; ++i) bn[i] = g.k3.binom[k][i] * nr[k - i];
            for (int m = 0; m <= pmax; ++m) {
                double vv = 0.0;
                const int im = m < k ? m : k;
                for (int i = 0; i <= im; ++i) vv = fma(bn[i], GD[m][i], vv);
                V[m][k] = hm[m] * vv;
            }
        }
        double wL = w0 * wL0;
        for (int iL = 0; iL < nL; ++iL) {
            const int L = Lmin + 2 * iL;
            const int pL = pmax - iL;
            const int J = (L < lb ? L : lb) + 1;
            const int kmaxL = L + lb + 1;
            double bj[kPmax + 1];
            for (int jj = 0; jj <= pL; ++jj) bj[jj] = g.k3.bj[L][pL][jj] * ia_p[jj];
            for (int j = 0; j <= J; ++j) {
                const int k = kmaxL - j;
                double s = 0.0;
                for (int jj = 0; jj <= pL; ++jj) s = fma(bj[jj], V[pL - jj][k], s);
                P[iL][j] = fma(wL, s, P[iL][j]);
            }
            wL *= i2ap2;
        }
    }

    double Rc[66], Rs[66];
    const int lR = Lmax > lb ? Lmax : lb;
    scaled_harmonics(v[0], v[1], v[2], lR, g.k, Rc, Rs);
    double dRc[3][66], dRs[3][66];
    harmonic_gradients3(Rc, Rs, lR, dRc, dRs);
    const int nb = 2 * lb + 1, nt = 2 * lt + 1;
    const int Jmax = (Lmax < lb ? Lmax : lb) + 1;
    double Wb[2 * kLmax2c + 1][kJmax * kJmax];
    for (int mb = -lb; mb <= lb; ++mb) w_row_rt(Rc, Rs, lb, mb, Jmax, Wb[mb + lb]);

    // U_L[M][mb]: upstream block projected through the Gaunt coefficients
    double Ust[(1 + 5 + 9 + 13 + 17 + 21) * (2 * kLmax2c + 1)];
    int ntot = 0;
    for (int iL = 0; iL < nL; ++iL) ntot += (2 * (Lmin + 2 * iL) + 1) * nb;
    for (int i = 0; i < ntot; ++i) Ust[i] = 0.0;
    const double *Wup = g.w + g.w_off[p];
    const int rbase = g.gaunt_base[la * 7 + lt];
    for (int ma = 0; ma < 2 * la + 1; ++ma)
        for (int mt = 0; mt < nt; ++mt) {
            const int r = rbase + ma * nt + mt;
            const double *u = Wup + (ma * nt + mt) * nb;
            for (int q = g.gaunt_row[r]; q < g.gaunt_row[r + 1]; ++q) {
                const GauntEnt ge = g.gaunt[q];
                const int iL = (ge.L - Lmin) / 2;
                double *ul = Ust + iL * (2 * Lmin + 1 + 2 * (iL - 1)) * nb + (ge.M + ge.L) * nb;
                for (int mb = 0; mb < nb; ++mb) ul[mb] = fma(ge.g, u[mb], ul[mb]);
            }
        }

    const double sgn_b = (lb & 1) ? -1.0 : 1.0;
    const double lam0 = 3.5449077018110320545963349666822903 / (g.k3.sqrt_int[2 * la + 1] * g.k3.sqrt_int[2 * lt + 1]);
    double G1 = 0.0, G2[3] = {0.0, 0.0, 0.0};
    for (int iL = 0; iL < nL; ++iL) {
        const int L = Lmin + 2 * iL;
        const int J = (L < lb ? L : lb) + 1;
        const int JJ = J * J;
        const double lamK = lam0 * g.k3.sqrt_int[2 * L + 1];
        double f0[kJmax * kJmax], f1[kJmax * kJmax];
        for (int j = 0; j < J; ++j) {
            const double b2 = lamK * g.k.pow2[L + lb - j];
            for (int kp = 0; kp <= j; ++kp) {
                const double bb = b2 * g.k.jB[j][kp];
                const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
                f0[e0] = bb * P[iL][j + 1];
                f1[e0] = bb * P[iL][j];
                if (kp) {
                    f0[e0 + 1] = f0[e0];
                    f1[e0 + 1] = f1[e0];
                }
            }
        }
        const double *UL = Ust + iL * (2 * Lmin + 1 + 2 * (iL - 1)) * nb;
        double Y[2 * kLmax2c + 1][kJmax * kJmax];
        for (int mb = 0; mb < nb; ++mb)
            for (int e = 0; e < JJ; ++e) Y[mb][e] = 0.0;
        for (int M = -L; M <= L; ++M) {
            double wa[kJmax * kJmax], z[kJmax * kJmax];
            w_row_rt(Rc, Rs, L, M, J, wa);
            const double Aa = g.k.A[L][M < 0 ? -M : M] * sgn_b;
            for (int e = 0; e < JJ; ++e) z[e] = 0.0;
            for (int mb = -lb; mb <= lb; ++mb) {
                const double ua = UL[(M + L) * nb + (mb + lb)] * Aa * g.k.A[lb][mb < 0 ? -mb : mb];
                for (int e = 0; e < JJ; ++e) {
                    z[e] = fma(ua, Wb[mb + lb][e], z[e]);
                    Y[mb + lb][e] = fma(ua, wa[e], Y[mb + lb][e]);
                }
            }
            for (int e = 0; e < JJ; ++e) G1 = fma(f1[e] * wa[e], z[e], G1);
            for (int d = 0; d < 3; ++d) {
                double dw[kJmax * kJmax];
                w_row_rt(dRc[d], dRs[d], L, M, J, dw);
                for (int e = 0; e < JJ; ++e) G2[d] = fma(f0[e] * dw[e], z[e], G2[d]);
            }
        }
        for (int mb = -lb; mb <= lb; ++mb)
            for (int d = 0; d < 3; ++d) {
                double dw[kJmax * kJmax];
                w_row_rt(dRc[d], dRs[d], lb, mb, J, dw);
                for (int e = 0; e < JJ; ++e) G2[d] = fma(f0[e] * dw[e], Y[mb + lb][e], G2[d]);
            }
    }
    for (int d = 0; d < 3; ++d) {
        const double gd = fma(2.0 * v[d], G1, G2[d]);
        g.grad_a[3 * (int64_t)p + d] = gd;
        if (g.grad_b) g.grad_b[3 * (int64_t)p + d] = -gd;
    }
}

__global__ void __launch_bounds__(128) k_3c_grad_fp64_persistent(const Args3c g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        const Tile tl = g.tiles[t];
        if (lane < tl.count) triple_aab_grad_fp64(g, g.perm[tl.start + lane]);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) k_3c_mixed_persistent(const Args3c g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        const Tile tl = g.tiles[t];
        if (lane < tl.count) triple_aab_mixed(g, g.perm[tl.start + lane]);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) k_3c_fp64_persistent(const Args3c g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        const Tile tl = g.tiles[t];
        if (lane < tl.count) triple_aab_fp64(g, g.perm[tl.start + lane]);
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_3c(const Args3c &a, int precision, int grid, cudaStream_t s)
{
    if (a.grad_a)
        k_3c_grad_fp64_persistent<<<grid, 128, 0, s>>>(a);
    else if (precision == 1)
        k_3c_mixed_persistent<<<grid, 128, 0, s>>>(a);
    else
        k_3c_fp64_persistent<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

int persistent_grid_3c(int precision)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = precision == 1
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_3c_mixed_persistent, 128, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_3c_grad_fp64_persistent, 128, 0);
    if (e != cudaSuccess || per < 1) per = 1;
    return (sms > 0 ? sms : 1) * per;
}

}  // namespace shg
