// Angular part of the two-center vector-Jacobian product (Sec. II E, Eq.
// dev_ab), shared by the FP64 and the mixed-precision gradient kernels: given
// the radial orders of one pair as the weights
//   f0[e] = 2^{kmax-j} (2j-1)!! B_{j,kappa} O^{(kmax-j)}
//   f1[e] = 2^{kmax-j} (2j-1)!! B_{j,kappa} O^{(kmax-j+1)}
// of the translation-matrix entries e = (j, kappa, z), it forms
//   g_i = 2 (R_a - R_b)_i <W, Q~(f1)> + <W, dQ~(f0)/dR_{a,i}>
// with dQ~ from the lowering rules of the regular scaled solid harmonics,
// and writes grad_a[p] (and grad_b[p] = -grad_a[p]).
#pragma once

#include "shg_device.cuh"

namespace shg {
namespace gradang {
using namespace dev;

constexpr int kNR = (kLmax2c + 1) * (kLmax2c + 2) / 2;

// derivative tables dR^{c/s}/dv_d, d = x, y, z, for 0 <= m <= l <= lmax
__device__ __forceinline__ void harmonic_gradients(const double *Rc, const double *Rs, int lmax, double (*dRc)[kNR],
                                                   double (*dRs)[kNR])
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

template <int J>
__device__ __forceinline__ void grad_from_orders(const Args2c &g, int p, int la, int lb, const double (&v)[3],
                                                 const double (&f0)[J * J], const double (&f1)[J * J])
{
    double Rc[kNR], Rs[kNR];
    const int lmax = la > lb ? la : lb;
    scaled_harmonics(v[0], v[1], v[2], lmax, g.k, Rc, Rs);
    double dRc[3][kNR], dRs[3][kNR];
    harmonic_gradients(Rc, Rs, lmax, dRc, dRs);

    const int nb = 2 * lb + 1;
    double Wb[2 * kLmax2c + 1][J * J];
    for (int mb = -lb; mb <= lb; ++mb) {
        double w[J * J];
        w_row<J>(Rc, Rs, lb, mb, w);
#pragma unroll
        for (int e = 0; e < J * J; ++e) Wb[mb + lb][e] = w[e];
    }
    const double *Wup = g.w + g.w_off[p];
    const double sgn_b = (lb & 1) ? -1.0 : 1.0;
    double Y[2 * kLmax2c + 1][J * J];
    for (int mb = 0; mb < nb; ++mb)
#pragma unroll
        for (int e = 0; e < J * J; ++e) Y[mb][e] = 0.0;
    double G1 = 0.0, G2[3] = {0.0, 0.0, 0.0};
    for (int ma = -la; ma <= la; ++ma) {
        double wa[J * J], z[J * J];
        w_row<J>(Rc, Rs, la, ma, wa);
        const double Aa = g.k.A[la][ma < 0 ? -ma : ma] * sgn_b;
#pragma unroll
        for (int e = 0; e < J * J; ++e) z[e] = 0.0;
        for (int mb = -lb; mb <= lb; ++mb) {
            const double ua = Wup[(ma + la) * nb + (mb + lb)] * Aa * g.k.A[lb][mb < 0 ? -mb : mb];
#pragma unroll
            for (int e = 0; e < J * J; ++e) {
                z[e] = fma(ua, Wb[mb + lb][e], z[e]);
                Y[mb + lb][e] = fma(ua, wa[e], Y[mb + lb][e]);
            }
        }
#pragma unroll
        for (int e = 0; e < J * J; ++e) G1 = fma(f1[e] * wa[e], z[e], G1);
        // compact (runtime-J) dW rows: six unrolled copies per J cost more in
        // instruction fetch than the loops do
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            double dw[kJmax * kJmax];
            w_row_rt(dRc[d], dRs[d], la, ma, J, dw);
#pragma unroll
            for (int e = 0; e < J * J; ++e) G2[d] = fma(f0[e] * dw[e], z[e], G2[d]);
        }
    }
    for (int mb = -lb; mb <= lb; ++mb)
        // compact (runtime-J) dW rows: six unrolled copies per J cost more in
        // instruction fetch than the loops do
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            double dw[kJmax * kJmax];
            w_row_rt(dRc[d], dRs[d], lb, mb, J, dw);
#pragma unroll
            for (int e = 0; e < J * J; ++e) G2[d] = fma(f0[e] * dw[e], Y[mb + lb][e], G2[d]);
        }
    for (int d = 0; d < 3; ++d) {
        const double gd = fma(2.0 * v[d], G1, G2[d]);
        g.grad_a[3 * (int64_t)p + d] = gd;
        if (g.grad_b) g.grad_b[3 * (int64_t)p + d] = -gd;
    }
}

}  // namespace gradang
}  // namespace shg
