// Double-float angular helpers shared by the mixed-precision kernels: the
// regular scaled solid harmonics R^{c/s}_{l,m}(v) (Sec. II E recursions) and
// rows of the real translation matrix W, with runtime l and J (one compact
// copy serves every class).
#pragma once

#include "shg_device.cuh"
#include "shg_df.cuh"

namespace shg {
namespace mixa {
namespace {
using namespace dfm;

__device__ __forceinline__ df ldf(float2 v) { return df{v.x, v.y}; }

__device__ __forceinline__ df rcm(const df *Rc, int L, int m)
{
    const int am = m < 0 ? -m : m;
    if (L < 0 || am > L) return df_f(0.0f);
    const df v = Rc[L * (L + 1) / 2 + am];
    return (m < 0 && (am & 1)) ? neg(v) : v;
}
__device__ __forceinline__ df rsm(const df *Rs, int L, int m)
{
    const int am = m < 0 ? -m : m;
    if (L < 0 || am > L) return df_f(0.0f);
    const df v = Rs[L * (L + 1) / 2 + am];
    return (m < 0 && !(am & 1)) ? neg(v) : v;
}

__device__ __noinline__ void scaled_harmonics_mix(df x, df y, df z, int lmax, const ConstsMix &k, df *Rc, df *Rs)
{
    const df r2 = add(add(mul(x, x), mul(y, y)), mul(z, z));
    Rc[0] = df_f(1.0f);
    Rs[0] = df_f(0.0f);
    for (int l = 0; l < lmax; ++l) {
        const int d0 = l * (l + 1) / 2, d1 = (l + 1) * (l + 2) / 2, dm = (l - 1) * l / 2;
        const df cll = Rc[d0 + l], sll = Rs[d0 + l];
        const df inv = ldf(k.inv_int[2 * l + 2]);
        Rc[d1 + l + 1] = neg(mul(sub(mul(x, cll), mul(y, sll)), inv));
        Rs[d1 + l + 1] = neg(mul(add(mul(y, cll), mul(x, sll)), inv));
        const df zl = mul_f(z, (float)(2 * l + 1));
        for (int m = 0; m <= l; ++m) {
            const df im = ldf(k.inv_int[(l + m + 1) * (l - m + 1)]);
            df vc = mul(zl, Rc[d0 + m]);
            if (m <= l - 1) vc = sub(vc, mul(r2, Rc[dm + m]));
            Rc[d1 + m] = mul(vc, im);
            if (m == 0) {
                Rs[d1] = df_f(0.0f);
            } else {
                df vs = mul(zl, Rs[d0 + m]);
                if (m <= l - 1) vs = sub(vs, mul(r2, Rs[dm + m]));
                Rs[d1 + m] = mul(vs, im);
            }
        }
    }
}

// Runtime-J row of W (compact code: one copy serves every class).
__device__ __noinline__ void w_row_mix_rt(const df *Rc, const df *Rs, int l, int m, int J, df *w)
{
    const int mu = m < 0 ? -m : m;
    const bool sine = m < 0;
    for (int j = 0; j < J; ++j) {
        const int L = l - j;
        w[j * j] = sine ? rsm(Rs, L, mu) : rcm(Rc, L, mu);
        for (int kp = 1; kp <= j; ++kp) {
            const int e0 = j * j + 2 * kp - 1;
            const df cm = rcm(Rc, L, mu - kp), cp = rcm(Rc, L, mu + kp);
            const df sm = rsm(Rs, L, mu - kp), sp = rsm(Rs, L, mu + kp);
            const bool odd = kp & 1;
            if (!sine) {
                w[e0] = odd ? sub(cm, cp) : add(cm, cp);
                w[e0 + 1] = odd ? neg(add(sm, sp)) : sub(sp, sm);
            } else {
                w[e0] = odd ? sub(sm, sp) : add(sm, sp);
                w[e0 + 1] = odd ? add(cm, cp) : sub(cm, cp);
            }
        }
    }
}

}  // namespace
}  // namespace mixa
}  // namespace shg
