// Double-float arithmetic (an unevaluated sum hi + lo of two FP32 numbers,
// |lo| <= ulp(hi)/2) for the mixed-precision kernels.  Built on the
// error-free transformations TwoSum (Knuth), FastTwoSum (Dekker) and the
// FMA-based TwoProd; relative error of one operation about 2^-44 of the
// operand magnitudes (the additions are the "sloppy" variant: their error is
// relative to |a| + |b|, which is the scale the parity bar of cancelling
// contractions is measured against).
#pragma once

namespace shg {
namespace dfm {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df make_df(float h, float l) { return df{h, l}; }
__device__ __forceinline__ df df_f(float a) { return df{a, 0.0f}; }

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = a + b;
    return df{s, b - (s - a)};
}

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return df{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }

__device__ __forceinline__ df add_f(df a, float b)
{
    df s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df mul(df a, df b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df mul_f(df a, float b)
{
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

// exact scaling by a power of two
__device__ __forceinline__ df scale2(df a, float p2) { return df{a.hi * p2, a.lo * p2}; }

// a*b + c
__device__ __forceinline__ df fma_df(df a, df b, df c) { return add(mul(a, b), c); }

// 1/sqrt(a), a > 0: FP32 estimate r (relative error ~2^-23) and one Newton
// step r + r (1 - a r^2) / 2.  a r^2 = q + s with q = fl(a.hi r^2) and the
// rest s from the exact FP32 products (FMA); q is within 2^-21 of 1, so 1 - q
// is exact and e = (1 - q) - s carries 1 - a r^2 to ~2^-46 absolute.  The
// correction r e / 2 (~2^-23 r) in FP32 then adds an error of ~2^-47 r.
__device__ __forceinline__ df rsqrt_df(df a)
{
    const float r = rsqrtf(a.hi);
    const float p = r * r;
    const float pe = fmaf(r, r, -p);                // r^2 = p + pe exactly
    const float q = a.hi * p;
    float t = fmaf(a.hi, p, -q);                    // a.hi p = q + t exactly
    t = fmaf(a.hi, pe, t);
    t = fmaf(a.lo, p, t);
    const float e = (1.0f - q) - t;
    return fast_two_sum(r, (0.5f * r) * e);
}

__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace dfm
}  // namespace shg
