// fl_ffmath.cuh -- elementary functions in float pairs (type ff of
// fl_common.cuh) for the FP64-accuracy form FL_FP64_FF, so that its gather and
// direct bands need no FP64 arithmetic (GB300 issues FP64 at 1/64 of the FP32
// rate).  Each function is written from its series definition with a
// classical argument reduction; accuracy is a few 2^-48 relative to the
// result (exp, sqrt, division) or absolute (sincospi), enough for the
// window values, barycentric weights and phases of a 1e-12 transform.
#pragma once

#include "fl_common.cuh"

namespace fl {

// hi = fl(hi + lo), lo the exact remainder (Knuth's error-free sum: any order).
__device__ __forceinline__ ff ff_norm(ff a) {
    const float s = a.hi + a.lo;
    const float bb = s - a.hi;
    return ff(s, (a.hi - (s - bb)) + (a.lo - bb));
}

// a / b: the float quotient q0 corrected by the remainder a - q0 b, formed
// with the error-free product q0 * b.hi (Newton's correction for division).
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    b = ff_norm(b);
    const float r = 1.0f / b.hi;
    const float q0 = a.hi * r;
    const float p = q0 * b.hi;
    const float e = fmaf(q0, b.hi, -p);
    const float rem = ((a.hi - p) - e) + fmaf(-q0, b.lo, a.lo);
    return ff(q0, rem * r);
}

// sqrt(a), a >= 0: r = sqrtf(a.hi) plus Newton's correction (a - r^2) / (2 r)
// with r^2 formed exactly; 0 for a <= 0.
__device__ __forceinline__ ff ff_sqrt(ff a) {
    a = ff_norm(a);
    if (!(a.hi > 0.f)) return ff(0.f);
    const float r = sqrtf(a.hi);
    const float p = r * r;
    const float e = fmaf(r, r, -p);
    const float d = ((a.hi - p) - e) + a.lo;
    return ff(r, d * (0.5f / r));
}

// e^x for x in [-104, 88].  Cody-Waite reduction x = k ln 2 + r, |r| <= ln2/2,
// with ln 2 split into three floats (16 + 24 + 24 significant bits, so k times
// the first is exact for |k| < 2^8 and the reduction error is below 2^-60), then
// the Taylor series of e^r to degree 12 (remainder below 2^-50) by Horner in
// float pairs, and the exact scaling by 2^k.
__device__ __forceinline__ ff ff_exp(ff x) {
    constexpr float kLn2a = 0x1.62e4p-1f;        // ln 2 to 16 bits
    constexpr float kLn2b = 0x1.7f7d1cp-20f;     // next 24 bits
    constexpr float kLn2c = 0x1.ef357ap-45f;     // next 24 bits
    x = ff_norm(x);
    const float k = rintf(x.hi * 1.44269504f);
    const float s1 = x.hi - k * kLn2a;           // exact (Sterbenz-type: |s1| < 1/2)
    const float p = k * kLn2b;
    const float pe = fmaf(k, kLn2b, -p);
    ff r = ff(s1, 0.f) + ff(-p, 0.f);
    r.lo += (x.lo - pe) - k * kLn2c;
    // 1/n!, n = 12 .. 1, rounded from double
    constexpr double kInvFact[13] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720,
                                     1.0 / 5040, 1.0 / 40320, 1.0 / 362880, 1.0 / 3628800,
                                     1.0 / 39916800, 1.0 / 479001600};
    ff y = ff(kInvFact[12]);
#pragma unroll
    for (int n = 11; n >= 0; --n) y = y * r + ff(kInvFact[n]);
    const int ki = (int)k;
    return ff(ldexpf(y.hi, ki), ldexpf(y.lo, ki));
}

// sin(pi a), cos(pi a) for a in [-1, 1]: reflections to |a| <= 1/2 and to
// |a| <= 1/4 (sin(pi (1/2 - b)) = cos(pi b)), then the Taylor series of sin t
// and cos t at t = pi a, |t| <= pi/4, to degree 17 / 16 (remainders below
// 2^-60), pi as a float pair.
__device__ __forceinline__ void ff_sincospi(ff a, ff* s, ff* c) {
    constexpr float kPiHi = 0x1.921fb6p+1f, kPiLo = -0x1.777a5cp-24f;
    a = ff_norm(a);
    float cs = 1.f;                     // sign of the cosine after the reflection about 1
    if (a.hi > 0.5f) {
        a = ff(1.f) - a;
        cs = -1.f;
    } else if (a.hi < -0.5f) {
        a = ff(-1.f) - a;
        cs = -1.f;
    }
    bool swap = false;
    float sg = 1.f;
    if (a.hi > 0.25f) {
        a = ff(0.5f) - a;
        swap = true;
    } else if (a.hi < -0.25f) {
        a = ff(-0.5f) - a;
        swap = true;
        sg = -1.f;
    }
    const ff t = a * ff(kPiHi, kPiLo);
    const ff t2 = t * t;
    // sin t = t sum_n (-1)^n t^(2n) / (2n+1)!, cos t = sum_n (-1)^n t^(2n) / (2n)!
    constexpr double kSin[9] = {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880,
                                -1.0 / 39916800, 1.0 / 6227020800.0, -1.0 / 1307674368000.0,
                                1.0 / 355687428096000.0};
    constexpr double kCos[9] = {1.0, -1.0 / 2, 1.0 / 24, -1.0 / 720, 1.0 / 40320,
                                -1.0 / 3628800, 1.0 / 479001600, -1.0 / 87178291200.0,
                                1.0 / 20922789888000.0};
    ff ps = ff(kSin[8]), pc = ff(kCos[8]);
#pragma unroll
    for (int n = 7; n >= 0; --n) {
        ps = ps * t2 + ff(kSin[n]);
        pc = pc * t2 + ff(kCos[n]);
    }
    ps = ps * t;
    ff sv = swap ? pc : ps, cv = swap ? ps : pc;
    sv = ff(sg * sv.hi, sg * sv.lo);
    cv = ff(sg * cs * cv.hi, sg * cs * cv.lo);
    *s = sv;
    *c = cv;
}

// Kaiser-Bessel window in grid units, phi(t) = sinh(b r) / r, r = sqrt(m^2 - t^2),
// |t| <= m (b at the edge), as in kb_window: sinh from one exponential,
// (e^u - 1/e^u) / 2.  Near the edge (small b r) the difference loses relative
// accuracy, but those taps are smaller than the centre tap by about e^(b m),
// so the error stays a few 2^-48 of the window sum.
__device__ __forceinline__ ff ff_kb_window(ff t, float m, ff b) {
    const ff s2 = ff(m * m) - t * t;
    const ff r = ff_sqrt(s2);
    if (!(r.hi > 0.f)) return b;
    const ff e = ff_exp(b * r);
    const ff sh = (e - ff_div(ff(1.f), e)) * ff(0.5f);
    return ff_div(sh, r);
}

}  // namespace fl
