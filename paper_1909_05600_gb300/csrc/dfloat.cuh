// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 2^-44 relative accuracy, computed on the FP32 pipe (this part
// runs FP64 at a small fraction of its FP32 rate).  The error-free transformations are
// Knuth's TwoSum, the fast TwoSum of Dekker (|a| >= |b|) and the product split by fused
// multiply-add; additions use the short form whose error is bounded relative to the
// operands (enough for sums whose cancellation is bounded separately).  Every rounding
// step uses an explicit round-to-nearest intrinsic so that no multiply-add is contracted.
#pragma once

#include <cuda_runtime.h>

namespace ffm {

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h) : hi(h), lo(0.f) {}
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dd(s, e);
}
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);  // exact rounding error of the product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}
__device__ __forceinline__ dd operator*(dd a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return dd_fast_two_sum(p, e);
}
// keep the FP32 / FP64 fma overloads visible beside the double-float ones in this namespace
using ::fma;
__device__ __forceinline__ dd fma(dd a, dd b, dd c) { return a * b + c; }
__device__ __forceinline__ dd fma(dd a, float b, dd c) { return a * b + c; }

struct dd2 {
    dd x, y;
};
struct dd4 {
    dd x, y, z, w;
};
struct dd3 {
    dd x, y, z;
};

// sin and cos of a double-float argument, to about 1e-13 absolute.  x = n pi/2 + r with
// |r| <= pi/4 (pi/2 split into three FP32 parts; n pi/2's leading product is split
// exactly), then r = a + b with a = j/64 taken from a table of sin a, cos a (entries
// j = -DD_SC_J..DD_SC_J, as (sin.hi, sin.lo, cos.hi, cos.lo)) and |b| <= 1/128, for
// which sin b = b - b^3/6 + b^5/120 and cos b = 1 - b^2/2 + b^4/24 (the first omitted
// terms are below 1e-17), then the angle-sum formulas and the quadrant's symmetry.
constexpr int DD_SC_J = 51;  // |r| * 64 <= 50.3

__device__ __forceinline__ void dd_sincos(dd x, dd &s, dd &c, const float4 *__restrict__ tab) {
    constexpr double PIO2 = 1.5707963267948966;
    constexpr float P0 = (float)PIO2;
    constexpr float P1 = (float)(PIO2 - (double)P0);
    constexpr float P2 = (float)(PIO2 - (double)P0 - (double)P1);
    constexpr float TWO_OVER_PI = (float)(2.0 / 3.14159265358979323846);
    // n = nearest integer of x 2/pi (1.5 2^23 shifter); its low bits give the quadrant
    float t = fmaf(x.hi, TWO_OVER_PI, 12582912.f);
    float n = __fsub_rn(t, 12582912.f);
    int q = __float_as_int(t) & 3;
    float p = __fmul_rn(n, P0);
    float pe = fmaf(n, P0, -p);
    float rh = __fsub_rn(x.hi, p);  // exact: x.hi and n P0 agree to within pi/4
    float rl = __fsub_rn(__fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(n, P1)), __fmul_rn(n, P2));
    dd r = dd_two_sum(rh, rl);
    float tj = fmaf(r.hi, 64.f, 12582912.f);
    float jf = __fsub_rn(tj, 12582912.f);
    int j = __float_as_int(tj) - 0x4B400000;  // tj = 1.5 2^23 + j, unit in the last place 1
    float a = __fmul_rn(jf, 0.015625f);
    dd b = dd_fast_two_sum(__fsub_rn(r.hi, a), r.lo);  // r.hi - a is exact (Sterbenz)
    float4 T = __ldg(tab + (j + DD_SC_J));
    float b2 = __fmul_rn(b.hi, b.hi);
    // sin b = b + b^3 (-1/6 + b^2/120)
    dd sb = b + dd(__fmul_rn(__fmul_rn(b.hi, b2), fmaf(b2, 1.f / 120.f, -1.f / 6.f)));
    // cos b = 1 - (b^2)/2 + b^4/24 with b^2 split exactly
    float b2e = fmaf(b.hi, b.hi, -b2);
    b2e = fmaf(2.f * b.hi, b.lo, b2e);
    dd cb = dd(1.f) + (dd(-0.5f * b2, -0.5f * b2e) + dd(__fmul_rn(__fmul_rn(b2, b2), 1.f / 24.f)));
    dd sa(T.x, T.y), ca(T.z, T.w);
    dd sr = sa * cb + ca * sb;
    dd cr = ca * cb - sa * sb;
    dd u = (q & 1) ? cr : sr, v = (q & 1) ? sr : cr;
    s = (q & 2) ? -u : u;
    c = ((q + 1) & 2) ? -v : v;
}

}  // namespace ffm
