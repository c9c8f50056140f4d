// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two float32 numbers with |lo| <= ulp(hi)/2, giving about 48
// significant bits on the float32 pipes.  GB300 issues float32 FMAs at 64x its
// float64 rate, so float64-accuracy FFTs run faster this way.  Error-free
// transformations: Knuth's two-sum, Dekker's fast two-sum, and the
// FMA-based two-product (a*b - fl(a*b) computed exactly by one fmaf).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace nufft45 {

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (exact for |x| in the float range to ~2^-48 relative)
    __host__ __device__ constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ constexpr dd(int x) : hi((float)x), lo(0.f) {}
};

__host__ __device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
    const float s = a + b;
    return dd(s, b - (s - a));
}

__host__ __device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    return dd(s, (a - (s - v)) + (b - v));
}

__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) { a = a + b; return a; }
__host__ __device__ __forceinline__ dd& operator-=(dd& a, dd b) { a = a - b; return a; }
__host__ __device__ __forceinline__ dd& operator*=(dd& a, dd b) { a = a * b; return a; }

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dd dd_from_double(double x) {
    const float h = __double2float_rn(x);
    return dd(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ dd dd_mul_f(dd a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return dd_fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_add_f(dd a, float b) {
    dd s = dd_two_sum(a.hi, b);
    s.lo += a.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}
// a / b: float quotient, then one correction from the double-float remainder
__device__ __forceinline__ dd dd_div(dd a, dd b) {
    const float q0 = a.hi / b.hi;
    const dd r = a - dd_mul_f(b, q0);
    return dd_fast_two_sum(q0, r.hi / b.hi);
}
// sqrt(a), a >= 0: one Newton step from the float square root; s0^2 is split
// exactly by an FMA and a.hi - s0^2 is exact (Sterbenz), so the step carries
// the error from 2^-24 to about 2^-47
__device__ __forceinline__ dd dd_sqrt(dd a) {
    if (a.hi <= 0.f) return dd(0.f, 0.f);
    const float s0 = sqrtf(a.hi);
    const float p = s0 * s0;
    const float pe = fmaf(s0, s0, -p);
    const float res = ((a.hi - p) - pe) + a.lo;
    return dd_fast_two_sum(s0, res / (2.0f * s0));
}

// 2^(j/64), j < 64, rounded to double-float (hi, lo)
#define NUFFT_EXP2_64_TABLE {                                                                                     \
    {1.0f, 0.0f}, {1.0108892917633057f, -5.7116054108519165e-09f}, \
    {1.0218971967697144f, -4.811559861650494e-08f}, {1.0330249071121216f, -2.809089316713198e-08f}, \
    {1.0442737340927124f, 4.8334701574503924e-08f}, {1.055645227432251f, -4.9071694263602694e-08f}, \
    {1.0671404600143433f, -5.9337519786595294e-08f}, {1.0787607431411743f, 5.4615945543901034e-08f}, \
    {1.0905077457427979f, -1.3077539939843064e-08f}, {1.1023825407028198f, 4.260501995645427e-08f}, \
    {1.114386796951294f, -5.435540018083884e-08f}, {1.1265215873718262f, 3.12364143439936e-08f}, \
    {1.1387885808944702f, 5.386222312608879e-08f}, {1.1511892080307007f, 2.1922282655850722e-08f}, \
    {1.1637248992919922f, -4.051441493402308e-08f}, {1.1763969659805298f, 2.566975076945255e-08f}, \
    {1.1892070770263672f, 3.797635272917432e-08f}, {1.2021567821502686f, -5.069756525699631e-08f}, \
    {1.215247392654419f, -3.267394887984665e-08f}, {1.228480577468872f, -4.136200359994291e-08f}, \
    {1.2418577671051025f, 4.496838101886169e-08f}, {1.2553807497024536f, 7.3222374830095305e-09f}, \
    {1.2690509557724f, 1.419333317542737e-09f}, {1.2828700542449951f, -3.816621685359678e-08f}, \
    {1.2968395948410034f, -4.018999533172973e-08f}, {1.3109612464904785f, -3.496571565619888e-08f}, \
    {1.3252366781234741f, -3.496373324196611e-08f}, {1.339667558670044f, -3.4616739696957666e-08f}, \
    {1.3542555570602417f, -1.0123349269974824e-08f}, {1.3690024614334106f, -3.845881835218279e-08f}, \
    {1.3839099407196045f, -5.875577357983275e-08f}, {1.398979663848877f, 8.689434061182055e-09f}, \
    {1.4142135381698608f, 2.4203234971764687e-08f}, {1.4296133518218994f, -1.3429929168751187e-08f}, \
    {1.4451807737350464f, 3.324199937537742e-08f}, {1.4609178304672241f, -3.628657552212644e-08f}, \
    {1.4768261909484863f, -4.500898853621038e-08f}, {1.4929077625274658f, -3.4236201429393986e-08f}, \
    {1.5091644525527954f, -2.4959373234878512e-08f}, {1.525598168373108f, -1.7628568826921764e-08f}, \
    {1.5422108173370361f, 8.070904833346049e-09f}, {1.5590044260025024f, -2.5764665068095383e-08f}, \
    {1.5759809017181396f, -5.661025426206834e-08f}, {1.5931421518325806f, -4.903136785472384e-10f}, \
    {1.610490322113037f, 9.836217174097328e-09f}, {1.6280274391174316f, -1.7260083140513416e-08f}, \
    {1.6457555294036865f, -5.124972091152813e-08f}, {1.6636766195297241f, -3.9202987522912736e-08f}, \
    {1.6817928552627563f, -2.4755326677450284e-08f}, {1.7001063823699951f, -2.8651472305796233e-08f}, \
    {1.7186193466186523f, -4.8496175963919086e-08f}, {1.73733389377594f, -5.850223416814515e-08f}, \
    {1.7562521696090698f, -9.235770370707996e-09f}, {1.7753764390945435f, 5.3431978841445016e-08f}, \
    {1.7947090864181519f, -1.141504490931311e-08f}, {1.8142521381378174f, 3.736258236131107e-08f}, \
    {1.8340080976486206f, -1.1239277952768134e-08f}, {1.8539791107177734f, 1.4365611811228973e-08f}, \
    {1.8741676807403564f, -4.663005626071026e-08f}, {1.8945759534835815f, 2.8103384508426643e-08f}, \
    {1.9152065515518188f, 9.845328108326612e-09f}, {1.9360617399215698f, 5.357072296874321e-08f}, \
    {1.9571441411972046f, -1.7021804410433106e-08f}, {1.9784560203552246f, 6.032726318494497e-09f} }

// e^x for -87 < x <= 0 in double-float, by P. T. P. Tang's table-driven
// method ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989) with a Cody-Waite style
// additive reduction (W. J. Cody and W. Waite, "Software Manual for the
// Elementary Functions", 1980): x = (64 m + j) ln2/64 + r with
// |r| <= ln2/128, the reduction constant ln2/64 split as C1 + C2 + C3 with
// C1 of 12 significant bits so that k C1 is exact; then
// e^x = 2^m 2^(j/64) (1 + S), S = e^r - 1 = r + r^2/2 in double-float plus
// the Taylor terms r^3/6 + r^4/24 + r^5/120 + r^6/720 in float (truncation
// below |r|^7/5040 < 1e-16).  tab: the 2^(j/64) table above.  Absolute error
// below 4e-15 over the range, about 2^-48, the precision of the double-float
// format itself (measured maximum 3.5e-15 against long-double host values
// through the nufft_debug_dd_exp test hook).
__device__ __forceinline__ dd dd_exp_nonpos(dd x, const float2* tab) {
    const float kf = rintf(x.hi * 92.33248138427734f);
    const int k = (int)kf;
    dd r = dd_add_f(x, -kf * 0.010829925537109375f);
    const float c2 = 4.991591140424134e-07f;
    const float p2 = kf * c2;
    r = r - dd(p2, fmaf(kf, c2, -p2));
    r = dd_add_f(r, -kf * 2.572804640231345e-14f);
    const float rh = r.hi;
    const float tail = rh * rh * rh * fmaf(rh, fmaf(rh, fmaf(rh, 1.f / 720.f, 1.f / 120.f), 1.f / 24.f), 1.f / 6.f);
    const dd S = dd_add_f(r + dd_mul_f(r * r, 0.5f), tail);
    const int j = k & 63, m = k >> 6;
    const dd t(tab[j].x, tab[j].y);
    const dd e = t + t * S;
    const float sc = __int_as_float((m + 127) << 23);   // 2^m, m >= -126
    return dd(e.hi * sc, e.lo * sc);
}

// phi(d) = exp(beta (sqrt(1 - z^2) - 1)), z = d / h, h = w/2, in
// double-float.  With h exact the exponent is formed without rounding a
// constant 2/w and without cancellation:
//   beta (sqrt(1 - z^2) - 1) = -beta d^2 / (h (h + sqrt((h - d)(h + d)))).
__device__ __forceinline__ dd es_kernel_dd(dd d, float h, dd beta, const float2* tab) {
    const dd num = dd_add_f(-d, h) * dd_add_f(d, h);
    if (num.hi <= 0.f) return dd(0.f, 0.f);
    const dd x = -dd_div(beta * (d * d), dd_mul_f(dd_add_f(dd_sqrt(num), h), h));
    return dd_exp_nonpos(x, tab);
}

// complex double-float: the layout of float4 (re.hi, re.lo, im.hi, im.lo)
struct __align__(16) cdd {
    dd x, y;
};
template <> struct C2<dd> { using type = cdd; };

template <> __device__ __forceinline__ cdd ldg<cdd>(const cdd* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    cdd r;
    r.x = dd(v.x, v.y);
    r.y = dd(v.z, v.w);
    return r;
}
template <> __device__ __forceinline__ dd ldg<dd>(const dd* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dd(v.x, v.y);
}

}  // namespace nufft45
