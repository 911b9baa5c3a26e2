// Shared device helpers: complex arithmetic on float2/double2, constants.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SCINT_DEV __device__ __forceinline__

namespace scint {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kKmPerPc = 3.0856775814913673e13;
constexpr double kKmPerNm = 1.0e-12;

// ---------------------------------------------------------------------------
// complex helpers (x = real, y = imaginary)
// ---------------------------------------------------------------------------
SCINT_DEV float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
SCINT_DEV float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
SCINT_DEV float2 operator*(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
SCINT_DEV double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
SCINT_DEV double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
SCINT_DEV double2 operator*(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

SCINT_DEV float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
SCINT_DEV double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
SCINT_DEV float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
SCINT_DEV double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
SCINT_DEV float2 conjc(float2 a) { return make_float2(a.x, -a.y); }
SCINT_DEV double2 conjc(double2 a) { return make_double2(a.x, -a.y); }

// multiply by (DIR * i): DIR = -1 gives -i, +1 gives +i
template <int DIR> SCINT_DEV float2 mul_i(float2 a) {
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <int DIR> SCINT_DEV double2 mul_i(double2 a) {
    return DIR > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename C> SCINT_DEV C make_c(double re, double im);
template <> SCINT_DEV float2 make_c<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> SCINT_DEV double2 make_c<double2>(double re, double im) { return make_double2(re, im); }

// ---------------------------------------------------------------------------
// Double-float arithmetic: a real is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, about 44 significant bits.  Sums use Knuth's
// two-sum and products Dekker's exact product (here through a fused multiply-
// add), the error-free transformations of the double-double literature (Hida,
// Li & Bailey 2001) on FP32 pairs.  The addition is the short form, whose error
// is bounded relative to the operands (not to the result), which is the
// normwise accuracy an FFT needs.  On GB300 these run on the FP32 pipes, which
// are 64 times wider than the FP64 pipe.
// ---------------------------------------------------------------------------
struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
SCINT_DEV dfl two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return dfl(s, (a - (s - bb)) + (b - bb));
}
SCINT_DEV dfl fast_two_sum(float a, float b) {   // requires |a| >= |b| or a == 0
    const float s = a + b;
    return dfl(s, b - (s - a));
}
SCINT_DEV dfl operator+(dfl a, dfl b) {
    const dfl s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
SCINT_DEV dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
SCINT_DEV dfl operator-(dfl a, dfl b) { return a + (-b); }
SCINT_DEV dfl operator*(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
    return fast_two_sum(p, e);
}
SCINT_DEV double to_double(dfl a) { return (double)a.hi + (double)a.lo; }
// a b + c d with one renormalisation: the two high products and their sum exactly (two
// products by FMA, one two-sum), the cross terms and errors folded into the low word
// (19 FP32 operations where two products and a sum take 25); the error stays of the
// order of 2^-44 (|a b| + |c d|), the normwise bound a transform needs.
SCINT_DEV dfl dot2(dfl a, dfl b, dfl c, dfl d) {
    const float p = a.hi * b.hi, q = c.hi * d.hi;
    const float ep = fmaf(a.hi, b.hi, -p), eq = fmaf(c.hi, d.hi, -q);
    const dfl s = two_sum(p, q);
    float lo = s.lo + ep + eq;
    lo = fmaf(a.hi, b.lo, lo);
    lo = fmaf(a.lo, b.hi, lo);
    lo = fmaf(c.hi, d.lo, lo);
    lo = fmaf(c.lo, d.hi, lo);
    return fast_two_sum(s.hi, lo);
}

// float -> double from the bits, with integer instructions only (exact for normal numbers
// and zero; a subnormal float, below 1.2e-38, becomes 0; no inf or NaN arises here)
SCINT_DEV double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |       // 1023 - 127
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double(e ? (long long)d : 0ll);
}
// s * a as a double: the product in double-float, then one FP64 addition (the FP64 pipe of
// GB300 is narrow; the conversions of to_double and an FP64 multiply would cost three more)
SCINT_DEV double scaled_to_double(dfl a, dfl s) {
    const dfl p = a * s;
    return f2d_bits(p.hi) + f2d_bits(p.lo);
}

// complex double-float (x real, y imaginary), 16 bytes like double2
struct __align__(16) dfc {
    dfl x, y;
};
SCINT_DEV dfc operator+(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
SCINT_DEV dfc operator-(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
SCINT_DEV dfc cmul(dfc a, dfc b) { return dfc{dot2(a.x, b.x, -a.y, b.y), dot2(a.x, b.y, a.y, b.x)}; }
SCINT_DEV dfc cmulc(dfc a, dfc b) { return dfc{dot2(a.x, b.x, a.y, b.y), dot2(a.y, b.x, -a.x, b.y)}; }
SCINT_DEV dfc conjc(dfc a) { return dfc{a.x, -a.y}; }
template <int DIR> SCINT_DEV dfc mul_i(dfc a) { return DIR > 0 ? dfc{-a.y, a.x} : dfc{a.y, -a.x}; }
template <> struct real_of<dfc> { using type = dfl; };
template <> SCINT_DEV dfc make_c<dfc>(double re, double im) { return dfc{dfl(re), dfl(im)}; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

SCINT_DEV u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

}  // namespace scint
