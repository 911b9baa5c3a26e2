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
