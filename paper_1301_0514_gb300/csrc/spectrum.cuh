// Shaped spectral values of the phase screen (Sect. 3.1, Eq. densite): the
// noise of FFT bin (kx, ky) from Philox4x32-10 with counter (kx, ky, screen_id,
// 0), Box-Muller, and the amplitude sqrt(L^2 S(q)).  Shared by the synthesis
// and by the screen check of Sect. 3.1.1, so both see the same F.
#pragma once

#include "kernels.cuh"

namespace scint {

// Uniform in (0,1) from the 64-bit word (hi:lo): top 53 bits plus one half, times 2^-53.
SCINT_DEV double uniform53(uint32_t hi, uint32_t lo) {
    const uint64_t w = ((uint64_t)hi << 32) | lo;
    return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

SCINT_DEV int signed_freq(int i, int n) { return i < n / 2 ? i : i - n; }

// -ln u_a of a bin's first uniform u_a = (top 53 bits of (w1:w0) + 1/2) 2^-53, in FP64.
SCINT_DEV double neg_log_ua64(const u32x4& w) { return -log(uniform53(w.y, w.x)); }

// The same in FP32: u_a rounded once to float; -ln u_a goes through
// log1p(-(1 - u_a)) when u_a >= 1/2 so that values near 1 keep their relative
// accuracy (1 - u_a uses the complemented bits exactly).
SCINT_DEV float neg_log_ua32(const u32x4& w) {
    if (w.y & 0x80000000u) {
        const float d = fmaf((float)((~w.x) >> 11), 0x1.0p-53f, (float)(~w.y) * 0x1.0p-32f) + 0x1.0p-54f;
        return -log1pf(-d);
    }
    const float ua = fmaf((float)(w.x >> 11), 0x1.0p-53f, (float)w.y * 0x1.0p-32f) + 0x1.0p-54f;
    return -logf(ua);
}

// Bins with |mx| <= K and |my| <= K (K = a.low_k) carry almost all of the phase
// variance (S ~ q^-beta): their noise and amplitude are computed in FP64.  The
// other bins have small amplitudes, so FP32 Box-Muller and pow give phase errors
// of ~1e-7 of their (small) rms contribution, which falls as K^((2 - beta)/2)
// with the square's size.  The host picks K per screen (32 to 256) from that rms
// (api.cu, fp64_square); with K = 32 everywhere the screens with the largest phases
// (rms 72 rad at 4096^2, R_diff = 30 km) were 2.4e-6 rad off the FP64 oracle.

// A bin's shaped value F[ky][kx] = sqrt(L^2 S(q)) (g_re + i g_im) / sqrt(2), in the
// precision it is computed in: FP64 for the low bins (low = true, d), FP32 for the
// others (f).  The DC bin is 0 (low = true).
struct BinValue {
    bool low;
    double2 d;
    float2 f;
};
SCINT_DEV u32x4 bin_words(const SynthArgs& a, int kx, int ky) {
    return philox4x32_10(u32x4{(uint32_t)kx, (uint32_t)ky, a.screen_id, 0u}, a.key0, a.key1);
}
// amplitude sqrt(L^2 S(q)) (with the 1/sqrt(2)) from m2 = mx^2 + my^2 > 0, in each precision
SCINT_DEV double amplitude_low(const SynthArgs& a, int m2) { return a.amp * pow((double)m2, a.neg_beta_4); }
// FP32: amp m2^(-beta/4) with the rounding of the constants undone to first order.  amp and
// -beta/4 are split as hi + lo (hi the FP32 value); m2 > 2^24 rounds to float as m2f, m2 = m2f + d.
// With x = amp_hi m2f^(y_hi), the amplitude is x (1 + amp_lo/amp_hi + y_lo ln m2f + y_hi d/m2f):
// the lo part of the exponent alone would otherwise err by up to 3e-8 ln m2 (5e-7 at m2 = 1e7),
// the same sign for every bin.
SCINT_DEV float amplitude_high(const SynthArgs& a, int m2) {
    const float m2f = (float)m2;
    const float d = (float)(m2 - (int)m2f);
    const float x = a.amp32 * powf(m2f, a.neg_beta_4_32);
    const float corr = fmaf(a.neg_beta_4_lo, __logf(m2f), fmaf(a.neg_beta_4_32, __fdividef(d, m2f), a.amp_rel_lo));
    return fmaf(x, corr, x);
}
// sig (g_re + i g_im) from a bin's Philox words, Box-Muller in FP64 ...
SCINT_DEV double2 shaped_low(const u32x4& w, double sig) {
    const double ub = uniform53(w.w, w.z);
    const double r = sqrt(2.0 * neg_log_ua64(w));
    double sn, cs;
    sincospi(2.0 * ub, &sn, &cs);
    return make_double2(sig * r * cs, sig * r * sn);
}
// ... and in FP32 with the same 53-bit uniforms, each rounded once to float
SCINT_DEV float2 shaped_high(const u32x4& w, float sig) {
    const float r = sqrtf(2.0f * neg_log_ua32(w));
    const float tb = fmaf((float)(w.z >> 11), 0x1.0p-52f, (float)w.w * 0x1.0p-31f) + 0x1.0p-53f;  // 2 u_b
    float sn, cs;
    sincospif(tb, &sn, &cs);
    return make_float2(sig * r * cs, sig * r * sn);
}

SCINT_DEV BinValue spectrum_value(const SynthArgs& a, int kx, int ky) {
    const u32x4 w = bin_words(a, kx, ky);
    const int mx = signed_freq(kx, a.n), my = signed_freq(ky, a.n);
    const int m2 = mx * mx + my * my;
    BinValue v;
    v.low = true;
    v.d = make_double2(0.0, 0.0);
    v.f = make_float2(0.0f, 0.0f);
    if (m2 == 0) return v;
    if (abs(mx) <= a.low_k && abs(my) <= a.low_k) {
        v.d = shaped_low(w, amplitude_low(a, m2));
        return v;
    }
    v.low = false;
    v.f = shaped_high(w, amplitude_high(a, m2));
    return v;
}

// F[ky][kx] in FP64 (the inspection hook's form)
SCINT_DEV double2 spectrum_bin(const SynthArgs& a, int kx, int ky) {
    const BinValue v = spectrum_value(a, kx, ky);
    return v.low ? v.d : make_double2((double)v.f.x, (double)v.f.y);
}

// F[ky][kx] as a double-float: FP32 bins are exact with lo = 0, so only the few
// low bins touch the FP64 pipe
SCINT_DEV dfc spectrum_bin_df(const SynthArgs& a, int kx, int ky) {
    const BinValue v = spectrum_value(a, kx, ky);
    if (v.low) return dfc{dfl(v.d.x), dfl(v.d.y)};
    return dfc{dfl(v.f.x, 0.0f), dfl(v.f.y, 0.0f)};
}

// F at (kx, ky) and at the mirror bin (-kx, -ky) mod n, as double-floats: the same values
// as two spectrum_bin_df calls, with the amplitude (which depends on |k| only, and so is the
// same for both) computed once.
SCINT_DEV void spectrum_pair_df(const SynthArgs& a, int kx, int ky, dfc& f, dfc& g) {
    const int n = a.n;
    const u32x4 w1 = bin_words(a, kx, ky), w2 = bin_words(a, (n - kx) & (n - 1), (n - ky) & (n - 1));
    const int mx = signed_freq(kx, n), my = signed_freq(ky, n);
    const int m2 = mx * mx + my * my;
    if (m2 == 0) {
        f = g = dfc{dfl(0.0f, 0.0f), dfl(0.0f, 0.0f)};
    } else if (abs(mx) <= a.low_k && abs(my) <= a.low_k) {
        const double sig = amplitude_low(a, m2);
        const double2 d1 = shaped_low(w1, sig), d2 = shaped_low(w2, sig);
        f = dfc{dfl(d1.x), dfl(d1.y)};
        g = dfc{dfl(d2.x), dfl(d2.y)};
    } else {
        const float sig = amplitude_high(a, m2);
        const float2 v1 = shaped_high(w1, sig), v2 = shaped_high(w2, sig);
        f = dfc{dfl(v1.x, 0.0f), dfl(v1.y, 0.0f)};
        g = dfc{dfl(v2.x, 0.0f), dfl(v2.y, 0.0f)};
    }
}

// F at (kx, ky) and at the mirror bin in FP32, for bins outside the FP64 square
// (|mx| > low_k or |my| > low_k): the values spectrum_pair_df gives them, lo = 0.
SCINT_DEV void spectrum_pair_high(const SynthArgs& a, int kx, int ky, float2& f, float2& g) {
    const int n = a.n;
    const u32x4 w1 = bin_words(a, kx, ky), w2 = bin_words(a, (n - kx) & (n - 1), (n - ky) & (n - 1));
    const int mx = signed_freq(kx, n), my = signed_freq(ky, n);
    const float sig = amplitude_high(a, mx * mx + my * my);
    f = shaped_high(w1, sig);
    g = shaped_high(w2, sig);
}

// |F[ky][kx]|^2 = sigma^2 (g_re^2 + g_im^2) / 2 = sigma^2 (-2 ln u_a) / 2 of a
// bin with Philox words w and m2 = mx^2 + my^2 > 0 (the Box-Muller angle
// cancels), in the precision spectrum_bin uses for it: FP64 for the low bins
// (|mx|, |my| <= a.low_k), FP32 for the others.
SCINT_DEV bool low_bin(const SynthArgs& a, int mx, int my) { return abs(mx) <= a.low_k && abs(my) <= a.low_k; }
SCINT_DEV double power_low(const SynthArgs& a, const u32x4& w, int m2) {
    const double sig = amplitude_low(a, m2);
    return sig * sig * (2.0 * neg_log_ua64(w));
}
SCINT_DEV float power_high(const SynthArgs& a, const u32x4& w, int m2) {
    const float sig = amplitude_high(a, m2);
    return sig * sig * (2.0f * neg_log_ua32(w));
}

}  // namespace scint
