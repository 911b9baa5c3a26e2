// Packed Stockham FFT: two independent lines of the same length and position (in the
// propagation passes: one line of the field at two wavelengths) transformed together
// with two-wide FP32 instructions.
//
// A value is cp2 {re, im}: lane 0 of re and im is the element of line a, lane 1 that
// of line b.  Every add, subtract and multiply of the butterflies is one packed
// instruction (__ffma2_rn / __fmul2_rn) acting on both lines, so a pair of lines costs
// about the instructions of one: the FP32 pipe does the same work, but the issue
// slots it needs halve.  Twiddle factors are the same for both lines; they are formed
// once in scalar FP32 (from the register bases of TwiddleRegs, products of depth <= 3,
// or from the block's shared table) and applied to both.
//
// Additions are packed FMAs with a (1, 1) or (-1, -1) multiplier: on GB300 a packed
// FMA runs at the full FP32 rate while a packed add runs at about two thirds of it.
// The constants come from a kernel argument (PK), so the compiler cannot turn the
// FMAs back into adds.
//
// The team layout, radix plan, shared-memory buffer (padded by one element per 16;
// the 16-byte elements keep the stage accesses conflict-free for the same reason as
// the 8-byte ones: consecutive threads touch consecutive elements) and the data
// distribution (thread t holds positions t + m T in registers on entry and exit) are
// those of fft_line in fft.cuh, so a forward transform, a pointwise multiply and an
// inverse transform chain in registers.
#pragma once

#include "fft.cuh"

namespace scint {

struct __align__(16) cp2 {
    float2 re, im;
};

// (1, 1) and (-1, -1), loaded from a kernel argument
struct PK {
    float2 one, mone;
};
SCINT_DEV PK make_pk(float one) { return PK{make_float2(one, one), make_float2(-one, -one)}; }

SCINT_DEV float2 padd(float2 a, float2 b, const PK& k) { return __ffma2_rn(a, k.one, b); }
SCINT_DEV float2 psub(float2 a, float2 b, const PK& k) { return __ffma2_rn(b, k.mone, a); }
SCINT_DEV cp2 add(cp2 a, cp2 b, const PK& k) { return cp2{padd(a.re, b.re, k), padd(a.im, b.im, k)}; }
SCINT_DEV cp2 sub(cp2 a, cp2 b, const PK& k) { return cp2{psub(a.re, b.re, k), psub(a.im, b.im, k)}; }

SCINT_DEV float2 bcast(float v) { return make_float2(v, v); }

// a * w (DIR < 0) or a * conj(w) (DIR > 0), w the same for both lines
template <int DIR>
SCINT_DEV cp2 twmul(cp2 a, float2 w, const PK& k) {
    const float2 wx = bcast(w.x), wy = bcast(w.y);
    if constexpr (DIR < 0) {
        return cp2{psub(__fmul2_rn(a.re, wx), __fmul2_rn(a.im, wy), k), __ffma2_rn(a.im, wx, __fmul2_rn(a.re, wy))};
    } else {
        return cp2{__ffma2_rn(a.im, wy, __fmul2_rn(a.re, wx)), psub(__fmul2_rn(a.im, wx), __fmul2_rn(a.re, wy), k)};
    }
}

// a * h with a different factor per line: h.re = (h_a.re, h_b.re), h.im likewise
SCINT_DEV cp2 lanemul(cp2 a, cp2 h, const PK& k) {
    return cp2{psub(__fmul2_rn(a.re, h.re), __fmul2_rn(a.im, h.im), k), __ffma2_rn(a.im, h.re, __fmul2_rn(a.re, h.im))};
}

// |a|^2 per line
SCINT_DEV float2 norm2(cp2 a) { return __ffma2_rn(a.re, a.re, __fmul2_rn(a.im, a.im)); }

SCINT_DEV cp2 pack2(float2 a, float2 b) { return cp2{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }

// a * exp(DIR 2 pi i J16 / 16), a compile-time multiple of 1/16 turn
template <int J16, int DIR>
SCINT_DEV cp2 rot16p(cp2 a, const PK& k) {
    constexpr int j = ((J16 % 16) + 16) % 16;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4 || j == 12) {
        // times +-i: (re, im) -> (-im, re) for +i, (im, -re) for -i
        constexpr int sgn = (j == 4 ? DIR : -DIR);
        if constexpr (sgn > 0) return cp2{__fmul2_rn(a.im, k.mone), a.re};
        else return cp2{a.im, __fmul2_rn(a.re, k.mone)};
    } else if constexpr (j == 8) {
        return cp2{__fmul2_rn(a.re, k.mone), __fmul2_rn(a.im, k.mone)};
    } else {
        constexpr float c = (float)cos16(j);
        constexpr float s = (float)(DIR * cos16(j - 4));
        return cp2{__ffma2_rn(a.im, bcast(-s), __fmul2_rn(a.re, bcast(c))),
                   __ffma2_rn(a.im, bcast(c), __fmul2_rn(a.re, bcast(s)))};
    }
}

// ---- in-register DFTs, natural order in and out ----------------------------------
template <int DIR>
SCINT_DEV void dft2p(cp2& a, cp2& b, const PK& k) {
    const cp2 t = sub(a, b, k);
    a = add(a, b, k);
    b = t;
}

// the multiplication by DIR i folds into the signs of the last additions
template <int DIR>
SCINT_DEV void dft4p(cp2& a0, cp2& a1, cp2& a2, cp2& a3, const PK& k) {
    const cp2 t0 = add(a0, a2, k), t1 = sub(a0, a2, k), t2 = add(a1, a3, k), d = sub(a1, a3, k);
    a0 = add(t0, t2, k);
    a2 = sub(t0, t2, k);
    // t1 +- DIR i d: re = t1.re -+ DIR d.im, im = t1.im +- DIR d.re
    if constexpr (DIR > 0) {
        a1 = cp2{psub(t1.re, d.im, k), padd(t1.im, d.re, k)};
        a3 = cp2{padd(t1.re, d.im, k), psub(t1.im, d.re, k)};
    } else {
        a1 = cp2{padd(t1.re, d.im, k), psub(t1.im, d.re, k)};
        a3 = cp2{psub(t1.re, d.im, k), padd(t1.im, d.re, k)};
    }
}

template <int R, int DIR>
SCINT_DEV void dftp(cp2* x, const PK& k) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2p<DIR>(x[0], x[1], k);
    } else if constexpr (R == 4) {
        dft4p<DIR>(x[0], x[1], x[2], x[3], k);
    } else if constexpr (R == 8) {
        // n = n1 + 2 n2, k = 4 k1 + k2
#pragma unroll
        for (int n1 = 0; n1 < 2; ++n1) dft4p<DIR>(x[n1], x[n1 + 2], x[n1 + 4], x[n1 + 6], k);
        x[3] = rot16p<2, DIR>(x[3], k);
        x[5] = rot16p<4, DIR>(x[5], k);
        x[7] = rot16p<6, DIR>(x[7], k);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) dft2p<DIR>(x[2 * k2], x[2 * k2 + 1], k);
        cp2 y[8];
#pragma unroll
        for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[4 * k1 + k2] = x[k1 + 2 * k2];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = y[i];
    } else if constexpr (R == 16) {
        // n = n1 + 4 n2, k = 4 k1 + k2
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) dft4p<DIR>(x[n1], x[n1 + 4], x[n1 + 8], x[n1 + 12], k);
        x[5] = rot16p<1, DIR>(x[5], k);
        x[9] = rot16p<2, DIR>(x[9], k);
        x[13] = rot16p<3, DIR>(x[13], k);
        x[6] = rot16p<2, DIR>(x[6], k);
        x[10] = rot16p<4, DIR>(x[10], k);
        x[14] = rot16p<6, DIR>(x[14], k);
        x[7] = rot16p<3, DIR>(x[7], k);
        x[11] = rot16p<6, DIR>(x[11], k);
        x[15] = rot16p<9, DIR>(x[15], k);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) dft4p<DIR>(x[4 * k2], x[4 * k2 + 1], x[4 * k2 + 2], x[4 * k2 + 3], k);
        cp2 y[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[4 * k1 + k2] = x[k1 + 4 * k2];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = y[i];
    }
}

// Apply the stage twiddles W^{r k}, r = 1..R-1, to one butterfly's inputs, each formed
// in scalar FP32 just before its use (few live registers): from the register bases
// (TWM 2, W^k and W^{4k}, products of depth <= 3) or from the block's shared table
// (TWM 1, entries [k][r - 1]).
template <int R, int DIR, int TWM>
SCINT_DEV void apply_twiddles(cp2* u, float2 w1, float2 w4, const float2* __restrict__ tws, const PK& k) {
    if constexpr (TWM == 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = twmul<DIR>(u[r], tws[r - 1], k);
    } else {
        float2 w[4];
        w[1] = w1;
        u[1] = twmul<DIR>(u[1], w[1], k);
        if constexpr (R >= 4) {
            w[2] = cmul(w1, w1);
            w[3] = cmul(w1, w[2]);
            u[2] = twmul<DIR>(u[2], w[2], k);
            u[3] = twmul<DIR>(u[3], w[3], k);
        }
        if constexpr (R >= 8) {
            u[4] = twmul<DIR>(u[4], w4, k);
#pragma unroll
            for (int r = 5; r < 8; ++r) u[r] = twmul<DIR>(u[r], cmul(w4, w[r - 4]), k);
        }
        if constexpr (R >= 16) {
            const float2 w8 = cmul(w4, w4);
            u[8] = twmul<DIR>(u[8], w8, k);
#pragma unroll
            for (int r = 9; r < 12; ++r) u[r] = twmul<DIR>(u[r], cmul(w8, w[r - 8]), k);
            const float2 w12 = cmul(w8, w4);
            u[12] = twmul<DIR>(u[12], w12, k);
#pragma unroll
            for (int r = 13; r < 16; ++r) u[r] = twmul<DIR>(u[r], cmul(w12, w[r - 12]), k);
        }
    }
}

// One stage of the packed transform (see fft_stage in fft.cuh for the indexing).
// LW lines of pairs share the buffer lane-interleaved (element e of lane w at
// pad16(e) LW + w; the caller offsets buf by w).
template <int N, int EPT, int DIR, int LW, int TWM, int S>
SCINT_DEV void fft2_stage(cp2 (&v)[FftPlan<N, EPT>::E], cp2* buf, int t, const float2* __restrict__ tw,
                          const TwiddleRegs<float2, N, EPT>* tr, const PK& k) {
    using Pl = FftPlan<N, EPT>;
    constexpr int E = Pl::E, T = Pl::T;
    constexpr int R = Pl::radix(S), P = Pl::span(S), NB = E / R;
    constexpr bool FIRST = (S == 0), LAST = (S == Pl::NSTAGE - 1);
    cp2 u[E];
    if constexpr (FIRST) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) u[b * R + r] = v[b + r * NB];
    } else {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) u[b * R + r] = buf[pad16(t + b * T) * LW + r * ((N / R) + (N / R) / 16) * LW];
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if constexpr (!FIRST) {
            const int kk = (t + b * T) & (P - 1);
            if constexpr (TWM == 1)
                apply_twiddles<R, DIR, 1>(&u[b * R], float2{}, float2{}, tw + Pl::twoff(S) + kk * (R - 1), k);
            else
                apply_twiddles<R, DIR, 2>(&u[b * R], tr->w[S][b][0], tr->w[S][b][1], nullptr, k);
        }
        dftp<R, DIR>(&u[b * R], k);
    }
    if constexpr (LAST) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * NB] = u[b * R + r];
    } else {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = t + b * T;
            const int kk = i & (P - 1);
            const int j = (i - kk) * R + kk;
            cp2* dst = buf + pad16(j) * LW;
#pragma unroll
            for (int r = 0; r < R; ++r)
                dst[(P >= 16 ? r * (P + P / 16) : (P == 1 ? r : pad16(j + r * P) - pad16(j))) * LW] = u[b * R + r];
        }
        __syncthreads();
        fft2_stage<N, EPT, DIR, LW, TWM, S + 1>(v, buf, t, tw, tr, k);
    }
}

// Transform the team's pair of lines in place.  TWM 2: register bases tr (tw unused);
// TWM 1: tw is the block's shared table (fill_twiddle_table).  Every thread of the
// block must call this the same number of times.
template <int N, int EPT, int DIR, int LW, int TWM>
SCINT_DEV void fft2_line(cp2 (&v)[FftPlan<N, EPT>::E], cp2* buf, int t, const float2* __restrict__ tw,
                         const TwiddleRegs<float2, N, EPT>* tr, const PK& k) {
    static_assert(TWM == 1 || TWM == 2, "shared table or register bases");
    static_assert(EPT != 8 || N >= 128, "8 values per thread: N >= 128");
    fft2_stage<N, EPT, DIR, LW, TWM, 0>(v, buf, t, tw, tr, k);
}

}  // namespace scint
