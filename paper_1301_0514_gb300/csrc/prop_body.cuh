// Bodies of the unsplit transfer-function passes (see propagate.cu for the method),
// shared by their kernels (propagate.cu) and the persistent batch kernel (persist.cu).
#pragma once

#include "propagate.cuh"

namespace scint {

// ---- row pass ------------------------------------------------------------------
// The pass bodies take the block index, the thread index and the block's shared memory
// as arguments, so that the persistent batch kernel (persist.cu) runs the same code as
// the kernels below.
// SUB: the barrier scope (fft.cuh team_sync): 0 the whole block, else the SUB-thread part
// of a larger block that runs this body.
template <int N, bool CONJ, int SUB = 0>
SCINT_DEV void prop_rows_body(const PropArgs& a, int bid, int tid, float2* smem32) {
    using Pl = FftPlan<N>;
    constexpr int TWM = prow_twm<N>();
    constexpr int T = Pl::T, E = Pl::E, B = prow_lines<N>(), W = pstrip<N>(), BUFL = Pl::BUF;
    const int team = tid / T, t = tid % T;    // line of the block, index in its team
    const int y = bid * B + team;
    float2* buf = smem32 + team * BUFL;
    // fixed-point phase of this thread's pixels, kept in shared memory across the
    // wavelength loop (each thread reads back only the entries it wrote)
    long long* P = reinterpret_cast<long long*>(smem32 + B * BUFL) + team * N + t;
    float2* tws = smem32 + B * BUFL + B * N;    // shared twiddle table (after P, 8 B per entry)
    const float2* twp = TWM == 1 ? tws : a.tw;
    constexpr bool PP = ppp_row<N>();            // second line buffers after the table
    float2* buf1 = smem32 + B * BUFL + B * N + (TWM == 1 ? Pl::TWS : 0) + team * BUFL;
    TwiddleRegs<float2, N, 16> tr;
    if constexpr (TWM == 2) tr.load(a.tw, t);
    else if constexpr (TWM == 1) fill_twiddle_table<float2, N>(tws, a.tw, tid, prow_threads<N>());
#pragma unroll
    for (int m = 0; m < E; ++m) P[m * T] = phase_fixed(a.phi[(size_t)y * N + t + m * T]);
    team_sync<SUB>();

#pragma unroll 1
    for (int l = 0; l < a.lam.count; ++l) {
        const unsigned long long S = a.lam.scale_fx[l];
        // the taper from its table; H_x from a scalar (its phase exact in fixed-point turns)
        const float* sf = a.sf + (size_t)l * N;
        // the inverse transform's 1/N rides on the taper of the row (a power of two: exact, so the
        // field equals that of H/N applied after the forward transform, bit for bit)
        const float sfy = CONJ ? sf[y] : sf[y] * (1.0f / N);
        float2 v[E];
        if constexpr (CONJ) {
            // G = SF SF exp(i (phi s + |x_1|^2 / 2 R_F^2)) (-1)^(x + y), Eq. Gxy
            const unsigned long long C = a.conj.chirp_fx[l];
            const unsigned long long cy = chirp_turns(C, y, N);
#pragma unroll
            for (int m = 0; m < E; ++m)
                v[m] = unit_phasor(P[m * T], S, cy + chirp_turns(C, t + m * T, N)) * (sfy * __ldg(sf + t + m * T));
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = unit_phasor(P[m * T], S) * (sfy * __ldg(sf + t + m * T));
        }
        if constexpr (PP && TWM == 2) fft_line_tr_pp<float2, N, -1, 16, 1, SUB>(v, buf, buf1, t, tr);
        else if constexpr (PP) fft_line_pp<float2, N, -1, 16, 1, TWM, SUB>(v, buf, buf1, t, twp);
        else if constexpr (TWM == 2) fft_line_tr<float2, N, -1, 16, 1, 1, SUB>(v, buf, t, tr);
        else fft_line<float2, N, -1, 16, 1, TWM, 1, 1, SUB>(v, buf, t, twp);
        if constexpr (!CONJ) {
            const unsigned long long hc = a.lam.h_fx[l];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer_phasor(hc, t + m * T, N));
            if constexpr (PP && TWM == 2) fft_line_tr_pp<float2, N, +1, 16, 1, SUB>(v, buf, buf1, t, tr);
            else if constexpr (PP) fft_line_pp<float2, N, +1, 16, 1, TWM, SUB>(v, buf, buf1, t, twp);
            else if constexpr (TWM == 2) fft_line_tr<float2, N, +1, 16, 1, 1, SUB>(v, buf, t, tr);
            else fft_line<float2, N, +1, 16, 1, TWM, 1, 1, SUB>(v, buf, t, twp);
        }
        float2* dst = a.work + (size_t)l * N * N;
#pragma unroll
        for (int m = 0; m < E; ++m) dst[strip_index<W>(y, t + m * T, N)] = v[m];
    }
}

// ---- column pass ---------------------------------------------------------------
// The fields are read through L2 only (ld.global.cg): in the persistent batch kernel a
// field slot is rewritten by other blocks between uses, and L1 is not coherent across
// SMs.  No element is read twice by a block, so L1 would not help here anyway.
template <int N, bool CONJ, int SUB = 0>
SCINT_DEV void prop_cols_body(const PropArgs& a, int bid, int tid, float2* smem32) {
    using Pl = FftPlan<N, kColEPT>;
    constexpr int TWM = pcol_twm<N>();
    constexpr int T = Pl::T, E = Pl::E, W = pcol_lines<N>(), WL = pstrip<N>(), BUFL = Pl::BUF;
    const int w = tid % W, t = tid / W;
    const int x0 = bid * W;    // first column of the block: strip x0 / WL, offset x0 % WL
    const int x = x0 + w;
    float2* buf = smem32 + w;     // W lines interleaved: element e of line w at pad16(e) * W + w
    // passband accumulator of this thread's pixels, in registers (a shared-memory
    // copy would add a read-modify-write per wavelength to the busiest queue)
    float acc[E];
    float2* tws = smem32 + W * BUFL;   // shared twiddle table (after the line buffers)
    const float2* twp = TWM == 1 ? tws : a.tw;
    constexpr bool PP = ppp_col<N>();   // second line buffers after the table
    float2* buf1 = smem32 + W * BUFL + (TWM == 1 ? Pl::TWS : 0) + w;
    TwiddleRegs<float2, N, kColEPT> tr;
    if constexpr (TWM == 2) tr.load(a.tw, t);
    else if constexpr (TWM == 1) fill_twiddle_table<float2, N>(tws, a.tw, tid, pcol_threads<N>());
#pragma unroll
    for (int m = 0; m < E; ++m) acc[m] = 0.0f;
    team_sync<SUB>();
#pragma unroll 1
    for (int l = 0; l < a.lam.count; ++l) {
        const float2* src = a.work + (size_t)l * N * N + (size_t)(x0 / WL) * N * WL + (x0 % WL);
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = __ldcg(src + (size_t)(t + m * T) * WL + w);
        if constexpr (PP && TWM == 2) fft_line_tr_pp<float2, N, -1, kColEPT, W, SUB>(v, buf, buf1, t, tr);
        else if constexpr (PP) fft_line_pp<float2, N, -1, kColEPT, W, TWM, SUB>(v, buf, buf1, t, twp);
        else if constexpr (TWM == 2) fft_line_tr<float2, N, -1, kColEPT, W, 1, SUB>(v, buf, t, tr);
        else fft_line<float2, N, -1, kColEPT, W, TWM, 1, 1, SUB>(v, buf, t, twp);
        if constexpr (CONJ) {
            // h = (Delta^2 / lambda z)^2 |FT G|^2 on the pattern grid of this wavelength (Eq. intens)
            const float nrm = a.conj.norm[l];
            if (a.conj.direct) {
                const float wn = a.lam.weight[l] * nrm;
#pragma unroll
                for (int m = 0; m < E; ++m) acc[m] = fmaf(wn, fmaf(v[m].x, v[m].x, v[m].y * v[m].y), acc[m]);
            } else {
                // column-major: this column's values are contiguous, so the stores coalesce
                float* pat = a.conj.pattern + (size_t)l * N * N + (size_t)x * N;
#pragma unroll
                for (int m = 0; m < E; ++m) pat[t + m * T] = nrm * fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
            }
            continue;
        } else {
            const unsigned long long hc = a.lam.h_fx[l];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer_phasor(hc, t + m * T, N));
            if constexpr (PP && TWM == 2) fft_line_tr_pp<float2, N, +1, kColEPT, W, SUB>(v, buf, buf1, t, tr);
            else if constexpr (PP) fft_line_pp<float2, N, +1, kColEPT, W, TWM, SUB>(v, buf, buf1, t, twp);
            else if constexpr (TWM == 2) fft_line_tr<float2, N, +1, kColEPT, W, 1, SUB>(v, buf, t, tr);
            else fft_line<float2, N, +1, kColEPT, W, TWM, 1, 1, SUB>(v, buf, t, twp);
        }
        // the 1/N of H_y, squared, rides on the weight (powers of two: the sums are unchanged bit for bit)
        const float wl = a.lam.weight[l] * (1.0f / ((float)N * (float)N));
#pragma unroll
        for (int m = 0; m < E; ++m) acc[m] = fmaf(wl, fmaf(v[m].x, v[m].x, v[m].y * v[m].y), acc[m]);
    }
    if constexpr (CONJ) {
        if (!a.conj.direct) return;
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float* o = a.intensity + (size_t)(t + m * T) * N + x;
        *o = a.accumulate ? *o + acc[m] : acc[m];
    }
}

}  // namespace scint
