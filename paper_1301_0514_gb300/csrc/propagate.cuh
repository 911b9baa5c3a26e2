// Block shapes and layouts shared by the propagation passes and their adjoints.
#pragma once

#include "fft.cuh"
#include "kernels.cuh"

// Twiddle source of the propagation FFTs (build-time tuning choices, measured on
// GB300 at 1024^2-4096^2 x 32 wavelengths): 1 = per-block shared table,
// 2 = per-thread register bases + products.  The row pass is faster with
// register bases (its 2 blocks/SM keep the shared-memory pipe busy), the column
// pass with the shared table (its single block/SM has registers to spare).
#ifndef SCINT_ROW_TWIDDLES
#define SCINT_ROW_TWIDDLES 2
#endif
#ifndef SCINT_COL_TWIDDLES
#define SCINT_COL_TWIDDLES 1
#endif

namespace scint {

// Ping-pong FFT buffers in the propagation passes (fft.cuh: one barrier per stage
// instead of two), off by default.  Measured on GB300 with 32 wavelengths, each pass
// alone is faster with them (rows 1.4 % at 4096 to 10 % at 1024, columns 1-4.5 %
// below 4096; 1.5 % slower at 4096, which would keep one buffer), but the batched
// step on four lanes is 7.6 % slower (123.1 -> 132.5 ms): at 102 KB per row block two
// blocks fill an SM's shared memory and the other lanes' kernels no longer share it.
#ifndef SCINT_PROP_PINGPONG
#define SCINT_PROP_PINGPONG 0
#endif

constexpr int kRowTw = SCINT_ROW_TWIDDLES;
constexpr int kColTw = SCINT_COL_TWIDDLES;
constexpr int kColEPT = 16;   // values per thread in the column passes
constexpr size_t kMaxSmem = 227 * 1024;

// Lines longer than one block's shared memory (N = 16384) go to a cluster of two
// blocks, split by one radix-2 step (prop_*_split_kernel and conj_*_split_kernel in
// propagate.cu, adj_*_split_kernel in adjoint.cu): each block transforms one parity
// as a whole N/2-point line.  The kernels below are the unsplit passes.
template <int N> __host__ __device__ constexpr int pcs() { return N >= kSplitN ? 2 : 1; }
template <int N> __host__ __device__ constexpr bool ppp_row() { return SCINT_PROP_PINGPONG; }
template <int N> __host__ __device__ constexpr bool ppp_col() { return SCINT_PROP_PINGPONG && N < 4096; }
template <int N> __host__ __device__ constexpr int prow_twm() { return kRowTw; }
template <int N> __host__ __device__ constexpr int pcol_twm();   // below: depends on the shared-memory budget

// rows per row-pass block, columns per column-pass block (all lines of a block
// are transformed together); threads are per block
template <int N> __host__ __device__ constexpr int prow_lines() { return N >= kTileRow32 ? 1 : (kTileRow32 / N < N ? kTileRow32 / N : N); }
template <int N> __host__ __device__ constexpr int prow_threads() { return prow_lines<N>() * FftPlan<N>::T; }
// Column-pass blocks take 256 threads (two blocks per SM, so a stage barrier idles
// half the SM, not all of it) wherever a block still holds two or more columns of
// a strip; at N = 4096 that would leave one column (a quarter of every 32-byte
// sector read), so there a block holds two columns in 512 threads.
template <int N> __host__ __device__ constexpr int pcol_lines() {
    return N >= 8192 ? 1 : (N >= 4096 ? 2 : (4096 / N < N ? 4096 / N : N));
}
template <int N> __host__ __device__ constexpr int pcol_threads() { return pcol_lines<N>() * FftPlan<N, kColEPT>::T; }
// Strip width of the intermediate: at least 4 columns, so that every row of the
// row pass writes whole 32-byte sectors; a column block then reads its
// pcol_lines() columns out of one strip (sibling blocks share the sectors in L2).
template <int N> __host__ __device__ constexpr int pstrip() { return pcol_lines<N>() >= 4 ? pcol_lines<N>() : (N >= 4 ? 4 : N); }

template <int N> constexpr size_t ptws_bytes(int twm) { return twm == 1 ? (size_t)FftPlan<N>::TWS * sizeof(float2) : 0; }
template <int N> constexpr size_t prow_smem() {
    return (size_t)prow_lines<N>() * ((ppp_row<N>() ? 2 : 1) * FftPlan<N>::BUF * sizeof(float2) + N * sizeof(long long)) +
           ptws_bytes<N>(prow_twm<N>());
}
// column pass: line buffers and (when it fits) the twiddle table
template <int N> __host__ __device__ constexpr size_t pcol_base_bytes() {
    return (size_t)pcol_lines<N>() * FftPlan<N>::BUF * sizeof(float2);
}
template <int N> __host__ __device__ constexpr int pcol_twm() {
    return (kColTw == 1 && pcol_base_bytes<N>() * (ppp_col<N>() ? 2 : 1) + (size_t)FftPlan<N>::TWS * sizeof(float2) > kMaxSmem
                ? 2 : kColTw);
}
template <int N> constexpr size_t pcol_smem() {
    return pcol_base_bytes<N>() * (ppp_col<N>() ? 2 : 1) + ptws_bytes<N>(pcol_twm<N>());
}

// signed FFT frequency index of bin i
SCINT_DEV int sfreq(int i, int n) { return i < n / 2 ? i : i - n; }

// element (y, x) of a strip-layout field
template <int WL> SCINT_DEV size_t strip_index(int y, int x, int n) {
    return (size_t)(x / WL) * n * WL + (size_t)y * WL + (x % WL);
}

// phi (radians) -> 64-bit fixed-point turns, P = round(phi 2^32 / 2 pi)
SCINT_DEV long long phase_fixed(double phi) { return __double2ll_rn(phi * (4294967296.0 / (2.0 * kPi))); }

// exp(i (phi s + add 2^-64 turns)) from P and S = round(s 2^32): the low 64
// bits of P S are the fractional turns of phi s times 2^64 (exact reduction
// mod 2 pi); the angle in [-pi, pi) goes to the hardware sine/cosine (abs.
// error ~4e-7 there).
SCINT_DEV float2 unit_phasor(long long P, unsigned long long S, unsigned long long add = 0ull) {
    const unsigned long long prod = (unsigned long long)P * S + add;   // + extra turns 2^-64
    const float ang = (float)(int)(prod >> 32) * (float)(2.0 * kPi * 0x1.0p-32);
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    return make_float2(cs, sn);
}

// H_x(k) = exp(-i pi lambda z k^2) at FFT index i, from C = frac(-lambda z / 2L^2) 2^64:
// the phase C m^2 mod 2^64 (m the signed frequency index) is exact in fixed-point turns.
SCINT_DEV float2 transfer_phasor(unsigned long long C, int i, int n) {
    const long long m = sfreq(i, n);
    return unit_phasor(0, 0ull, C * (unsigned long long)(m * m));
}
// H_x(k)/n (the inverse transform's normalisation)
SCINT_DEV float2 transfer_at(unsigned long long C, int i, int n) { return transfer_phasor(C, i, n) * (1.0f / n); }

// One-FFT mode: chirp |x_1|^2 / (2 R_F^2) with x_1 = (i - n/2) Delta in fixed-point
// turns, C (i - n/2)^2 mod 2^64 (exact), plus half a turn for odd i: the factor
// (-1)^i that centres the transform on the optical axis (the sum over
// (i - n/2)(k - n/2) is the plain DFT times (-1)^(i + k) and a constant).
SCINT_DEV unsigned long long chirp_turns(unsigned long long C, int i, int n) {
    const long long d = (long long)i - n / 2;
    return C * (unsigned long long)(d * d) + ((unsigned long long)(i & 1) << 63);
}

}  // namespace scint
