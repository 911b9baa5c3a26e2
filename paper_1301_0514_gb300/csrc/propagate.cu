// Fresnel propagation of a phase screen by the transfer function (Eq. hxy)
// with the edge taper of Sect. 3.2.1 and passband co-addition (Sect. 3.2.4).
//
// The transfer function H(k) = exp(-i pi lambda z (kx^2 + ky^2)) factors into
// H_x(kx) H_y(ky), so the 2D propagator is a 1D propagator along x followed by
// one along y.  Each 1D propagator is FFT -> multiply -> inverse FFT on a line
// held in registers and shared memory, so a wavelength costs two HBM passes:
//   row pass:    phi (read once per wavelength group) -> exact phase reduction
//                -> sin/cos -> taper -> FFT_x -> H_x/N -> IFFT_x -> field (write);
//                H_x and H_y come from one scalar per wavelength (no table
//                loads), their phases exact in fixed-point turns like the screen phase
//   column pass: field (read) -> FFT_y -> H_y/N -> IFFT_y -> w |A|^2, summed over
//                the group in registers -> intensity (one write per group)
//
// Phase reduction: phi is converted once per pixel to 64-bit fixed point in
// turns, P = round(phi 2^32 / 2 pi); for each wavelength the low 64 bits of
// P * round(s 2^32) (s = lambda_ref / lambda) are the fractional turns of
// phi s scaled by 2^64, so the reduction modulo 2 pi is exact integer
// arithmetic (error |phi s| 2^-33 / 2 pi turns from rounding s) and only the
// reduced angle goes to the FP32 sine/cosine.
#include <algorithm>

#include "dispatch.cuh"
#include "prop_body.cuh"
#include "propagate.cuh"

namespace scint {

// ---- taper table --------------------------------------------------------------
// raised-sine taper SF at the pixel centre (i + 1/2), symmetric about the centre
// (Sect. 3.2.1); H is not tabulated: the passes compute it from one fixed-point
// constant per wavelength (transfer_at)
__global__ void prop_tables_kernel(TableArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (i >= a.n) return;
    const int n = a.n;
    const double lm = a.margin_px[l];
    double sf = 1.0;
    if (lm > 0.0) {
        const double u = fmin((double)i + 0.5, (double)n - (double)i - 0.5);
        if (u <= lm) {
            const double sn = sinpi(u / (2.0 * lm));
            sf = sn * sn;
        }
    }
    a.sf[(size_t)l * n + i] = (float)sf;
}

cudaError_t launch_prop_tables(const TableArgs& a, cudaStream_t s) {
    dim3 grid((a.n + 255) / 256, a.count);
    prop_tables_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Resident row blocks per SM the register budget is set for (build-time choice, 2 by default;
// 3 caps the pass at 80 registers).
#ifndef SCINT_ROW_MIN_BLOCKS
#define SCINT_ROW_MIN_BLOCKS 2
#endif
template <int N, bool CONJ>
__global__ void __launch_bounds__(prow_threads<N>(), (prow_threads<N>() <= 256 ? SCINT_ROW_MIN_BLOCKS : 1))
prop_rows_kernel(PropArgs a) {
    extern __shared__ float2 smem32[];
    prop_rows_body<N, CONJ>(a, blockIdx.x, threadIdx.x, smem32);
}

template <int N, bool CONJ>
__global__ void __launch_bounds__(pcol_threads<N>(), (pcol_threads<N>() <= 256 ? 2 : 1))
prop_cols_kernel(PropArgs a) {
    extern __shared__ float2 smem32[];
    prop_cols_body<N, CONJ>(a, blockIdx.x, threadIdx.x, smem32);
}

// ---- lines split over a two-block cluster (N = 16384) -------------------------------
// One radix-2 step on each side of the line transforms divides them between the two
// blocks of a cluster (n < N/2, W = exp(-2 pi i / N)):
//   forward, decimation in frequency: a_n = x_n + x_{n+N/2}, b_n = (x_n - x_{n+N/2}) W^n,
//     X_{2k} = FFT_{N/2}(a)_k, X_{2k+1} = FFT_{N/2}(b)_k;
//   inverse, decimation in time: A' = IFFT_{N/2}(Y_{2k}), B' = IFFT_{N/2}(Y_{2k+1}),
//     y_n = A'_n + W^{-n} B'_n, y_{n+N/2} = A'_n - W^{-n} B'_n.
// Block r takes the parity-r half-problem, a whole N/2-point line in its own shared
// memory with block barriers only, and H at the frequencies 2k + r.  Each block forms
// its a or b from both halves of the input (row pass: the whole line's phases sit in
// both blocks; column pass: both blocks read the whole column, the second read from
// L2).  The halves meet once per wavelength: each block publishes its A' or B' and
// fetches the half of the other one that its outputs need (block 0 makes y_n and
// y_{n+N/2} for n < N/4, block 1 for N/4 <= n < N/2).  The fetch is followed by a
// split arrive/wait, so the next wavelength's input is formed while the partner
// finishes reading.
template <int N> __host__ __device__ constexpr int psplit_threads() { return FftPlan<N / 2>::T; }
template <int N> constexpr size_t prow_split_smem() {
    return (size_t)FftPlan<N / 2>::BUF * sizeof(float2) + (size_t)N * sizeof(long long);
}
template <int N> constexpr size_t pcol_split_smem() {
    return (size_t)(FftPlan<N / 2>::BUF + FftPlan<N / 2>::TWS) * sizeof(float2);
}

template <int N>
__global__ void __launch_bounds__(psplit_threads<N>(), 1) prop_rows_split_kernel(PropArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E, W = pstrip<N>();
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    // the whole line's fixed-point phases: this block converts its half (FP64) and copies
    // the partner's; each thread reads back only the entries it wrote
    long long* P = reinterpret_cast<long long*>(smem32 + Pl::BUF);
    TwiddleRegs<float2, H2, 16> tr;
    tr.load(a.tw, t, 2);    // the N-point table at even indices
    // persistent: the cluster takes rows y, y + clusters, ...
#pragma unroll 1
    for (int y = blockIdx.x / 2; y < N; y += gridDim.x / 2) {
        const double* phi = a.phi + (size_t)y * N + r * H2;
#pragma unroll
        for (int m = 0; m < E; ++m) P[r * H2 + t + m * T] = phase_fixed(phi[t + m * T]);
        line_sync<2>();
        const unsigned pp = cluster_addr(P, (unsigned)(r ^ 1)) + (unsigned)(((r ^ 1) * H2 + t) * sizeof(long long));
#pragma unroll
        for (int m = 0; m < E; ++m)
            P[(r ^ 1) * H2 + t + m * T] = ld_cluster<long long>(pp + (unsigned)(m * T * sizeof(long long)));
        cluster_arrive();
#pragma unroll 1
        for (int l = 0; l < a.lam.count; ++l) {
            const unsigned long long S = a.lam.scale_fx[l];
            const float* sf = a.sf + (size_t)l * N;
            const float sfy = sf[y];
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int e = t + m * T;
                const float2 x0 = unit_phasor(P[e], S) * (sfy * __ldg(sf + e));
                const float2 x1 = unit_phasor(P[e + H2], S) * (sfy * __ldg(sf + e + H2));
                v[m] = r == 0 ? x0 + x1 : cmul(x0 - x1, __ldg(a.tw + e));
            }
            cluster_wait();      // the partner has read this block's buffer
            fft_line_tr<float2, H2, -1, 16, 1>(v, buf, t, tr);
            const unsigned long long hc = a.lam.h_fx[l];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer_at(hc, 2 * (t + m * T) + r, N));
            fft_line_tr<float2, H2, +1, 16, 1>(v, buf, t, tr);
            float2* dst = a.work + (size_t)l * N * N;
            split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int, int n, float2 y0, float2 y1) {
                dst[strip_index<W>(y, n, N)] = y0;
                dst[strip_index<W>(y, n + H2, N)] = y1;
            });
        }
        cluster_wait();    // the partner is done with this block's buffers (no block leaves before)
    }
}

template <int N>
__global__ void __launch_bounds__(psplit_threads<N>(), 1) prop_cols_split_kernel(PropArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E, WL = pstrip<N>();
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    float2* tws = smem32 + Pl::BUF;
    fill_twiddle_table<float2, H2>(tws, a.tw, t, T, 2);
    // persistent: the cluster takes columns x, x + clusters, ...
#pragma unroll 1
    for (int x = blockIdx.x / 2; x < N; x += gridDim.x / 2) {
        float acc[E];
#pragma unroll
        for (int m = 0; m < E; ++m) acc[m] = 0.0f;
        cluster_arrive();    // the first wait below also publishes the twiddle table to the block
#pragma unroll 1
        for (int l = 0; l < a.lam.count; ++l) {
            const float2* src = a.work + (size_t)l * N * N + (size_t)(x / WL) * N * WL + (x % WL);
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int e = t + m * T;
                const float2 x0 = src[(size_t)e * WL], x1 = src[(size_t)(e + H2) * WL];
                v[m] = r == 0 ? x0 + x1 : cmul(x0 - x1, __ldg(a.tw + e));
            }
            cluster_wait();
            fft_line<float2, H2, -1, 16, 1, 1, 1>(v, buf, t, tws);
            const unsigned long long hc = a.lam.h_fx[l];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer_at(hc, 2 * (t + m * T) + r, N));
            fft_line<float2, H2, +1, 16, 1, 1, 1>(v, buf, t, tws);
            const float wl = a.lam.weight[l];
            split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int j, int, float2 y0, float2 y1) {
                acc[2 * j] = fmaf(wl, fmaf(y0.x, y0.x, y0.y * y0.y), acc[2 * j]);
                acc[2 * j + 1] = fmaf(wl, fmaf(y1.x, y1.x, y1.y * y1.y), acc[2 * j + 1]);
            });
        }
        cluster_wait();
        // column-major, so that the stores coalesce; transpose_add_kernel puts it in place
        float* col = a.scratch + (size_t)x * N;
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
            const int n = t + (j + r * (E / 2)) * T;
            col[n] = acc[2 * j];
            col[n + H2] = acc[2 * j + 1];
        }
    }
}

// One-FFT mode (Eq. intens, Eq. Gxy) at N = 16384: forward transforms only, so the
// decimation-in-frequency split alone divides them (block r makes the frequencies
// 2k + r).  The row pass copies the partner's half of the row's phases once per row
// (split arrive/wait around the next row's fill) and writes X(2k + r); the column pass
// needs nothing from its partner: both blocks read the whole column (the second read
// from L2) and each writes its parity's pattern rows, column-major.
template <int N>
__global__ void __launch_bounds__(psplit_threads<N>(), 1) conj_rows_split_kernel(PropArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E, W = pstrip<N>();
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    long long* P = reinterpret_cast<long long*>(smem32 + Pl::BUF);
    TwiddleRegs<float2, H2, 16> tr;
    tr.load(a.tw, t, 2);
    bool first = true;
#pragma unroll 1
    for (int y = blockIdx.x / 2; y < N; y += gridDim.x / 2) {
        if (!first) cluster_wait();     // the partner has copied this block's previous phases
        first = false;
        const double* phi = a.phi + (size_t)y * N + r * H2;
#pragma unroll
        for (int m = 0; m < E; ++m) P[r * H2 + t + m * T] = phase_fixed(phi[t + m * T]);
        line_sync<2>();
        const unsigned pp = cluster_addr(P, (unsigned)(r ^ 1)) + (unsigned)(((r ^ 1) * H2 + t) * sizeof(long long));
#pragma unroll
        for (int m = 0; m < E; ++m)
            P[(r ^ 1) * H2 + t + m * T] = ld_cluster<long long>(pp + (unsigned)(m * T * sizeof(long long)));
        cluster_arrive();
#pragma unroll 1
        for (int l = 0; l < a.lam.count; ++l) {
            const unsigned long long S = a.lam.scale_fx[l], C = a.conj.chirp_fx[l];
            const float* sf = a.sf + (size_t)l * N;
            const float sfy = sf[y];
            const unsigned long long cy = chirp_turns(C, y, N);
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int e = t + m * T;
                // G = SF SF exp(i (phi s + |x_1|^2 / 2 R_F^2)) (-1)^(x + y), Eq. Gxy
                const float2 x0 = unit_phasor(P[e], S, cy + chirp_turns(C, e, N)) * (sfy * __ldg(sf + e));
                const float2 x1 = unit_phasor(P[e + H2], S, cy + chirp_turns(C, e + H2, N)) * (sfy * __ldg(sf + e + H2));
                v[m] = split_dif(x0, x1, r, e, a.tw);
            }
            fft_line_tr<float2, H2, -1, 16, 1>(v, buf, t, tr);
            float2* dst = a.work + (size_t)l * N * N;
#pragma unroll
            for (int m = 0; m < E; ++m) dst[strip_index<W>(y, 2 * (t + m * T) + r, N)] = v[m];
        }
    }
    if (!first) cluster_wait();
}

template <int N>
__global__ void __launch_bounds__(psplit_threads<N>(), 1) conj_cols_split_kernel(PropArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E, WL = pstrip<N>();
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    float2* tws = smem32 + Pl::BUF;
    fill_twiddle_table<float2, H2>(tws, a.tw, t, T, 2);
    __syncthreads();
#pragma unroll 1
    for (int x = blockIdx.x / 2; x < N; x += gridDim.x / 2) {
        float acc[E];
#pragma unroll
        for (int m = 0; m < E; ++m) acc[m] = 0.0f;
#pragma unroll 1
        for (int l = 0; l < a.lam.count; ++l) {
            const float2* src = a.work + (size_t)l * N * N + (size_t)(x / WL) * N * WL + (x % WL);
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int e = t + m * T;
                v[m] = split_dif(src[(size_t)e * WL], src[(size_t)(e + H2) * WL], r, e, a.tw);
            }
            fft_line<float2, H2, -1, 16, 1, 1, 1>(v, buf, t, tws);
            // h = (Delta^2 / lambda z)^2 |FT G|^2 on the pattern grid of this wavelength (Eq. intens)
            const float nrm = a.conj.norm[l];
            if (a.conj.direct) {
                const float wn = a.lam.weight[l] * nrm;
#pragma unroll
                for (int m = 0; m < E; ++m) acc[m] = fmaf(wn, fmaf(v[m].x, v[m].x, v[m].y * v[m].y), acc[m]);
            } else {
                float* pat = a.conj.pattern + (size_t)l * N * N + (size_t)x * N;
#pragma unroll
                for (int m = 0; m < E; ++m) pat[2 * (t + m * T) + r] = nrm * fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
            }
        }
        if (a.conj.direct) {
            // column-major, transposed into place by transpose_add_kernel
            float* col = a.scratch + (size_t)x * N;
#pragma unroll
            for (int m = 0; m < E; ++m) col[2 * (t + m * T) + r] = acc[m];
        }
    }
}

// intensity (+)= the transpose of the column-major map src, in 32 x 32 tiles through
// shared memory (reads and writes both coalesced); n is a multiple of 32
__global__ void __launch_bounds__(256) transpose_add_kernel(const float* __restrict__ src, float* dst, int n,
                                                            int accumulate) {
    __shared__ float tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
    for (int k = ty; k < 32; k += 8) tile[k][tx] = src[(size_t)(x0 + k) * n + y0 + tx];   // [x][y]
    __syncthreads();
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
        float* o = dst + (size_t)(y0 + k) * n + x0 + tx;
        const float v = tile[tx][k];
        *o = accumulate ? *o + v : v;
    }
}

template <bool CONJ>
cudaError_t launch_rows(const PropArgs& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (pcs<N>() == 2) {
            static_assert(prow_split_smem<N>() <= kMaxSmem, "split row pass does not fit");
            auto k = CONJ ? conj_rows_split_kernel<N> : prop_rows_split_kernel<N>;
            cudaError_t e = set_smem(k, prow_split_smem<N>());
            int nc = 0;
            if (e == cudaSuccess) e = active_clusters(k, 2, psplit_threads<N>(), prow_split_smem<N>(), &nc);
            if (e != cudaSuccess) return e;
            return launch_k(k, 2, dim3(2 * std::min(nc, N)), dim3(psplit_threads<N>()), prow_split_smem<N>(), s, a);
        } else if constexpr (prow_smem<N>() > kMaxSmem || pcol_smem<N>() > kMaxSmem) {
            return cudaErrorNotSupported;
        } else {
            cudaError_t e = set_smem(prop_rows_kernel<N, CONJ>, prow_smem<N>());
            if (e != cudaSuccess) return e;
            prop_rows_kernel<N, CONJ><<<N / prow_lines<N>(), prow_threads<N>(), prow_smem<N>(), s>>>(a);
            return cudaGetLastError();
        }
    });
}

template <bool CONJ>
cudaError_t launch_cols(const PropArgs& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (pcs<N>() == 2) {
            static_assert(pcol_split_smem<N>() <= kMaxSmem, "split column pass does not fit");
            const bool to_scratch = !CONJ || a.conj.direct;    // intensity through the transpose
            if (to_scratch && !a.scratch) return cudaErrorInvalidValue;
            auto k = CONJ ? conj_cols_split_kernel<N> : prop_cols_split_kernel<N>;
            cudaError_t e = set_smem(k, pcol_split_smem<N>());
            int nc = 0;
            if (e == cudaSuccess) e = active_clusters(k, 2, psplit_threads<N>(), pcol_split_smem<N>(), &nc);
            if (e != cudaSuccess) return e;
            e = launch_k(k, 2, dim3(2 * std::min(nc, N)), dim3(psplit_threads<N>()), pcol_split_smem<N>(), s, a);
            if (e != cudaSuccess || !to_scratch) return e;
            transpose_add_kernel<<<dim3(N / 32, N / 32), 256, 0, s>>>(a.scratch, a.intensity, N, a.accumulate);
            return cudaGetLastError();
        } else if constexpr (prow_smem<N>() > kMaxSmem || pcol_smem<N>() > kMaxSmem) {
            return cudaErrorNotSupported;
        } else {
            cudaError_t e = set_smem(prop_cols_kernel<N, CONJ>, pcol_smem<N>());
            if (e != cudaSuccess) return e;
            prop_cols_kernel<N, CONJ><<<N / pcol_lines<N>(), pcol_threads<N>(), pcol_smem<N>(), s>>>(a);
            return cudaGetLastError();
        }
    });
}

cudaError_t launch_prop_rows(const PropArgs& a, bool conj, cudaStream_t s) {
    return conj ? launch_rows<true>(a, s) : launch_rows<false>(a, s);
}
cudaError_t launch_prop_cols(const PropArgs& a, bool conj, cudaStream_t s) {
    return conj ? launch_cols<true>(a, s) : launch_cols<false>(a, s);
}

// ---- passband of one-FFT patterns --------------------------------------------------
// Output pixel (X, Y) samples pattern l at (X - n/2) r_l + n/2 and (Y - n/2) r_l + n/2
// pattern pixels; the products are exact in 32.32 fixed point (|X - n/2| r_l < 2^47).
// Patterns are column-major (element (x, y) at x n + y).
struct Sample {
    int i0;       // integer part, not yet wrapped
    float f;      // fraction
};
SCINT_DEV Sample sample_at(int X, int n, long long r_fx) {
    const long long u = (long long)(X - n / 2) * r_fx + ((long long)(n / 2) << 32);
    return Sample{(int)(u >> 32), (float)(unsigned)(u & 0xFFFFFFFFll) * 0x1.0p-32f};
}

// Tiled form: a block makes a 32 x 32 output tile and keeps it in registers over
// all wavelengths.  Lanes take consecutive output rows of one column, so the
// four bilinear taps of a warp read consecutive elements of two pattern columns
// (patterns are column-major); the tile goes out through shared memory as rows.
constexpr int kResTile = 32;
__global__ void __launch_bounds__(256) resample_tiled_kernel(ResampleArgs a) {
    __shared__ float tile[kResTile][kResTile + 1];   // [x][y]
    const int n = a.n;
    const int X0 = blockIdx.x * kResTile, Y0 = blockIdx.y * kResTile;
    const int ly = threadIdx.x % kResTile, lx = threadIdx.x / kResTile;   // lx in [0, 8)
    float acc[kResTile / 8] = {};
    for (int l = 0; l < a.count; ++l) {
        const long long r = a.r_fx[l];
        const float* h = a.pattern + (size_t)l * n * n;
        const Sample sy = sample_at(Y0 + ly, n, r);
        const int y0 = sy.i0 & (n - 1), y1 = (y0 + 1) & (n - 1);
        const float wl = a.weight[l];
#pragma unroll
        for (int q = 0; q < kResTile / 8; ++q) {
            const Sample sx = sample_at(X0 + lx + 8 * q, n, r);
            const int x0 = sx.i0 & (n - 1), x1 = (x0 + 1) & (n - 1);
            const float* c0 = h + (size_t)x0 * n;
            const float* c1 = h + (size_t)x1 * n;
            const float h00 = __ldg(c0 + y0), h01 = __ldg(c0 + y1), h10 = __ldg(c1 + y0), h11 = __ldg(c1 + y1);
            const float left = fmaf(sy.f, h01 - h00, h00), right = fmaf(sy.f, h11 - h10, h10);
            acc[q] = fmaf(wl, fmaf(sx.f, right - left, left), acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kResTile / 8; ++q) tile[lx + 8 * q][ly] = acc[q];
    __syncthreads();
    // rows out: lanes take consecutive x of one row
#pragma unroll
    for (int q = 0; q < kResTile / 8; ++q) {
        const int oy = lx + 8 * q, ox = ly;
        float* o = a.intensity + (size_t)(Y0 + oy) * n + X0 + ox;
        const float v = tile[ox][oy];
        *o = a.accumulate ? *o + v : v;
    }
}

// Plain form for grids below one tile and scale factors beyond the patch.
__global__ void resample_kernel(ResampleArgs a) {
    const int n = a.n;
    const size_t total = (size_t)n * n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % n), Y = (int)(i / n);
        float acc = 0.0f;
        for (int l = 0; l < a.count; ++l) {
            const Sample sx = sample_at(X, n, a.r_fx[l]), sy = sample_at(Y, n, a.r_fx[l]);
            const int x0 = sx.i0 & (n - 1), y0 = sy.i0 & (n - 1);
            const int x1 = (x0 + 1) & (n - 1), y1 = (y0 + 1) & (n - 1);
            const float* h = a.pattern + (size_t)l * total;
            const float h00 = __ldg(h + (size_t)x0 * n + y0), h10 = __ldg(h + (size_t)x1 * n + y0);
            const float h01 = __ldg(h + (size_t)x0 * n + y1), h11 = __ldg(h + (size_t)x1 * n + y1);
            const float top = fmaf(sx.f, h10 - h00, h00), bot = fmaf(sx.f, h11 - h01, h01);
            acc = fmaf(a.weight[l], fmaf(sy.f, bot - top, top), acc);
        }
        a.intensity[i] = a.accumulate ? a.intensity[i] + acc : acc;
    }
}

cudaError_t launch_resample(const ResampleArgs& a, cudaStream_t s) {
    const bool tiled = a.n >= kResTile;
    if (tiled) {
        resample_tiled_kernel<<<dim3(a.n / kResTile, a.n / kResTile), 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t total = (size_t)a.n * a.n;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)sms * 8);
    resample_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace scint
