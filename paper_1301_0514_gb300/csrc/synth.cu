// Phase-screen synthesis (Sect. 3.1, Eq. spectre, Eq. densite), to FP64 accuracy where
// the phase variance lies.
//
// phi = sqrt(2)/L^2 Re sum_k F_k e^{+2 pi i k.x}; the real part of the inverse
// transform of F equals the inverse transform of its Hermitian part
// F_h(k) = (F(k) + conj F(-k)) / 2, whose transform is real.  So:
// Row pass (spectral rows ky = 0..N/2 only): each team generates F_h of one
//   row in registers (for every bin the noise of (ky, kx) and of the mirror
//   bin (-ky, -kx), Philox4x32-10 + Box-Muller, amplitude sqrt(L^2 S(q))),
//   inverse-transforms it along x and writes the row G(ky, x); rows N/2+1..N-1
//   are conj G(N-ky, x) and are never formed.
// Column pass: two real columns per complex transform: Z(ky) = G_a(ky) + i
//   G_b(ky) over all ky (Hermitian extension), inverse transform along y, and
//   phi_a = sqrt(2)/L^2 Re, phi_b = sqrt(2)/L^2 Im.
// This halves the transform work and the intermediate ((N/2+1) x N values, kept
// column pair by column pair: synth_idx below).
// The noise is never stored, except up to N = 512, where the bins are drawn by a kernel of
// their own before the row pass (synth_draw_kernel).
//
// Precision: the transforms run in double-float arithmetic (dfc: pairs of FP32
// numbers, ~44 significant bits; common.cuh) on the FP32 pipes, which on GB300
// are 64 times wider than the FP64 pipe, except the x transforms of the rows
// outside the FP64 square (synth_row32), which run in FP32; the low bins are
// drawn in FP64 and the phase is written in FP64.
#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "pairs.cuh"
#include "spectrum.cuh"

namespace scint {

__global__ void twiddles32_kernel(float2* tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)n, &s, &c);
        tw[j] = make_float2((float)c, (float)s);
    }
}
__global__ void twiddles64_kernel(double2* tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)n, &s, &c);
        tw[j] = make_double2(c, s);
    }
}
__global__ void twiddles_df_kernel(dfc* tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)n, &s, &c);
        tw[j] = dfc{dfl(c), dfl(s)};
    }
}
cudaError_t launch_twiddles_df(dfc* tw, int n, cudaStream_t s) {
    twiddles_df_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
    return cudaGetLastError();
}
cudaError_t launch_twiddles32(float2* tw, int n, cudaStream_t s) {
    twiddles32_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
    return cudaGetLastError();
}
cudaError_t launch_twiddles64(double2* tw, int n, cudaStream_t s) {
    twiddles64_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
    return cudaGetLastError();
}

// Lines per block (all transformed together); N = 16384 lines (256 KB in
// double-float) go to a cluster of two blocks (the split kernels below).
template <int N> __host__ __device__ constexpr int synth_cs() { return N >= kSplitN ? 2 : 1; }
template <int N> __host__ __device__ constexpr int synth_tile_lines() { return N >= kTile64 ? 1 : (kTile64 / N < N ? kTile64 / N : N); }
// Rows per row-pass block: the tile, but no more than leaves about two blocks per SM (the
// N/2 + 1 rows over 304 blocks).  Up to N = 512 every bin is drawn in FP64, whose pipe is
// narrow: at 256^2 sixteen rows per block had kept 9 SMs busy for 0.30 ms.
template <int N> __host__ __device__ constexpr int synth_lines() {
    constexpr int spread = (N / 2 + 1) / 304 > 1 ? (N / 2 + 1) / 304 : 1;
    return synth_tile_lines<N>() < spread ? synth_tile_lines<N>() : spread;
}
template <int N> __host__ __device__ constexpr int synth_threads() { return synth_lines<N>() * FftPlan<N>::T / synth_cs<N>(); }
// column pass: complex lines (each two real output columns) per block, at most N/2
// (two at N = 4096, 139 KB of shared memory: 0.236 -> 0.201 ms per 4096^2 pass against one)
template <int N> __host__ __device__ constexpr int synth_col_lines() {
    return N == 4096 ? 2 : (synth_tile_lines<N>() < N / 2 ? synth_tile_lines<N>() : N / 2);
}
template <int N> __host__ __device__ constexpr int synth_col_threads() { return synth_col_lines<N>() * FftPlan<N>::T / synth_cs<N>(); }
template <int N> constexpr size_t synth_smem() { return (size_t)synth_lines<N>() * FftPlan<N>::BUF * sizeof(dfc) / synth_cs<N>(); }
template <int N> constexpr size_t synth_col_smem() { return (size_t)synth_col_lines<N>() * FftPlan<N>::BUF * sizeof(dfc) / synth_cs<N>(); }

// The intermediate G(ky, x), ky = 0..N/2, is stored in strips of one column pair
// p = x/2 (synth_strip<N>() values each), so that a column pass reads contiguous memory:
// below the split size the rows follow each other (two values per row); at N >= kSplitN
// the rows of each parity are grouped (N/4 + 1 rows each), since block r of a column
// cluster reads the rows of parity r.  The row pass's stores are whole 32-byte sectors.
template <int N> __host__ __device__ constexpr int synth_strip() { return N + 4; }
template <int N> SCINT_DEV size_t synth_idx(int ky, int x) {
    const size_t strip = (size_t)(x >> 1) * synth_strip<N>() + (x & 1);
    if constexpr (N >= kSplitN) return strip + (size_t)(ky & 1) * (synth_strip<N>() / 2) + (size_t)(ky >> 1) * 2;
    else return strip + (size_t)ky * 2;
}

template <int CS> SCINT_DEV int synth_rank() {
    if constexpr (CS == 1) return 0;
    else return (int)cooperative_groups::this_cluster().block_rank();
}

// F_h(ky, kx) = (F(ky, kx) + conj F(-ky, -kx)) / 2 (the halving is exact)
SCINT_DEV dfl half(dfl v) { return dfl(0.5f * v.hi, 0.5f * v.lo); }
SCINT_DEV dfc hermitian_bin(const SynthArgs& a, int kx, int ky) {
    dfc f, g;
    spectrum_pair_df(a, kx, ky, f, g);
    return dfc{half(f.x + g.x), half(f.y - g.y)};
}

// Rows outside the FP64 square (|my| > low_k) hold only bins drawn in FP32, whose
// phase contribution is small (an rms below ~0.5 rad for every screen, by the choice
// of low_k), so their x transform runs in FP32: its rounding is ~1e-7 of that small
// contribution.  The rows inside the square carry nearly all of the phase variance and
// keep the double-float transform; the column pass, where every row's contribution
// meets, stays in double-float.  Outputs go to the same double-float rows (lo = 0).
SCINT_DEV float2 hermitian_bin32(const SynthArgs& a, int kx, int ky) {
    float2 f, g;
    spectrum_pair_high(a, kx, ky, f, g);
    return make_float2(0.5f * (f.x + g.x), 0.5f * (f.y - g.y));
}
SCINT_DEV dfc widen(float2 v) { return dfc{dfl(v.x, 0.0f), dfl(v.y, 0.0f)}; }

template <int N>
SCINT_DEV void synth_row32(const SynthArgs& a, int ky, bool live, int t, float2* buf) {
    using Pl = FftPlan<N>;
    constexpr int T = Pl::T, E = Pl::E;
    float2 v[E];
    // drawn in a loop that is not unrolled and staged in the line buffer (as in the rows below)
#pragma unroll 1
    for (int m = 0; m < E; ++m) buf[pad16(t + m * T)] = live ? hermitian_bin32(a, t + m * T, ky) : make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = buf[pad16(t + m * T)];
    TwiddleRegs<float2, N, 16> tr;
    tr.load(a.tw32, t);
    __syncthreads();
    fft_line_tr<float2, N, +1, 16, 1>(v, buf, t, tr);
    if (live) {
#pragma unroll
        for (int m = 0; m < E; ++m) a.work[synth_idx<N>(ky, t + m * T)] = widen(v[m]);
    }
}

// Up to N = 512 every bin is drawn in FP64 on the narrow FP64 pipe; a row's team there has
// only N/16 threads, so the Hermitian bins of rows 0..N/2 are drawn first, one per thread of
// this kernel, into a.drawn (row-major), and the row pass reads them.
__global__ void __launch_bounds__(256) synth_draw_kernel(SynthArgs a) {
    const int n = a.n;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= (n / 2 + 1) * n) return;
    a.drawn[i] = hermitian_bin(a, i % n, i / n);
}

template <int N>
__global__ void __launch_bounds__(synth_threads<N>())
synth_rows_kernel(SynthArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = synth_cs<N>();
    constexpr int T = Pl::T, E = Pl::E, B = synth_lines<N>(), TL = T / CS;
    extern __shared__ dfc smem_df[];
    const int team = threadIdx.x / TL;
    const int t = synth_rank<CS>() * TL + threadIdx.x % TL;
    const int ky = (blockIdx.x / CS) * B + team;
    const bool live = ky <= N / 2;                 // rows above N/2 are the conjugates of rows below
    if constexpr (CS == 1) {
        // every row of the block outside the square (the choice is uniform over the block)
        if ((blockIdx.x / CS) * B > a.low_k) {
            synth_row32<N>(a, ky, live, t, reinterpret_cast<float2*>(smem_df) + team * Pl::BUF);
            return;
        }
    }
    dfc v[E];
    dfc* buf = smem_df + team * (Pl::BUF / CS);
    if constexpr (CS == 1) {
        if (a.drawn) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = live ? a.drawn[(size_t)ky * N + t + m * T] : make_c<dfc>(0.0, 0.0);
        } else {
            // the bins are drawn in a loop that is not unrolled (one copy of the Philox and
            // Box-Muller code: unrolled sixteen times it overflowed the instruction cache) and
            // staged in the line buffer, where each thread reads back its own entries
#pragma unroll 1
            for (int m = 0; m < E; ++m)
                buf[pad16(t + m * T)] = live ? hermitian_bin(a, t + m * T, ky) : make_c<dfc>(0.0, 0.0);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = buf[pad16(t + m * T)];
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = live ? hermitian_bin(a, t + m * T, ky) : make_c<dfc>(0.0, 0.0);
    }
    line_sync<CS>();
    fft_line<dfc, N, +1, 16, 1, 0, CS>(v, buf, t, a.tw);
    if (live) {
#pragma unroll
        for (int m = 0; m < E; ++m) a.work[synth_idx<N>(ky, t + m * T)] = v[m];
    }
    if constexpr (CS == 2) line_sync<CS>();
}

// two real output columns (xa, xa + 1) per complex line
template <int N>
__global__ void __launch_bounds__(synth_col_threads<N>())
synth_cols_kernel(SynthArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = synth_cs<N>();
    constexpr int T = Pl::T, E = Pl::E, W = synth_col_lines<N>(), TL = T / CS;
    extern __shared__ dfc smem_df[];
    const int w = threadIdx.x % W;
    const int t = synth_rank<CS>() * TL + threadIdx.x / W;
    const int xa = ((blockIdx.x / CS) * W + w) * 2;
    dfc v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int ky = t + m * T;
        const bool lo = ky <= N / 2;
        const dfc* g = a.work + synth_idx<N>(lo ? ky : N - ky, xa);
        const dfc ga = g[0], gb = g[1];
        // G(ky) = conj G(N - ky) above N/2; Z = G_a + i G_b
        const dfc za = lo ? ga : conjc(ga), zb = lo ? gb : conjc(gb);
        v[m] = dfc{za.x - zb.y, za.y + zb.x};
    }
    line_sync<CS>();
    fft_line<dfc, N, +1, 16, W, 0, CS>(v, smem_df + w, t, a.tw);     // W lines interleaved
    // columns xa, xa + 1 of a row are adjacent (xa even): one 16-byte store per row
#pragma unroll
    for (int m = 0; m < E; ++m)
        *reinterpret_cast<double2*>(a.phi + (size_t)(t + m * T) * N + xa) =
            make_double2(scaled_to_double(v[m].x, a.out_scale_df), scaled_to_double(v[m].y, a.out_scale_df));
    if constexpr (CS == 2) line_sync<CS>();
}

// ---- N = 16384: lines split by one radix-2 step over a two-block cluster --------------
// Both passes are inverse transforms, so each block r of a cluster takes the spectral
// values of parity r (f = 2k + r), inverse-transforms them as a whole 8192-point line in
// its own shared memory, and the decimation-in-time step combines the two halves through
// the partner's buffer (fft.cuh, split_combine): no value is generated or read twice.
// Twiddles come from the N-point double-float table at even indices.  Persistent grids.
template <int N> __host__ __device__ constexpr int synth_split_threads() { return FftPlan<N / 2>::T; }
template <int N> constexpr size_t synth_split_smem() { return (size_t)FftPlan<N / 2>::BUF * sizeof(dfc); }

template <int N>
__global__ void __launch_bounds__(synth_split_threads<N>(), 1) synth_rows_split_kernel(SynthArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ dfc smem_df[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    dfc* buf = smem_df;
    cluster_arrive();
#pragma unroll 1
    for (int ky = blockIdx.x / 2; ky <= N / 2; ky += gridDim.x / 2) {
        cluster_wait();
        if (ky > a.low_k) {    // outside the FP64 square: FP32 transform (see synth_row32)
            float2* b32 = reinterpret_cast<float2*>(buf);
            float2 u[E];
#pragma unroll 1
            for (int m = 0; m < E; ++m) b32[pad16(t + m * T)] = hermitian_bin32(a, 2 * (t + m * T) + r, ky);
#pragma unroll
            for (int m = 0; m < E; ++m) u[m] = b32[pad16(t + m * T)];
            TwiddleRegs<float2, H2, 16> tr;
            tr.load(a.tw32, t, 2);    // the N-point table at even indices
            __syncthreads();
            fft_line_tr<float2, H2, +1, 16, 1>(u, b32, t, tr);
            split_combine<float2, H2>(u, b32, t, r, a.tw32, [&](int, int n, float2 y0, float2 y1) {
                a.work[synth_idx<N>(ky, n)] = widen(y0);
                a.work[synth_idx<N>(ky, n + H2)] = widen(y1);
            });
            continue;
        }
        dfc v[E];
        // bins drawn in a loop that is not unrolled and staged in the line buffer (see synth_rows_kernel)
#pragma unroll 1
        for (int m = 0; m < E; ++m) buf[pad16(t + m * T)] = hermitian_bin(a, 2 * (t + m * T) + r, ky);
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = buf[pad16(t + m * T)];
        __syncthreads();
        fft_line<dfc, H2, +1, 16, 1, 0, 1, 2>(v, buf, t, a.tw);
        split_combine<dfc, H2>(v, buf, t, r, a.tw, [&](int, int n, dfc y0, dfc y1) {
            a.work[synth_idx<N>(ky, n)] = y0;
            a.work[synth_idx<N>(ky, n + H2)] = y1;
        });
    }
    cluster_wait();
}

// two real output columns (xa, xa + 1) per complex line
template <int N>
__global__ void __launch_bounds__(synth_split_threads<N>(), 1) synth_cols_split_kernel(SynthArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ dfc smem_df[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    dfc* buf = smem_df;
    cluster_arrive();
#pragma unroll 1
    for (int xa = (blockIdx.x / 2) * 2; xa < N; xa += gridDim.x) {
        dfc v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int ky = 2 * (t + m * T) + r;
            const bool lo = ky <= N / 2;
            const dfc* g = a.work + synth_idx<N>(lo ? ky : N - ky, xa);
            const dfc ga = g[0], gb = g[1];
            // G(ky) = conj G(N - ky) above N/2; Z = G_a + i G_b
            const dfc za = lo ? ga : conjc(ga), zb = lo ? gb : conjc(gb);
            v[m] = dfc{za.x - zb.y, za.y + zb.x};
        }
        cluster_wait();
        fft_line<dfc, H2, +1, 16, 1, 0, 1, 2>(v, buf, t, a.tw);
        // the column pair goes out column-major (consecutive rows of a warp are consecutive 16-byte
        // entries); a tiled transpose (pairs.cuh) puts it in place: row-major stores of one 16-byte pair
        // per row had cost 2.6 of this pass's 6.9 ms at 16384^2
        double2* col = a.pairs + (size_t)(xa / 2) * N;
        split_combine<dfc, H2>(v, buf, t, r, a.tw, [&](int, int n, dfc y0, dfc y1) {
            col[n] = make_double2(scaled_to_double(y0.x, a.out_scale_df), scaled_to_double(y0.y, a.out_scale_df));
            col[n + H2] = make_double2(scaled_to_double(y1.x, a.out_scale_df), scaled_to_double(y1.y, a.out_scale_df));
        });
    }
    cluster_wait();
}

template <bool ROWS>
cudaError_t launch_synth_pass(const SynthArgs& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (synth_smem<N>() > 227 * 1024) {
            return cudaErrorNotSupported;
        } else {
            constexpr int CS = synth_cs<N>();
            cudaError_t e;
            if constexpr (CS == 2) {
                static_assert(synth_split_smem<N>() <= 227 * 1024, "split synthesis pass does not fit");
                auto k = ROWS ? synth_rows_split_kernel<N> : synth_cols_split_kernel<N>;
                int nc = 0;
                if ((e = set_smem(k, synth_split_smem<N>())) != cudaSuccess) return e;
                if ((e = active_clusters(k, 2, synth_split_threads<N>(), synth_split_smem<N>(), &nc)) != cudaSuccess)
                    return e;
                const int lines = ROWS ? N / 2 + 1 : N / 2;
                if (!ROWS && !a.pairs) return cudaErrorInvalidValue;
                e = launch_k(k, 2, dim3(2 * std::min(nc, lines)), dim3(synth_split_threads<N>()),
                             synth_split_smem<N>(), s, a);
                if (e != cudaSuccess || ROWS) return e;
                return launch_pairs_to_rows(a.pairs, a.phi, N, s);
            } else if (ROWS) {
                if ((e = set_smem(synth_rows_kernel<N>, synth_smem<N>())) != cudaSuccess) return e;
                if (a.drawn) {
                    const int bins = (N / 2 + 1) * N;
                    synth_draw_kernel<<<(bins + 255) / 256, 256, 0, s>>>(a);
                    if ((e = cudaGetLastError()) != cudaSuccess) return e;
                }
                const int rows = N / 2 + 1;
                return launch_k(synth_rows_kernel<N>, CS, dim3((rows + synth_lines<N>() - 1) / synth_lines<N>() * CS),
                                dim3(synth_threads<N>()), synth_smem<N>(), s, a);
            } else {
                if ((e = set_smem(synth_cols_kernel<N>, synth_col_smem<N>())) != cudaSuccess) return e;
                return launch_k(synth_cols_kernel<N>, CS, dim3(N / (2 * synth_col_lines<N>()) * CS),
                                dim3(synth_col_threads<N>()), synth_col_smem<N>(), s, a);
            }
        }
    });
}
cudaError_t launch_synth_rows(const SynthArgs& a, cudaStream_t s) { return launch_synth_pass<true>(a, s); }
cudaError_t launch_synth_cols(const SynthArgs& a, cudaStream_t s) { return launch_synth_pass<false>(a, s); }

// ---- test hooks --------------------------------------------------------------
__global__ void noise_words_kernel(int n, uint32_t sid, uint32_t k0, uint32_t k1, uint32_t* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n * n) return;
    const int kx = (int)(i % n), ky = (int)(i / n);
    const u32x4 w = philox4x32_10(u32x4{(uint32_t)kx, (uint32_t)ky, sid, 0u}, k0, k1);
    reinterpret_cast<uint4*>(out)[i] = make_uint4(w.x, w.y, w.z, w.w);
}
__global__ void noise_spectrum_kernel(SynthArgs a, double2* F) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)a.n * a.n) return;
    F[i] = spectrum_bin(a, (int)(i % a.n), (int)(i / a.n));
}
cudaError_t launch_noise_words(int n, uint32_t sid, uint32_t k0, uint32_t k1, uint32_t* words,
                               cudaStream_t s) {
    const size_t tot = (size_t)n * n;
    noise_words_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, sid, k0, k1, words);
    return cudaGetLastError();
}
cudaError_t launch_noise_spectrum(const SynthArgs& a, double2* F, cudaStream_t s) {
    const size_t tot = (size_t)a.n * a.n;
    noise_spectrum_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a, F);
    return cudaGetLastError();
}

}  // namespace scint
