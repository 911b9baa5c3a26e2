// Extended-source smoothing (Sect. 3.2.3, Eq. iprh): periodic convolution of a
// real N x N intensity map with the uniform disk of radius R_s, done as
//   column pass: two real columns packed as one complex line, FFT_y, split into
//                the two half spectra (ky = 0..N/2) -> spec[ky][x]
//   row pass:    each half-spectrum row: FFT_x, times K(q)/N^2, IFFT_x, in place
//   column pass: rebuild the full ky range from Hermitian symmetry, pack two
//                columns, IFFT_y, unpack real and imaginary parts -> intensity
// with K(q) = 2 J1(2 pi q R_s) / (2 pi q R_s), K(0) = 1.
#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "pairs.cuh"

namespace scint {

// N = 16384 lines go to a cluster of two blocks (the split kernels below)
template <int N> __host__ __device__ constexpr int scs() { return N >= kSplitN ? 2 : 1; }
// column passes: packed column pairs per block, 16384 / N below N = 8192 (1024 threads), so that
// a block's row accesses are whole 32-byte sectors (four pairs at 4096): the passes are bound by
// scattered sector requests, not latency (two 512-thread blocks per SM were slower).  Measured
// against two pairs per block: 4096^2 forward 79 -> 66 us, inverse 91 -> 62 us; 2048^2 19 -> 16,
// 18.5 -> 15 us.
// From N = kSmoothPairsN (8192) a block holds one pair, and the map is read and written as
// column pairs through the transposes of pairs.cuh (one 8-byte value per row otherwise).
template <int N> __host__ __device__ constexpr int scol_lines() { return N >= kSmoothPairsN ? 1 : (16384 / N < N / 2 ? 16384 / N : N / 2); }
template <int N> __host__ __device__ constexpr int scol_threads() { return scol_lines<N>() * FftPlan<N>::T / scs<N>(); }
template <int N> __host__ __device__ constexpr int srow_lines() { return N >= kTileRow32 ? 1 : (kTileRow32 / N < N / 2 ? kTileRow32 / N : N / 2); }
template <int N> __host__ __device__ constexpr int srow_threads() { return srow_lines<N>() * FftPlan<N>::T / scs<N>(); }

// shared twiddle table below the split size (after the line buffers)
template <int N> __host__ __device__ constexpr int stwm() { return scs<N>() == 1 ? 1 : 0; }
template <int N> constexpr size_t stws_bytes() { return stwm<N>() == 1 ? (size_t)FftPlan<N>::TWS * sizeof(float2) : 0; }

template <int CS> SCINT_DEV int srank() {
    if constexpr (CS == 1) return 0;
    else return (int)cooperative_groups::this_cluster().block_rank();
}

// forward: two real columns (xa, xa+1) -> half spectra rows 0..N/2 of spec
template <int N>
__global__ void __launch_bounds__(scol_threads<N>(), (scol_threads<N>() <= 256 ? 2 : 1))
smooth_fwd_cols_kernel(SmoothArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = scs<N>();
    constexpr int T = Pl::T, E = Pl::E, W = scol_lines<N>(), TL = T / CS, HALF = N / 2;
    extern __shared__ float2 smem32[];
    const int w = threadIdx.x % W;
    const int t = srank<CS>() * TL + threadIdx.x / W;
    const int xa = ((blockIdx.x / CS) * W + w) * 2;
    float2* buf = smem32 + w;     // W lines interleaved
    constexpr int TWM = stwm<N>();
    float2* tws = smem32 + W * (Pl::BUF / CS);
    if constexpr (TWM == 1) fill_twiddle_table<float2, N>(tws, a.tw, threadIdx.x, blockDim.x);
    const float2* twp = TWM == 1 ? tws : a.tw;
    float2 v[E];
    if constexpr (N >= kSmoothPairsN) {
        // one pair per block: the map as column pairs (consecutive rows, consecutive 8-byte values)
        static_assert(W == 1 && CS == 1, "column pairs with one pair per unsplit block");
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = a.pairs[(size_t)(xa / 2) * N + t + m * T];
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = *reinterpret_cast<const float2*>(a.intensity + (size_t)(t + m * T) * N + xa);
    }
    line_sync<CS>();
    fft_line<float2, N, -1, 16, W, TWM, CS>(v, buf, t, twp);
    // Z[N-k] lives in another thread: go through shared memory (natural order)
    float2* bufs[CS];
    if constexpr (CS == 1) {
        bufs[0] = buf;
    } else {
        bufs[0] = cooperative_groups::this_cluster().map_shared_rank(buf, 0);
        bufs[1] = cooperative_groups::this_cluster().map_shared_rank(buf, 1);
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int e = t + m * T, o = CS == 2 && e >= HALF ? 1 : 0;
        bufs[o][pad16(e - o * HALF) * W] = v[m];
    }
    line_sync<CS>();
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * T;
        if (k <= N / 2) {
            const int e = (N - k) & (N - 1), o = CS == 2 && e >= HALF ? 1 : 0;
            const float2 z = v[m];
            const float2 zc = conjc(bufs[o][pad16(e - o * HALF) * W]);
            // X_a = (Z + conj Z(-k))/2, X_b = (Z - conj Z(-k))/(2i)
            const float2 xa_ = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y + zc.y));
            const float2 xb_ = make_float2(0.5f * (z.y - zc.y), -0.5f * (z.x - zc.x));
            *reinterpret_cast<float4*>(a.spec + (size_t)k * N + xa) = make_float4(xa_.x, xa_.y, xb_.x, xb_.y);
        }
    }
    line_sync<CS>();
}

// rows of the half spectrum: FFT_x, times K/N^2, IFFT_x
// register twiddle bases below the split size (the row pass's loads stay in registers)
template <int N> __host__ __device__ constexpr int srow_twm() { return scs<N>() == 1 ? 2 : 0; }

template <int N>
__global__ void __launch_bounds__(srow_threads<N>(), (srow_threads<N>() <= 256 ? 2 : 1))
smooth_rows_kernel(SmoothArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = scs<N>();
    constexpr int T = Pl::T, E = Pl::E, B = srow_lines<N>(), TL = T / CS;
    extern __shared__ float2 smem32[];
    const int team = threadIdx.x / TL;
    const int t = srank<CS>() * TL + threadIdx.x % TL;
    const int ky = (blockIdx.x / CS) * B + team;
    const bool live = ky <= N / 2;
    float2* row = a.spec + (size_t)(live ? ky : 0) * N;
    constexpr int TWM = srow_twm<N>();
    TwiddleRegs<float2, N, 16> tr;
    if constexpr (TWM == 2) tr.load(a.tw, t);
    float2* buf = smem32 + team * (Pl::BUF / CS);
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = live ? row[t + m * T] : make_float2(0.f, 0.f);
    line_sync<CS>();
    if constexpr (TWM == 2) fft_line_tr<float2, N, -1, 16, 1>(v, buf, t, tr);
    else fft_line<float2, N, -1, 16, 1, TWM, CS>(v, buf, t, a.tw);
    // mx^2 + my^2 <= N^2/2 is exact in FP32 for N <= 4096 and within one rounding above
    const float inv = 1.0f / ((float)N * (float)N);
    const float twopi_r = (float)(2.0 * kPi * a.radius_over_L);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int kx = t + m * T;
        const int mx = kx < N / 2 ? kx : kx - N;
        const float u = twopi_r * sqrtf((float)(mx * mx + ky * ky));
        const float K = u > 0.0f ? 2.0f * j1f(u) / u : 1.0f;
        v[m] = v[m] * (K * inv);
    }
    if constexpr (TWM == 2) fft_line_tr<float2, N, +1, 16, 1>(v, buf, t, tr);
    else fft_line<float2, N, +1, 16, 1, TWM, CS>(v, buf, t, a.tw);
    if (live) {
#pragma unroll
        for (int m = 0; m < E; ++m) row[t + m * T] = v[m];
    }
    if constexpr (CS == 2) line_sync<CS>();
}

// inverse: half spectra -> two real columns
template <int N>
__global__ void __launch_bounds__(scol_threads<N>(), (scol_threads<N>() <= 256 ? 2 : 1))
smooth_inv_cols_kernel(SmoothArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = scs<N>();
    constexpr int T = Pl::T, E = Pl::E, W = scol_lines<N>(), TL = T / CS;
    extern __shared__ float2 smem32[];
    const int w = threadIdx.x % W;
    const int t = srank<CS>() * TL + threadIdx.x / W;
    const int xa = ((blockIdx.x / CS) * W + w) * 2;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * T;
        const bool lo = k <= N / 2;
        const float4 q = *reinterpret_cast<const float4*>(a.spec + (size_t)(lo ? k : N - k) * N + xa);
        // X(k) for k > N/2 is conj X(N-k) (real columns)
        const float2 Xa = lo ? make_float2(q.x, q.y) : make_float2(q.x, -q.y);
        const float2 Xb = lo ? make_float2(q.z, q.w) : make_float2(q.z, -q.w);
        v[m] = make_float2(Xa.x - Xb.y, Xa.y + Xb.x);   // Z = X_a + i X_b
    }
    constexpr int TWM = stwm<N>();
    float2* tws = smem32 + W * (Pl::BUF / CS);
    if constexpr (TWM == 1) fill_twiddle_table<float2, N>(tws, a.tw, threadIdx.x, blockDim.x);
    const float2* twp = TWM == 1 ? tws : a.tw;
    line_sync<CS>();
    fft_line<float2, N, +1, 16, W, TWM, CS>(v, smem32 + w, t, twp);
    if constexpr (N >= kSmoothPairsN) {
#pragma unroll
        for (int m = 0; m < E; ++m) a.pairs[(size_t)(xa / 2) * N + t + m * T] = v[m];
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m)
            *reinterpret_cast<float2*>(a.intensity + (size_t)(t + m * T) * N + xa) = v[m];
    }
    if constexpr (CS == 2) line_sync<CS>();
}

// ---- N = 16384: lines split by one radix-2 step over a two-block cluster --------------
// Block r of a cluster transforms the parity-r half of every line as a whole 8192-point
// line in its own shared memory (fft.cuh: split_dif, split_combine):
//   forward column pass: the frequencies f = 2k + r of the packed column pair, by
//     decimation in frequency from both halves of the columns (both blocks read them);
//     Z(N - f) has the parity of f, so the half-spectrum split stays in the block;
//   row pass: decimation in frequency from the whole row, K at the frequencies 2k + r,
//     inverse, decimation in time through the partner's buffer, written in place
//     (the partner read the row before it reached the exchange);
//   inverse column pass: block r reads the spectrum rows of its parity, inverse,
//     decimation in time.
// Grids are persistent: as many clusters as fit, each looping over lines.
//   The map enters and leaves as column pairs (pairs.cuh: a.pairs, column-major, through
//   tiled transposes), so that the column passes read and write consecutive 8-byte values:
//   one 8-byte value per 64 KB row of the map had cost about half of their time (16384^2,
//   measured without the map accesses: forward 1.87 -> 0.81 ms, inverse 2.18 -> 1.14 ms;
//   with the transposes 1.41 and 1.53 ms).  The half spectrum stays row-major: in strips of
//   four columns the column passes gained 0.25 ms each but the row pass lost 0.85 ms.
template <int N> __host__ __device__ constexpr int ssplit_threads() { return FftPlan<N / 2>::T; }
template <int N> constexpr size_t ssplit_smem() {
    return (size_t)(FftPlan<N / 2>::BUF + FftPlan<N / 2>::TWS) * sizeof(float2);
}

template <int N>
__global__ void __launch_bounds__(ssplit_threads<N>(), 1) smooth_fwd_cols_split_kernel(SmoothArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    float2* tws = smem32 + Pl::BUF;
    fill_twiddle_table<float2, H2>(tws, a.tw, t, T, 2);
    __syncthreads();
#pragma unroll 1
    for (int xa = (blockIdx.x / 2) * 2; xa < N; xa += gridDim.x) {
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = t + m * T;
            const float2* col = a.pairs + (size_t)(xa / 2) * N;
            v[m] = split_dif(col[e], col[e + H2], r, e, a.tw);
        }
        fft_line<float2, H2, -1, 16, 1, 1, 1>(v, buf, t, tws);     // v[m] = Z(2k + r), k = t + m T
#pragma unroll
        for (int m = 0; m < E; ++m) buf[pad16(t + m * T)] = v[m];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + m * T, f = 2 * k + r;
            if (f <= N / 2) {
                const float2 z = v[m];
                const float2 zc = conjc(buf[pad16((H2 - r - k) & (H2 - 1))]);   // conj Z(N - f)
                // X_a = (Z + conj Z(-f))/2, X_b = (Z - conj Z(-f))/(2i)
                *reinterpret_cast<float4*>(a.spec + (size_t)f * N + xa) =
                    make_float4(0.5f * (z.x + zc.x), 0.5f * (z.y + zc.y), 0.5f * (z.y - zc.y), -0.5f * (z.x - zc.x));
            }
        }
        __syncthreads();    // the next pair's first stage rewrites buf
    }
}

template <int N>
__global__ void __launch_bounds__(ssplit_threads<N>(), 1) smooth_rows_split_kernel(SmoothArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    float2* tws = smem32 + Pl::BUF;
    fill_twiddle_table<float2, H2>(tws, a.tw, t, T, 2);
    const float inv = 1.0f / ((float)N * (float)N);
    const float twopi_r = (float)(2.0 * kPi * a.radius_over_L);
    cluster_arrive();    // the first wait also publishes the twiddle table to the block
#pragma unroll 1
    for (int ky = blockIdx.x / 2; ky <= N / 2; ky += gridDim.x / 2) {
        float2* row = a.spec + (size_t)ky * N;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = split_dif(row[t + m * T], row[t + m * T + H2], r, t + m * T, a.tw);
        cluster_wait();
        fft_line<float2, H2, -1, 16, 1, 1, 1>(v, buf, t, tws);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int kx = 2 * (t + m * T) + r;
            const int mx = kx < N / 2 ? kx : kx - N;
            const float u = twopi_r * sqrtf((float)(mx * mx + ky * ky));
            const float K = u > 0.0f ? 2.0f * j1f(u) / u : 1.0f;
            v[m] = v[m] * (K * inv);
        }
        fft_line<float2, H2, +1, 16, 1, 1, 1>(v, buf, t, tws);
        split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int, int n, float2 y0, float2 y1) {
            row[n] = y0;
            row[n + H2] = y1;
        });
    }
    cluster_wait();
}

template <int N>
__global__ void __launch_bounds__(ssplit_threads<N>(), 1) smooth_inv_cols_split_kernel(SmoothArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    float2* tws = smem32 + Pl::BUF;
    fill_twiddle_table<float2, H2>(tws, a.tw, t, T, 2);
    cluster_arrive();
#pragma unroll 1
    for (int xa = (blockIdx.x / 2) * 2; xa < N; xa += gridDim.x) {
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int f = 2 * (t + m * T) + r;
            const bool lo = f <= N / 2;
            const float4 q = *reinterpret_cast<const float4*>(a.spec + (size_t)(lo ? f : N - f) * N + xa);
            // X(f) for f > N/2 is conj X(N-f) (real columns); Z = X_a + i X_b
            const float2 Xa = lo ? make_float2(q.x, q.y) : make_float2(q.x, -q.y);
            const float2 Xb = lo ? make_float2(q.z, q.w) : make_float2(q.z, -q.w);
            v[m] = make_float2(Xa.x - Xb.y, Xa.y + Xb.x);
        }
        cluster_wait();
        fft_line<float2, H2, +1, 16, 1, 1, 1>(v, buf, t, tws);
        float2* col = a.pairs + (size_t)(xa / 2) * N;
        split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int, int n, float2 y0, float2 y1) {
            col[n] = y0;
            col[n + H2] = y1;
        });
    }
    cluster_wait();
}

template <int N> constexpr size_t scol_smem() { return (size_t)scol_lines<N>() * FftPlan<N>::BUF * sizeof(float2) / scs<N>() + stws_bytes<N>(); }
template <int N> constexpr size_t srow_smem() { return (size_t)srow_lines<N>() * FftPlan<N>::BUF * sizeof(float2) / scs<N>(); }

// which = 0: forward column pass, 1: row pass, 2: inverse column pass
cudaError_t launch_smooth_pass(const SmoothArgs& a, int which, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (N < 32) {
            return cudaErrorNotSupported;
        } else {
            constexpr int CS = scs<N>();
            cudaError_t e;
            if constexpr (CS == 2) {
                static_assert(ssplit_smem<N>() <= 227 * 1024, "split smoothing pass does not fit");
                auto k = which == 0 ? smooth_fwd_cols_split_kernel<N>
                                    : (which == 1 ? smooth_rows_split_kernel<N> : smooth_inv_cols_split_kernel<N>);
                int nc = 0;
                if ((e = set_smem(k, ssplit_smem<N>())) != cudaSuccess) return e;
                if ((e = active_clusters(k, 2, ssplit_threads<N>(), ssplit_smem<N>(), &nc)) != cudaSuccess) return e;
                const int lines = which == 1 ? N / 2 + 1 : N / 2;
                if (!a.pairs) return cudaErrorInvalidValue;
                if (which == 0 && (e = launch_rows_to_pairs(a.intensity, a.pairs, N, s)) != cudaSuccess) return e;
                e = launch_k(k, 2, dim3(2 * std::min(nc, lines)), dim3(ssplit_threads<N>()), ssplit_smem<N>(), s, a);
                if (e != cudaSuccess || which != 2) return e;
                return launch_pairs_to_rows(a.pairs, a.intensity, N, s);
            } else {
            // every block (cluster) of the column passes holds W line pairs = 2W real columns
            const int col_blocks = N / (2 * scol_lines<N>()) * CS;
            if (N >= kSmoothPairsN && !a.pairs) return cudaErrorInvalidValue;
            if (which == 0) {
                if ((e = set_smem(smooth_fwd_cols_kernel<N>, scol_smem<N>())) != cudaSuccess) return e;
                if (N >= kSmoothPairsN && (e = launch_rows_to_pairs(a.intensity, a.pairs, N, s)) != cudaSuccess) return e;
                return launch_k(smooth_fwd_cols_kernel<N>, CS, dim3(col_blocks), dim3(scol_threads<N>()), scol_smem<N>(), s, a);
            } else if (which == 1) {
                if ((e = set_smem(smooth_rows_kernel<N>, srow_smem<N>())) != cudaSuccess) return e;
                const int rows = N / 2 + 1;
                return launch_k(smooth_rows_kernel<N>, CS, dim3((rows + srow_lines<N>() - 1) / srow_lines<N>() * CS),
                                dim3(srow_threads<N>()), srow_smem<N>(), s, a);
            } else {
                if ((e = set_smem(smooth_inv_cols_kernel<N>, scol_smem<N>())) != cudaSuccess) return e;
                e = launch_k(smooth_inv_cols_kernel<N>, CS, dim3(col_blocks), dim3(scol_threads<N>()), scol_smem<N>(), s, a);
                if (e != cudaSuccess || N < kSmoothPairsN) return e;
                return launch_pairs_to_rows(a.pairs, a.intensity, N, s);
            }
            }
        }
    });
}

}  // namespace scint
