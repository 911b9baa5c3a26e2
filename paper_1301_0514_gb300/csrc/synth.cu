// FP64 phase-screen synthesis (Sect. 3.1, Eq. spectre, Eq. densite).
//
// Pass 1 (rows of the spectrum): each team generates the shaped Gaussian noise
// F[ky][kx] of one spectral row in registers (Philox4x32-10 + Box-Muller,
// amplitude sqrt(L^2 S_phi(q))), inverse-transforms it along x and writes the
// half-transformed row into the strip-layout intermediate.  The noise is never
// stored.
// Pass 2 (columns): inverse transform along y and write phi = sqrt(2)/L^2 Re(.).
#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"

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
cudaError_t launch_twiddles32(float2* tw, int n, cudaStream_t s) {
    twiddles32_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
    return cudaGetLastError();
}
cudaError_t launch_twiddles64(double2* tw, int n, cudaStream_t s) {
    twiddles64_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
    return cudaGetLastError();
}

// Uniform in (0,1) from the 64-bit word (hi:lo): top 53 bits plus one half, times 2^-53.
SCINT_DEV double uniform53(uint32_t hi, uint32_t lo) {
    const uint64_t w = ((uint64_t)hi << 32) | lo;
    return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

SCINT_DEV int signed_freq(int i, int n) { return i < n / 2 ? i : i - n; }

// Bins with |mx| <= kLowK and |my| <= kLowK carry almost all of the phase
// variance (S ~ q^-beta): their noise and amplitude are computed in FP64.  The
// other bins have small amplitudes, so FP32 Box-Muller and pow give phase errors
// of ~1e-7 of their (small) rms contribution.
constexpr int kLowK = 32;

// Shaped spectral value F[ky][kx] = sqrt(L^2 S(q)) (g_re + i g_im) / sqrt(2).
SCINT_DEV double2 spectrum_bin(const SynthArgs& a, int kx, int ky) {
    const u32x4 w = philox4x32_10(u32x4{(uint32_t)kx, (uint32_t)ky, a.screen_id, 0u}, a.key0, a.key1);
    const int mx = signed_freq(kx, a.n), my = signed_freq(ky, a.n);
    const int m2 = mx * mx + my * my;
    if (m2 == 0) return make_double2(0.0, 0.0);
    if (abs(mx) <= kLowK && abs(my) <= kLowK) {
        const double ua = uniform53(w.y, w.x);
        const double ub = uniform53(w.w, w.z);
        const double r = sqrt(-2.0 * log(ua));
        double sn, cs;
        sincospi(2.0 * ub, &sn, &cs);
        const double sig = a.amp * pow((double)m2, a.neg_beta_4);
        return make_double2(sig * r * cs, sig * r * sn);
    }
    // FP32 with the same 53-bit uniforms, u = (top 53 bits + 1/2) 2^-53, rounded
    // once to float; -ln u_a goes through log1p(-(1 - u_a)) when u_a >= 1/2 so
    // that values near 1 keep their relative accuracy (1 - u_a uses the
    // complemented bits exactly).
    float nl;
    if (w.y & 0x80000000u) {
        const float d = fmaf((float)((~w.x) >> 11), 0x1.0p-53f, (float)(~w.y) * 0x1.0p-32f) + 0x1.0p-54f;
        nl = -log1pf(-d);
    } else {
        const float ua = fmaf((float)(w.x >> 11), 0x1.0p-53f, (float)w.y * 0x1.0p-32f) + 0x1.0p-54f;
        nl = -logf(ua);
    }
    const float r = sqrtf(2.0f * nl);
    const float tb = fmaf((float)(w.z >> 11), 0x1.0p-52f, (float)w.w * 0x1.0p-31f) + 0x1.0p-53f;  // 2 u_b
    float sn, cs;
    sincospif(tb, &sn, &cs);
    const float sig = a.amp32 * powf((float)m2, a.neg_beta_4_32);
    return make_double2((double)(sig * r * cs), (double)(sig * r * sn));
}

// Lines per block (all transformed together); N = 16384 lines (256 KB in FP64)
// are split over a cluster of two blocks (fft.cuh, CS = 2).
template <int N> __host__ __device__ constexpr int synth_cs() { return N >= 16384 ? 2 : 1; }
template <int N> __host__ __device__ constexpr int synth_lines() { return N >= kTile64 ? 1 : (kTile64 / N < N ? kTile64 / N : N); }
template <int N> __host__ __device__ constexpr int synth_threads() { return synth_lines<N>() * FftPlan<N>::T / synth_cs<N>(); }
// strip width of the intermediate: at least 2 complex128 columns (whole 32-byte sectors per row)
template <int N> __host__ __device__ constexpr int synth_strip() { return synth_lines<N>() >= 2 ? synth_lines<N>() : 2; }
template <int N> constexpr size_t synth_smem() { return (size_t)synth_lines<N>() * FftPlan<N>::BUF * sizeof(double2) / synth_cs<N>(); }

template <int CS> SCINT_DEV int synth_rank() {
    if constexpr (CS == 1) return 0;
    else return (int)cooperative_groups::this_cluster().block_rank();
}

template <int N>
__global__ void __launch_bounds__(synth_threads<N>())
synth_rows_kernel(SynthArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = synth_cs<N>();
    constexpr int T = Pl::T, E = Pl::E, B = synth_lines<N>(), W = synth_strip<N>(), TL = T / CS;
    extern __shared__ double2 smem64[];
    const int team = threadIdx.x / TL;
    const int t = synth_rank<CS>() * TL + threadIdx.x % TL;
    const int ky = (blockIdx.x / CS) * B + team;
    double2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = spectrum_bin(a, t + m * T, ky);
    if constexpr (CS == 2) line_sync<CS>();       // the partner block is running before its buffer is touched
    fft_line<double2, N, +1, 16, 1, 0, CS>(v, smem64 + team * (Pl::BUF / CS), t, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int x = t + m * T;
        a.work[(size_t)(x / W) * N * W + (size_t)ky * W + (x % W)] = v[m];
    }
    if constexpr (CS == 2) line_sync<CS>();
}

template <int N>
__global__ void __launch_bounds__(synth_threads<N>())
synth_cols_kernel(SynthArgs a) {
    using Pl = FftPlan<N>;
    constexpr int CS = synth_cs<N>();
    constexpr int T = Pl::T, E = Pl::E, W = synth_lines<N>(), WL = synth_strip<N>(), TL = T / CS;
    extern __shared__ double2 smem64[];
    const int w = threadIdx.x % W;
    const int t = synth_rank<CS>() * TL + threadIdx.x / W;
    const int x0 = (blockIdx.x / CS) * W;
    const int x = x0 + w;
    const double2* src = a.work + (size_t)(x0 / WL) * N * WL + (x0 % WL);
    double2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = src[(size_t)(t + m * T) * WL + w];
    if constexpr (CS == 2) line_sync<CS>();
    fft_line<double2, N, +1, 16, W, 0, CS>(v, smem64 + w, t, a.tw);     // W lines interleaved
#pragma unroll
    for (int m = 0; m < E; ++m) a.phi[(size_t)(t + m * T) * N + x] = a.out_scale * v[m].x;
    if constexpr (CS == 2) line_sync<CS>();
}

template <bool ROWS>
cudaError_t launch_synth_pass(const SynthArgs& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (synth_smem<N>() > 227 * 1024) {
            return cudaErrorNotSupported;
        } else {
            auto k = ROWS ? synth_rows_kernel<N> : synth_cols_kernel<N>;
            cudaError_t e = set_smem(k, synth_smem<N>());
            if (e != cudaSuccess) return e;
            return launch_k(k, synth_cs<N>(), dim3(N / synth_lines<N>() * synth_cs<N>()), dim3(synth_threads<N>()),
                            synth_smem<N>(), s, a);
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
