// Light-curve time analysis (Sect. 5): the time power spectrum of each curve,
// whose slope breaks near 1/t_ref, and the correlation of curves taken along
// parallel tracks (two telescopes a distance apart).
//
// Periodogram P_k = |sum_s (c_s - mean c) e^{-2 pi i k s / n}|^2 / n, k = 0..n/2:
// a team of n/16 threads holds one curve (16 values per thread), removes the
// curve's mean (FP64 sum) before the FP32 transform so that the rounding of
// a large mean does not leak into the weak bins, and writes |X_k|^2 / n.
// Correlation: one block per pair, mean then centred sums, FP64; pairs come in
// groups that share one row of a (a reference curve against its parallels).
#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"

namespace scint {

template <int N> __host__ __device__ constexpr int ps_lines() {
    return N >= kTileRow32 ? 1 : (kTileRow32 / N < 64 ? kTileRow32 / N : 64);
}

template <int N>
__global__ void __launch_bounds__(ps_lines<N>() * FftPlan<N>::T)
power_spectrum_kernel(const float* curves, int n_curves, float* power, const float2* tw) {
    using Pl = FftPlan<N>;
    constexpr int T = Pl::T, E = Pl::E, B = ps_lines<N>(), NW = (T + 31) / 32;
    extern __shared__ __align__(16) float2 ps_smem[];
    __shared__ double wsum[B][NW];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int c = blockIdx.x * B + team;
    const bool live = c < n_curves;
    const float* src = curves + (size_t)(live ? c : 0) * N;
    float x[E];
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        x[m] = live ? src[t + m * T] : 0.0f;
        s += x[m];
    }
    // team sum: warps of the team, then the team's warps in order
    if constexpr (T >= 32) {
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((t & 31) == 0) wsum[team][t >> 5] = s;
    } else {
        // teams smaller than a warp: T lanes of one team are contiguous in the warp
        for (int o = T / 2; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
        if (t == 0) wsum[team][0] = s;
    }
    __syncthreads();
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) tot += wsum[team][w];
    const float mean = (float)(tot / N);
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = make_float2(x[m] - mean, 0.0f);
    fft_line<float2, N, -1, 16, 1, 0, 1>(v, ps_smem + team * Pl::BUF, t, tw);
    if (live) {
        float* out = power + (size_t)c * (N / 2 + 1);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + m * T;
            if (k <= N / 2) out[k] = k == 0 ? 0.0f : fmaf(v[m].x, v[m].x, v[m].y * v[m].y) * (1.0f / N);
        }
    }
}

cudaError_t launch_power_spectrum(const float* curves, int n_curves, int n, float* power, const float2* tw,
                                  cudaStream_t s) {
    if (n_curves <= 0) return cudaSuccess;
    return dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (N > 8192) {
            return cudaErrorNotSupported;
        } else {
            constexpr int B = ps_lines<N>();
            constexpr size_t smem = (size_t)B * FftPlan<N>::BUF * sizeof(float2);
            cudaError_t e = set_smem(power_spectrum_kernel<N>, smem);
            if (e != cudaSuccess) return e;
            power_spectrum_kernel<N><<<(n_curves + B - 1) / B, B * FftPlan<N>::T, smem, s>>>(curves, n_curves,
                                                                                              power, tw);
            return cudaGetLastError();
        }
    });
}

// FP64 block sum (blockDim.x == 256), result in every thread
__device__ double block_sum_all(double v) {
    __shared__ double part[8];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) correlation_kernel(const float* a, int group, long long a_stride,
                                                          const float* b, int n, double* r) {
    const int i = blockIdx.x;
    const float* x = a + (size_t)(i / group) * a_stride;
    const float* y = b + (size_t)i * n;
    double sx = 0.0, sy = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        sx += x[s];
        sy += y[s];
    }
    const double mx = block_sum_all(sx) / n, my = block_sum_all(sy) / n;
    double sxy = 0.0, sxx = 0.0, syy = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const double dx = x[s] - mx, dy = y[s] - my;
        sxy = fma(dx, dy, sxy);
        sxx = fma(dx, dx, sxx);
        syy = fma(dy, dy, syy);
    }
    sxy = block_sum_all(sxy);
    sxx = block_sum_all(sxx);
    syy = block_sum_all(syy);
    if (threadIdx.x == 0) r[i] = sxy / sqrt(sxx * syy);
}

cudaError_t launch_correlation(const float* a, int a_rows, long long a_stride, const float* b, int n_pairs, int n,
                               double* r, cudaStream_t s) {
    if (n_pairs <= 0) return cudaSuccess;
    correlation_kernel<<<n_pairs, 256, 0, s>>>(a, n_pairs / a_rows, a_stride, b, n, r);
    return cudaGetLastError();
}

}  // namespace scint
