// Standalone line FFTs for the inspection entry points (same device code as the
// propagation and synthesis passes).
#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"

namespace scint {

template <typename C> __host__ __device__ constexpr int lines_tile() { return sizeof(C) == 8 ? kTileRow32 : kTile64; }

template <typename C, int N>
__host__ __device__ constexpr int tl_lines() {
    return N >= lines_tile<C>() ? 1 : (lines_tile<C>() / N < N ? lines_tile<C>() / N : N);
}

template <typename C, int N, int DIR>
__global__ void __launch_bounds__(tl_lines<C, N>() * FftPlan<N>::T)
fft_lines_kernel(C* data, int n_lines, const C* tw) {
    using Pl = FftPlan<N>;
    constexpr int T = Pl::T, E = Pl::E, B = tl_lines<C, N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int line = blockIdx.x * B + team;
    const bool live = line < n_lines;
    C* p = data + (size_t)(live ? line : 0) * N;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = live ? p[t + m * T] : make_c<C>(0, 0);
    fft_line<C, N, DIR>(v, smem + team * Pl::BUF, t, tw);
    if (live) {
#pragma unroll
        for (int m = 0; m < E; ++m) p[t + m * T] = v[m];
    }
}

template <typename C>
cudaError_t launch_fft_lines(int n, int dir, C* data, int n_lines, const C* tw, cudaStream_t s) {
    return dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        constexpr int B = tl_lines<C, N>();
        constexpr size_t smem = (size_t)B * FftPlan<N>::BUF * sizeof(C);
        if constexpr (smem > 200 * 1024) {
            return cudaErrorNotSupported;
        } else {
            const int blocks = (n_lines + B - 1) / B;
            cudaError_t e;
            if (dir < 0) {
                if ((e = set_smem(fft_lines_kernel<C, N, -1>, smem)) != cudaSuccess) return e;
                fft_lines_kernel<C, N, -1><<<blocks, B * FftPlan<N>::T, smem, s>>>(data, n_lines, tw);
            } else {
                if ((e = set_smem(fft_lines_kernel<C, N, +1>, smem)) != cudaSuccess) return e;
                fft_lines_kernel<C, N, +1><<<blocks, B * FftPlan<N>::T, smem, s>>>(data, n_lines, tw);
            }
            return cudaGetLastError();
        }
    });
}

cudaError_t launch_fft_lines32(int n, int dir, float2* data, int n_lines, const float2* tw, cudaStream_t s) {
    return launch_fft_lines<float2>(n, dir, data, n_lines, tw, s);
}
cudaError_t launch_fft_lines64(int n, int dir, double2* data, int n_lines, const double2* tw, cudaStream_t s) {
    return launch_fft_lines<double2>(n, dir, data, n_lines, tw, s);
}

}  // namespace scint
