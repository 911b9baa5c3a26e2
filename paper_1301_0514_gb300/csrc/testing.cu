// Standalone line FFTs for the inspection entry points (same device code as the
// propagation and synthesis passes).
#include <algorithm>

#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "propagate.cuh"

namespace scint {

template <typename C> __host__ __device__ constexpr int lines_tile() { return sizeof(C) == 8 ? kTileRow32 : kTile64; }
template <int N> __host__ __device__ constexpr int tl_cs() { return N >= 16384 ? 2 : 1; }

template <typename C, int N>
__host__ __device__ constexpr int tl_lines() {
    return N >= lines_tile<C>() ? 1 : (lines_tile<C>() / N < N ? lines_tile<C>() / N : N);
}

template <typename C, int N, int DIR>
__global__ void __launch_bounds__(tl_lines<C, N>() * FftPlan<N>::T / tl_cs<N>())
fft_lines_kernel(C* data, int n_lines, const C* tw) {
    using Pl = FftPlan<N>;
    constexpr int CS = tl_cs<N>();
    constexpr int T = Pl::T, E = Pl::E, B = tl_lines<C, N>(), TL = T / CS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int team = threadIdx.x / TL;
    int rank = 0;
    if constexpr (CS == 2) rank = (int)cooperative_groups::this_cluster().block_rank();
    const int t = rank * TL + threadIdx.x % TL;
    const int line = (blockIdx.x / CS) * B + team;
    const bool live = line < n_lines;
    C* p = data + (size_t)(live ? line : 0) * N;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = live ? p[t + m * T] : make_c<C>(0, 0);
    if constexpr (CS == 2) line_sync<CS>();
    fft_line<C, N, DIR, 16, 1, 0, CS>(v, smem + team * (Pl::BUF / CS), t, tw);
    if (live) {
#pragma unroll
        for (int m = 0; m < E; ++m) p[t + m * T] = v[m];
    }
    if constexpr (CS == 2) line_sync<CS>();
}

template <typename C>
cudaError_t launch_fft_lines(int n, int dir, C* data, int n_lines, const C* tw, cudaStream_t s) {
    return dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        constexpr int B = tl_lines<C, N>(), CS = tl_cs<N>();
        constexpr size_t smem = (size_t)B * FftPlan<N>::BUF * sizeof(C) / CS;
        if constexpr (smem > 200 * 1024) {
            return cudaErrorNotSupported;
        } else {
            const dim3 grid((n_lines + B - 1) / B * CS), block(B * FftPlan<N>::T / CS);
            cudaError_t e;
            if (dir < 0) {
                if ((e = set_smem(fft_lines_kernel<C, N, -1>, smem)) != cudaSuccess) return e;
                return launch_k(fft_lines_kernel<C, N, -1>, CS, grid, block, smem, s, data, n_lines, tw);
            } else {
                if ((e = set_smem(fft_lines_kernel<C, N, +1>, smem)) != cudaSuccess) return e;
                return launch_k(fft_lines_kernel<C, N, +1>, CS, grid, block, smem, s, data, n_lines, tw);
            }
        }
    });
}

cudaError_t launch_fft_lines32(int n, int dir, float2* data, int n_lines, const float2* tw, cudaStream_t s) {
    return launch_fft_lines<float2>(n, dir, data, n_lines, tw, s);
}
cudaError_t launch_fft_lines64(int n, int dir, double2* data, int n_lines, const double2* tw, cudaStream_t s) {
    return launch_fft_lines<double2>(n, dir, data, n_lines, tw, s);
}

__global__ void phase_fixed_kernel(const double* phi, long long* P, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        P[i] = phase_fixed(phi[i]);
}
cudaError_t launch_phase_fixed(const double* phi, long long* P, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    phase_fixed_kernel<<<(unsigned)blocks, 256, 0, s>>>(phi, P, n);
    return cudaGetLastError();
}

}  // namespace scint
