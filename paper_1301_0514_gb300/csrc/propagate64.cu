// Fresnel propagation of one screen at one wavelength entirely in FP64 (the paper's
// plain method, Eq. hxy, with the edge taper of Sect. 3.2.1): the reference-precision
// form of the FP32 passes in propagate.cu, for grids up to 4096^2.
//
// Row pass:    A_in = SF(x) SF(y) exp(i phi s) (FP64 sine and cosine of phi s), FFT_x,
//              times H_x(kx)/N, IFFT_x -> field (complex128, row-major).
// Column pass: field column -> FFT_y -> H_y(ky)/N -> IFFT_y -> |A|^2 (FP64 map).
// H(k) = exp(-i pi lambda z k^2) with k = m/L: the phase in turns is c m^2 with
// c = lambda z / (2 L^2); c is split as c_hi + c_lo with c_hi holding 31 significant
// bits, so that c_hi m^2 is exact in FP64 for |m| <= 2048 and its fractional part
// carries no rounding; c_lo m^2 adds the rest.
#include <cmath>

#include "dispatch.cuh"
#include "fft.cuh"
#include "kernels.cuh"

namespace scint {

// taper at pixel centre i + 1/2 (raised sine over the margin, 1 inside), FP64
SCINT_DEV double taper64(int i, int n, double margin_px) {
    if (margin_px <= 0.0) return 1.0;
    const double u = fmin((double)i + 0.5, (double)n - (double)i - 0.5);
    if (u > margin_px) return 1.0;
    const double sn = sinpi(u / (2.0 * margin_px));
    return sn * sn;
}

// H(m)/n for the signed frequency index m: exp(-2 pi i frac(c m^2)) / n
SCINT_DEV double2 transfer64(const Prop64Args& a, int i) {
    const int n = a.n;
    const long long m = i < n / 2 ? i : i - n;
    const double m2 = (double)(m * m);
    const double hi = a.c_hi * m2;                  // exact: 31 + 22 bits
    double turns = (hi - floor(hi)) + a.c_lo * m2;
    turns -= floor(turns);
    double sn, cs;
    sincospi(-2.0 * turns, &sn, &cs);
    return make_double2(cs / n, sn / n);
}

template <int N> __host__ __device__ constexpr size_t p64_smem() { return (size_t)FftPlan<N>::BUF * sizeof(double2); }
// values per thread: 8 up to N = 1024, so that a line has N/8 threads (at 256^2 sixteen values
// per thread left less than one warp per SM on the FP64 pipe's latency)
template <int N> __host__ __device__ constexpr int p64_ept() { return N <= 1024 ? 8 : 16; }

template <int N>
__global__ void __launch_bounds__(FftPlan<N, p64_ept<N>()>::T) prop64_rows_kernel(Prop64Args a) {
    constexpr int EPT = p64_ept<N>();
    using Pl = FftPlan<N, EPT>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ double2 smem64[];
    const int y = blockIdx.x, t = threadIdx.x;
    const double sfy = taper64(y, N, a.margin_px);
    double2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int x = t + m * T;
        double sn, cs;
        sincos(a.phi[(size_t)y * N + x] * a.scale, &sn, &cs);
        const double w = sfy * taper64(x, N, a.margin_px);
        v[m] = make_double2(w * cs, w * sn);
    }
    fft_line<double2, N, -1, EPT, 1, 0>(v, smem64, t, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer64(a, t + m * T));
    fft_line<double2, N, +1, EPT, 1, 0>(v, smem64, t, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) a.field[(size_t)y * N + t + m * T] = v[m];
}

template <int N>
__global__ void __launch_bounds__(FftPlan<N, p64_ept<N>()>::T) prop64_cols_kernel(Prop64Args a) {
    constexpr int EPT = p64_ept<N>();
    using Pl = FftPlan<N, EPT>;
    constexpr int T = Pl::T, E = Pl::E;
    extern __shared__ double2 smem64[];
    const int x = blockIdx.x, t = threadIdx.x;
    double2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = a.field[(size_t)(t + m * T) * N + x];
    fft_line<double2, N, -1, EPT, 1, 0>(v, smem64, t, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer64(a, t + m * T));
    fft_line<double2, N, +1, EPT, 1, 0>(v, smem64, t, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) a.intensity[(size_t)(t + m * T) * N + x] = v[m].x * v[m].x + v[m].y * v[m].y;
}

cudaError_t launch_prop64(const Prop64Args& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (N > kMax64N) {
            return cudaErrorNotSupported;
        } else {
            cudaError_t e = set_smem(prop64_rows_kernel<N>, p64_smem<N>());
            if (e == cudaSuccess) e = set_smem(prop64_cols_kernel<N>, p64_smem<N>());
            if (e != cudaSuccess) return e;
            constexpr int T = FftPlan<N, p64_ept<N>()>::T;
            prop64_rows_kernel<N><<<N, T, p64_smem<N>(), s>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            prop64_cols_kernel<N><<<N, T, p64_smem<N>(), s>>>(a);
            return cudaGetLastError();
        }
    });
}

}  // namespace scint
