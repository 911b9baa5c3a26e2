// Transfer-function propagation passes (Eq. hxy) with two wavelengths per thread.
// Kernel templates; propagate2_16.cu and propagate2_8.cu instantiate them for 16 and 8
// values per thread (two translation units, compiled in parallel).
//
// The same two passes as in propagate.cu (row pass: phase -> taper -> FFT_x -> H_x/N ->
// IFFT_x -> field; column pass: field -> FFT_y -> H_y/N -> IFFT_y -> w |A|^2 summed over
// the group), but wavelengths 2q and 2q + 1 of a group travel together as the two lanes
// of packed values (fft2.cuh): every butterfly instruction works on both, and the
// twiddle factors, which depend on the position only, are formed once for both.  The
// row pass converts the screen phase to fixed point once per pixel and forms both
// wavelengths' phasors from it; H_x and H_y differ per wavelength and are applied lane
// by lane.
//
// The field of pair q is one N x N array of cp2 (16 bytes per pixel: re and im of both
// wavelengths), in strip layout with pstrip2 columns per strip, so the bytes per
// pixel and wavelength crossing HBM are those of the one-wavelength passes.  A group
// of odd size ends with a pair whose second lane repeats the last wavelength with
// weight 0 (its field slot is allocated; its intensity contribution is zero).
#pragma once

#include <algorithm>

#include "dispatch.cuh"
#include "fft2.cuh"
#include "propagate.cuh"

namespace scint {

template <int N> __host__ __device__ constexpr int pstrip2() { return pcol_lines<N>() >= 2 ? pcol_lines<N>() : 2; }
// EPT: values per thread, 16 (radix-16 stages, the blocks of the one-wavelength passes) or
// 8 (radix-8 stages: twice the threads per line, half the registers per thread)
template <int N, int EPT> constexpr bool packed_size() { return N >= (EPT == 8 ? 128 : 64) && N < kSplitN; }
template <int N, int EPT> __host__ __device__ constexpr int prow2_threads() {
    return prow_lines<N>() * FftPlan<N, EPT>::T;
}
template <int N, int EPT> __host__ __device__ constexpr int pcol2_threads() {
    return pcol_lines<N>() * FftPlan<N, EPT>::T;
}
// blocks per SM the register budget is set for: 8 values per thread aim at 64 registers
template <int EPT> __host__ __device__ constexpr int p2_min_blocks(int threads) {
    return EPT == 8 ? (threads <= 512 ? 2 : 1) : (threads <= 256 ? 2 : 1);
}
template <int N, int TWM, int EPT> constexpr size_t prow2_smem() {
    return (size_t)prow_lines<N>() * (FftPlan<N, EPT>::BUF * sizeof(cp2) + N * sizeof(long long)) +
           (TWM == 1 ? (size_t)FftPlan<N, EPT>::TWS * sizeof(float2) : 0);
}
template <int N, int TWM, int EPT> constexpr size_t pcol2_smem() {
    return (size_t)pcol_lines<N>() * FftPlan<N, EPT>::BUF * sizeof(cp2) +
           (TWM == 1 ? (size_t)FftPlan<N, EPT>::TWS * sizeof(float2) : 0);
}

// ---- row pass --------------------------------------------------------------------
template <int N, int TWM, int EPT>
__global__ void __launch_bounds__(prow2_threads<N, EPT>(), p2_min_blocks<EPT>(prow2_threads<N, EPT>()))
prop_rows2_kernel(PropArgs a) {
    using Pl = FftPlan<N, EPT>;
    constexpr int T = Pl::T, E = Pl::E, B = prow_lines<N>(), W = pstrip2<N>(), BUFL = Pl::BUF;
    extern __shared__ float4 smem_v4[];
    cp2* const sm = reinterpret_cast<cp2*>(smem_v4);
    const int team = threadIdx.x / T, t = threadIdx.x % T;    // line of the block, index in its team
    const int y = blockIdx.x * B + team;
    cp2* buf = sm + team * BUFL;
    // fixed-point phase of this thread's pixels (each thread reads back only its own entries)
    long long* P = reinterpret_cast<long long*>(sm + B * BUFL) + team * N + t;
    float2* tws = reinterpret_cast<float2*>(reinterpret_cast<long long*>(sm + B * BUFL) + B * N);
    const PK k = make_pk(a.one);
    TwiddleRegs<float2, N, EPT> tr;
    if constexpr (TWM == 2) tr.load(a.tw, t);
    else fill_twiddle_table<float2, N, EPT>(tws, a.tw, threadIdx.x, blockDim.x);
#pragma unroll
    for (int m = 0; m < E; ++m) P[m * T] = phase_fixed(a.phi[(size_t)y * N + t + m * T]);
    __syncthreads();
    const int nl = a.lam.count;
    cp2* const work = reinterpret_cast<cp2*>(a.work);
#pragma unroll 1
    for (int la = 0; la < nl; la += 2) {
        const int lb = la + 1 < nl ? la + 1 : la;
        const unsigned long long Sa = a.lam.scale_fx[la], Sb = a.lam.scale_fx[lb];
        const float* sfa = a.sf + (size_t)la * N;
        const float* sfb = a.sf + (size_t)lb * N;
        const float sya = sfa[y], syb = sfb[y];
        cp2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = t + m * T;
            const long long p = P[m * T];
            v[m] = pack2(unit_phasor(p, Sa) * (sya * __ldg(sfa + e)), unit_phasor(p, Sb) * (syb * __ldg(sfb + e)));
        }
        fft2_line<N, EPT, -1, 1, TWM>(v, buf, t, tws, &tr, k);
        const unsigned long long ha = a.lam.h_fx[la], hb = a.lam.h_fx[lb];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = t + m * T;
            v[m] = lanemul(v[m], pack2(transfer_at(ha, e, N), transfer_at(hb, e, N)), k);
        }
        fft2_line<N, EPT, +1, 1, TWM>(v, buf, t, tws, &tr, k);
        cp2* dst = work + (size_t)(la / 2) * N * N;
#pragma unroll
        for (int m = 0; m < E; ++m) dst[strip_index<W>(y, t + m * T, N)] = v[m];
    }
}

// ---- column pass -----------------------------------------------------------------
template <int N, int TWM, int EPT>
__global__ void __launch_bounds__(pcol2_threads<N, EPT>(), p2_min_blocks<EPT>(pcol2_threads<N, EPT>()))
prop_cols2_kernel(PropArgs a) {
    using Pl = FftPlan<N, EPT>;
    constexpr int T = Pl::T, E = Pl::E, W = pcol_lines<N>(), WL = pstrip2<N>(), BUFL = Pl::BUF;
    extern __shared__ float4 smem_v4[];
    cp2* const sm = reinterpret_cast<cp2*>(smem_v4);
    const int w = threadIdx.x % W, t = threadIdx.x / W;
    const int x0 = blockIdx.x * W;    // first column of the block: strip x0 / WL, offset x0 % WL
    const int x = x0 + w;
    cp2* buf = sm + w;                // W lines interleaved: element e of line w at pad16(e) * W + w
    float2* tws = reinterpret_cast<float2*>(sm + W * BUFL);
    const PK k = make_pk(a.one);
    TwiddleRegs<float2, N, EPT> tr;
    if constexpr (TWM == 2) tr.load(a.tw, t);
    else fill_twiddle_table<float2, N, EPT>(tws, a.tw, threadIdx.x, blockDim.x);
    float acc[E];
#pragma unroll
    for (int m = 0; m < E; ++m) acc[m] = 0.0f;
    __syncthreads();
    const int nl = a.lam.count;
    const cp2* const work = reinterpret_cast<const cp2*>(a.work);
#pragma unroll 1
    for (int la = 0; la < nl; la += 2) {
        const int lb = la + 1 < nl ? la + 1 : la;
        const cp2* src = work + (size_t)(la / 2) * N * N + (size_t)(x0 / WL) * N * WL + (x0 % WL);
        cp2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = src[(size_t)(t + m * T) * WL + w];
        fft2_line<N, EPT, -1, W, TWM>(v, buf, t, tws, &tr, k);
        const unsigned long long ha = a.lam.h_fx[la], hb = a.lam.h_fx[lb];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = t + m * T;
            v[m] = lanemul(v[m], pack2(transfer_at(ha, e, N), transfer_at(hb, e, N)), k);
        }
        fft2_line<N, EPT, +1, W, TWM>(v, buf, t, tws, &tr, k);
        const float wa = a.lam.weight[la], wb = la + 1 < nl ? a.lam.weight[lb] : 0.0f;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const float2 q = norm2(v[m]);
            acc[m] = fmaf(wb, q.y, fmaf(wa, q.x, acc[m]));
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float* o = a.intensity + (size_t)(t + m * T) * N + x;
        *o = a.accumulate ? *o + acc[m] : acc[m];
    }
}

// ---- launchers -------------------------------------------------------------------
template <int N, int TWM, int EPT> constexpr bool rows2_fits() {
    if constexpr (!packed_size<N, EPT>()) return false;
    else return prow2_smem<N, TWM, EPT>() <= kMaxSmem;
}
template <int N, int TWM, int EPT> constexpr bool cols2_fits() {
    if constexpr (!packed_size<N, EPT>()) return false;
    else return pcol2_smem<N, TWM, EPT>() <= kMaxSmem && pcol2_threads<N, EPT>() <= 1024;
}

template <int N, int TWM, int EPT>
cudaError_t rows2_at(const PropArgs& a, cudaStream_t s) {
    if constexpr (!rows2_fits<N, TWM, EPT>()) {
        return cudaErrorNotSupported;
    } else {
        constexpr size_t smem = prow2_smem<N, TWM, EPT>();
        cudaError_t e = set_smem(prop_rows2_kernel<N, TWM, EPT>, smem);
        if (e != cudaSuccess) return e;
        prop_rows2_kernel<N, TWM, EPT><<<N / prow_lines<N>(), prow2_threads<N, EPT>(), smem, s>>>(a);
        return cudaGetLastError();
    }
}

template <int N, int TWM, int EPT>
cudaError_t cols2_at(const PropArgs& a, cudaStream_t s) {
    if constexpr (!cols2_fits<N, TWM, EPT>()) {
        return cudaErrorNotSupported;
    } else {
        constexpr size_t smem = pcol2_smem<N, TWM, EPT>();
        cudaError_t e = set_smem(prop_cols2_kernel<N, TWM, EPT>, smem);
        if (e != cudaSuccess) return e;
        prop_cols2_kernel<N, TWM, EPT><<<N / pcol_lines<N>(), pcol2_threads<N, EPT>(), smem, s>>>(a);
        return cudaGetLastError();
    }
}


// per values-per-thread variant (propagate2_8.cu / propagate2_16.cu)
bool packed_prop_supported_p8(int n, int row_twm, int col_twm);
cudaError_t launch_prop_rows2_p8(const PropArgs& a, int twm, cudaStream_t s);
cudaError_t launch_prop_cols2_p8(const PropArgs& a, int twm, cudaStream_t s);

}  // namespace scint
