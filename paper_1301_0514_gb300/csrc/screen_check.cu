// Screen check of Sect. 3.1.1: the phase spectrum and structure function
// recomputed from the generated F_phi, and R_diff^rec.
//
//   S_rec(q_j) = sum_{annulus j} |F|^2 / (count_j L^2), annulus j = bins with
//                j - 1/2 <= |m| < j + 1/2 (nearest integer to |m|);
//   D_rec(r)   = 2 (xi_rec(0) - xi_rec(r)) with Eq. crec on the annuli,
//              = 4 pi dq sum_{j=1}^{J} q_j S_rec(q_j) (1 - J0(2 pi q_j r)),
//                q_j = j dq, dq = 1/L, J = min(n_bins - 1, N/2) (q_max = 1/(2 Delta));
//   R_diff^rec = root of D_rec(R) = 1, bisection on (0, L/2].
//
// The annulus sums run as one persistent pass: each block keeps a histogram of
// every annulus in shared memory, walks whole spectral rows (each thread a
// contiguous run of columns, adding into its current annulus until it changes,
// so a run of equal annuli costs one shared atomic), and adds its histogram
// into the global one at the end.  The sums are 64-bit fixed point (see
// annulus_shift), hence exact and independent of the order of the additions;
// the hot loop has no FP64 operation (GB300's FP64 pipe is narrow).  The noise is regenerated per bin
// (spectrum.cuh), never stored.  The bisection launches one kernel per step;
// within a step the blocks' partial sums are combined in block order by the
// last block to finish, so the result does not depend on scheduling.
#include <math_constants.h>

#include "dispatch.cuh"
#include "kernels.cuh"
#include "spectrum.cuh"

namespace scint {

// Nearest integer to sqrt(m2), exactly: j with j^2 - j + 1 <= m2 <= j^2 + j.
// m2 <= 2 (N/2)^2 < 2^31 for N <= 32768, so 32-bit integers suffice (64-bit
// conversions would run on the narrow FP64 pipe).
SCINT_DEV int annulus_of(int m2) {
    // any estimate within +-1 will do: the integer tests below make j exact
    const float f = (float)m2;
    int j = m2 > 0 ? __float2int_rn(f * rsqrtf(f)) : 0;
    while (j * j + j < m2) ++j;
    while (j > 0 && j * j - j + 1 > m2) --j;
    return j;
}

// Annulus sums in 64-bit fixed point.  Annulus j's values are scaled by 2^s_j
// with s_j chosen so that the expected bin power amp^2 j^-beta lands in
// [2^36, 2^37); a bin holds at most ~120 times that (the -2 ln u tail and the
// spread of |m| within an annulus) and an annulus at most ~1.5e5 bins, so a sum
// stays below 2^62.  Truncating each value to the fixed-point grid costs at
// most 2^-36 of the annulus' scale per bin.  Integer sums are exact, so the
// result does not depend on the order of the additions.
// Any shift near the target range is valid as long as the sums and the final
// normalisation use the same one, so the fast hardware log2 serves (the same
// j gives the same shift in every kernel).
SCINT_DEV int annulus_shift(const SynthArgs& a, int j) {
    const float l2 = 2.0f * __log2f(a.amp32) + 4.0f * a.neg_beta_4_32 * __log2f((float)max(j, 1));
    return 36 - (int)floorf(l2);
}
// v 2^s truncated to an integer, from the bits of a positive normal float / double
SCINT_DEV unsigned long long to_fixed(float v, int s) {
    const uint32_t b = __float_as_uint(v);
    if ((b >> 23) == 0u) return 0ull;
    const int e = (int)(b >> 23) - 150 + s;
    const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
    return e >= 0 ? m << e : (e > -24 ? m >> -e : 0ull);
}
SCINT_DEV unsigned long long to_fixed(double v, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if ((b >> 52) == 0ull) return 0ull;
    const int e = (int)(b >> 52) - 1075 + s;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return e >= 0 ? m << e : (e > -53 ? m >> -e : 0ull);
}

// COUNT: bins per annulus.  Otherwise: fixed-point sums of |F|^2 (high bins from
// their FP32 value, low bins from their FP64 value, as the synthesis draws them);
// a thread adds a run of bins of one annulus in a register and the run into the
// block's shared histogram with one atomic.
template <bool COUNT>
__global__ void __launch_bounds__(kRadialThreads)
radial_kernel(SynthArgs a, int n_hist, unsigned long long* sums, unsigned long long* counts) {
    extern __shared__ __align__(16) unsigned char radial_smem[];
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(radial_smem);
    unsigned* hc = reinterpret_cast<unsigned*>(radial_smem);
    for (int j = threadIdx.x; j < n_hist; j += blockDim.x) {
        if (COUNT) hc[j] = 0u;
        else hs[j] = 0ull;
    }
    __syncthreads();
    const int n = a.n;
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int x0 = threadIdx.x * chunk, x1 = min(n, x0 + chunk);
    for (int ky = blockIdx.x; ky < n; ky += gridDim.x) {
        const int my = signed_freq(ky, n);
        int cur = -1, shift = 0;
        unsigned long long acc = 0ull;
        unsigned cnt = 0u;
        for (int kx = x0; kx < x1; ++kx) {
            const int mx = signed_freq(kx, n);
            const int m2 = mx * mx + my * my;
            const int j = annulus_of(m2);
            if (j != cur) {
                if (cur >= 0 && cur < n_hist) {
                    if (COUNT) atomicAdd(hc + cur, cnt);
                    else atomicAdd(hs + cur, acc);
                }
                cur = j;
                acc = 0ull;
                cnt = 0u;
                if (!COUNT) shift = annulus_shift(a, j);
            }
            if (COUNT) {
                ++cnt;
            } else if (j < n_hist && m2 > 0) {
                const u32x4 w = philox4x32_10(u32x4{(uint32_t)kx, (uint32_t)ky, a.screen_id, 0u}, a.key0, a.key1);
                acc += low_bin(a, mx, my) ? to_fixed(power_low(a, w, m2), shift) : to_fixed(power_high(a, w, m2), shift);
            }
        }
        if (cur >= 0 && cur < n_hist) {
            if (COUNT) atomicAdd(hc + cur, cnt);
            else atomicAdd(hs + cur, acc);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n_hist; j += blockDim.x) {
        if (COUNT) {
            if (hc[j]) atomicAdd(counts + j, (unsigned long long)hc[j]);
        } else {
            if (hs[j]) atomicAdd(sums + j, hs[j]);
        }
    }
}

// s_rec holds the fixed-point sums on entry (as integers); S_rec = sum 2^-s_j / count / L^2
__global__ void radial_finish_kernel(SynthArgs a, int n_hist, double inv_l2, double* s,
                                     const unsigned long long* counts) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_hist) return;
    const unsigned long long fx = reinterpret_cast<const unsigned long long*>(s)[j];
    s[j] = counts[j] ? ldexp((double)fx, -annulus_shift(a, j)) / (double)counts[j] * inv_l2 : 0.0;
}

cudaError_t launch_radial_spectrum(const SynthArgs& a, double inv_l2, int n_hist, double* s_rec,
                                   unsigned long long* counts, int blocks, cudaStream_t s) {
    const size_t bytes_s = (size_t)n_hist * sizeof(unsigned long long), bytes_c = (size_t)n_hist * sizeof(unsigned);
    cudaError_t e;
    if ((e = set_smem(radial_kernel<false>, bytes_s)) != cudaSuccess) return e;
    if ((e = set_smem(radial_kernel<true>, bytes_c)) != cudaSuccess) return e;
    unsigned long long* fx = reinterpret_cast<unsigned long long*>(s_rec);
    radial_kernel<true><<<blocks, kRadialThreads, bytes_c, s>>>(a, n_hist, fx, counts);
    radial_kernel<false><<<blocks, kRadialThreads, bytes_s, s>>>(a, n_hist, fx, counts);
    radial_finish_kernel<<<(n_hist + 255) / 256, 256, 0, s>>>(a, n_hist, inv_l2, s_rec, counts);
    return cudaGetLastError();
}

// ---- Eq. crec ------------------------------------------------------------------
// sum_{j = j0 + 1, j0 + 1 + stride, ...} q_j S_j (1 - J0(2 pi q_j r)) for this thread
SCINT_DEV double crec_terms(const double* __restrict__ s, int J, double dq, double r, int first, int stride) {
    double acc = 0.0;
    for (int j = first; j <= J; j += stride) {
        const double q = j * dq;
        acc += q * s[j] * (1.0 - j0(2.0 * kPi * q * r));
    }
    return acc;
}

// block sum in a fixed order (the result is the same on every run)
SCINT_DEV double block_sum_fixed(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double t = red[0];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kCrecThreads) crec_kernel(CrecArgs a, const double* r_km, int n_r, double* d) {
    __shared__ double red[kCrecThreads];
    const int i = blockIdx.x;
    const double acc = crec_terms(a.s, a.J, a.dq, r_km[i], 1 + threadIdx.x, blockDim.x);
    const double t = block_sum_fixed(acc, red);
    if (threadIdx.x == 0) d[i] = 4.0 * kPi * a.dq * t;
}

cudaError_t launch_crec(const CrecArgs& a, const double* r_km, int n_r, double* d, cudaStream_t s) {
    crec_kernel<<<n_r, kCrecThreads, 0, s>>>(a, r_km, n_r, d);
    return cudaGetLastError();
}

// One bisection step.  Step -1 evaluates D_rec(L/2) and opens the bracket (or
// marks "no root"); step k >= 0 evaluates D_rec at the midpoint and keeps the
// half that brackets the root.  The last step writes the result.
__global__ void __launch_bounds__(kCrecThreads) bisect_kernel(CrecArgs a, BisectState* st, int step, int last,
                                                            double* out) {
    __shared__ double red[kCrecThreads];
    __shared__ bool is_last;
    if (st->no_root) {   // uniform across the grid: nothing left to do
        if (blockIdx.x == 0 && threadIdx.x == 0 && step == last) *out = CUDART_NAN;
        return;
    }
    const double r = step < 0 ? a.half_L : 0.5 * (st->lo + st->hi);
    const int stride = gridDim.x * blockDim.x;
    const double acc = crec_terms(a.s, a.J, a.dq, r, 1 + blockIdx.x * blockDim.x + threadIdx.x, stride);
    const double t = block_sum_fixed(acc, red);
    if (threadIdx.x == 0) {
        st->partial[blockIdx.x] = t;
        __threadfence();
        is_last = atomicAdd(&st->arrived, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    __threadfence();
    double tot = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) tot += *((volatile double*)&st->partial[b]);
    const double D = 4.0 * kPi * a.dq * tot;
    if (step < 0) {
        st->lo = 0.0;
        st->hi = a.half_L;
        st->no_root = D < 1.0;
    } else if (D < 1.0) {
        st->lo = r;
    } else {
        st->hi = r;
    }
    st->arrived = 0u;
    if (step == last) *out = st->no_root ? CUDART_NAN : 0.5 * (st->lo + st->hi);
}

cudaError_t launch_bisect(const CrecArgs& a, BisectState* st, int iterations, double* out, cudaStream_t s) {
    const int blocks = kBisectBlocks;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(BisectState), s);
    if (e != cudaSuccess) return e;
    for (int step = -1; step < iterations; ++step) {
        bisect_kernel<<<blocks, kCrecThreads, 0, s>>>(a, st, step, iterations - 1, out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace scint
