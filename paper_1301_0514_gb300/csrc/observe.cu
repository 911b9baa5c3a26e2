// Light curves (Sect. 3.3) and the modulation index m = sigma_I / mean(I) (Sect. 4).
#include "kernels.cuh"

namespace scint {

// One thread per sample: bilinear interpolation with periodic wrap; positions
// in FP64 so that the fractional offsets stay exact on large grids.
__global__ void lightcurve_kernel(CurveArgs a) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (s >= a.n_samples || c >= a.n_tracks) return;
    const Track tr = a.tr[c];
    const double d = (double)s * tr.ds;
    const double x = fma(d, tr.c, tr.x0);
    const double y = fma(d, tr.s, tr.y0);
    const double fx = floor(x), fy = floor(y);
    const float tx = (float)(x - fx), ty = (float)(y - fy);
    const int n = a.n;
    long long ix = (long long)fx % n, iy = (long long)fy % n;
    if (ix < 0) ix += n;
    if (iy < 0) iy += n;
    const int ix1 = (int)(ix + 1 == n ? 0 : ix + 1), iy1 = (int)(iy + 1 == n ? 0 : iy + 1);
    const float* I = a.intensity;
    const float i00 = __ldg(I + iy * n + ix), i01 = __ldg(I + iy * n + ix1);
    const float i10 = __ldg(I + (size_t)iy1 * n + ix), i11 = __ldg(I + (size_t)iy1 * n + ix1);
    const float top = fmaf(tx, i01 - i00, i00);
    const float bot = fmaf(tx, i11 - i10, i10);
    a.curves[(size_t)c * a.n_samples + s] = fmaf(ty, bot - top, top);
}

cudaError_t launch_lightcurve(const CurveArgs& a, cudaStream_t s) {
    if (a.n_tracks <= 0 || a.n_samples <= 0) return cudaSuccess;
    dim3 grid((a.n_samples + 255) / 256, a.n_tracks);
    lightcurve_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// block-wide FP64 sum of two values (blockDim.x == 256)
__device__ void block_sum2(double& a, double& b) {
    __shared__ double sa[8], sb[8];
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        a = l < 8 ? sa[l] : 0.0;
        b = l < 8 ? sb[l] : 0.0;
        for (int o = 4; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

// Pass 1: block b sums rows r0 + b, r0 + b + gridDim.x, ...; each thread a
// strided share of a row's columns.  The sums are of d = v - v0 and d^2, with v0
// the region's first pixel: shifted by a value inside the data, they cancel
// little when the variance is formed, so a thread may add one row's share in
// FP32 (a few dozen values) and fold it into its FP64 sums once per row; the
// FP64 pipe then sees two additions per row share instead of per pixel.
__global__ void __launch_bounds__(256) map_moments_kernel(const float* map, int n, int r0, int r1,
                                                          int c0, int c1, double* partial) {
    const float v0 = __ldg(map + (size_t)r0 * n + c0);
    double s = 0.0, s2 = 0.0;
    for (int r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const float* row = map + (size_t)r * n;
        // four independent loads in flight per iteration (one would leave the pass latency-bound)
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, a2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int c = c0 + threadIdx.x;
        for (; c + 3 * (int)blockDim.x < c1; c += 4 * blockDim.x) {
            float d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = __ldg(row + c + k * blockDim.x) - v0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] += d[k];
                a2[k] = fmaf(d[k], d[k], a2[k]);
            }
        }
        for (; c < c1; c += blockDim.x) {
            const float d = __ldg(row + c) - v0;
            a[0] += d;
            a2[0] = fmaf(d, d, a2[0]);
        }
        s += (double)((a[0] + a[1]) + (a[2] + a[3]));
        s2 += (double)((a2[0] + a2[1]) + (a2[2] + a2[3]));
    }
    block_sum2(s, s2);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s;
        partial[2 * blockIdx.x + 1] = s2;
    }
}

// Pass 2: one block reduces the partial sums (fixed order: deterministic).
__global__ void __launch_bounds__(256) moments_final_kernel(const double* partial, int nblocks,
                                                            double count, const float* v0p, double* out) {
    double s = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        s += partial[2 * i];
        s2 += partial[2 * i + 1];
    }
    block_sum2(s, s2);
    if (threadIdx.x == 0) {
        const double md = s / count;                        // mean of d = v - v0
        const double var = fmax(s2 / count - md * md, 0.0);
        const double sd = sqrt(var);
        const double mean = (double)*v0p + md;
        out[0] = sd / mean;
        out[1] = mean;
        out[2] = sd;
        out[3] = count;
    }
}

cudaError_t launch_map_moments(const float* map, int n, int r0, int r1, int c0, int c1,
                               double* partial, double* out, cudaStream_t s) {
    map_moments_kernel<<<kMomentBlocks, 256, 0, s>>>(map, n, r0, r1, c0, c1, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_final_kernel<<<1, 256, 0, s>>>(partial, kMomentBlocks, (double)(r1 - r0) * (c1 - c0),
                                           map + (size_t)r0 * n + c0, out);
    return cudaGetLastError();
}

// One block per curve.
__global__ void __launch_bounds__(256) curve_moments_kernel(const float* curves, int n_samples,
                                                            double* out) {
    const float* c = curves + (size_t)blockIdx.x * n_samples;
    double s = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < n_samples; i += blockDim.x) {
        const double v = (double)c[i];
        s += v;
        s2 = fma(v, v, s2);
    }
    block_sum2(s, s2);
    if (threadIdx.x == 0) {
        const double mean = s / n_samples;
        const double sd = sqrt(fmax(s2 / n_samples - mean * mean, 0.0));
        out[3 * blockIdx.x] = sd / mean;
        out[3 * blockIdx.x + 1] = mean;
        out[3 * blockIdx.x + 2] = sd;
    }
}

cudaError_t launch_curve_moments(const float* curves, int n_curves, int n_samples, double* out,
                                 cudaStream_t s) {
    if (n_curves <= 0) return cudaSuccess;
    curve_moments_kernel<<<n_curves, 256, 0, s>>>(curves, n_samples, out);
    return cudaGetLastError();
}

}  // namespace scint
