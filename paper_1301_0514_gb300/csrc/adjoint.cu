// Reverse-mode gradient of a light-curve misfit with respect to the phase
// screen: the adjoint of  phi -> A_in = SF exp(i s phi) -> A_out = P A_in ->
// I = sum_l w_l |A_out|^2 -> (disk filter) -> bilinear light curves.
//
// Given g_c = dL/dcurves:
//   g_I      = B^T g_c                   (bilinear scatter, this file)
//   g_I     <- K g_I                     (disk filter is real and even: self-adjoint; smooth.cu)
//   G_out    = 2 w_l g_I A_out           (complex gradient of |A|^2)
//   G_in     = P^H G_out = IDFT(DFT(G_out) conj(H))
//   g_phi   += s_l Im(conj(A_in) G_in)
// P = P_y P_x is separable, so P^H = P_x^H P_y^H.  Per wavelength group:
//   forward row pass (propagate.cu) -> field F in the strip layout;
//   adjoint column pass: FFT_y H_y IFFT_y -> A_out; G_out; FFT_y conj(H_y)
//                        IFFT_y, written back over F;
//   adjoint row pass:    FFT_x conj(H_x) IFFT_x -> G_in; A_in recomputed from
//                        the fixed-point phase; g_phi accumulated over the group.
// The forward fields are recomputed, never stored.
#include <algorithm>

#include "dispatch.cuh"
#include "propagate.cuh"

namespace scint {

// ---- bilinear scatter (transpose of lightcurve_kernel) ---------------------------
__global__ void lightcurve_adjoint_kernel(CurveAdjArgs a) {
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
    const float g = a.grad_curves[(size_t)c * a.n_samples + s];
    atomicAdd(a.grad_map + iy * n + ix, g * (1.0f - tx) * (1.0f - ty));
    atomicAdd(a.grad_map + iy * n + ix1, g * tx * (1.0f - ty));
    atomicAdd(a.grad_map + (size_t)iy1 * n + ix, g * (1.0f - tx) * ty);
    atomicAdd(a.grad_map + (size_t)iy1 * n + ix1, g * tx * ty);
}

cudaError_t launch_lightcurve_adjoint(const CurveAdjArgs& a, cudaStream_t s) {
    if (a.n_tracks <= 0 || a.n_samples <= 0) return cudaSuccess;
    dim3 grid((a.n_samples + 255) / 256, a.n_tracks);
    lightcurve_adjoint_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---- adjoint column pass ----------------------------------------------------------
// buffers, the g_I columns (in place of the accumulator) and the twiddle table
template <int N> constexpr size_t acol_smem() {
    return (size_t)pcol_lines<N>() * FftPlan<N, kColEPT>::BUF * sizeof(float2) + (size_t)FftPlan<N>::TWS * sizeof(float2);
}

template <int N>
__global__ void __launch_bounds__(pcol_threads<N>(), (pcol_threads<N>() <= 256 ? 2 : 1))
adj_cols_kernel(AdjArgs a) {
    using Pl = FftPlan<N, kColEPT>;
    constexpr int TWM = 1;   // the shared twiddle table
    constexpr int T = Pl::T, E = Pl::E, W = pcol_lines<N>(), WL = pstrip<N>(), BUFL = Pl::BUF;
    extern __shared__ float2 smem32[];
    const int w = threadIdx.x % W, t = threadIdx.x / W;
    const int x0 = blockIdx.x * W;
    const int x = x0 + w;
    float2* buf = smem32 + w;
    float gi[E];                                  // g_I of this column (own entries), in registers
    float2* tws = smem32 + W * BUFL;
    const float2* twp = TWM == 1 ? tws : a.tw;
    if constexpr (TWM == 1) fill_twiddle_table<float2, N>(tws, a.tw, threadIdx.x, blockDim.x);
#pragma unroll
    for (int m = 0; m < E; ++m) gi[m] = a.grad_map[(size_t)(t + m * T) * N + x];
    __syncthreads();
#pragma unroll 1
    for (int l = 0; l < a.lam.count; ++l) {
        float2* f = a.work + (size_t)l * N * N + (size_t)(x0 / WL) * N * WL + (x0 % WL);
        const unsigned long long hc = a.lam.h_fx[l];    // H_y from its fixed-point phase
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = f[(size_t)(t + m * T) * WL + w];
        fft_line<float2, N, -1, kColEPT, W, TWM>(v, buf, t, twp);
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer_at(hc, t + m * T, N));
        fft_line<float2, N, +1, kColEPT, W, TWM>(v, buf, t, twp);          // A_out of this column
        const float c2w = 2.0f * a.lam.weight[l];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = v[m] * (c2w * gi[m]);          // G_out
        fft_line<float2, N, -1, kColEPT, W, TWM>(v, buf, t, twp);
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cmulc(v[m], transfer_at(hc, t + m * T, N));
        fft_line<float2, N, +1, kColEPT, W, TWM>(v, buf, t, twp);          // P_y^H G_out
#pragma unroll
        for (int m = 0; m < E; ++m) f[(size_t)(t + m * T) * WL + w] = v[m];
    }
}

// ---- adjoint row pass --------------------------------------------------------------
// buffers and fixed-point phases (the g_phi sums and the twiddle bases live in registers)
template <int N> constexpr size_t arow_smem() {
    return (size_t)prow_lines<N>() * (FftPlan<N>::BUF * sizeof(float2) + N * sizeof(long long));
}

template <int N>
__global__ void __launch_bounds__(prow_threads<N>(), (prow_threads<N>() <= 256 ? 2 : 1))
adj_rows_kernel(AdjArgs a) {
    using Pl = FftPlan<N>;
    constexpr int T = Pl::T, E = Pl::E, B = prow_lines<N>(), WL = pstrip<N>(), BUFL = Pl::BUF;
    extern __shared__ float2 smem32[];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int y = blockIdx.x * B + team;
    float2* buf = smem32 + team * BUFL;
    long long* P = reinterpret_cast<long long*>(smem32 + B * BUFL) + team * N + t;
    float acc[E];                                 // g_phi of this row (own entries)
    TwiddleRegs<float2, N, 16> tr;
    tr.load(a.tw, t);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        P[m * T] = phase_fixed(a.phi[(size_t)y * N + t + m * T]);
        acc[m] = 0.0f;
    }
    __syncthreads();
#pragma unroll 1
    for (int l = 0; l < a.lam.count; ++l) {
        const float2* f = a.work + (size_t)l * N * N;
        const unsigned long long hc = a.lam.h_fx[l];    // H_x from its fixed-point phase
        const float* sf = a.sf + (size_t)l * N;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = f[strip_index<WL>(y, t + m * T, N)];
        fft_line_tr<float2, N, -1, 16, 1>(v, buf, t, tr);
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cmulc(v[m], transfer_at(hc, t + m * T, N));
        fft_line_tr<float2, N, +1, 16, 1>(v, buf, t, tr);   // G_in of this row
        const unsigned long long S = a.lam.scale_fx[l];
        const float s_l = a.lam.scale[l], sfy = sf[y];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const float2 A = unit_phasor(P[m * T], S) * (sfy * __ldg(sf + t + m * T));
            // s Im(conj(A_in) G_in)
            acc[m] = fmaf(s_l, A.x * v[m].y - A.y * v[m].x, acc[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
        double* o = a.grad_phi + (size_t)y * N + t + m * T;
        *o = a.accumulate ? *o + (double)acc[m] : (double)acc[m];
    }
}

// ---- N = 16384: the adjoint passes on the radix-2 cluster split --------------------
// Block r of a cluster transforms the parity-r half of every line as a whole 8192-point
// line in its own shared memory (fft.cuh: split_dif, split_combine), as the forward
// passes do.  The column pass chains two transform pairs per wavelength: after the first
// (A_out) each block holds G_out at its quarter of the outputs, n and n + N/2, i.e. both
// halves of the decimation-in-frequency pairs for those n; it keeps its parity's a_n or
// b_n and hands the other to its partner through shared memory.  Grids are persistent.
template <int N> __host__ __device__ constexpr int asplit_threads() { return FftPlan<N / 2>::T; }
template <int N> constexpr size_t asplit_col_smem() {
    return (size_t)(FftPlan<N / 2>::BUF + FftPlan<N / 2>::TWS) * sizeof(float2);
}
template <int N> constexpr size_t asplit_row_smem() {
    return (size_t)FftPlan<N / 2>::BUF * sizeof(float2) + (size_t)N * sizeof(long long);
}

template <int N>
__global__ void __launch_bounds__(asplit_threads<N>(), 1) adj_cols_split_kernel(AdjArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E, WL = pstrip<N>();
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    float2* tws = smem32 + Pl::BUF;
    fill_twiddle_table<float2, H2>(tws, a.tw, t, T, 2);
    cluster_arrive();    // the first wait also publishes the twiddle table to the block
#pragma unroll 1
    for (int x = blockIdx.x / 2; x < N; x += gridDim.x / 2) {
        float gi[E];     // g_I at this block's outputs: n (2j) and n + N/2 (2j + 1), n = t + (j + r E/2) T
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
            const int n = t + (j + r * (E / 2)) * T;
            gi[2 * j] = a.grad_map[(size_t)n * N + x];
            gi[2 * j + 1] = a.grad_map[(size_t)(n + H2) * N + x];
        }
#pragma unroll 1
        for (int l = 0; l < a.lam.count; ++l) {
            float2* f = a.work + (size_t)l * N * N + (size_t)(x / WL) * N * WL + (x % WL);
            const unsigned long long hc = a.lam.h_fx[l];    // H_y from its fixed-point phase
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int e = t + m * T;
                v[m] = split_dif(f[(size_t)e * WL], f[(size_t)(e + H2) * WL], r, e, a.tw);
            }
            cluster_wait();
            fft_line<float2, H2, -1, 16, 1, 1, 1>(v, buf, t, tws);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmul(v[m], transfer_at(hc, 2 * (t + m * T) + r, N));
            fft_line<float2, H2, +1, 16, 1, 1, 1>(v, buf, t, tws);
            const float c2w = 2.0f * a.lam.weight[l];
            float2 gq[E];                                    // G_out at n and n + N/2
            split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int j, int, float2 y0, float2 y1) {
                gq[2 * j] = y0 * (c2w * gi[2 * j]);
                gq[2 * j + 1] = y1 * (c2w * gi[2 * j + 1]);
            });
            // decimation in frequency of G_out: keep this block's parity, hand over the other
            cluster_wait();                                  // the partner has read this block's buffer
#pragma unroll
            for (int j = 0; j < E / 2; ++j) {
                const int e = t + (j + r * (E / 2)) * T;
                const float2 own = split_dif(gq[2 * j], gq[2 * j + 1], r, e, a.tw);
                buf[pad16(e)] = split_dif(gq[2 * j], gq[2 * j + 1], r ^ 1, e, a.tw);
                if (r == 0) v[j] = own;
                else v[j + E / 2] = own;
            }
            line_sync<2>();
            const unsigned pb = cluster_addr(buf, (unsigned)(r ^ 1)) +
                                (unsigned)(pad16(t + (r ^ 1) * (E / 2) * T) * sizeof(float2));
#pragma unroll
            for (int j = 0; j < E / 2; ++j) {
                const float2 q = ld_cluster<float2>(pb + (unsigned)(j * (T + T / 16) * sizeof(float2)));
                if (r == 0) v[j + E / 2] = q;
                else v[j] = q;
            }
            line_sync<2>();                                  // the partner is done with this block's buffer
            fft_line<float2, H2, -1, 16, 1, 1, 1>(v, buf, t, tws);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmulc(v[m], transfer_at(hc, 2 * (t + m * T) + r, N));
            fft_line<float2, H2, +1, 16, 1, 1, 1>(v, buf, t, tws);
            // P_y^H G_out over the field (the partner read this column before its first exchange)
            split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int, int n, float2 y0, float2 y1) {
                f[(size_t)n * WL] = y0;
                f[(size_t)(n + H2) * WL] = y1;
            });
        }
    }
    cluster_wait();
}

template <int N>
__global__ void __launch_bounds__(asplit_threads<N>(), 1) adj_rows_split_kernel(AdjArgs a) {
    constexpr int H2 = N / 2;
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E, WL = pstrip<N>();
    extern __shared__ float2 smem32[];
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int t = threadIdx.x;
    float2* buf = smem32;
    // the whole row's fixed-point phases (each thread reads back only the entries it wrote)
    long long* P = reinterpret_cast<long long*>(smem32 + Pl::BUF);
    TwiddleRegs<float2, H2, 16> tr;
    tr.load(a.tw, t, 2);
#pragma unroll 1
    for (int y = blockIdx.x / 2; y < N; y += gridDim.x / 2) {
        const double* phi = a.phi + (size_t)y * N + r * H2;
#pragma unroll
        for (int m = 0; m < E; ++m) P[r * H2 + t + m * T] = phase_fixed(phi[t + m * T]);
        line_sync<2>();
        const unsigned pp = cluster_addr(P, (unsigned)(r ^ 1)) + (unsigned)(((r ^ 1) * H2 + t) * sizeof(long long));
#pragma unroll
        for (int m = 0; m < E; ++m)
            P[(r ^ 1) * H2 + t + m * T] = ld_cluster<long long>(pp + (unsigned)(m * T * sizeof(long long)));
        cluster_arrive();
        float acc[E];    // g_phi at n (2j) and n + N/2 (2j + 1), n = t + (j + r E/2) T
#pragma unroll
        for (int m = 0; m < E; ++m) acc[m] = 0.0f;
#pragma unroll 1
        for (int l = 0; l < a.lam.count; ++l) {
            const float2* f = a.work + (size_t)l * N * N;
            const unsigned long long hc = a.lam.h_fx[l];    // H_x from its fixed-point phase
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int e = t + m * T;
                v[m] = split_dif(f[strip_index<WL>(y, e, N)], f[strip_index<WL>(y, e + H2, N)], r, e, a.tw);
            }
            cluster_wait();
            fft_line_tr<float2, H2, -1, 16, 1>(v, buf, t, tr);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cmulc(v[m], transfer_at(hc, 2 * (t + m * T) + r, N));
            fft_line_tr<float2, H2, +1, 16, 1>(v, buf, t, tr);     // G_in of this row
            const unsigned long long S = a.lam.scale_fx[l];
            const float s_l = a.lam.scale[l];
            const float* sf = a.sf + (size_t)l * N;
            const float sfy = sf[y];
            split_combine<float2, H2>(v, buf, t, r, a.tw, [&](int j, int n, float2 g0, float2 g1) {
                // s Im(conj(A_in) G_in), A_in recomputed from the fixed-point phase
                const float2 A0 = unit_phasor(P[n], S) * (sfy * __ldg(sf + n));
                const float2 A1 = unit_phasor(P[n + H2], S) * (sfy * __ldg(sf + n + H2));
                acc[2 * j] = fmaf(s_l, A0.x * g0.y - A0.y * g0.x, acc[2 * j]);
                acc[2 * j + 1] = fmaf(s_l, A1.x * g1.y - A1.y * g1.x, acc[2 * j + 1]);
            });
        }
        cluster_wait();
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
            const int n = t + (j + r * (E / 2)) * T;
            double* o0 = a.grad_phi + (size_t)y * N + n;
            double* o1 = o0 + H2;
            *o0 = a.accumulate ? *o0 + (double)acc[2 * j] : (double)acc[2 * j];
            *o1 = a.accumulate ? *o1 + (double)acc[2 * j + 1] : (double)acc[2 * j + 1];
        }
    }
}

cudaError_t launch_adj_cols(const AdjArgs& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (pcs<N>() == 2) {
            static_assert(asplit_col_smem<N>() <= kMaxSmem, "split adjoint pass does not fit");
            cudaError_t e = set_smem(adj_cols_split_kernel<N>, asplit_col_smem<N>());
            int nc = 0;
            if (e == cudaSuccess)
                e = active_clusters(adj_cols_split_kernel<N>, 2, asplit_threads<N>(), asplit_col_smem<N>(), &nc);
            if (e != cudaSuccess) return e;
            return launch_k(adj_cols_split_kernel<N>, 2, dim3(2 * std::min(nc, N)), dim3(asplit_threads<N>()),
                            asplit_col_smem<N>(), s, a);
        } else if constexpr (acol_smem<N>() > kMaxSmem || arow_smem<N>() > kMaxSmem) {
            return cudaErrorNotSupported;
        } else {
            cudaError_t e = set_smem(adj_cols_kernel<N>, acol_smem<N>());
            if (e != cudaSuccess) return e;
            adj_cols_kernel<N><<<N / pcol_lines<N>(), pcol_threads<N>(), acol_smem<N>(), s>>>(a);
            return cudaGetLastError();
        }
    });
}

cudaError_t launch_adj_rows(const AdjArgs& a, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (pcs<N>() == 2) {
            static_assert(asplit_row_smem<N>() <= kMaxSmem, "split adjoint pass does not fit");
            cudaError_t e = set_smem(adj_rows_split_kernel<N>, asplit_row_smem<N>());
            int nc = 0;
            if (e == cudaSuccess)
                e = active_clusters(adj_rows_split_kernel<N>, 2, asplit_threads<N>(), asplit_row_smem<N>(), &nc);
            if (e != cudaSuccess) return e;
            return launch_k(adj_rows_split_kernel<N>, 2, dim3(2 * std::min(nc, N)), dim3(asplit_threads<N>()),
                            asplit_row_smem<N>(), s, a);
        } else if constexpr (acol_smem<N>() > kMaxSmem || arow_smem<N>() > kMaxSmem) {
            return cudaErrorNotSupported;
        } else {
            cudaError_t e = set_smem(adj_rows_kernel<N>, arow_smem<N>());
            if (e != cudaSuccess) return e;
            adj_rows_kernel<N><<<N / prow_lines<N>(), prow_threads<N>(), arow_smem<N>(), s>>>(a);
            return cudaGetLastError();
        }
    });
}

// ---- dL/dR_diff = ((2 - beta) / (2 R_diff)) sum phi g_phi (FP64) ----------------------
// Block partials of sum a_i b_i, each thread over a fixed strided set of i with four loads
// of each array in flight (one dependent load-FMA chain per thread left the loop latency-bound).
__global__ void __launch_bounds__(256) dot_partial_kernel(const double* a, const double* b, long long n,
                                                          double* partial) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const double a0 = __ldg(a + i), a1 = __ldg(a + i + stride), a2 = __ldg(a + i + 2 * stride),
                     a3 = __ldg(a + i + 3 * stride);
        const double b0 = __ldg(b + i), b1 = __ldg(b + i + stride), b2 = __ldg(b + i + 2 * stride),
                     b3 = __ldg(b + i + 3 * stride);
        s0 = fma(a0, b0, s0);
        s1 = fma(a1, b1, s1);
        s2 = fma(a2, b2, s2);
        s3 = fma(a3, b3, s3);
    }
    for (; i < n; i += stride) s0 = fma(__ldg(a + i), __ldg(b + i), s0);
    double s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double sw[8];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sw[i];
        partial[blockIdx.x] = t;
    }
}

// fixed-order reduction of the block partials (the same bits on every run)
__global__ void __launch_bounds__(256) dot_final_kernel(const double* partial, int nb, double scale, double* out) {
    __shared__ double red[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) t += partial[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = scale * red[0];
}

cudaError_t launch_scaled_dot(const double* a, const double* b, long long n, double scale, double* partial,
                              double* out, cudaStream_t s) {
    dot_partial_kernel<<<kMomentBlocks, 256, 0, s>>>(a, b, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dot_final_kernel<<<1, 256, 0, s>>>(partial, kMomentBlocks, scale, out);
    return cudaGetLastError();
}

}  // namespace scint
