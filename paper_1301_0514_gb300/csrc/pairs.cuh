// Column pairs of an N x N real map held column-major: pairs[p * N + y] holds the
// values (y, 2p) and (y, 2p + 1).  The passes that transform one pair of columns per
// block (at N = 16384) read and write this form, where consecutive rows are
// consecutive 8- or 16-byte values, and these two tiled transposes convert it from
// and to the row-major map (32 pairs x 32 rows per block through shared memory, reads
// and writes both coalesced).  n is a multiple of 64.
#pragma once

#include "kernels.cuh"

namespace scint {

// out[y][2p + c] = pairs[p][y].c
template <typename P, typename S>
__global__ void __launch_bounds__(256) pairs_to_rows_kernel(const P* __restrict__ pairs, S* out, int n) {
    __shared__ P tile[32][33];
    const int p0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
    for (int k = ty; k < 32; k += 8) tile[k][tx] = pairs[(size_t)(p0 + k) * n + y0 + tx];   // [pair][y]
    __syncthreads();
#pragma unroll
    for (int k = ty; k < 32; k += 8) reinterpret_cast<P*>(out + (size_t)(y0 + k) * n)[p0 + tx] = tile[tx][k];
}

// pairs[p][y] = (in[y][2p], in[y][2p + 1])
template <typename P, typename S>
__global__ void __launch_bounds__(256) rows_to_pairs_kernel(const S* __restrict__ in, P* pairs, int n) {
    __shared__ P tile[32][33];
    const int p0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
    for (int k = ty; k < 32; k += 8) tile[k][tx] = reinterpret_cast<const P*>(in + (size_t)(y0 + k) * n)[p0 + tx];   // [y][pair]
    __syncthreads();
#pragma unroll
    for (int k = ty; k < 32; k += 8) pairs[(size_t)(p0 + k) * n + y0 + tx] = tile[tx][k];
}

template <typename P, typename S>
cudaError_t launch_pairs_to_rows(const P* pairs, S* out, int n, cudaStream_t s) {
    pairs_to_rows_kernel<P, S><<<dim3(n / 64, n / 32), 256, 0, s>>>(pairs, out, n);
    return cudaGetLastError();
}
template <typename P, typename S>
cudaError_t launch_rows_to_pairs(const S* in, P* pairs, int n, cudaStream_t s) {
    rows_to_pairs_kernel<P, S><<<dim3(n / 64, n / 32), 256, 0, s>>>(in, pairs, n);
    return cudaGetLastError();
}

}  // namespace scint
