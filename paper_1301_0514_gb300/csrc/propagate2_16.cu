// Packed transfer-function passes with 16 values per thread (kernels in propagate2.cuh).
#include "propagate2.cuh"

namespace scint {

template <int TWM>
static bool fits_16(int n, bool rows) {
    bool ok = false;
    dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        ok = rows ? rows2_fits<N, TWM, 16>() : cols2_fits<N, TWM, 16>();
        return cudaSuccess;
    });
    return ok;
}

static bool supported_16(int n, int row_twm, int col_twm) {
    if ((row_twm != 1 && row_twm != 2) || (col_twm != 1 && col_twm != 2)) return false;
    return (row_twm == 1 ? fits_16<1>(n, true) : fits_16<2>(n, true)) &&
           (col_twm == 1 ? fits_16<1>(n, false) : fits_16<2>(n, false));
}

static cudaError_t rows_16(const PropArgs& a, int twm, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        return twm == 1 ? rows2_at<N, 1, 16>(a, s) : rows2_at<N, 2, 16>(a, s);
    });
}

static cudaError_t cols_16(const PropArgs& a, int twm, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        return twm == 1 ? cols2_at<N, 1, 16>(a, s) : cols2_at<N, 2, 16>(a, s);
    });
}

// the entry points of kernels.cuh: 16 values per thread here, 8 in propagate2_8.cu
bool packed_prop_supported(int n, int points, int row_twm, int col_twm) {
    if (points == 8) return packed_prop_supported_p8(n, row_twm, col_twm);
    return points == 16 && supported_16(n, row_twm, col_twm);
}

cudaError_t launch_prop_rows2(const PropArgs& a, int points, int twm, cudaStream_t s) {
    return points == 8 ? launch_prop_rows2_p8(a, twm, s) : rows_16(a, twm, s);
}

cudaError_t launch_prop_cols2(const PropArgs& a, int points, int twm, cudaStream_t s) {
    return points == 8 ? launch_prop_cols2_p8(a, twm, s) : cols_16(a, twm, s);
}

}  // namespace scint
