// Packed transfer-function passes with 8 values per thread (kernels in propagate2.cuh).
#include "propagate2.cuh"

namespace scint {

template <int TWM>
static bool fits_8(int n, bool rows) {
    bool ok = false;
    dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        ok = rows ? rows2_fits<N, TWM, 8>() : cols2_fits<N, TWM, 8>();
        return cudaSuccess;
    });
    return ok;
}

static bool supported_8(int n, int row_twm, int col_twm) {
    if ((row_twm != 1 && row_twm != 2) || (col_twm != 1 && col_twm != 2)) return false;
    return (row_twm == 1 ? fits_8<1>(n, true) : fits_8<2>(n, true)) &&
           (col_twm == 1 ? fits_8<1>(n, false) : fits_8<2>(n, false));
}

static cudaError_t rows_8(const PropArgs& a, int twm, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        return twm == 1 ? rows2_at<N, 1, 8>(a, s) : rows2_at<N, 2, 8>(a, s);
    });
}

static cudaError_t cols_8(const PropArgs& a, int twm, cudaStream_t s) {
    return dispatch_n(a.n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        return twm == 1 ? cols2_at<N, 1, 8>(a, s) : cols2_at<N, 2, 8>(a, s);
    });
}

bool packed_prop_supported_p8(int n, int row_twm, int col_twm) { return supported_8(n, row_twm, col_twm); }
cudaError_t launch_prop_rows2_p8(const PropArgs& a, int twm, cudaStream_t s) { return rows_8(a, twm, s); }
cudaError_t launch_prop_cols2_p8(const PropArgs& a, int twm, cudaStream_t s) { return cols_8(a, twm, s); }

}  // namespace scint
