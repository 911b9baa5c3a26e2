// Internal launch interface between the C-ABI layer (api.cu) and the kernel
// translation units.  Every launcher enqueues on `stream` and returns the
// cudaError_t of the launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace scint {

constexpr int kMaxLambda = 128;

// Line-tile sizes (complex elements staged in shared memory per block).
constexpr int kTileRow32 = 4096;    // FP32 line passes over rows
constexpr int kSplitN = 16384;      // lines this long are split over a two-block cluster
constexpr int kTile64 = 4096;       // double-float synthesis passes

// Intermediates between a row pass and a column pass use the "strip layout":
// element (y, x) of an N x N field sits at (x / W) * N * W + y * W + x % W, so
// that the column pass reads contiguous strips; W is at least the number of
// columns one column-pass block holds, and for FP32 fields at least 4 (whole
// 32-byte sectors per row written by the row pass).

// -------- tables ------------------------------------------------------------
// tw[j] = exp(-2 pi i j / n), j < n, rounded from FP64.
cudaError_t launch_twiddles32(float2* tw, int n, cudaStream_t s);
cudaError_t launch_twiddles64(double2* tw, int n, cudaStream_t s);

// -------- synthesis (FP64) -------------------------------------------------
struct SynthArgs {
    int n;
    int low_k;           // bins with |mx|, |my| <= low_k are drawn in FP64, the others in FP32
    uint32_t screen_id, key0, key1;
    double amp;          // sigma(k) = amp * (mx^2 + my^2)^(-beta/4), includes 1/sqrt(2)
    double neg_beta_4;   // -beta/4
    float amp32, neg_beta_4_32;   // the same in FP32 for the high-frequency bins
    float amp_rel_lo;             // (amp - amp32) / amp32
    float neg_beta_4_lo;          // -beta/4 - neg_beta_4_32
    double out_scale;    // sqrt(2) / L^2
    dfl out_scale_df;    // the same as a double-float
    const dfc* tw;       // double-float twiddles for n
    const float2* tw32;  // FP32 twiddles for n (the transforms of rows outside the FP64 square)
    dfc* work;           // rows ky = 0..n/2 after the x transform, n/2 strips of one column pair (n + 4 values each)
    double* phi;         // n*n, row-major
    double2* pairs;      // n >= kSplitN: n*n doubles, the column pairs column-major before the transpose
    dfc* drawn;          // n <= kDrawN: the Hermitian bins of rows 0..n/2, row-major, drawn before the row pass
};
constexpr int kDrawN = 512;   // up to this size every bin is FP64 and the bins are drawn by their own kernel
cudaError_t launch_twiddles_df(dfc* tw, int n, cudaStream_t s);
cudaError_t launch_synth_rows(const SynthArgs& a, cudaStream_t s);
cudaError_t launch_synth_cols(const SynthArgs& a, cudaStream_t s);

// Test hooks: raw Philox words and the shaped spectrum F (row-major, FFT order).
cudaError_t launch_noise_words(int n, uint32_t screen_id, uint32_t k0, uint32_t k1,
                               uint32_t* words, cudaStream_t s);
cudaError_t launch_noise_spectrum(const SynthArgs& a, double2* F, cudaStream_t s);

// -------- propagation (FP32 with fixed-point phase reduction) --------------
struct LambdaSet {
    int count;                       // wavelengths in this group
    uint64_t scale_fx[kMaxLambda];   // round(lambda_ref/lambda * 2^32)
    uint64_t h_fx[kMaxLambda];       // frac(-lambda z / (2 L^2)) 2^64: H_x phase turns per index^2
    float weight[kMaxLambda];        // passband weight w_l
    float scale[kMaxLambda];         // s = lambda_ref/lambda (the adjoint's d(phase)/d(phi))
};

// One-FFT (conjugate-plane) mode of the propagation passes (Eq. intens, Eq. Gxy).
struct ConjSet {
    unsigned long long chirp_fx[kMaxLambda];   // frac(Delta^2 / (2 lambda z)) 2^64: chirp turns per pixel^2
    float norm[kMaxLambda];                    // (Delta^2 / (lambda z))^2
    int direct;                                // 1: w norm |A|^2 is summed into intensity
    float* pattern;                            // 0: per lambda n*n floats norm |A|^2, row-major
};

struct PropArgs {
    int n;
    const double* phi;       // n*n radians at lambda_ref
    const float2* tw;        // FP32 twiddles
    const float* sf;         // per lambda: n taper values
    float2* work;            // per lambda: n*n complex64, strip layout
    float* intensity;        // n*n
    int accumulate;          // add to intensity instead of overwriting
    float* scratch;          // n = 16384: the column pass's column-major intensity (n*n)
    LambdaSet lam;
    ConjSet conj;            // used by the one-FFT mode only
    float one;               // 1.0f: the multiplier of the packed passes' additions (fft2.cuh)
};
// The taper table of a wavelength group (SF at the pixel centres, per wavelength).
struct TableArgs {
    int n, count;
    double margin_px[kMaxLambda];     // taper margin in pixels (0 = no taper)
    float* sf;
};
cudaError_t launch_prop_tables(const TableArgs& a, cudaStream_t s);
// conj = false: transfer function (FFT, H, IFFT per axis); true: one-FFT method.
cudaError_t launch_prop_rows(const PropArgs& a, bool conj, cudaStream_t s);
cudaError_t launch_prop_cols(const PropArgs& a, bool conj, cudaStream_t s);
// Transfer-function passes with two wavelengths per thread (propagate2.cu): the field
// of wavelengths 2q, 2q + 1 is one array of 16-byte pixels at work + q N^2 (as cp2);
// points: values per thread (16: radix-16 stages; 8: radix-8 stages, twice the threads);
// twm: twiddles from register bases (2) or the block's shared table (1).
bool packed_prop_supported(int n, int points, int row_twm, int col_twm);
cudaError_t launch_prop_rows2(const PropArgs& a, int points, int twm, cudaStream_t s);
cudaError_t launch_prop_cols2(const PropArgs& a, int points, int twm, cudaStream_t s);
// Passband of one-FFT patterns: intensity (+)= sum_l w_l pattern_l resampled
// bilinearly (periodic) at (k - n/2) r_l + n/2, r_l in 32.32 fixed point.
struct ResampleArgs {
    int n, count, accumulate;
    const float* pattern;    // count patterns of n*n floats
    float* intensity;
    long long r_fx[kMaxLambda];
    float weight[kMaxLambda];
};
cudaError_t launch_resample(const ResampleArgs& a, cudaStream_t s);

// -------- FP64 propagation of one screen at one wavelength (propagate64.cu) ------
constexpr int kMax64N = 4096;
struct Prop64Args {
    int n;
    const double* phi;       // n*n radians at lambda_ref
    const double2* tw;       // FP64 twiddles of n
    double scale;            // s = lambda_ref / lambda
    double margin_px;        // taper margin in pixels (0: no taper)
    double c_hi, c_lo;       // frac(lambda z / (2 L^2)) = c_hi + c_lo, c_hi with 31 bits after the point
    double2* field;          // n*n complex128 scratch
    double* intensity;       // n*n
};
cudaError_t launch_prop64(const Prop64Args& a, cudaStream_t s);

// -------- source smoothing ---------------------------------------------------
struct SmoothArgs {
    int n;
    double radius_over_L;    // R_s / L: K depends on 2 pi R_s sqrt(mx^2 + my^2) / L
    const float2* tw;
    float2* spec;            // (n/2 + 1) x n complex64, row-major [ky][x]
    float* intensity;        // n*n in/out
    float2* pairs;           // n >= kSmoothPairsN: n*n floats, the map as column pairs (pairs.cuh)
};
// From this size a smoothing column block holds one column pair, and the map enters and
// leaves the column passes as column pairs (pairs.cuh); floats of that scratch:
constexpr int kSmoothPairsN = 8192;
__host__ __device__ constexpr size_t smooth_pairs_floats(int n) { return n >= kSmoothPairsN ? (size_t)n * n : 0; }
// which = 0: forward column pass, 1: row pass, 2: inverse column pass
cudaError_t launch_smooth_pass(const SmoothArgs& a, int which, cudaStream_t s);

// -------- observables --------------------------------------------------------
struct Track { double x0, y0, c, s, ds; };
constexpr int kTracksPerLaunch = 64;
struct CurveArgs {
    int n, n_tracks, n_samples;
    const float* intensity;
    float* curves;           // n_tracks * n_samples (this launch's slice)
    Track tr[kTracksPerLaunch];
};
cudaError_t launch_lightcurve(const CurveArgs& a, cudaStream_t s);

// -------- adjoint -------------------------------------------------------------
struct CurveAdjArgs {
    int n, n_tracks, n_samples;
    const float* grad_curves;  // this launch's slice, n_tracks * n_samples
    float* grad_map;           // n*n, accumulated with atomics
    Track tr[kTracksPerLaunch];
};
cudaError_t launch_lightcurve_adjoint(const CurveAdjArgs& a, cudaStream_t s);

struct AdjArgs {
    int n;
    const double* phi;
    const float2* tw;
    const float* sf;           // per lambda: taper
    float2* work;              // per lambda: forward row-pass field, overwritten by P_y^H G_out
    const float* grad_map;     // dL/dI after the disk filter
    double* grad_phi;          // n*n, written or accumulated
    int accumulate;
    LambdaSet lam;
};
cudaError_t launch_adj_cols(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_rows(const AdjArgs& a, cudaStream_t s);
// out[0] = scale * sum_i a_i b_i (FP64); partial: kMomentBlocks doubles
cudaError_t launch_scaled_dot(const double* a, const double* b, long long n, double scale, double* partial,
                              double* out, cudaStream_t s);

// FP64 moments of a rectangular region [r0, r1) x [c0, c1) of an n x n map;
// out = {m, mean, sigma, count}.  partial: workspace of >= kMomentBlocks*2 doubles.
constexpr int kMomentBlocks = 1216;     // 8 per SM of a 152-SM GPU
cudaError_t launch_map_moments(const float* map, int n, int r0, int r1, int c0, int c1,
                               double* partial, double* out, cudaStream_t s);
// per-curve {m, mean, sigma}
cudaError_t launch_curve_moments(const float* curves, int n_curves, int n_samples,
                                 double* out, cudaStream_t s);


// ---- screen check of Sect. 3.1.1 (screen_check.cu) --------------------------------
constexpr int kRadialThreads = 512;
constexpr int kCrecThreads = 256;
constexpr int kBisectBlocks = 128;
// Annulus sums of |F|^2 and bin counts (rows walked by `blocks` persistent
// blocks, n_hist annuli in shared memory), then S_rec = sum / count * inv_l2.
// s_rec and counts must be zero on entry.
cudaError_t launch_radial_spectrum(const SynthArgs& a, double inv_l2, int n_hist, double* s_rec,
                                   unsigned long long* counts, int blocks, cudaStream_t s);
struct CrecArgs {
    const double* s;     // S_rec(q_j), j = 0..J
    int J;               // last annulus of the integral
    double dq;           // 1/L
    double half_L;       // upper end of the bisection bracket
};
struct BisectState {
    double lo, hi;
    int no_root;
    unsigned arrived;
    double partial[kBisectBlocks];
};
cudaError_t launch_crec(const CrecArgs& a, const double* r_km, int n_r, double* d, cudaStream_t s);
cudaError_t launch_bisect(const CrecArgs& a, BisectState* st, int iterations, double* out, cudaStream_t s);


// ---- light-curve time analysis (timeseries.cu) -------------------------------------
// Periodogram |DFT(c - mean c)|^2 / n, k = 0..n/2, of n_curves curves of n samples
// (n a power of two up to 8192); tw: FP32 twiddles of n.
cudaError_t launch_power_spectrum(const float* curves, int n_curves, int n, float* power, const float2* tw,
                                  cudaStream_t s);
// Pearson correlation of row i of b with row i / (n_pairs / a_rows) of a (rows of a
// a_stride floats apart); a_rows divides n_pairs.
cudaError_t launch_correlation(const float* a, int a_rows, long long a_stride, const float* b, int n_pairs, int n,
                               double* r, cudaStream_t s);

}  // namespace scint
