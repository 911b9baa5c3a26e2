/*
 * scint.h -- C ABI of the GB300 Fresnel-scintillation library (libscint.so).
 *
 * The library computes the data-parallel hot path of the optical interstellar
 * scintillation simulation of Habibi, Moniez, Ansari & Rahvar (A&A 2013,
 * arXiv:1301.0514): a power-law phase screen synthesised from seeded Gaussian
 * noise (Sect. 3.1, Eq. spectre, Eq. densite), its Fresnel propagation to the
 * observer plane (Eq. hxy) with the edge taper of Sect. 3.2.1, the intensity
 * |A|^2 co-added over a passband (Sect. 3.2.4), smoothed by the projected
 * stellar disk (Sect. 3.2.3, Eq. iprh), and sampled along straight tracks
 * (Sect. 3.3), plus the modulation index m = sigma_I / mean(I) (Sect. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grids are square, N x N, N a power of two (the screen check of Sect.
 *    3.1.1 takes any even N); arrays are row-major with the
 *    row index y: element (y, x) sits at [y * N + x].  Pixel (ix, iy) has its
 *    centre at ((ix + 1/2) Delta, (iy + 1/2) Delta) on the screen.
 *  - Lengths are in km, wavelengths in nm, distances in pc.
 *  - Pointers named "device" must be CUDA device memory of the current device;
 *    pointers named "host" are ordinary host memory read before the call
 *    returns.  The caller owns every buffer it passes; the library never
 *    frees or keeps caller memory past the call.
 *  - Every call is asynchronous and ordered on `stream` (a cudaStream_t, NULL
 *    for the legacy default stream).  Inputs are never modified unless the
 *    argument is documented as in/out.
 *  - Return value: SCINT_OK, or an error code; scint_last_error() then gives a
 *    message for the calling thread.  Parameter errors are detected on the host
 *    before anything is launched, so a failing call leaves outputs untouched.
 *  - Workspace: entry points taking (workspace, workspace_bytes) need device
 *    scratch memory.  Pass a device buffer of scint_workspace_bytes() bytes for
 *    the call's parameters, or a smaller one (>= the minimum that call
 *    reports), in which case wavelengths are processed in groups that fit.
 *    Passing workspace == NULL makes the library use its own per-device pool,
 *    grown with cudaMalloc on first need (not allowed inside stream capture).
 */
#ifndef SCINT_H
#define SCINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SCINT_OK           0
#define SCINT_EINVAL       1   /* invalid argument (checked on the host) */
#define SCINT_ENOMEM       2   /* workspace too small or allocation failed */
#define SCINT_ECUDA        3   /* a CUDA runtime call failed */
#define SCINT_ETIMEOUT     4   /* reserved for a bounded device-side wait that gives up;
                                  no kernel of this version waits on a flag or a peer */
#define SCINT_EUNSUPPORTED 5   /* valid parameters this build does not support */

#define SCINT_MAX_LAMBDA   128 /* wavelengths per passband call */
#define SCINT_MIN_N        16
#define SCINT_MAX_N        16384
#define SCINT_MAX_CHECK_N  32768 /* grid size limit of the screen check (any even N) */

/*
 * Parameters of one screen and observation.
 *   n                 grid size N (power of two, SCINT_MIN_N..SCINT_MAX_N)
 *   pixel_km          pixel side Delta_1 (km)
 *   r_diff_km         diffraction radius R_diff at lambda_ref_nm (Eq. dphi)
 *   beta              spectral index of S_phi, 2 < beta < 4 (11/3 = Kolmogorov)
 *   lambda_nm         wavelength of single-wavelength calls (and of the
 *                     fiducial zone of scint_modulation_index)
 *   lambda_ref_nm     wavelength at which the screen phase is defined; the
 *                     phase at lambda is phi * lambda_ref / lambda (Eq. phiNl)
 *   z_pc              screen-observer distance z_0
 *   source_radius_km  projected source radius R_s (Eq. iprh); 0 = point source
 *   margin_km         taper margin L_m of Sect. 3.2.1: < 0 selects the default
 *                     min(10 R_F(lambda), L/4); 0 switches the taper off
 *   seed, screen_id   select the Philox4x32-10 noise stream of the screen
 */
typedef struct scint_params {
    int32_t  n;
    int32_t  reserved0;        /* must be 0 */
    double   pixel_km;
    double   r_diff_km;
    double   beta;
    double   lambda_nm;
    double   lambda_ref_nm;
    double   z_pc;
    double   source_radius_km;
    double   margin_km;
    uint64_t seed;
    uint32_t screen_id;
    uint32_t reserved1;        /* must be 0 */
} scint_params;

/* Library version as 10000*major + 100*minor + patch. */
int scint_version(void);

/* Message describing the last error on the calling thread ("" if none). */
const char* scint_last_error(void);

/*
 * Sampling condition of Sect. 3.2.2: the pixel must resolve the screen's phase
 * variations, pixel_km < R_diff(lambda)/2, with R_diff(lambda) =
 * r_diff_km (lambda / lambda_ref_nm)^(2/(beta-2)) (the phase scales as
 * lambda_ref/lambda, Sect. 3.2.4).  Returns the worst ratio
 * 2 pixel_km / R_diff(lambda) over lambdas_nm[0..n_lambda) (host array; NULL or
 * n_lambda <= 0: p->lambda_nm), >= 1 meaning violated; -1 on invalid arguments
 * (scint_last_error() says why).  Host only.
 */
double scint_sampling_ratio(const scint_params* p, const double* lambdas_nm, int n_lambda);

/* Warning left by the last propagating call on the calling thread
 * (scint_propagate*, scint_sum_passband*, scint_lightcurve_adjoint,
 * scint_run_batch): "" when its parameters meet the sampling condition above,
 * else a message naming the wavelength (and, for a batch, the first item) that
 * violates it.  Such a call still runs and returns SCINT_OK. */
const char* scint_last_warning(void);

/* Device scratch bytes that the calls below need for grid p->n when a passband
 * of n_lambda wavelengths is processed in one group (n_lambda >= 1). */
size_t scint_workspace_bytes(const scint_params* p, int n_lambda);

/*
 * Phase screen synthesis (Sect. 3.1, Eq. spectre, Eq. densite).
 * For every FFT bin k (row ky, column kx) draws two normals from
 * Philox4x32-10 with counter (kx, ky, screen_id, 0) and key (seed low word,
 * seed high word) by the Box-Muller transform, forms
 *   F_k = sqrt(L^2 S_phi(q_k)) (g_re + i g_im) / sqrt(2),  F_0 = 0,
 * and writes phi_j = sqrt(2)/L^2 Re sum_k F_k exp(+2 pi i k.x_j)  (radians, at
 * lambda_ref).  Precision: the bins in a square |kx|, |ky| <= K around the
 * origin (nearly all of the phase variance, since S ~ q^-beta) draw their normals
 * and amplitude in FP64; every other bin draws them in FP32 from the same 53-bit
 * uniforms.  Up to N = 512 every bin is drawn in FP64; above, K in {32, 64, 128,
 * 256} is chosen per screen: the smallest square whose outside carries an rms
 * phase of at most 0.45 rad (the FP32 draws err by ~1e-7 of that), 256 when none
 * does.  The
 * inverse 2D transform runs in double-float arithmetic (pairs of FP32 numbers,
 * about 44 significant bits), except the x transforms of the spectral rows with
 * |ky| > K (FP32 bins only, a small share of the phase), which run in FP32; phi
 * is written in FP64.  Against the FP64
 * oracle the screen agrees to better than 2e-6 rad (the measured worst cases are
 * stated with the tests of the full-size workloads).
 *   phi   device, N*N doubles, written; 16-byte aligned (SCINT_EINVAL otherwise).
 * Needs workspace (scint_workspace_bytes): about 8 N^2 bytes for (N/2 + 1) N
 * double-float values and the twiddle tables, 16 N^2 at N = 16384 (the column
 * pairs before their transpose) and up to N = 512 (the drawn bins).
 */
int scint_make_screen(const scint_params* p, double* phi,
                      void* workspace, size_t workspace_bytes, void* stream);

/*
 * Screen check of Sect. 3.1.1, part 1: the spectral density recomputed from the
 * generated F_phi (the same F as scint_make_screen draws),
 *   S_rec(q_j) = sum_{annulus j} |F_k|^2 / (count_j L_x L_y),  q_j = j / L,
 * where annulus j holds the FFT bins whose integer wave vector m (k = m / L)
 * has j - 1/2 <= |m| < j + 1/2 (the paper averages over the circle |k| = q
 * without naming a width; annuli of width 1/L are this library's reading).
 * The noise is regenerated bin by bin, never stored.  p->n may be any even
 * number in [SCINT_MIN_N, SCINT_MAX_CHECK_N] (the paper's check uses N ~ 14000);
 * only n, pixel_km, r_diff_km, beta, seed and screen_id are used.
 *   s_rec    device, n_bins doubles written: S_rec(q_j) for j < n_bins (0 for
 *            annuli without bins: j = 0 holds only the DC bin, where F = 0, and
 *            j > sqrt(2) N/2 lies outside the grid).
 *   counts   device, n_bins uint64 written: bins per annulus.
 * The annulus sums are 64-bit fixed point with a per-annulus scale (each bin
 * truncated to 2^-36 of the annulus' expected bin power), so they are exact
 * and the result is the same bit for bit on every run.
 */
int scint_spectrum_rec(const scint_params* p, double* s_rec, uint64_t* counts, int n_bins, void* stream);

/*
 * Screen check of Sect. 3.1.1, part 2 (Eq. crec): the structure function
 *   D_rec(r) = 2 (xi_rec(0) - xi_rec(r))
 *            = 2 sum_{j=1}^{J} 2 pi q_j S_rec(q_j) (1 - J0(2 pi q_j r)) dq,
 * dq = 1/L, J = min(n_bins - 1, N/2): the integral of Eq. crec between the
 * paper's q_min = 1/L and q_max = 1/(2 Delta_1) by the midpoint rule on the
 * annuli, with J0 from the CUDA math library; and R_diff^rec, the root of
 * D_rec(R) = 1, by 64 bisection steps on (0, L/2] (NaN if D_rec(L/2) < 1).
 * s_rec may be scint_spectrum_rec's output or any spectrum sampled at q_j
 * (e.g. the theoretical S_phi, as in the paper's comparison).
 *   s_rec   device, n_bins >= 2 doubles, read.
 *   r_km    device, n_r lags (km), read; d_rec device, n_r doubles written
 *           (both may be NULL when n_r == 0).
 *   r_rec   device, 1 double written, or NULL to skip the root.
 * Each D_rec value is summed in a fixed order (reproducible bit for bit).
 * Needs workspace (< 1 KB) when r_rec != NULL.
 */
int scint_structure_function_rec(const scint_params* p, const double* s_rec, int n_bins,
                                 const double* r_km, int n_r, double* d_rec, double* r_rec,
                                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Monochromatic point-source intensity at p->lambda_nm (Eq. hxy, Sect. 3.2.1):
 *   A_in  = SF(x) SF(y) exp(i phi lambda_ref/lambda),
 *   A_out = IDFT(DFT(A_in) H),  H(k) = exp(-i pi lambda z |k|^2),
 *   I     = |A_out|^2   (1 for an unobstructed plane wave).
 * The phase is reduced modulo 2 pi exactly (64-bit fixed point) before the
 * FP32 sine/cosine; FFTs and intensity are FP32.
 *   phi        device, N*N doubles (radians at lambda_ref), read.
 *   intensity  device, N*N floats, written.
 */
int scint_propagate(const scint_params* p, const double* phi, float* intensity,
                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * The plain method in FP64 (Eq. hxy, Sect. 3.2.1): scint_propagate with every step in
 * double precision, for grids n <= 4096 (SCINT_EUNSUPPORTED above).  The field is
 * A_in = SF(x) SF(y) exp(i phi lambda_ref / lambda), propagated by the transfer function
 * (FFT, H = exp(-i pi lambda z |k|^2), inverse FFT, along x then y) with FP64 sines,
 * cosines and line transforms; the chirp phase is reduced exactly (its constant split so
 * that the product with m^2 carries no rounding).  One wavelength (p->lambda_nm).
 *   phi        device, N*N doubles (radians at lambda_ref).
 *   intensity  device, N*N doubles, written (|A_out|^2, the unobstructed wave = 1).
 * Needs workspace (16 N^2 + 16 N bytes).  Much slower than the FP32 path on GB300
 * (its FP64 pipe is narrow); it is the reference-precision form of config-1 sizes.
 */
int scint_propagate64(const scint_params* p, const double* phi, double* intensity,
                      void* workspace, size_t workspace_bytes, void* stream);

/*
 * scint_propagate without any device allocation.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc and cannot pass
 * a workspace either, e.g. hosts that forbid device allocation once running
 * (fixed-budget real-time loops) or plugins inside a framework that owns all
 * device memory.  The caller still passes phi and intensity exactly as for
 * scint_propagate, and gets the same result.
 *   - Scratch comes from one static device array of 8 MiB + 64 KiB inside the
 *     library, so n is limited to 1024; larger n returns SCINT_EINVAL.  Every
 *     GPU that loads the library holds the array until the process exits.
 *   - The first call on each device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - All calls share the array, and each call leaves its scratch contents
 *     behind; nothing in it needs clearing between calls.  Calls whose
 *     executions overlap on the GPU (different streams, or several host
 *     threads) race on the array: serialise them.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.  The
 *     twiddle table is computed into the array on every call, with the same
 *     kernel that fills the table scint_propagate keeps, so the two calls give
 *     bit-identical intensities.
 *   - The looked-up address is forgotten by scint_release; call scint_release
 *     before a device reset (cudaDeviceReset) if this entry point is used
 *     again afterwards.
 */
int scint_propagate_noalloc(const scint_params* p, const double* phi, float* intensity, void* stream);

/*
 * Passband co-addition (Sect. 3.2.4): intensity = sum_l w_l I(lambda_l) with
 * the same screen phase scaled by lambda_ref/lambda_l.
 *   lambdas_nm  host, n_lambda wavelengths (1..SCINT_MAX_LAMBDA).
 *   weights     host, n_lambda weights, or NULL for 1/n_lambda each.
 *   intensity   device, N*N floats, written (accumulate == 0) or added to
 *               (accumulate != 0).
 */
int scint_sum_passband(const scint_params* p, const double* phi,
                       const double* lambdas_nm, const double* weights, int n_lambda,
                       float* intensity, int accumulate,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * The paper's own propagator (Eq. intens with Eq. Gxy): one 2D Fourier
 * transform of G = SF(x_1) SF(y_1) exp(i (phi lambda_ref/lambda + |x_1|^2/2R_F^2)),
 *   h(x_0) = |FT[G](x_0 / (lambda z))|^2 / (lambda z)^2     (1 for a uniform screen),
 * on the observer grid of the conjugate variable: x_0 = (k - N/2) Delta_0 with
 * Delta_0 = lambda z / (N Delta_1) (scint_conjugate_pixel_km), screen pixels at
 * x_1 = (i - N/2) Delta_1 about the optical axis (integer pixel centres, Sect.
 * 3.2.1).  Unlike the transfer function this is the plain, non-periodic Fresnel
 * sum over the screen; at critical sampling N Delta_1^2 = lambda z (the paper's
 * N Delta^2 = 2 pi R_F^2) both give the same pattern pixel for pixel.  Half the
 * FFT work of scint_propagate (one transform per axis instead of two).
 *   phi        device, N*N doubles, read.   intensity  device, N*N floats, written,
 *              row-major with the optical axis at element (N/2, N/2).
 * Workspace: as scint_propagate.
 */
int scint_propagate_conjugate(const scint_params* p, const double* phi, float* intensity,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Observer-plane pixel Delta_0 = lambda z / (N Delta_1) of the one-FFT method at
 * lambda_nm (km); NaN for invalid arguments. */
double scint_conjugate_pixel_km(const scint_params* p, double lambda_nm);

/*
 * Passband co-addition (Sect. 3.2.4) of one-FFT patterns.  The pattern of
 * wavelength l has pixel Delta_0(lambda_l), so each is resampled onto the grid
 * of p->lambda_nm about the optical axis, a pixel centre of every grid: output
 * pixel k samples pattern l bilinearly (periodic, like the discrete transform)
 * at (k - N/2) lambda_nm/lambda_l + N/2 of its pixels, and
 *   intensity (+)= sum_l w_l h_l(resampled).
 * Arguments as scint_sum_passband.  Workspace: that of the transfer-function
 * passband plus 4 N^2 bytes per
 * wavelength of a group (smaller workspaces give smaller groups).
 */
int scint_sum_passband_conjugate(const scint_params* p, const double* phi,
                                 const double* lambdas_nm, const double* weights, int n_lambda,
                                 float* intensity, int accumulate,
                                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Extended source (Sect. 3.2.3, Eq. iprh): periodic convolution of the
 * intensity with the uniform disk of radius p->source_radius_km, applied in
 * Fourier space as K(q) = 2 J1(2 pi q R_s)/(2 pi q R_s).  R_s = 0 leaves the
 * map unchanged.
 *   intensity  device, N*N floats, in/out.
 */
int scint_smooth_source(const scint_params* p, float* intensity,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * Light curves (Sect. 3.3): sample the map along straight tracks at constant
 * speed, bilinear interpolation with periodic wrap.  Pixel (ix, iy) sits at
 * integer coordinates (ix, iy).
 *   tracks   host, n_tracks records of 4 doubles (x0, y0, theta, ds) in pixels
 *            and radians; sample s is at (x0 + s ds cos theta, y0 + s ds sin theta).
 *   curves   device, n_tracks * n_samples floats, written row by row.
 * With n_tracks == 0 or n_samples == 0 nothing is read or written and the
 * pointers may be NULL.
 */
int scint_lightcurve(const scint_params* p, const float* intensity,
                     const double* tracks, int n_tracks, int n_samples,
                     float* curves, void* stream);

/*
 * Modulation index m = sigma_I / mean(I) (Sect. 4, population sigma) of a map
 * over its fiducial zone: pixels whose centres are at least
 * L_m + R_ref(lambda)/2 + R_s from every border (Sect. 3.2.1, 3.2.3), with
 * lambda = p->lambda_nm and R_ref = lambda z / R_diff(lambda).  The whole map
 * is used when the taper is off or that zone is empty.
 *   out   device, 4 doubles written: m, mean, sigma, pixel count.
 * Accumulation is FP64.  Needs workspace (a few KB).
 */
int scint_modulation_index(const scint_params* p, const float* intensity, double* out,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * The fiducial zone that scint_modulation_index uses: pixel index range
 * [*i0, *i1) on both axes whose centres lie at least L_m + R_ref/2 + R_s from
 * every border (Sect. 3.2.1, 3.2.3), with lambda = p->lambda_nm; *r_ref_km
 * (may be NULL) receives R_ref = lambda z / R_diff(lambda).  Host only.
 * Returns SCINT_EUNSUPPORTED (with [0, N)) when the zone is empty, SCINT_OK
 * otherwise (also when the taper is off: the whole map).
 */
int scint_fiducial_zone(const scint_params* p, int32_t* i0, int32_t* i1, double* r_ref_km);

/*
 * Modulation index of each light curve: out[c] = {m, mean, sigma} for curve c
 * of curves (n_curves x n_samples, row-major).
 *   out   device, 3 * n_curves doubles, written.
 */
int scint_curve_modulation(const float* curves, int n_curves, int n_samples,
                           double* out, void* stream);

/*
 * Time power spectrum of light curves (Sect. 5: its slope breaks near 1/t_ref,
 * t_ref = R_ref / V_T), the periodogram
 *   power[c][k] = |sum_s (c_s - mean c) exp(-2 pi i k s / n)|^2 / n,  k = 0..n/2,
 * with n = n_samples a power of two in [SCINT_MIN_N, 8192].  The mean is
 * removed in FP64 before the FP32 transform.
 *   curves   device, n_curves x n_samples floats, read.
 *   power    device, n_curves x (n_samples/2 + 1) floats, written.
 * Needs workspace (8 n_samples bytes).
 */
int scint_curve_power_spectrum(const float* curves, int n_curves, int n_samples, float* power,
                               void* workspace, size_t workspace_bytes, void* stream);

/*
 * Correlation coefficient of pairs of light curves (Sect. 5: two telescopes a
 * distance apart see decorrelated curves once it exceeds 2 max(R_ref, R_s)):
 *   r[i] = sum (a_j - mean a_j)(b_i - mean b_i) / sqrt(sum (a_j - ..)^2 sum (b_i - ..)^2),
 * FP64, where b_i is row i of b and a_j row j = i / (n_pairs / a_rows) of a: the
 * pairs come in a_rows equal groups, each against one curve of a (a reference
 * telescope against its parallels).
 *   a  device, a_rows rows of n_samples floats, a_stride floats apart (ignored
 *      when a_rows == 1);  b  device, n_pairs x n_samples floats;
 *   r  device, n_pairs doubles, written.   a_rows must divide n_pairs.
 */
int scint_curve_correlation(const float* a, int a_rows, int64_t a_stride, const float* b, int n_pairs,
                            int n_samples, double* r, void* stream);

/*
 * Batch of independent screens, each run through the whole forward path of the
 * paper's polychromatic extended-source simulation (Sect. 3.1 synthesis,
 * Sect. 3.2 propagation with taper, Sect. 3.2.4 passband co-addition,
 * Sect. 3.2.3 disk smoothing, Sect. 3.3 light curves, Sect. 4 modulation
 * index), as in the paper's sweeps over R_diff, source radius and spectral
 * index.  For item i, with its own params:
 *   phi  = make_screen(params)                                  (if phi != NULL, kept)
 *   I    = smooth_source(sum_passband(phi, lambdas, weights))   (if intensity != NULL, kept)
 *   curves   = lightcurve(I, tracks)                             (if n_tracks, n_samples > 0)
 *   m_map    = modulation_index(I)                               (if m_map != NULL)
 *   m_curves = curve_modulation(curves)                          (if m_curves != NULL)
 * Each result equals that of the single-screen calls above.  Fields:
 *   params      the screen (its lambda_nm only selects the fiducial zone of m_map)
 *   phi         device, N*N doubles written, or NULL (the screen lives in scratch)
 *   intensity   device, N*N floats written, or NULL (scratch)
 *   tracks      host, 4 * n_tracks doubles as in scint_lightcurve (read before
 *               the call returns)
 *   curves      device, n_tracks * n_samples floats written; may be NULL only
 *               when n_tracks or n_samples is 0
 *   m_map       device, 4 doubles (m, mean, sigma, count) or NULL
 *   m_curves    device, 3 * n_tracks doubles or NULL; needs curves
 */
typedef struct scint_batch_item {
    scint_params  params;
    double*       phi;
    float*        intensity;
    const double* tracks;
    int32_t       n_tracks;
    int32_t       n_samples;
    float*        curves;
    double*       m_map;
    double*       m_curves;
} scint_batch_item;

#define SCINT_MAX_LANES 8

/*
 * Workspace for scint_run_batch with n_lanes lanes when each screen's passband
 * of n_lambda wavelengths runs in one group: n_lanes equal slices, each the
 * forward workspace of the largest screen plus, when any item leaves phi or
 * intensity NULL, scratch maps of that size.  0 on invalid arguments.
 */
size_t scint_batch_workspace_bytes(const scint_batch_item* items, int n_items, int n_lambda, int n_lanes);

/*
 * Run a batch (see scint_batch_item).  The library schedules the items on
 * n_lanes internal CUDA streams (1..SCINT_MAX_LANES; <= 0 selects 2), the
 * costliest first, each to the lane with the least work queued
 * (longest-processing-time rule with cost N^2 log2 N (n_lambda + 8)), so that
 * kernels of small screens fill the tail waves of large ones.  The lanes start
 * after the work already queued on `stream` and `stream` waits for all of
 * them, so the call is ordered on `stream` like every other entry point and can
 * be captured into a CUDA graph (the lanes join the capture).
 *   items        host array of n_items records (n_items >= 0).
 *   lambdas_nm   host, n_lambda wavelengths shared by every item; weights host
 *                or NULL (1/n_lambda), as in scint_sum_passband.
 *   workspace    device, >= n_lanes * (the minimum slice for one wavelength
 *                group); a slice smaller than the one-group size makes the
 *                passbands run in groups.  NULL: the per-device pool.
 * Every item is checked on the host before anything is launched.  Concurrent
 * calls from several host threads are serialised while they enqueue.
 */
int scint_run_batch(const scint_batch_item* items, int n_items,
                    const double* lambdas_nm, const double* weights, int n_lambda,
                    int n_lanes, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Gradient of a light-curve misfit with respect to the phase screen (reverse
 * mode through Sect. 3.2-3.3; the paper states no gradient, this is the
 * adjoint of the forward path of this library).  The forward map is
 *   curves = lightcurve(smooth_source(sum_passband(phi)))
 * with the same parameters; given grad_curves = dL/dcurves this computes
 *   grad_phi = dL/dphi = sum_l s_l Im(conj(A_in,l) P_l^H (2 w_l g_I A_out,l)),
 *   g_I = K B^T grad_curves  (B: bilinear sampling, K: disk filter, both as in
 *   the forward calls), s_l = lambda_ref/lambda_l.
 * The forward fields are recomputed (never stored).
 *   lambdas_nm, weights, tracks  host, as in scint_sum_passband / scint_lightcurve.
 *   grad_curves  device, n_tracks * n_samples floats.
 *   grad_phi     device, N*N doubles, written (accumulate == 0) or added to.
 * Workspace: scint_workspace_bytes(p, n_lambda) covers it.
 */
int scint_lightcurve_adjoint(const scint_params* p, const double* phi,
                             const double* lambdas_nm, const double* weights, int n_lambda,
                             const double* tracks, int n_tracks, int n_samples,
                             const float* grad_curves, double* grad_phi, int accumulate,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * dL/dR_diff from dL/dphi: at a fixed seed the synthesised screen scales as
 * R_diff^((2 - beta)/2) (Eq. spectre: sigma ~ R_diff^(1 - beta/2)), so
 *   out[0] = ((2 - beta) / (2 R_diff)) sum_j phi_j grad_phi_j   (FP64).
 *   out  device, 1 double.  Needs workspace (a few KB).
 */
int scint_rdiff_gradient(const scint_params* p, const double* phi, const double* grad_phi, double* out,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * Propagation plans and the autotuner (build-side; the paper has no counterpart).
 * The transfer-function passes of scint_propagate, scint_sum_passband,
 * scint_run_batch and the batch's passbands exist in several compiled variants
 * that compute the same intensity to FP32 rounding (they differ in the last bits):
 *   packed        1: two wavelengths per thread (packed two-wide FP32 arithmetic),
 *                 used for groups of >= 2 wavelengths at 64 <= N <= 8192;
 *                 0: one wavelength per thread.
 *   points        values per thread of the packed passes: 16 (radix-16 stages) or
 *                 8 (radix-8 stages, twice the threads per line, N >= 128).
 *   row_twiddles  FFT twiddle source of the packed row pass: 1 the block's shared
 *                 table, 2 register bases and products.
 *   col_twiddles  the same for the packed column pass.
 * (the one-wavelength passes and N = 16384 have one variant each).  A plan is
 * kept per (device, N).  Until one is set or tuned, a default built from
 * measurements on GB300 is used.  A call that runs while the plan of its N
 * changes may use either plan; results of one plan are reproducible bit for bit.
 */
typedef struct scint_plan {
    int32_t packed;
    int32_t points;
    int32_t row_twiddles;
    int32_t col_twiddles;
    int32_t tuned;      /* out: 1 if scint_tune measured this plan, 0 otherwise */
    int32_t reserved;   /* 0 */
    double  ms;         /* out: scint_tune's best time for its test passband, else 0 */
} scint_plan;

/* The plan used for grid n on the current device (SCINT_EINVAL for an invalid n). */
int scint_get_plan(int n, scint_plan* out);

/* Fix the plan of grid n on the current device.  SCINT_EUNSUPPORTED when the
 * variant is not built for n (e.g. a shared table that does not fit in shared
 * memory); the plan is then unchanged.  tuned and ms are ignored. */
int scint_set_plan(int n, const scint_plan* plan);

/*
 * Autotuner: time every built variant of the propagation passes for grid n on a
 * test passband of n_lambda wavelengths (clamped to [2, 32]) on the current
 * device, three times each after one warm-up, with CUDA events on `stream`, and
 * keep the fastest as the plan of n (returned in *out when out != NULL).  The
 * test passband's fields are limited to 1 GiB (fewer wavelengths at large n).
 * Allocates its own test buffers (a phase screen of zeros, the intensity and the
 * workspace) with cudaMalloc and frees them before returning; synchronous.  Not
 * allowed while `stream` is being captured (SCINT_EINVAL).
 */
int scint_tune(int n, int n_lambda, scint_plan* out, void* stream);

/*
 * Batch execution form (build-side; the paper has no counterpart).
 *   0  lanes (default): every screen through the single-screen entry points on
 *      up to n_lanes internal streams.
 *   1  persistent propagation: the screens' syntheses on the lanes, then the
 *      propagation passes of every screen in ONE persistent launch (one block per
 *      SM walking a work list of (screen, pass, block of lines) items; a screen's
 *      column work waits for its row work, and a screen's row work for the column
 *      work of the screen that used its field slot before it, through counters in
 *      the workspace), then smoothing and observables on the lanes.  Used when every
 *      grid size is in [256, 4096], at most 256 screens, and every size's plan is
 *      the one-wavelength passes; otherwise the call runs on lanes.  Results equal
 *      the single-screen calls bit for bit.  It needs a larger workspace
 *      (scint_batch_workspace_bytes accounts for it while the mode is 1): one field
 *      slot per lane for the whole passband, plus each screen's phase and intensity
 *      map where the item leaves them NULL.
 * Every wait of the persistent kernel is bounded: after about 2 s it gives up, sets
 * a status word to SCINT_ETIMEOUT and ends the launch (the outputs are then
 * incomplete).  scint_batch_status reads that word.  Returns the previous mode, or
 * -1 (SCINT_EINVAL in scint_last_error) for a mode other than 0 or 1.
 */
int scint_batch_mode(int mode);

/* Waits for `stream`, then returns SCINT_OK, or SCINT_ETIMEOUT if the last persistent
 * batch launched on the current device gave up a dependency wait (SCINT_ECUDA if the
 * stream reports an error). */
int scint_batch_status(void* stream);

/*
 * Batch autotuner: the plans that win alone are not always the fastest when
 * several screens run at once on the batch executor's lanes (blocks that need
 * more shared memory leave less room for the other lanes' kernels).  This times
 * scint_run_batch on the given batch under each candidate: on lanes, plan sets
 * {the per-size winners of scint_tune, every size on the one-wavelength passes,
 * every size on the packed passes}, and the persistent form (scint_batch_mode 1,
 * one-wavelength passes) where the batch allows it; each with lanes {4, 8} (those
 * the workspace holds, at most n_items), one warm-up and two timed runs with CUDA
 * events on `stream`.  It keeps the fastest: its plans become the plans of the
 * batch's grid sizes (tuned = 1, ms = the batch time), its form the batch mode
 * (*out_mode, may be NULL), and its lane count is returned in *out_lanes (*out_ms:
 * its time).  Runs the batch's whole forward path about 25 times; writes the
 * items' outputs.  Synchronous; not allowed during capture.
 *   workspace, workspace_bytes  as for scint_run_batch (NULL: the pool); the
 *   persistent candidate is skipped when the workspace is too small for it.
 */
int scint_tune_batch(const scint_batch_item* items, int n_items, const double* lambdas_nm, const double* weights,
                     int n_lambda, void* workspace, size_t workspace_bytes, int* out_lanes, double* out_ms,
                     int* out_mode, void* stream);

/* Autotuning on first use (off by default): while on, scint_run_batch calls
 * scint_tune for every grid size of its items that has no plan on the current
 * device yet, before it launches anything, unless `stream` is being captured.
 * Returns the previous setting. */
int scint_autotune(int on);

/* Release the library's internal per-device workspace pools, the twiddle tables
 * it keeps per (device, grid size) after their first use, and the batch
 * executor's streams, and forget the device addresses that
 * scint_propagate_noalloc looked up (the next call looks them up again).  Waits
 * for the work that may still read them.  Call it before a device reset if the
 * library is used again afterwards. */
void scint_release(void);

/*
 * Kernel profiler (instrumentation; the paper has no counterpart).  While
 * enabled, every kernel launch is bracketed by two CUDA events recorded on the
 * launching stream (event nodes when the stream is being captured into a
 * graph), tagged with the launch's algorithmic DRAM bytes (each input read
 * once, each output written once) and FFT flops (5 n log2 n per complex line
 * transform of n points).
 *   scint_profile_enable(on)  clears the records and turns recording on/off.
 *   scint_profile_read        waits for the recorded events and sums them per
 *                             kernel class into stats[0..max_stats); *n_stats
 *                             receives the number of classes written.  For
 *                             events inside a graph, the last replay counts.
 */
typedef struct scint_kernel_stat {
    char    name[32];
    int64_t launches;   /* kernel launches recorded */
    double  total_ms;
    double  bytes;
    double  flops;
} scint_kernel_stat;
int scint_profile_enable(int on);
int scint_profile_read(scint_kernel_stat* stats, int max_stats, int* n_stats);

#ifdef __cplusplus
}
#endif

#endif /* SCINT_H */
