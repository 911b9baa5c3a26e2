// C-ABI entry points: host-side parameter checks, derived physical scalars,
// workspace carving and kernel sequencing.  Declarations and the contract of
// every function are in include/scint.h and include/scint_testing.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/scint.h"
#include "../../include/scint_testing.h"
#include "api_internal.h"
#include "kernels.cuh"
#include "persist.cuh"

namespace scint {
cudaError_t launch_fft_lines32(int n, int dir, float2* data, int n_lines, const float2* tw, cudaStream_t s);
cudaError_t launch_fft_lines64(int n, int dir, double2* data, int n_lines, const double2* tw, cudaStream_t s);
cudaError_t launch_phase_fixed(const double* phi, long long* P, long long n, cudaStream_t s);
}

using namespace scint;

namespace {

thread_local std::string g_error;
thread_local std::string g_warning;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int ok() {
    g_error.clear();
    return SCINT_OK;
}

#define SCINT_CUDA(call)                                                                      \
    do {                                                                                      \
        const cudaError_t e_ = (call);                                                        \
        if (e_ == cudaErrorNotSupported)                                                      \
            return fail(SCINT_EUNSUPPORTED, "%s: not supported for this grid size", #call);   \
        if (e_ != cudaSuccess) return fail(SCINT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int check_params(const scint_params* p) {
    if (!p) return fail(SCINT_EINVAL, "params is NULL");
    if (!pow2(p->n) || p->n < SCINT_MIN_N || p->n > SCINT_MAX_N)
        return fail(SCINT_EINVAL, "n=%d must be a power of two in [%d, %d]", p->n, SCINT_MIN_N, SCINT_MAX_N);
    if (p->reserved0 || p->reserved1) return fail(SCINT_EINVAL, "reserved fields must be 0");
    if (!(p->pixel_km > 0) || !std::isfinite(p->pixel_km)) return fail(SCINT_EINVAL, "pixel_km must be > 0");
    if (!(p->r_diff_km > 0) || !std::isfinite(p->r_diff_km)) return fail(SCINT_EINVAL, "r_diff_km must be > 0");
    if (!(p->beta > 2.0 && p->beta < 4.0)) return fail(SCINT_EINVAL, "beta=%g must be in (2, 4)", p->beta);
    if (!(p->lambda_nm > 0) || !std::isfinite(p->lambda_nm)) return fail(SCINT_EINVAL, "lambda_nm must be > 0");
    if (!(p->lambda_ref_nm > 0) || !std::isfinite(p->lambda_ref_nm))
        return fail(SCINT_EINVAL, "lambda_ref_nm must be > 0");
    if (!(p->z_pc > 0) || !std::isfinite(p->z_pc)) return fail(SCINT_EINVAL, "z_pc must be > 0");
    if (!(p->source_radius_km >= 0) || !std::isfinite(p->source_radius_km))
        return fail(SCINT_EINVAL, "source_radius_km must be >= 0");
    if (!std::isfinite(p->margin_km)) return fail(SCINT_EINVAL, "margin_km must be finite");
    if (p->margin_km > 0.5 * p->n * p->pixel_km) return fail(SCINT_EINVAL, "margin_km exceeds half the screen");
    return SCINT_OK;
}

// ---- physics scalars (same formulas as the paper; units km) ----------------------
double lz_km2(double lambda_nm, double z_pc) { return lambda_nm * kKmPerNm * z_pc * kKmPerPc; }
double fresnel_radius(double lambda_nm, double z_pc) { return std::sqrt(lz_km2(lambda_nm, z_pc) / (2.0 * kPi)); }
double screen_len(const scint_params* p) { return p->n * p->pixel_km; }
// taper margin L_m (Sect. 3.2.1): default 10 R_F clamped to L/4
double taper_margin(const scint_params* p, double lambda_nm) {
    if (p->margin_km >= 0.0) return p->margin_km;
    return std::fmin(10.0 * fresnel_radius(lambda_nm, p->z_pc), screen_len(p) / 4.0);
}
double diffraction_radius(const scint_params* p, double lambda_nm) {
    return p->r_diff_km * std::pow(lambda_nm / p->lambda_ref_nm, 2.0 / (p->beta - 2.0));
}
// Sampling condition of Sect. 3.2.2: the pixel must resolve the phase variations,
// Delta < R_diff(lambda) / 2.  Worst ratio 2 Delta / R_diff(lambda) over the wavelengths
// (the smallest wavelength has the smallest R_diff); >= 1 violates it.
double sampling_ratio(const scint_params* p, const double* lambdas, int n_lambda) {
    double worst = 0.0;
    for (int i = 0; i < n_lambda; ++i) worst = std::fmax(worst, 2.0 * p->pixel_km / diffraction_radius(p, lambdas[i]));
    return worst;
}
// Record a warning (the call still succeeds) when the condition is violated.
void note_sampling(const scint_params* p, const double* lambdas, int n_lambda, int item = -1) {
    int worst = 0;
    for (int i = 1; i < n_lambda; ++i)
        if (diffraction_radius(p, lambdas[i]) < diffraction_radius(p, lambdas[worst])) worst = i;
    const double rd = diffraction_radius(p, lambdas[worst]);
    if (2.0 * p->pixel_km < rd) return;
    char buf[320];
    snprintf(buf, sizeof buf,
             "%spixel %.6g km >= R_diff/2 = %.6g km at %.6g nm: the screen does not resolve its phase "
             "variations (Sect. 3.2.2 needs pixel < R_diff/2)",
             item >= 0 ? (std::string("item ") + std::to_string(item) + ": ").c_str() : "", p->pixel_km, 0.5 * rd,
             lambdas[worst]);
    g_warning = buf;
}
double refraction_radius(const scint_params* p, double lambda_nm) {
    return lz_km2(lambda_nm, p->z_pc) / diffraction_radius(p, lambda_nm);
}
double f_beta(double beta) {
    return std::pow(2.0, -beta) * beta * std::tgamma(-beta / 2.0) / std::tgamma(beta / 2.0);
}

// ---- workspace ------------------------------------------------------------------
constexpr size_t kAlign = 256;
constexpr int kRdiffRecIterations = 64;   // bisection steps for R_diff^rec (resolution L 2^-65)
size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

size_t ws_synth(int n) {
    return up((size_t)n * 16) + up((size_t)n * 8) + up((size_t)(n / 2) * (n + 4) * 16) +
           (n >= kSplitN ? up((size_t)n * n * 8) : 0) + (n <= kDrawN ? up((size_t)(n / 2 + 1) * n * 16) : 0);
}
// twiddles, the taper table per wavelength, one field per wavelength of the group, and at
// n = 16384 the column pass's column-major intensity
// (a group of g > 1 wavelengths holds fields for g rounded up to even: the packed passes
// process wavelengths in pairs)
int field_slots(int g) { return g > 1 ? (g + 1) / 2 * 2 : g; }
size_t ws_prop(int n, int g) {
    return up((size_t)n * 8) + up((size_t)g * n * 4) + up((size_t)field_slots(g) * n * n * 8) +
           (n >= kSplitN ? up((size_t)n * n * 4) : 0);
}
size_t ws_prop64(int n) { return n <= kMax64N ? up((size_t)n * 16) + up((size_t)n * n * 16) : 0; }
size_t ws_smooth(int n) {
    return up((size_t)n * 8) + up((size_t)(n / 2 + 1) * n * 8) + up(smooth_pairs_floats(n) * 4);
}
// adjoint: twiddles, g_I map, half spectrum for its disk filter, then the propagation group buffers
size_t ws_adjoint(int n, int g) {
    return up((size_t)n * n * 4) + up((size_t)(n / 2 + 1) * n * 8) + up(smooth_pairs_floats(n) * 4) + ws_prop(n, g);
}
size_t ws_moments() { return up((size_t)kMomentBlocks * 2 * sizeof(double)); }

struct Carver {
    char* base;
    size_t size, used = 0;
    template <typename T> T* take(size_t bytes) {
        T* r = reinterpret_cast<T*>(base + used);
        used += up(bytes);
        return r;
    }
};

// per-device pool used when the caller passes no workspace
struct Pool {
    std::mutex mu;
    std::vector<void*> ptr;
    std::vector<size_t> size;
};
Pool g_pool;

int pool_get(size_t bytes, cudaStream_t stream, void** out) {
    int dev = 0;
    SCINT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_pool.mu);
    if ((int)g_pool.ptr.size() <= dev) {
        g_pool.ptr.resize(dev + 1, nullptr);
        g_pool.size.resize(dev + 1, 0);
    }
    if (g_pool.size[dev] < bytes) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        SCINT_CUDA(cudaStreamIsCapturing(stream, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(SCINT_ENOMEM, "internal workspace must grow to %zu bytes during stream capture; "
                                      "pass a workspace or call once before capturing", bytes);
        if (g_pool.ptr[dev]) {
            SCINT_CUDA(cudaDeviceSynchronize());
            SCINT_CUDA(cudaFree(g_pool.ptr[dev]));
            g_pool.ptr[dev] = nullptr;
            g_pool.size[dev] = 0;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(SCINT_ENOMEM, "cudaMalloc of %zu bytes for the internal workspace failed", bytes);
        }
        g_pool.ptr[dev] = p;
        g_pool.size[dev] = bytes;
    }
    *out = g_pool.ptr[dev];
    return SCINT_OK;
}

// Resolve (workspace, bytes) against a requirement; NULL -> pool.
int resolve_ws(void* ws, size_t bytes, size_t need, cudaStream_t s, Carver* c) {
    if (!ws) {
        const int rc = pool_get(need, s, &ws);
        if (rc) return rc;
        bytes = need;
    } else if (bytes < need) {
        return fail(SCINT_ENOMEM, "workspace of %zu bytes is smaller than the %zu bytes needed", bytes, need);
    }
    if (reinterpret_cast<uintptr_t>(ws) % kAlign)
        return fail(SCINT_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    *c = Carver{static_cast<char*>(ws), bytes};
    return SCINT_OK;
}

// ---- twiddle tables kept per (device, size, kind) -----------------------------------
// A table is computed once, outside stream capture, synchronously (so every stream
// may read it at once), and kept until scint_release.  A call that is capturing and
// finds no table, or that must not allocate, computes one in its own workspace.
enum TwKind { kTw32 = 0, kTwDf = 1 };
struct TwCache {
    std::mutex mu;
    std::map<std::tuple<int, int, int>, void*> tab;
};
TwCache g_tw;

int cached_twiddles(int n, int kind, cudaStream_t s, const void** out) {
    *out = nullptr;
    int dev = 0;
    SCINT_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, n, kind);
    {
        std::lock_guard<std::mutex> lk(g_tw.mu);
        const auto it = g_tw.tab.find(key);
        if (it != g_tw.tab.end()) {
            *out = it->second;
            return SCINT_OK;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SCINT_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SCINT_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)n * (kind == kTwDf ? 16 : 8)) != cudaSuccess) {
        cudaGetLastError();
        return SCINT_OK;   // no room: the caller uses its workspace
    }
    cudaError_t e = kind == kTwDf ? launch_twiddles_df(static_cast<dfc*>(p), n, s)
                                  : launch_twiddles32(static_cast<float2*>(p), n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(p);
        return fail(SCINT_ECUDA, "twiddle table: %s", cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(g_tw.mu);
    const auto ins = g_tw.tab.emplace(key, p);
    if (!ins.second) cudaFree(p);   // another thread made it first
    *out = ins.first->second;
    return SCINT_OK;
}

// ---- kernel profiler -------------------------------------------------------------
// When enabled, every kernel launch is bracketed by two CUDA events recorded on
// its stream (they become event nodes when the stream is being captured), and
// the algorithmic bytes and FFT flops of the launch are attached.
enum KClass {
    K_TWIDDLES, K_SYNTH_ROWS, K_SYNTH_COLS, K_PROP_TABLES, K_PROP_ROWS, K_PROP_COLS,
    K_SMOOTH_FWD, K_SMOOTH_ROWS, K_SMOOTH_INV, K_LIGHTCURVE, K_MOMENTS,
    K_LC_ADJ, K_ADJ_COLS, K_ADJ_ROWS, K_DOT, K_RADIAL, K_CREC, K_CONJ_ROWS, K_CONJ_COLS, K_RESAMPLE, K_POWER, K_CORR,
    K_PROP64, K_PERSIST, K_COUNT
};
const char* const kClassName[K_COUNT] = {
    "twiddles", "synth_rows", "synth_cols", "prop_tables", "prop_rows", "prop_cols",
    "smooth_fwd_cols", "smooth_rows", "smooth_inv_cols", "lightcurve", "moments",
    "lightcurve_adjoint", "adj_cols", "adj_rows", "dot", "radial_spectrum", "structure_rec",
    "conj_rows", "conj_cols", "resample", "power_spectrum", "correlation", "prop64", "prop_persistent"};

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;
    int kernels;
};
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRec> recs;
};
Profiler g_prof;

double fft_flops(int n) { return 5.0 * n * std::log2((double)n); }   // per complex line of n points

template <typename F>
int launch_timed(KClass c, double bytes, double flops, cudaStream_t s, F&& launch, int kernels = 1) {
    bool on;
    {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        on = g_prof.on;
    }
    ProfRec r{c, nullptr, nullptr, bytes, flops, kernels};
    // while capturing, the records must be external event nodes to time graph replays
    unsigned rec_flags = cudaEventRecordDefault;
    if (on) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        SCINT_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
        SCINT_CUDA(cudaEventCreate(&r.a));
        SCINT_CUDA(cudaEventCreate(&r.b));
        SCINT_CUDA(cudaEventRecordWithFlags(r.a, s, rec_flags));
    }
    SCINT_CUDA(launch());
    if (on) {
        SCINT_CUDA(cudaEventRecordWithFlags(r.b, s, rec_flags));
        std::lock_guard<std::mutex> lk(g_prof.mu);
        g_prof.recs.push_back(r);
    }
    return SCINT_OK;
}
#define SCINT_LAUNCH(cls, bytes, flops, stream, call)                                     \
    do {                                                                                  \
        const int rc_ = launch_timed(cls, bytes, flops, stream, [&] { return (call); }); \
        if (rc_) return rc_;                                                              \
    } while (0)

// FP32 twiddles of n: the kept table, else (capturing, no room, or cache off)
// computed into the slot reserved for it in the workspace
int twiddles32(int n, bool use_cache, cudaStream_t s, float2* slot, const float2** tw) {
    const void* kept = nullptr;
    if (use_cache) {
        const int rc = cached_twiddles(n, kTw32, s, &kept);
        if (rc) return rc;
    }
    if (kept) {
        *tw = static_cast<const float2*>(kept);
        return SCINT_OK;
    }
    SCINT_LAUNCH(K_TWIDDLES, 8.0 * n, 0.0, s, launch_twiddles32(slot, n, s));
    *tw = slot;
    return SCINT_OK;
}

void prof_clear_locked() {
    for (auto& r : g_prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof.recs.clear();
}

int check_passband(const scint_params* p, const double* lambdas, const double* weights, int n_lambda) {
    const int rc = check_params(p);
    if (rc) return rc;
    if (!lambdas || n_lambda < 1 || n_lambda > SCINT_MAX_LAMBDA)
        return fail(SCINT_EINVAL, "n_lambda=%d must be in [1, %d]", n_lambda, SCINT_MAX_LAMBDA);
    for (int i = 0; i < n_lambda; ++i) {
        if (!(lambdas[i] > 0) || !std::isfinite(lambdas[i])) return fail(SCINT_EINVAL, "lambda %d must be > 0", i);
        if (weights && !std::isfinite(weights[i])) return fail(SCINT_EINVAL, "weight %d is not finite", i);
        if (taper_margin(p, lambdas[i]) > 0.5 * screen_len(p))
            return fail(SCINT_EINVAL, "taper margin exceeds half the screen");
    }
    return SCINT_OK;
}

// ---- propagation plans (variants of the transfer-function passes) ----------------
// Default: the one-wavelength passes.  Measured on GB300 (1024^2-8192^2, 8 and 32
// wavelengths), the packed passes with 16 values per thread and register twiddle bases in
// both passes are 1-4 % faster when a screen runs alone, but 2.5 % slower when eight
// screens share the GPU on the batch executor's lanes (their blocks need more shared
// memory), and the persistent batch kernel runs the one-wavelength passes only.  scint_tune
// picks a size's fastest variant alone, scint_tune_batch the fastest set for a batch.
std::mutex g_plan_mu;
std::map<std::pair<int, int>, scint_plan> g_plans;   // (device, n) -> plan

scint_plan default_plan(int n) {
    (void)n;
    scint_plan pl{};
    pl.packed = 0;
    pl.points = 16;
    pl.row_twiddles = 2;
    pl.col_twiddles = 1;
    return pl;
}

// the packed plan measured fastest alone (a tuner candidate)
scint_plan packed_plan(int n) {
    scint_plan pl = default_plan(n);
    pl.packed = packed_prop_supported(n, 16, 2, 2) ? 1 : 0;
    pl.col_twiddles = pl.packed ? 2 : 1;
    return pl;
}

int plan_for(int n, scint_plan* out) {
    int dev = 0;
    SCINT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const auto it = g_plans.find(std::make_pair(dev, n));
    *out = it != g_plans.end() ? it->second : default_plan(n);
    return SCINT_OK;
}

bool plan_known(int n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    return g_plans.count(std::make_pair(dev, n)) > 0;
}

void erase_plan(int n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.erase(std::make_pair(dev, n));
}

std::atomic<int> g_autotune{0};

int store_plan(int n, const scint_plan& pl) {
    int dev = 0;
    SCINT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[std::make_pair(dev, n)] = pl;
    return SCINT_OK;
}

// Per-wavelength scalars of the propagation passes (slot i of a group).
void fill_lambda(LambdaSet& ls, int i, const scint_params* p, double lam, double w) {
    const double L = screen_len(p);
    ls.scale_fx[i] = (uint64_t)std::llround(p->lambda_ref_nm / lam * 4294967296.0);
    ls.weight[i] = (float)w;
    ls.scale[i] = (float)(p->lambda_ref_nm / lam);
    // H_x = exp(-2 pi i c m^2), c = lambda z / (2 L^2): -frac(c) in 0.64 fixed point (52 bits kept)
    const double c = lz_km2(lam, p->z_pc) / (2.0 * L * L);
    ls.h_fx[i] = 0ull - ((uint64_t)std::llround(std::ldexp(c - std::floor(c), 52)) << 12);
}

// Propagate one wavelength group [l0, l0 + g) into the intensity map.
int run_group(const scint_params* p, const double* phi, const double* lam, const double* wts,
              int l0, int g, float* intensity, int accumulate, Carver& c, const float2* tw,
              cudaStream_t s) {
    const int n = p->n;
    static_assert(kMaxLambda >= SCINT_MAX_LAMBDA, "lambda table size");
    TableArgs ta{};
    ta.n = n;
    ta.count = g;
    PropArgs pa{};
    pa.n = n;
    pa.phi = phi;
    pa.tw = tw;
    pa.lam.count = g;
    for (int i = 0; i < g; ++i) {
        const double l = lam[l0 + i];
        ta.margin_px[i] = taper_margin(p, l) / p->pixel_km;
        fill_lambda(pa.lam, i, p, l, wts[l0 + i]);
    }
    Carver cg = c;   // group buffers restart at the same offset for every group
    ta.sf = cg.take<float>((size_t)g * n * 4);
    pa.sf = ta.sf;
    pa.work = cg.take<float2>((size_t)field_slots(g) * n * n * 8);
    pa.scratch = n >= kSplitN ? cg.take<float>((size_t)n * n * 4) : nullptr;
    pa.intensity = intensity;
    pa.accumulate = accumulate;
    pa.one = 1.0f;
    scint_plan pl{};
    int rc = plan_for(n, &pl);
    if (rc) return rc;
    const bool packed = pl.packed && g > 1 && packed_prop_supported(n, pl.points, pl.row_twiddles, pl.col_twiddles);
    const double nn = (double)n * n;
    SCINT_LAUNCH(K_PROP_TABLES, 4.0 * g * n, 0.0, s, launch_prop_tables(ta, s));
    // rows: phi read once, one complex64 field written per wavelength; FFT_x + IFFT_x per row
    SCINT_LAUNCH(K_PROP_ROWS, 8.0 * nn + 8.0 * g * nn, 2.0 * g * n * fft_flops(n), s,
                 packed ? launch_prop_rows2(pa, pl.points, pl.row_twiddles, s) : launch_prop_rows(pa, false, s));
    // columns: fields read, intensity written once (and read when accumulating)
    SCINT_LAUNCH(K_PROP_COLS, 8.0 * g * nn + (accumulate ? 8.0 : 4.0) * nn, 2.0 * g * n * fft_flops(n), s,
                 packed ? launch_prop_cols2(pa, pl.points, pl.col_twiddles, s) : launch_prop_cols(pa, false, s));
    return SCINT_OK;
}

int passband_impl(const scint_params* p, const double* phi, const double* lambdas, const double* weights,
                  int n_lambda, float* intensity, int accumulate, void* ws, size_t ws_bytes,
                  cudaStream_t s, bool keep_tables = true) {
    int rc = check_passband(p, lambdas, weights, n_lambda);
    if (rc) return rc;
    if (!phi || !intensity) return fail(SCINT_EINVAL, "phi and intensity must be device pointers");
    g_warning.clear();
    note_sampling(p, lambdas, n_lambda);
    std::vector<double> w(n_lambda, 1.0 / n_lambda);
    if (weights) w.assign(weights, weights + n_lambda);
    const int n = p->n;
    // group size: all wavelengths if the workspace allows, else the largest that fits
    int g = n_lambda;
    if (ws) {
        while (g > 1 && ws_prop(n, g) > ws_bytes) --g;
    }
    Carver c{};
    rc = resolve_ws(ws, ws_bytes, ws_prop(n, g), s, &c);
    if (rc) return rc;
    const float2* tw = nullptr;
    rc = twiddles32(n, keep_tables, s, c.take<float2>((size_t)n * 8), &tw);
    if (rc) return rc;
    for (int l0 = 0; l0 < n_lambda; l0 += g) {
        const int gg = std::min(g, n_lambda - l0);
        rc = run_group(p, phi, lambdas, w.data(), l0, gg, intensity, accumulate || l0 > 0, c, tw, s);
        if (rc) return rc;
    }
    return ok();
}

// ---- the paper's one-FFT propagator (Eq. intens, Eq. Gxy) -----------------------
double conj_pixel(const scint_params* p, double lambda_nm) {
    return lz_km2(lambda_nm, p->z_pc) / (p->n * p->pixel_km);
}
size_t ws_conj(int n, int g, bool direct) {
    return ws_prop(n, g) + (direct ? 0 : up((size_t)g * n * n * 4));
}

int conj_impl(const scint_params* p, const double* phi, const double* lambdas, const double* weights,
              int n_lambda, float* intensity, int accumulate, void* ws, size_t ws_bytes, cudaStream_t s) {
    int rc = check_passband(p, lambdas, weights, n_lambda);
    if (rc) return rc;
    if (!phi || !intensity) return fail(SCINT_EINVAL, "phi and intensity must be device pointers");
    g_warning.clear();
    note_sampling(p, lambdas, n_lambda);
    const int n = p->n;
    std::vector<double> w(n_lambda, 1.0 / n_lambda);
    if (weights) w.assign(weights, weights + n_lambda);
    // one wavelength on the output grid: the column pass writes the pattern itself
    const bool direct = n_lambda == 1 && lambdas[0] == p->lambda_nm;
    int g = n_lambda;
    if (ws) {
        while (g > 1 && ws_conj(n, g, direct) > ws_bytes) --g;
    }
    Carver c{};
    rc = resolve_ws(ws, ws_bytes, ws_conj(n, g, direct), s, &c);
    if (rc) return rc;
    const float2* tw = nullptr;
    rc = twiddles32(n, true, s, c.take<float2>((size_t)n * 8), &tw);
    if (rc) return rc;
    const double nn = (double)n * n, d1 = p->pixel_km;
    for (int l0 = 0; l0 < n_lambda; l0 += g) {
        const int gg = std::min(g, n_lambda - l0);
        TableArgs ta{};
        ta.n = n;
        ta.count = gg;
        PropArgs pa{};
        pa.n = n;
        pa.phi = phi;
        pa.tw = tw;
        pa.lam.count = gg;
        ResampleArgs ra{};
        ra.n = n;
        ra.count = gg;
        ra.intensity = intensity;
        ra.accumulate = accumulate || l0 > 0;
        for (int i = 0; i < gg; ++i) {
            const double l = lambdas[l0 + i], lz = lz_km2(l, p->z_pc);
            ta.margin_px[i] = taper_margin(p, l) / p->pixel_km;
            fill_lambda(pa.lam, i, p, l, w[l0 + i]);
            // chirp turns per pixel^2, Delta^2 / (2 lambda z), reduced mod 1 and in 0.64 fixed point
            const double c_turns = d1 * d1 / (2.0 * lz);
            const double frac = c_turns - std::floor(c_turns);
            pa.conj.chirp_fx[i] = (unsigned long long)std::llround(std::ldexp(frac, 52)) << 12;   // 1 turn wraps to 0
            pa.conj.norm[i] = (float)((d1 * d1 / lz) * (d1 * d1 / lz));
            ra.r_fx[i] = std::llround(p->lambda_nm / l * 4294967296.0);
            ra.weight[i] = (float)w[l0 + i];
        }
        Carver cg = c;
        ta.sf = cg.take<float>((size_t)gg * n * 4);
        pa.sf = ta.sf;
        pa.work = cg.take<float2>((size_t)gg * n * n * 8);
        pa.scratch = n >= kSplitN ? cg.take<float>((size_t)n * n * 4) : nullptr;
        pa.intensity = intensity;
        pa.accumulate = accumulate || l0 > 0;
        pa.conj.direct = direct ? 1 : 0;
        pa.conj.pattern = direct ? nullptr : cg.take<float>((size_t)gg * n * n * 4);
        ra.pattern = pa.conj.pattern;
        SCINT_LAUNCH(K_PROP_TABLES, 4.0 * gg * n, 0.0, s, launch_prop_tables(ta, s));
        // one FFT per row and per column and wavelength
        SCINT_LAUNCH(K_CONJ_ROWS, 8.0 * nn + 8.0 * gg * nn, 1.0 * gg * n * fft_flops(n), s,
                     launch_prop_rows(pa, true, s));
        SCINT_LAUNCH(K_CONJ_COLS, 8.0 * gg * nn + (direct ? (pa.accumulate ? 8.0 : 4.0) * nn : 4.0 * gg * nn),
                     1.0 * gg * n * fft_flops(n), s, launch_prop_cols(pa, true, s));
        if (!direct)
            SCINT_LAUNCH(K_RESAMPLE, 4.0 * gg * nn + (ra.accumulate ? 8.0 : 4.0) * nn, 0.0, s, launch_resample(ra, s));
    }
    return ok();
}

// Fiducial zone: pixel centres at least L_m + R_ref/2 + R_s from both borders
// (Sect. 3.2.1, 3.2.3); the whole map when the taper is off or the zone is
// empty.  Returns 1 when the zone exists (or the taper is off), 0 when empty.
int fiducial_zone(const scint_params* p, int* i0, int* i1) {
    const int n = p->n;
    *i0 = 0;
    *i1 = n;
    if (p->margin_km == 0.0) return 1;
    const double L = screen_len(p);
    const double m = taper_margin(p, p->lambda_nm) + 0.5 * refraction_radius(p, p->lambda_nm) + p->source_radius_km;
    int a = -1, b = -1;
    for (int i = 0; i < n; ++i) {
        const double x = (i + 0.5) * p->pixel_km;
        if (x >= m && x <= L - m) {
            if (a < 0) a = i;
            b = i;
        }
    }
    if (a < 0) return 0;
    *i0 = a;
    *i1 = b + 1;
    return 1;
}

// rms phase (rad) that the FFT bins outside the square |mx|, |my| <= K carry: the
// spectrum's variance outside the disk |q| <= K/L (a bound for the square's outside),
// 2 pi int_{K/L}^inf S(q) q dq = 2 pi C R_diff^-beta (K/L)^(2 - beta) / (beta - 2).
double outer_phase_rms(double r_diff, double beta, double L, int K) {
    const double C = r_diff * r_diff / (2.0 * std::pow(2.0 * kPi, beta - 1.0) * f_beta(beta));
    return std::sqrt(2.0 * kPi * C * std::pow(r_diff, -beta) * std::pow(K / L, 2.0 - beta) / (beta - 2.0));
}

// The FP64 square of a screen: up to 512^2 all bins; above, the smallest K in {32, 64, 128, 256} whose outside
// carries no more phase than the outside of K = 256 on the worst screen validated
// against the oracle at full size (4096^2, 10 km pixels, R_diff = 30 km, Kolmogorov:
// 2.6e-7 rad); 256 when none does.  The FP32 bins' phase error scales with that rms.
int fp64_square(const scint_params* p) {
    // up to 512^2 every bin is drawn in FP64 (the whole spectrum is the square; at most 2.6e5 bins)
    if (p->n <= kDrawN) return p->n / 2;
    static const double target = outer_phase_rms(30.0, 11.0 / 3.0, 40960.0, 256);
    const double L = screen_len(p);
    for (int K = 32; K < 256; K *= 2)
        if (outer_phase_rms(p->r_diff_km, p->beta, L, K) <= target) return K;
    return 256;
}

SynthArgs synth_args(const scint_params* p) {
    SynthArgs a{};
    a.low_k = fp64_square(p);
    const double L = screen_len(p);
    const double rd = p->r_diff_km, beta = p->beta;
    const double C = rd * rd / (2.0 * std::pow(2.0 * kPi, beta - 1.0) * f_beta(beta));
    a.n = p->n;
    a.screen_id = p->screen_id;
    a.key0 = (uint32_t)(p->seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(p->seed >> 32);
    // sigma_k = sqrt(L^2 S(q_k)) with q_k = sqrt(m2)/L, times the 1/sqrt(2) of Eq. densite
    a.amp = L * std::sqrt(C) * std::pow(rd / L, -beta / 2.0) / std::sqrt(2.0);
    a.neg_beta_4 = -beta / 4.0;
    a.amp32 = (float)a.amp;
    a.neg_beta_4_32 = (float)a.neg_beta_4;
    a.amp_rel_lo = (float)((a.amp - (double)a.amp32) / (double)a.amp32);
    a.neg_beta_4_lo = (float)(a.neg_beta_4 - (double)a.neg_beta_4_32);
    a.out_scale = std::sqrt(2.0) / (L * L);
    a.out_scale_df.hi = (float)a.out_scale;
    a.out_scale_df.lo = (float)(a.out_scale - (double)a.out_scale_df.hi);
    return a;
}

}  // namespace

// ---- helpers shared with the batch executor (csrc/batch.cu) ----------------------
namespace scint {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
int clear_error() { return ok(); }
const char* last_error() { return g_error.c_str(); }
void sampling_warning(const scint_params* p, const double* lambdas, int n_lambda, int item, bool clear) {
    if (clear) g_warning.clear();
    if (g_warning.empty()) note_sampling(p, lambdas, n_lambda, item);
}
int validate_params(const scint_params* p) { return check_params(p); }
int validate_passband(const scint_params* p, const double* lambdas, const double* weights, int n_lambda) {
    return check_passband(p, lambdas, weights, n_lambda);
}
size_t aligned_bytes(size_t b) { return up(b); }
size_t forward_workspace_bytes(int n, int g) {
    return std::max(std::max(ws_synth(n), ws_prop(n, g)), std::max(ws_smooth(n), ws_moments()));
}
int pool_workspace(size_t bytes, cudaStream_t s, void** out) { return pool_get(bytes, s, out); }
bool autotune_on() { return g_autotune.load() != 0; }
bool has_plan(int n) { return plan_known(n); }
int plan_of(int n, scint_plan* out) { return plan_for(n, out); }
int set_tuned_plan(int n, scint_plan pl, double ms) {
    pl.tuned = 1;
    pl.ms = ms;
    return store_plan(n, pl);
}
scint_plan one_wavelength_plan() {
    scint_plan pl{};
    pl.points = 16;
    pl.row_twiddles = 2;
    pl.col_twiddles = 1;
    return pl;
}
scint_plan packed_default_plan(int n) { return packed_plan(n); }

static_assert(kPersistMaxScreensHost == kPersistMaxScreens, "screen limit of the persistent launch");

bool persist_batch_supported(const int* sizes, int n) {
    if (n < 1 || n > kPersistMaxScreens) return false;
    for (int i = 0; i < n; ++i) {
        if (!persist_supported(sizes[i])) return false;
        scint_plan pl{};
        if (plan_for(sizes[i], &pl) || pl.packed) return false;   // the persistent kernel runs the unpacked bodies
    }
    return true;
}

PersistLayout persist_layout(const int* sizes, int n, int n_lambda, int n_slots) {
    PersistLayout L;
    int nmax = 0;
    for (int i = 0; i < n; ++i) nmax = std::max(nmax, sizes[i]);
    size_t off = up(kPersistCounterBytes);
    L.args = off;
    off += up((size_t)n * sizeof(PropArgs));
    L.tw = off;
    off += (size_t)n * up((size_t)nmax * 8);     // one twiddle slot per screen (used only without kept tables)
    L.sf = off;
    for (int i = 0; i < n; ++i) off += up((size_t)n_lambda * sizes[i] * 4);
    L.slots = off;
    L.slot_bytes = std::max(up((size_t)field_slots(n_lambda) * nmax * nmax * 8), forward_workspace_bytes(nmax, 1));
    off += (size_t)n_slots * L.slot_bytes;
    L.total = off;
    return L;
}

std::atomic<int> g_persist_withhold{-1};
std::atomic<int> g_persist_wait_limit{0};
void persist_testing(int withhold, int wait_limit) {
    g_persist_withhold = withhold;
    g_persist_wait_limit = wait_limit;
}

int persist_propagate(const scint_params* const* params, const double* const* phis, float* const* intensities,
                      int n, const double* lambdas, const double* weights, int n_lambda, char* ws, int n_slots,
                      int** status_out, cudaStream_t s) {
    std::vector<int> sizes(n);
    for (int i = 0; i < n; ++i) sizes[i] = params[i]->n;
    const PersistLayout L = persist_layout(sizes.data(), n, n_lambda, n_slots);
    const size_t tw_stride = up((size_t)*std::max_element(sizes.begin(), sizes.end()) * 8);
    std::vector<double> w(n_lambda, 1.0 / n_lambda);
    if (weights) w.assign(weights, weights + n_lambda);
    // largest screens first; slot k holds order positions k, k + n_slots, ...
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sizes[a] > sizes[b]; });
    PersistPlan pl{};
    pl.withhold = g_persist_withhold.load();
    const int lim = g_persist_wait_limit.load();
    pl.wait_limit = lim > 0 ? lim : (1 << 23);    // about 2 s of 200 ns pauses
    pl.screens = reinterpret_cast<const PropArgs*>(ws + L.args);
    pl.counters = reinterpret_cast<unsigned*>(ws);
    pl.status = reinterpret_cast<int*>(ws + sizeof(unsigned) * (1 + 2 * kPersistMaxScreens));
    size_t smem = 0;
    char* sf_cur = ws + L.sf;
    std::vector<char*> sf_of(n);
    for (int i = 0; i < n; ++i) {
        sf_of[i] = sf_cur;
        sf_cur += up((size_t)n_lambda * sizes[i] * 4);
    }
    SCINT_CUDA(cudaMemsetAsync(ws, 0, kPersistCounterBytes, s));
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        const scint_params* p = params[i];
        const int nn = p->n;
        smem = std::max(smem, persist_smem(nn));
        pl.slot_prev[i] = (short)(k >= n_slots ? order[k - n_slots] : -1);
        pl.row_items[i] = persist_items(nn, 0);
        pl.col_items[i] = persist_items(nn, 1);
        // the screen's arguments, exactly as run_group forms them for one group
        const float2* tw = nullptr;
        int rc = twiddles32(nn, true, s, reinterpret_cast<float2*>(ws + L.tw + (size_t)i * tw_stride), &tw);
        if (rc) return rc;
        TableArgs ta{};
        ta.n = nn;
        ta.count = n_lambda;
        PropArgs pa{};
        pa.n = nn;
        pa.phi = phis[i];
        pa.tw = tw;
        pa.lam.count = n_lambda;
        for (int l = 0; l < n_lambda; ++l) {
            ta.margin_px[l] = taper_margin(p, lambdas[l]) / p->pixel_km;
            fill_lambda(pa.lam, l, p, lambdas[l], w[l]);
        }
        ta.sf = reinterpret_cast<float*>(sf_of[i]);
        pa.sf = ta.sf;
        pa.work = reinterpret_cast<float2*>(ws + L.slots + (size_t)(k % n_slots) * L.slot_bytes);
        pa.scratch = nullptr;
        pa.intensity = intensities[i];
        pa.accumulate = 0;
        pa.one = 1.0f;
        SCINT_LAUNCH(K_PROP_TABLES, 4.0 * n_lambda * nn, 0.0, s, launch_prop_tables(ta, s));
        SCINT_CUDA(launch_persist_args(pa, reinterpret_cast<PropArgs*>(ws + L.args) + i, s));
    }
    // phases: R(o0), R(o1), C(o0), R(o2), C(o1), ..., C(o_last)
    int ph = 0, first = 0;
    auto push = [&](int scr, int pass) {
        pl.phase_screen[ph] = (short)scr;
        pl.phase_pass[ph] = (unsigned char)pass;
        pl.phase_first[ph] = first;
        first += pass == 0 ? pl.row_items[scr] : pl.col_items[scr];
        ++ph;
    };
    for (int k = 0; k < n; ++k) {
        push(order[k], 0);
        if (k >= 1) push(order[k - 1], 1);
    }
    push(order[n - 1], 1);
    pl.n_phases = ph;
    pl.phase_first[ph] = first;
    double bytes = 0.0, flops = 0.0;
    for (int i = 0; i < n; ++i) {
        const double nn = (double)sizes[i] * sizes[i];
        bytes += 8.0 * nn + 16.0 * n_lambda * nn + 4.0 * nn;
        flops += 4.0 * n_lambda * sizes[i] * fft_flops(sizes[i]);
    }
    SCINT_LAUNCH(K_PERSIST, bytes, flops, s, launch_persist_prop(pl, smem, s));
    *status_out = pl.status;
    return SCINT_OK;
}
}  // namespace scint

namespace {

// ---- propagation from a static scratch array ------------------------------------
// For callers that cannot allocate device memory themselves and cannot hand the
// library a workspace (hosts that forbid device allocation once running, such
// as fixed-budget real-time loops, or plugins inside a framework that owns all
// device memory).  Scratch lives in this fixed array instead; every GPU that
// loads the library keeps it for the life of the process.
constexpr int kStaticMaxN = 1024;
constexpr size_t kStaticScratchBytes = (size_t)8 * 1024 * 1024 + 64 * 1024;   // >= ws_prop(1024, 1)
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
std::vector<void*> g_static_addr;   // device address of g_static_scratch, per device

// The array's name in host code is only a host-side handle: its device address
// is looked up once per device, with that device current.
int static_scratch_address(void** out) {
    int dev = 0;
    SCINT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_static_mu);
    if ((int)g_static_addr.size() <= dev) g_static_addr.resize(dev + 1, nullptr);
    if (!g_static_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(SCINT_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_static_addr[dev] = ptr;
    }
    *out = g_static_addr[dev];
    return SCINT_OK;
}

}  // namespace

extern "C" {

int scint_version(void) { return 100; }

const char* scint_last_error(void) { return g_error.c_str(); }

const char* scint_last_warning(void) { return g_warning.c_str(); }

double scint_sampling_ratio(const scint_params* p, const double* lambdas_nm, int n_lambda) {
    if (check_params(p)) return -1.0;
    if (!lambdas_nm || n_lambda <= 0) return sampling_ratio(p, &p->lambda_nm, 1);
    for (int i = 0; i < n_lambda; ++i)
        if (!(lambdas_nm[i] > 0) || !std::isfinite(lambdas_nm[i])) {
            fail(SCINT_EINVAL, "lambda %d must be > 0", i);
            return -1.0;
        }
    ok();
    return sampling_ratio(p, lambdas_nm, n_lambda);
}

size_t scint_workspace_bytes(const scint_params* p, int n_lambda) {
    if (check_params(p) || n_lambda < 1) return 0;
    const int n = p->n;
    size_t b = ws_synth(n);
    b = std::max(b, ws_prop(n, std::min(n_lambda, SCINT_MAX_LAMBDA)));
    b = std::max(b, ws_smooth(n));
    b = std::max(b, ws_moments());
    b = std::max(b, ws_adjoint(n, std::min(n_lambda, SCINT_MAX_LAMBDA)));
    b = std::max(b, ws_prop64(n));
    return b;
}

int scint_make_screen(const scint_params* p, double* phi, void* workspace, size_t workspace_bytes,
                      void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!phi) return fail(SCINT_EINVAL, "phi must be a device pointer");
    if (reinterpret_cast<uintptr_t>(phi) % 16) return fail(SCINT_EINVAL, "phi must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    rc = resolve_ws(workspace, workspace_bytes, ws_synth(p->n), s, &c);
    if (rc) return rc;
    SynthArgs a = synth_args(p);
    dfc* tw_slot = c.take<dfc>((size_t)p->n * 16);
    const void* kept = nullptr;
    rc = cached_twiddles(p->n, kTwDf, s, &kept);
    if (rc) return rc;
    a.tw = kept ? static_cast<const dfc*>(kept) : tw_slot;
    float2* tw32_slot = c.take<float2>((size_t)p->n * 8);
    a.work = c.take<dfc>((size_t)(p->n / 2) * (p->n + 4) * 16);
    a.pairs = p->n >= kSplitN ? c.take<double2>((size_t)p->n * p->n * 8) : nullptr;
    a.drawn = p->n <= kDrawN ? c.take<dfc>((size_t)(p->n / 2 + 1) * p->n * 16) : nullptr;
    a.phi = phi;
    const double nn = (double)p->n * p->n;
    if (!kept) SCINT_LAUNCH(K_TWIDDLES, 16.0 * p->n, 0.0, s, launch_twiddles_df(tw_slot, p->n, s));
    rc = twiddles32(p->n, true, s, tw32_slot, &a.tw32);
    if (rc) return rc;
    const double half = (double)(p->n / 2 + 1) * p->n * 16.0;
    // rows: the noise is generated in registers, rows 0..n/2 of the x-transformed field are written
    SCINT_LAUNCH(K_SYNTH_ROWS, half, (p->n / 2 + 1) * fft_flops(p->n), s, launch_synth_rows(a, s));
    // columns: two real columns per complex transform (at n >= kSplitN through a column-major
    // scratch and a transpose, timed with the pass)
    SCINT_LAUNCH(K_SYNTH_COLS, half + 8.0 * nn, (p->n / 2) * fft_flops(p->n), s, launch_synth_cols(a, s));
    return ok();
}

int scint_propagate(const scint_params* p, const double* phi, float* intensity, void* workspace,
                    size_t workspace_bytes, void* stream) {
    if (!p) return fail(SCINT_EINVAL, "params is NULL");
    const double lam = p->lambda_nm, w = 1.0;
    return passband_impl(p, phi, &lam, &w, 1, intensity, 0, workspace, workspace_bytes,
                         static_cast<cudaStream_t>(stream));
}

int scint_propagate64(const scint_params* p, const double* phi, double* intensity, void* workspace,
                      size_t workspace_bytes, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!phi || !intensity) return fail(SCINT_EINVAL, "phi and intensity must be device pointers");
    if (p->n > kMax64N)
        return fail(SCINT_EUNSUPPORTED, "scint_propagate64 supports n <= %d (n=%d)", kMax64N, p->n);
    const double lam = p->lambda_nm;
    rc = check_passband(p, &lam, nullptr, 1);
    if (rc) return rc;
    g_warning.clear();
    note_sampling(p, &lam, 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    rc = resolve_ws(workspace, workspace_bytes, ws_prop64(p->n), s, &c);
    if (rc) return rc;
    Prop64Args a{};
    a.n = p->n;
    a.phi = phi;
    double2* tw = c.take<double2>((size_t)p->n * 16);
    a.tw = tw;
    a.field = c.take<double2>((size_t)p->n * p->n * 16);
    a.intensity = intensity;
    a.scale = p->lambda_ref_nm / lam;
    a.margin_px = taper_margin(p, lam) / p->pixel_km;
    const double L = screen_len(p);
    const double cc = lz_km2(lam, p->z_pc) / (2.0 * L * L);
    const double cf = cc - std::floor(cc);
    a.c_hi = std::ldexp(std::nearbyint(std::ldexp(cf, 31)), -31);
    a.c_lo = cf - a.c_hi;
    const double nn = (double)p->n * p->n;
    SCINT_LAUNCH(K_TWIDDLES, 16.0 * p->n, 0.0, s, launch_twiddles64(tw, p->n, s));
    // rows: phi read, complex128 field written; columns: field read, FP64 map written
    SCINT_LAUNCH(K_PROP64, 8.0 * nn + 16.0 * nn + 16.0 * nn + 8.0 * nn, 4.0 * p->n * fft_flops(p->n), s,
                 launch_prop64(a, s));
    return ok();
}

int scint_propagate_noalloc(const scint_params* p, const double* phi, float* intensity, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (p->n > kStaticMaxN || ws_prop(p->n, 1) > kStaticScratchBytes)
        return fail(SCINT_EINVAL, "n=%d exceeds the static scratch limit n <= %d (%zu bytes) of "
                                  "scint_propagate_noalloc; use scint_propagate with a workspace",
                    p->n, kStaticMaxN, kStaticScratchBytes);
    void* scratch = nullptr;
    rc = static_scratch_address(&scratch);
    if (rc) return rc;
    // Everything in the scratch (twiddles, tables, field) is written before it is
    // read, so stale contents from the previous call need no clearing.
    const double lam = p->lambda_nm, w = 1.0;
    return passband_impl(p, phi, &lam, &w, 1, intensity, 0, scratch, kStaticScratchBytes,
                         static_cast<cudaStream_t>(stream), false);
}

int scint_autotune(int on) { return g_autotune.exchange(on ? 1 : 0); }

int scint_get_plan(int n, scint_plan* out) {
    if (!out) return fail(SCINT_EINVAL, "out is NULL");
    if (!pow2(n) || n < SCINT_MIN_N || n > SCINT_MAX_N)
        return fail(SCINT_EINVAL, "n=%d must be a power of two in [%d, %d]", n, SCINT_MIN_N, SCINT_MAX_N);
    const int rc = plan_for(n, out);
    return rc ? rc : ok();
}

int scint_set_plan(int n, const scint_plan* plan) {
    if (!plan) return fail(SCINT_EINVAL, "plan is NULL");
    if (!pow2(n) || n < SCINT_MIN_N || n > SCINT_MAX_N)
        return fail(SCINT_EINVAL, "n=%d must be a power of two in [%d, %d]", n, SCINT_MIN_N, SCINT_MAX_N);
    const bool tw_ok = (plan->row_twiddles == 1 || plan->row_twiddles == 2) &&
                       (plan->col_twiddles == 1 || plan->col_twiddles == 2);
    if ((plan->packed != 0 && plan->packed != 1) || !tw_ok || (plan->points != 8 && plan->points != 16) ||
        plan->reserved)
        return fail(SCINT_EINVAL, "packed must be 0 or 1, points 8 or 16, the twiddle sources 1 or 2, "
                                  "reserved 0");
    if (plan->packed && !packed_prop_supported(n, plan->points, plan->row_twiddles, plan->col_twiddles))
        return fail(SCINT_EUNSUPPORTED, "the packed passes with %d points per thread and twiddle sources (%d, %d) "
                                        "are not built for n=%d", plan->points, plan->row_twiddles,
                    plan->col_twiddles, n);
    scint_plan pl = *plan;
    pl.tuned = 0;
    pl.ms = 0.0;
    const int rc = store_plan(n, pl);
    return rc ? rc : ok();
}

int scint_tune(int n, int n_lambda, scint_plan* out, void* stream) {
    if (!pow2(n) || n < SCINT_MIN_N || n > SCINT_MAX_N)
        return fail(SCINT_EINVAL, "n=%d must be a power of two in [%d, %d]", n, SCINT_MIN_N, SCINT_MAX_N);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SCINT_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return fail(SCINT_EINVAL, "scint_tune cannot run during stream capture");
    std::vector<scint_plan> cand;
    scint_plan one{};
    one.points = 16;
    one.row_twiddles = 2;
    one.col_twiddles = 1;
    cand.push_back(one);     // the one-wavelength passes
    for (int pts : {16, 8})
        for (int r = 1; r <= 2; ++r)
            for (int c = 1; c <= 2; ++c)
                if (packed_prop_supported(n, pts, r, c)) cand.push_back(scint_plan{1, pts, r, c, 0, 0, 0.0});
    // test passband: n_lambda in [2, 32], fields within 1 GiB
    int g = std::max(2, std::min(n_lambda, 32));
    const size_t field = (size_t)n * n * 8;
    while (g > 2 && (size_t)field_slots(g) * field > ((size_t)1 << 30)) --g;
    scint_plan best = cand[0];
    best.ms = 0.0;
    const bool had = plan_known(n);
    scint_plan prev{};
    if (had) plan_for(n, &prev);
    if (cand.size() > 1) {
        const size_t wsb = ws_prop(n, g);
        void *phi = nullptr, *inten = nullptr, *ws = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        auto cleanup = [&] {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            cudaFree(phi);
            cudaFree(inten);
            cudaFree(ws);
        };
        if (cudaMalloc(&phi, field) != cudaSuccess || cudaMalloc(&inten, (size_t)n * n * 4) != cudaSuccess ||
            cudaMalloc(&ws, wsb) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(SCINT_ENOMEM, "scint_tune: cudaMalloc of its test buffers failed");
        }
        if (cudaMemsetAsync(phi, 0, field, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(SCINT_ECUDA, "scint_tune: setting up its test buffers failed");
        }
        scint_params p{};
        p.n = n;
        p.pixel_km = 10.0;
        p.r_diff_km = 100.0 * n;   // resolved at every test wavelength
        p.beta = 11.0 / 3.0;
        p.lambda_nm = p.lambda_ref_nm = 550.0;
        p.z_pc = 160.0;
        p.margin_km = -1.0;
        std::vector<double> lams(g), wts(g, 1.0 / g);
        for (int i = 0; i < g; ++i) lams[i] = 400.0 + 300.0 * i / (g - 1);
        double best_ms = 1e300;
        int rc = SCINT_OK;
        for (const scint_plan& c : cand) {
            if ((rc = store_plan(n, c))) break;
            double t = 1e300;
            for (int rep = 0; rep < 4 && !rc; ++rep) {
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = fail(SCINT_ECUDA, "scint_tune: event record");
                if (!rc) rc = passband_impl(&p, static_cast<const double*>(phi), lams.data(), wts.data(), g,
                                            static_cast<float*>(inten), 0, ws, wsb, s);
                if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                    rc = fail(SCINT_ECUDA, "scint_tune: timing");
                float ms = 0.0f;
                if (!rc && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t = std::min(t, (double)ms);
            }
            if (rc) break;
            if (t < best_ms) {
                best_ms = t;
                best = c;
                best.ms = t;
            }
        }
        cleanup();
        if (rc) {   // leave the plan as it was
            if (had) store_plan(n, prev);
            else erase_plan(n);
            return rc;
        }
    }
    best.tuned = 1;
    const int rc = store_plan(n, best);
    if (rc) return rc;
    if (out) *out = best;
    g_warning.clear();
    return ok();
}

double scint_conjugate_pixel_km(const scint_params* p, double lambda_nm) {
    if (check_params(p) || !(lambda_nm > 0) || !std::isfinite(lambda_nm)) return std::nan("");
    return conj_pixel(p, lambda_nm);
}

int scint_propagate_conjugate(const scint_params* p, const double* phi, float* intensity, void* workspace,
                              size_t workspace_bytes, void* stream) {
    if (!p) return fail(SCINT_EINVAL, "params is NULL");
    const double lam = p->lambda_nm, w = 1.0;
    return conj_impl(p, phi, &lam, &w, 1, intensity, 0, workspace, workspace_bytes,
                     static_cast<cudaStream_t>(stream));
}

int scint_sum_passband_conjugate(const scint_params* p, const double* phi, const double* lambdas_nm,
                                 const double* weights, int n_lambda, float* intensity, int accumulate,
                                 void* workspace, size_t workspace_bytes, void* stream) {
    return conj_impl(p, phi, lambdas_nm, weights, n_lambda, intensity, accumulate, workspace, workspace_bytes,
                     static_cast<cudaStream_t>(stream));
}

int scint_sum_passband(const scint_params* p, const double* phi, const double* lambdas_nm,
                       const double* weights, int n_lambda, float* intensity, int accumulate,
                       void* workspace, size_t workspace_bytes, void* stream) {
    return passband_impl(p, phi, lambdas_nm, weights, n_lambda, intensity, accumulate, workspace,
                         workspace_bytes, static_cast<cudaStream_t>(stream));
}

int scint_smooth_source(const scint_params* p, float* intensity, void* workspace, size_t workspace_bytes,
                        void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!intensity) return fail(SCINT_EINVAL, "intensity must be a device pointer");
    if (p->source_radius_km == 0.0) return ok();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    rc = resolve_ws(workspace, workspace_bytes, ws_smooth(p->n), s, &c);
    if (rc) return rc;
    SmoothArgs a{};
    a.n = p->n;
    a.radius_over_L = p->source_radius_km / screen_len(p);
    float2* tw_slot = c.take<float2>((size_t)p->n * 8);
    a.spec = c.take<float2>((size_t)(p->n / 2 + 1) * p->n * 8);
    a.pairs = smooth_pairs_floats(p->n) ? c.take<float2>(smooth_pairs_floats(p->n) * 4) : nullptr;
    a.intensity = intensity;
    const int n = p->n;
    const double half = (double)(n / 2 + 1) * n * 8.0, nn = (double)n * n;
    rc = twiddles32(n, true, s, tw_slot, &a.tw);
    if (rc) return rc;
    SCINT_LAUNCH(K_SMOOTH_FWD, 4.0 * nn + half, (n / 2) * fft_flops(n), s, launch_smooth_pass(a, 0, s));
    SCINT_LAUNCH(K_SMOOTH_ROWS, 2.0 * half, 2.0 * (n / 2 + 1) * fft_flops(n), s, launch_smooth_pass(a, 1, s));
    SCINT_LAUNCH(K_SMOOTH_INV, half + 4.0 * nn, (n / 2) * fft_flops(n), s, launch_smooth_pass(a, 2, s));
    return ok();
}

int scint_lightcurve(const scint_params* p, const float* intensity, const double* tracks, int n_tracks,
                     int n_samples, float* curves, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (n_tracks < 0 || n_samples < 0) return fail(SCINT_EINVAL, "negative track or sample count");
    if (n_tracks == 0 || n_samples == 0) return ok();   // nothing to sample: pointers may be NULL
    if (!intensity || !curves) return fail(SCINT_EINVAL, "intensity and curves must be device pointers");
    if (n_tracks > 0 && !tracks) return fail(SCINT_EINVAL, "tracks is NULL");
    for (int i = 0; i < 4 * n_tracks; ++i)
        if (!std::isfinite(tracks[i])) return fail(SCINT_EINVAL, "track parameters must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int t0 = 0; t0 < n_tracks; t0 += kTracksPerLaunch) {
        CurveArgs a{};
        a.n = p->n;
        a.n_tracks = std::min(kTracksPerLaunch, n_tracks - t0);
        a.n_samples = n_samples;
        a.intensity = intensity;
        a.curves = curves + (size_t)t0 * n_samples;
        for (int i = 0; i < a.n_tracks; ++i) {
            const double* tr = tracks + 4 * (t0 + i);
            a.tr[i] = Track{tr[0], tr[1], std::cos(tr[2]), std::sin(tr[2]), tr[3]};
        }
        SCINT_LAUNCH(K_LIGHTCURVE, 20.0 * a.n_tracks * (double)n_samples, 0.0, s, launch_lightcurve(a, s));
    }
    return ok();
}

int scint_modulation_index(const scint_params* p, const float* intensity, double* out, void* workspace,
                           size_t workspace_bytes, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!intensity || !out) return fail(SCINT_EINVAL, "intensity and out must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    rc = resolve_ws(workspace, workspace_bytes, ws_moments(), s, &c);
    if (rc) return rc;
    const int n = p->n;
    int i0 = 0, i1 = n;
    fiducial_zone(p, &i0, &i1);
    double* partial = c.take<double>((size_t)kMomentBlocks * 2 * sizeof(double));
    // two kernels: per-block partial sums, then the final reduction
    const int rc2 = launch_timed(K_MOMENTS, 4.0 * (double)(i1 - i0) * (i1 - i0), 0.0, s,
                                 [&] { return launch_map_moments(intensity, n, i0, i1, i0, i1, partial, out, s); }, 2);
    if (rc2) return rc2;
    return ok();
}

int scint_curve_power_spectrum(const float* curves, int n_curves, int n_samples, float* power, void* workspace,
                               size_t workspace_bytes, void* stream) {
    if (n_curves < 0) return fail(SCINT_EINVAL, "n_curves must be >= 0");
    if (!pow2(n_samples) || n_samples < SCINT_MIN_N || n_samples > 8192)
        return fail(SCINT_EINVAL, "n_samples=%d must be a power of two in [%d, 8192]", n_samples, SCINT_MIN_N);
    if (n_curves == 0) return ok();
    if (!curves || !power) return fail(SCINT_EINVAL, "curves and power must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    int rc = resolve_ws(workspace, workspace_bytes, up((size_t)n_samples * 8), s, &c);
    if (rc) return rc;
    const float2* tw = nullptr;
    rc = twiddles32(n_samples, true, s, c.take<float2>((size_t)n_samples * 8), &tw);
    if (rc) return rc;
    SCINT_LAUNCH(K_POWER, 4.0 * n_curves * (double)n_samples + 4.0 * n_curves * (n_samples / 2 + 1),
                 n_curves * fft_flops(n_samples), s, launch_power_spectrum(curves, n_curves, n_samples, power, tw, s));
    return ok();
}

int scint_curve_correlation(const float* a, int a_rows, int64_t a_stride, const float* b, int n_pairs,
                            int n_samples, double* r, void* stream) {
    if (n_pairs < 0 || n_samples < 2) return fail(SCINT_EINVAL, "need n_pairs >= 0 and n_samples >= 2");
    if (n_pairs == 0) return ok();
    if (a_rows < 1 || n_pairs % a_rows) return fail(SCINT_EINVAL, "a_rows=%d must divide n_pairs=%d", a_rows, n_pairs);
    if (a_rows > 1 && a_stride < n_samples) return fail(SCINT_EINVAL, "a_stride must be >= n_samples");
    if (!a || !b || !r) return fail(SCINT_EINVAL, "a, b and r must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SCINT_LAUNCH(K_CORR, 4.0 * (double)n_samples * (n_pairs + a_rows) + 8.0 * n_pairs, 0.0, s,
                 launch_correlation(a, a_rows, a_stride, b, n_pairs, n_samples, r, s));
    return ok();
}

int scint_fiducial_zone(const scint_params* p, int32_t* i0, int32_t* i1, double* r_ref_km) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!i0 || !i1) return fail(SCINT_EINVAL, "i0 and i1 must be host pointers");
    int a = 0, b = 0;
    const int has = fiducial_zone(p, &a, &b);
    *i0 = a;
    *i1 = b;
    if (r_ref_km) *r_ref_km = refraction_radius(p, p->lambda_nm);
    if (!has) return fail(SCINT_EUNSUPPORTED, "the fiducial zone is empty (margin exceeds half the screen)");
    return ok();
}

int scint_curve_modulation(const float* curves, int n_curves, int n_samples, double* out, void* stream) {
    if (n_curves < 0 || n_samples < 1) return fail(SCINT_EINVAL, "need n_curves >= 0 and n_samples >= 1");
    if (n_curves > 0 && (!curves || !out)) return fail(SCINT_EINVAL, "curves and out must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SCINT_LAUNCH(K_MOMENTS, 4.0 * (double)n_curves * n_samples, 0.0, s,
                 launch_curve_moments(curves, n_curves, n_samples, out, s));
    return ok();
}

int scint_lightcurve_adjoint(const scint_params* p, const double* phi, const double* lambdas_nm,
                             const double* weights, int n_lambda, const double* tracks, int n_tracks,
                             int n_samples, const float* grad_curves, double* grad_phi, int accumulate,
                             void* workspace, size_t workspace_bytes, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!phi || !grad_phi) return fail(SCINT_EINVAL, "phi and grad_phi must be device pointers");
    if (!lambdas_nm || n_lambda < 1 || n_lambda > SCINT_MAX_LAMBDA)
        return fail(SCINT_EINVAL, "n_lambda=%d must be in [1, %d]", n_lambda, SCINT_MAX_LAMBDA);
    if (n_tracks < 0 || n_samples < 0) return fail(SCINT_EINVAL, "negative track or sample count");
    if (n_tracks > 0 && n_samples > 0 && (!tracks || !grad_curves))
        return fail(SCINT_EINVAL, "tracks (host) and grad_curves (device) are required");
    for (int i = 0; i < 4 * n_tracks && n_samples > 0; ++i)
        if (!std::isfinite(tracks[i])) return fail(SCINT_EINVAL, "track parameters must be finite");
    std::vector<double> w(n_lambda, 1.0 / n_lambda);
    for (int i = 0; i < n_lambda; ++i) {
        if (!(lambdas_nm[i] > 0) || !std::isfinite(lambdas_nm[i])) return fail(SCINT_EINVAL, "lambda %d must be > 0", i);
        if (weights) {
            if (!std::isfinite(weights[i])) return fail(SCINT_EINVAL, "weight %d is not finite", i);
            w[i] = weights[i];
        }
        if (taper_margin(p, lambdas_nm[i]) > 0.5 * screen_len(p))
            return fail(SCINT_EINVAL, "taper margin exceeds half the screen");
    }
    g_warning.clear();
    note_sampling(p, lambdas_nm, n_lambda);
    const int n = p->n;
    int g = n_lambda;
    if (workspace) {
        while (g > 1 && ws_adjoint(n, g) > workspace_bytes) --g;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    rc = resolve_ws(workspace, workspace_bytes, ws_adjoint(n, g), s, &c);
    if (rc) return rc;
    float* gmap = c.take<float>((size_t)n * n * 4);
    float2* spec = c.take<float2>((size_t)(n / 2 + 1) * n * 8);
    float2* spairs = smooth_pairs_floats(n) ? c.take<float2>(smooth_pairs_floats(n) * 4) : nullptr;
    Carver cp = c;                       // propagation buffers: twiddles, then group tables and fields
    const float2* tw = nullptr;
    rc = twiddles32(n, true, s, cp.take<float2>((size_t)n * 8), &tw);
    if (rc) return rc;
    const double nn = (double)n * n;
    // g_I = B^T g_c
    SCINT_CUDA(cudaMemsetAsync(gmap, 0, (size_t)n * n * 4, s));
    for (int t0 = 0; t0 < n_tracks && n_samples > 0; t0 += kTracksPerLaunch) {
        CurveAdjArgs a{};
        a.n = n;
        a.n_tracks = std::min(kTracksPerLaunch, n_tracks - t0);
        a.n_samples = n_samples;
        a.grad_curves = grad_curves + (size_t)t0 * n_samples;
        a.grad_map = gmap;
        for (int i = 0; i < a.n_tracks; ++i) {
            const double* tr = tracks + 4 * (t0 + i);
            a.tr[i] = Track{tr[0], tr[1], std::cos(tr[2]), std::sin(tr[2]), tr[3]};
        }
        SCINT_LAUNCH(K_LC_ADJ, 20.0 * a.n_tracks * (double)n_samples, 0.0, s, launch_lightcurve_adjoint(a, s));
    }
    // the disk filter is real and even, hence self-adjoint
    if (p->source_radius_km > 0.0) {
        SmoothArgs sa{};
        sa.n = n;
        sa.radius_over_L = p->source_radius_km / screen_len(p);
        sa.tw = tw;
        sa.spec = spec;
        sa.pairs = spairs;
        sa.intensity = gmap;
        const double half = (double)(n / 2 + 1) * n * 8.0;
        SCINT_LAUNCH(K_SMOOTH_FWD, 4.0 * nn + half, (n / 2) * fft_flops(n), s, launch_smooth_pass(sa, 0, s));
        SCINT_LAUNCH(K_SMOOTH_ROWS, 2.0 * half, 2.0 * (n / 2 + 1) * fft_flops(n), s, launch_smooth_pass(sa, 1, s));
        SCINT_LAUNCH(K_SMOOTH_INV, half + 4.0 * nn, (n / 2) * fft_flops(n), s, launch_smooth_pass(sa, 2, s));
    }
    for (int l0 = 0; l0 < n_lambda; l0 += g) {
        const int gg = std::min(g, n_lambda - l0);
        TableArgs ta{};
        ta.n = n;
        ta.count = gg;
        PropArgs pa{};
        pa.n = n;
        pa.phi = phi;
        pa.tw = tw;
        pa.lam.count = gg;
        for (int i = 0; i < gg; ++i) {
            const double l = lambdas_nm[l0 + i];
            ta.margin_px[i] = taper_margin(p, l) / p->pixel_km;
            fill_lambda(pa.lam, i, p, l, w[l0 + i]);
        }
        Carver cg = cp;
        ta.sf = cg.take<float>((size_t)gg * n * 4);
        pa.sf = ta.sf;
        pa.work = cg.take<float2>((size_t)gg * n * n * 8);
        AdjArgs aa{};
        aa.n = n;
        aa.phi = phi;
        aa.tw = tw;
        aa.sf = ta.sf;
        aa.work = pa.work;
        aa.grad_map = gmap;
        aa.grad_phi = grad_phi;
        aa.accumulate = accumulate || l0 > 0;
        aa.lam = pa.lam;
        SCINT_LAUNCH(K_PROP_TABLES, 4.0 * gg * n, 0.0, s, launch_prop_tables(ta, s));
        SCINT_LAUNCH(K_PROP_ROWS, 8.0 * nn + 8.0 * gg * nn, 2.0 * gg * n * fft_flops(n), s, launch_prop_rows(pa, false, s));
        SCINT_LAUNCH(K_ADJ_COLS, 16.0 * gg * nn + 4.0 * nn, 4.0 * gg * n * fft_flops(n), s, launch_adj_cols(aa, s));
        SCINT_LAUNCH(K_ADJ_ROWS, 8.0 * gg * nn + 8.0 * nn + (aa.accumulate ? 16.0 : 8.0) * nn,
                     2.0 * gg * n * fft_flops(n), s, launch_adj_rows(aa, s));
    }
    return ok();
}

int scint_rdiff_gradient(const scint_params* p, const double* phi, const double* grad_phi, double* out,
                         void* workspace, size_t workspace_bytes, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!phi || !grad_phi || !out) return fail(SCINT_EINVAL, "phi, grad_phi and out must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c{};
    rc = resolve_ws(workspace, workspace_bytes, ws_moments(), s, &c);
    if (rc) return rc;
    double* partial = c.take<double>((size_t)kMomentBlocks * 2 * sizeof(double));
    const long long nn = (long long)p->n * p->n;
    // phi ~ R_diff^((2 - beta)/2) at a fixed seed
    const double scale = (2.0 - p->beta) / (2.0 * p->r_diff_km);
    SCINT_LAUNCH(K_DOT, 16.0 * (double)nn, 0.0, s, launch_scaled_dot(phi, grad_phi, nn, scale, partial, out, s));
    return ok();
}

// ---- screen check of Sect. 3.1.1 ------------------------------------------------
namespace {
int check_screen_check_params(const scint_params* p) {
    if (!p) return fail(SCINT_EINVAL, "params is NULL");
    if (p->n < SCINT_MIN_N || p->n > SCINT_MAX_CHECK_N || (p->n & 1))
        return fail(SCINT_EINVAL, "n=%d must be even in [%d, %d]", p->n, SCINT_MIN_N, SCINT_MAX_CHECK_N);
    if (p->reserved0 || p->reserved1) return fail(SCINT_EINVAL, "reserved fields must be 0");
    if (!(p->pixel_km > 0) || !std::isfinite(p->pixel_km)) return fail(SCINT_EINVAL, "pixel_km must be > 0");
    if (!(p->r_diff_km > 0) || !std::isfinite(p->r_diff_km)) return fail(SCINT_EINVAL, "r_diff_km must be > 0");
    if (!(p->beta > 2.0 && p->beta < 4.0)) return fail(SCINT_EINVAL, "beta=%g must be in (2, 4)", p->beta);
    return SCINT_OK;
}
int max_annulus(int n) { return (int)std::floor(std::sqrt(2.0 * (double)(n / 2) * (n / 2)) + 0.5); }
}  // namespace

int scint_spectrum_rec(const scint_params* p, double* s_rec, uint64_t* counts, int n_bins, void* stream) {
    int rc = check_screen_check_params(p);
    if (rc) return rc;
    if (n_bins < 1) return fail(SCINT_EINVAL, "n_bins=%d must be >= 1", n_bins);
    if (!s_rec || !counts) return fail(SCINT_EINVAL, "s_rec and counts must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_hist = std::min(n_bins, max_annulus(p->n) + 1);
    int dev = 0, sms = 0;
    SCINT_CUDA(cudaGetDevice(&dev));
    SCINT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t hist_bytes = (size_t)n_hist * sizeof(uint64_t);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(200 * 1024) / hist_bytes));
    const int blocks = std::min(p->n, sms * per_sm);
    SCINT_CUDA(cudaMemsetAsync(s_rec, 0, (size_t)n_bins * sizeof(double), s));
    SCINT_CUDA(cudaMemsetAsync(counts, 0, (size_t)n_bins * sizeof(uint64_t), s));
    SynthArgs a = synth_args(p);
    const double L = screen_len(p);
    // three kernels: bin counts, |F|^2 sums, normalisation; only the histograms touch memory
    rc = launch_timed(K_RADIAL, 16.0 * n_hist * 2, 0.0, s, [&] {
        return launch_radial_spectrum(a, 1.0 / (L * L), n_hist, s_rec, reinterpret_cast<unsigned long long*>(counts),
                                      blocks, s);
    }, 3);
    if (rc) return rc;
    return ok();
}

int scint_structure_function_rec(const scint_params* p, const double* s_rec, int n_bins, const double* r_km,
                                 int n_r, double* d_rec, double* r_rec, void* workspace, size_t workspace_bytes,
                                 void* stream) {
    int rc = check_screen_check_params(p);
    if (rc) return rc;
    if (n_bins < 2 || !s_rec) return fail(SCINT_EINVAL, "need s_rec with n_bins >= 2");
    if (n_r < 0 || (n_r > 0 && (!r_km || !d_rec))) return fail(SCINT_EINVAL, "r_km and d_rec must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CrecArgs a{};
    a.s = s_rec;
    a.J = std::min(n_bins - 1, p->n / 2);
    a.dq = 1.0 / screen_len(p);
    a.half_L = 0.5 * screen_len(p);
    if (n_r > 0) SCINT_LAUNCH(K_CREC, 8.0 * (a.J + n_r), 0.0, s, launch_crec(a, r_km, n_r, d_rec, s));
    if (r_rec) {
        Carver c{};
        rc = resolve_ws(workspace, workspace_bytes, up(sizeof(BisectState)), s, &c);
        if (rc) return rc;
        BisectState* st = c.take<BisectState>(sizeof(BisectState));
        const int rc2 = launch_timed(K_CREC, 8.0 * a.J, 0.0, s,
                                     [&] { return launch_bisect(a, st, kRdiffRecIterations, r_rec, s); },
                                     kRdiffRecIterations + 1);
        if (rc2) return rc2;
    }
    return ok();
}

int scint_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    prof_clear_locked();
    g_prof.on = on != 0;
    return ok();
}

int scint_profile_read(scint_kernel_stat* stats, int max_stats, int* n_stats) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    scint_kernel_stat acc[K_COUNT];
    memset(acc, 0, sizeof acc);
    for (int c = 0; c < K_COUNT; ++c) snprintf(acc[c].name, sizeof acc[c].name, "%s", kClassName[c]);
    for (auto& r : g_prof.recs) {
        float ms = 0.0f;
        const cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return fail(SCINT_ECUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
        const cudaError_t e2 = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e2 != cudaSuccess) return fail(SCINT_ECUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e2));
        acc[r.cls].launches += r.kernels;
        acc[r.cls].total_ms += ms;
        acc[r.cls].bytes += r.bytes;
        acc[r.cls].flops += r.flops;
    }
    int k = 0;
    for (int c = 0; c < K_COUNT; ++c)
        if (acc[c].launches && k < max_stats) stats[k++] = acc[c];
    if (n_stats) *n_stats = k;
    return ok();
}

void scint_release(void) {
    scint::release_lanes();
    {
        // a device reset would invalidate them; the next noalloc call looks them up again
        std::lock_guard<std::mutex> lk(g_static_mu);
        g_static_addr.clear();
    }
    {
        std::lock_guard<std::mutex> lk(g_tw.mu);
        int cur = 0;
        cudaGetDevice(&cur);
        for (auto& kv : g_tw.tab) {
            cudaSetDevice(std::get<0>(kv.first));
            cudaDeviceSynchronize();
            cudaFree(kv.second);
        }
        g_tw.tab.clear();
        cudaSetDevice(cur);
    }
    std::lock_guard<std::mutex> lk(g_pool.mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_pool.ptr.size(); ++d) {
        if (g_pool.ptr[d]) {
            cudaSetDevice((int)d);
            cudaDeviceSynchronize();
            cudaFree(g_pool.ptr[d]);
            g_pool.ptr[d] = nullptr;
            g_pool.size[d] = 0;
        }
    }
    cudaSetDevice(cur);
}

// ---- inspection entry points ----------------------------------------------------
int scint_noise_words(const scint_params* p, uint32_t* words, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!words) return fail(SCINT_EINVAL, "words must be a device pointer");
    SCINT_CUDA(launch_noise_words(p->n, p->screen_id, (uint32_t)(p->seed & 0xFFFFFFFFu),
                                  (uint32_t)(p->seed >> 32), words, static_cast<cudaStream_t>(stream)));
    return ok();
}

int scint_noise_spectrum(const scint_params* p, double* F, void* stream) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!F) return fail(SCINT_EINVAL, "F must be a device pointer");
    SCINT_CUDA(launch_noise_spectrum(synth_args(p), reinterpret_cast<double2*>(F),
                                     static_cast<cudaStream_t>(stream)));
    return ok();
}

int scint_phase_fixed(const double* phi, int64_t* P, int64_t n, void* stream) {
    if (n < 0) return fail(SCINT_EINVAL, "n=%lld must be >= 0", (long long)n);
    if (n > 0 && (!phi || !P)) return fail(SCINT_EINVAL, "phi and P must be device pointers");
    SCINT_CUDA(launch_phase_fixed(phi, reinterpret_cast<long long*>(P), (long long)n, static_cast<cudaStream_t>(stream)));
    return ok();
}

int scint_fft_lines32(int n, int dir, float* data, int n_lines, void* stream) {
    if (!pow2(n) || n < SCINT_MIN_N || n > SCINT_MAX_N) return fail(SCINT_EINVAL, "bad n=%d", n);
    if (dir != -1 && dir != 1) return fail(SCINT_EINVAL, "dir must be -1 or +1");
    if (!data || n_lines < 0) return fail(SCINT_EINVAL, "bad data or n_lines");
    if (n_lines == 0) return ok();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* ws = nullptr;
    int rc = pool_get(up((size_t)n * 8), s, &ws);
    if (rc) return rc;
    float2* tw = static_cast<float2*>(ws);
    SCINT_CUDA(launch_twiddles32(tw, n, s));
    SCINT_CUDA(launch_fft_lines32(n, dir, reinterpret_cast<float2*>(data), n_lines, tw, s));
    return ok();
}

int scint_fft_lines64(int n, int dir, double* data, int n_lines, void* stream) {
    if (!pow2(n) || n < SCINT_MIN_N || n > SCINT_MAX_N) return fail(SCINT_EINVAL, "bad n=%d", n);
    if (dir != -1 && dir != 1) return fail(SCINT_EINVAL, "dir must be -1 or +1");
    if (!data || n_lines < 0) return fail(SCINT_EINVAL, "bad data or n_lines");
    if (n_lines == 0) return ok();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* ws = nullptr;
    int rc = pool_get(up((size_t)n * 16), s, &ws);
    if (rc) return rc;
    double2* tw = static_cast<double2*>(ws);
    SCINT_CUDA(launch_twiddles64(tw, n, s));
    SCINT_CUDA(launch_fft_lines64(n, dir, reinterpret_cast<double2*>(data), n_lines, tw, s));
    return ok();
}

}  // extern "C"
