// Batch executor: many independent screens through the forward path on a few
// internal CUDA streams ("lanes").
//
// Each item is one screen taken through synthesis (Sect. 3.1), propagation and
// passband co-addition (Sect. 3.2, 3.2.4), disk smoothing (Sect. 3.2.3), light
// curves (Sect. 3.3) and the modulation index (Sect. 4) by the single-screen
// entry points, so a batch gives exactly their results.  What the executor adds
// is scheduling: a 1024^2 screen's passes fill fewer than one wave of the GPU,
// and every pass ends in a partial wave, so running screens on several streams
// lets one screen's blocks fill the SMs another leaves idle.
//
// Items are sorted by an estimated cost and each goes to the lane with the
// least queued cost (the longest-processing-time rule).  The lanes fork from
// the caller's stream through an event and join back through one event per
// lane, which keeps the call stream-ordered and capturable into a graph.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"

namespace {

using scint::set_error;

struct Lanes {
    bool ready = false;
    cudaStream_t s[SCINT_MAX_LANES] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[SCINT_MAX_LANES] = {};
};

std::mutex g_lanes_mu;                    // guards g_lanes and serialises enqueueing
std::vector<Lanes> g_lanes;               // per device

int cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(SCINT_ECUDA, m.c_str());
}

// Streams and events of device dev (created once; called with g_lanes_mu held).
int lanes_of(int dev, Lanes** out) {
    if ((int)g_lanes.size() <= dev) g_lanes.resize(dev + 1);
    Lanes& L = g_lanes[dev];
    if (!L.ready) {
        cudaError_t e = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreateWithFlags");
        for (int i = 0; i < SCINT_MAX_LANES; ++i) {
            if ((e = cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreateWithFlags");
            if ((e = cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreateWithFlags");
        }
        L.ready = true;
    }
    *out = &L;
    return SCINT_OK;
}

int lanes_or_default(int n_lanes) { return n_lanes <= 0 ? 2 : n_lanes; }

// Estimated cost of one item: FFT work N^2 log2 N per propagated wavelength, and
// about 8 wavelengths' worth for the FP64 synthesis and the smoothing.
double item_cost(const scint_batch_item& it, int n_lambda) {
    const double n = it.params.n;
    return n * n * std::log2(n) * (n_lambda + 8.0);
}

struct Sizes {
    int n_max = 0;
    bool scratch_phi = false, scratch_i = false;
};

Sizes batch_sizes(const scint_batch_item* items, int n_items) {
    Sizes z;
    for (int i = 0; i < n_items; ++i) {
        z.n_max = std::max(z.n_max, items[i].params.n);
        z.scratch_phi |= items[i].phi == nullptr;
        z.scratch_i |= items[i].intensity == nullptr;
    }
    return z;
}

// Bytes of one lane's slice when passbands run in groups of g wavelengths.
size_t lane_bytes(const Sizes& z, int g) {
    const size_t nn = (size_t)z.n_max * z.n_max;
    return (z.scratch_phi ? scint::aligned_bytes(nn * 8) : 0) + (z.scratch_i ? scint::aligned_bytes(nn * 4) : 0) +
           scint::forward_workspace_bytes(z.n_max, g);
}

// Host checks of the whole batch, before anything is launched.
int check_batch(const scint_batch_item* items, int n_items, const double* lambdas, const double* weights,
                int n_lambda, int n_lanes) {
    char msg[160];
    if (n_items < 0 || (n_items > 0 && !items)) return set_error(SCINT_EINVAL, "items is NULL or n_items < 0");
    if (n_lanes > SCINT_MAX_LANES) {
        snprintf(msg, sizeof msg, "n_lanes=%d exceeds %d", n_lanes, SCINT_MAX_LANES);
        return set_error(SCINT_EINVAL, msg);
    }
    for (int i = 0; i < n_items; ++i) {
        const scint_batch_item& it = items[i];
        int rc = scint::validate_passband(&it.params, lambdas, weights, n_lambda);
        if (rc) {
            snprintf(msg, sizeof msg, "item %d: %s", i, scint::last_error());
            return set_error(rc, msg);
        }
        const char* bad = nullptr;
        if (it.n_tracks < 0 || it.n_samples < 0) bad = "negative track or sample count";
        const bool sampled = it.n_tracks > 0 && it.n_samples > 0;
        if (!bad && sampled && (!it.tracks || !it.curves)) bad = "tracks and curves are needed when sampling";
        if (!bad && sampled)
            for (int k = 0; k < 4 * it.n_tracks; ++k)
                if (!std::isfinite(it.tracks[k])) bad = "track parameters must be finite";
        if (!bad && it.m_curves && it.n_tracks > 0 && (!it.curves || it.n_samples < 1))
            bad = "m_curves needs curves with n_samples >= 1";
        if (bad) {
            snprintf(msg, sizeof msg, "item %d: %s", i, bad);
            return set_error(SCINT_EINVAL, msg);
        }
    }
    return SCINT_OK;
}

// The forward path of one item on lane stream s with the lane's slice.
int run_item(const scint_batch_item& it, const double* lambdas, const double* weights, int n_lambda,
             const Sizes& z, char* slice, size_t slice_bytes, cudaStream_t s) {
    const size_t nn = (size_t)z.n_max * z.n_max;
    char* cur = slice;
    double* phi = it.phi;
    float* inten = it.intensity;
    if (z.scratch_phi) {
        if (!phi) phi = reinterpret_cast<double*>(cur);
        cur += scint::aligned_bytes(nn * 8);
    }
    if (z.scratch_i) {
        if (!inten) inten = reinterpret_cast<float*>(cur);
        cur += scint::aligned_bytes(nn * 4);
    }
    void* ws = cur;
    const size_t wsb = slice_bytes - (size_t)(cur - slice);
    const scint_params* p = &it.params;
    int rc;
    if ((rc = scint_make_screen(p, phi, ws, wsb, s))) return rc;
    if ((rc = scint_sum_passband(p, phi, lambdas, weights, n_lambda, inten, 0, ws, wsb, s))) return rc;
    if ((rc = scint_smooth_source(p, inten, ws, wsb, s))) return rc;
    if (it.n_tracks > 0 && it.n_samples > 0) {
        if ((rc = scint_lightcurve(p, inten, it.tracks, it.n_tracks, it.n_samples, it.curves, s))) return rc;
    }
    if (it.m_map) {
        if ((rc = scint_modulation_index(p, inten, it.m_map, ws, wsb, s))) return rc;
    }
    if (it.m_curves && it.n_tracks > 0) {
        if ((rc = scint_curve_modulation(it.curves, it.n_tracks, it.n_samples, it.m_curves, s))) return rc;
    }
    return SCINT_OK;
}

// ---- persistent mode ---------------------------------------------------------------
std::atomic<int> g_mode{0};              // 0: lanes, 1: persistent propagation
std::mutex g_status_mu;
std::vector<int*> g_last_status;         // per device: status word of the last persistent launch

bool persistent_ok(const scint_batch_item* items, int n_items) {
    if (g_mode.load() != 1 || n_items < 1 || n_items > scint::kPersistMaxScreensHost) return false;
    std::vector<int> sizes(n_items);
    for (int i = 0; i < n_items; ++i) sizes[i] = items[i].params.n;
    return scint::persist_batch_supported(sizes.data(), n_items);
}

int persist_slots(int n_lanes, int n_items) { return std::max(1, std::min(std::min(std::max(n_lanes, 2), 8), n_items)); }

// bytes of the persistent form: the propagation region, then the screens' own phase and
// intensity maps where the items leave them NULL (they live from synthesis to smoothing)
size_t persistent_bytes(const scint_batch_item* items, int n_items, int n_lambda, int n_slots) {
    std::vector<int> sizes(n_items);
    for (int i = 0; i < n_items; ++i) sizes[i] = items[i].params.n;
    size_t b = scint::persist_layout(sizes.data(), n_items, n_lambda, n_slots).total;
    for (int i = 0; i < n_items; ++i) {
        const size_t nn = (size_t)sizes[i] * sizes[i];
        if (!items[i].phi) b += scint::aligned_bytes(nn * 8);
        if (!items[i].intensity) b += scint::aligned_bytes(nn * 4);
    }
    return b;
}

// smoothing, light curves and m of one item (the tail of run_item)
int finish_item(const scint_batch_item& it, float* inten, void* ws, size_t wsb, cudaStream_t s) {
    const scint_params* p = &it.params;
    int rc;
    if ((rc = scint_smooth_source(p, inten, ws, wsb, s))) return rc;
    if (it.n_tracks > 0 && it.n_samples > 0) {
        if ((rc = scint_lightcurve(p, inten, it.tracks, it.n_tracks, it.n_samples, it.curves, s))) return rc;
    }
    if (it.m_map) {
        if ((rc = scint_modulation_index(p, inten, it.m_map, ws, wsb, s))) return rc;
    }
    if (it.m_curves && it.n_tracks > 0) {
        if ((rc = scint_curve_modulation(it.curves, it.n_tracks, it.n_samples, it.m_curves, s))) return rc;
    }
    return SCINT_OK;
}

// Synthesis on the lanes, the propagation of every screen in one persistent launch on
// the caller's stream, then smoothing and observables on the lanes.  Lane l uses field
// slot l as its scratch in the first and last phase.
int run_persistent(const scint_batch_item* items, int n_items, const double* lambdas, const double* weights,
                   int n_lambda, int n_lanes, void* workspace, size_t workspace_bytes, cudaStream_t caller) {
    const int n_slots = persist_slots(n_lanes, n_items);
    std::vector<int> sizes(n_items);
    for (int i = 0; i < n_items; ++i) sizes[i] = items[i].params.n;
    const scint::PersistLayout PL = scint::persist_layout(sizes.data(), n_items, n_lambda, n_slots);
    const size_t need = persistent_bytes(items, n_items, n_lambda, n_slots);
    int rc;
    if (workspace) {
        if (reinterpret_cast<uintptr_t>(workspace) % 256)
            return set_error(SCINT_EINVAL, "workspace must be 256-byte aligned");
        if (workspace_bytes < need) {
            char msg[200];
            snprintf(msg, sizeof msg, "workspace of %zu bytes is smaller than the %zu bytes of the persistent batch",
                     workspace_bytes, need);
            return set_error(SCINT_ENOMEM, msg);
        }
    } else if ((rc = scint::pool_workspace(need, caller, &workspace))) {
        return rc;
    }
    char* ws = static_cast<char*>(workspace);
    char* cur = ws + PL.total;
    std::vector<const scint_params*> prm(n_items);
    std::vector<const double*> phc(n_items);
    std::vector<double*> ph(n_items);
    std::vector<float*> in(n_items);
    for (int i = 0; i < n_items; ++i) {
        const size_t nn = (size_t)sizes[i] * sizes[i];
        prm[i] = &items[i].params;
        ph[i] = items[i].phi;
        if (!ph[i]) {
            ph[i] = reinterpret_cast<double*>(cur);
            cur += scint::aligned_bytes(nn * 8);
        }
        phc[i] = ph[i];
        in[i] = items[i].intensity;
        if (!in[i]) {
            in[i] = reinterpret_cast<float*>(cur);
            cur += scint::aligned_bytes(nn * 4);
        }
    }
    std::lock_guard<std::mutex> lk(g_lanes_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Lanes* L = nullptr;
    if ((rc = lanes_of(dev, &L))) return rc;
    // one lane phase: fork from the caller, work(lane, item) for item = lane, lane + n_slots, ..., join
    auto lane_phase = [&](auto&& work) -> int {
        cudaError_t e1 = cudaEventRecord(L->fork, caller);
        if (e1 != cudaSuccess) return cuda_fail(e1, "cudaEventRecord");
        int first = SCINT_OK, forked = 0;
        std::string msg;
        for (int l = 0; l < n_slots && !first; ++l) {
            if ((e1 = cudaStreamWaitEvent(L->s[l], L->fork, 0)) != cudaSuccess) {
                first = cuda_fail(e1, "cudaStreamWaitEvent");
                msg = scint::last_error();
                break;
            }
            forked = l + 1;
            char* slot = ws + PL.slots + (size_t)l * PL.slot_bytes;
            for (int i = l; i < n_items; i += n_slots) {
                const int r = work(i, slot, L->s[l]);
                if (r) {
                    first = r;
                    msg = std::string("item ") + std::to_string(i) + ": " + scint::last_error();
                    break;
                }
            }
        }
        for (int l = 0; l < forked; ++l) {
            cudaError_t a = cudaEventRecord(L->join[l], L->s[l]);
            cudaError_t b = a == cudaSuccess ? cudaStreamWaitEvent(caller, L->join[l], 0) : a;
            if (b != cudaSuccess && !first) {
                first = cuda_fail(b, "joining a lane");
                msg = scint::last_error();
            }
        }
        if (first) return set_error(first, msg.c_str());
        return SCINT_OK;
    };
    rc = lane_phase([&](int i, char* slot, cudaStream_t st) {
        return scint_make_screen(prm[i], ph[i], slot, PL.slot_bytes, st);
    });
    if (rc) return rc;
    int* status = nullptr;
    if ((rc = scint::persist_propagate(prm.data(), phc.data(), in.data(), n_items, lambdas, weights, n_lambda, ws,
                                       n_slots, &status, caller)))
        return rc;
    {
        std::lock_guard<std::mutex> sl(g_status_mu);
        if ((int)g_last_status.size() <= dev) g_last_status.resize(dev + 1, nullptr);
        g_last_status[dev] = status;
    }
    rc = lane_phase([&](int i, char* slot, cudaStream_t st) { return finish_item(items[i], in[i], slot, PL.slot_bytes, st); });
    if (rc) return rc;
    for (int i = 0; i < n_items; ++i) scint::sampling_warning(&items[i].params, lambdas, n_lambda, i, i == 0);
    return scint::clear_error();
}

}  // namespace

extern "C" {

int scint_batch_mode(int mode) {
    if (mode != 0 && mode != 1) {
        set_error(SCINT_EINVAL, "batch mode must be 0 (lanes) or 1 (persistent propagation)");
        return -1;
    }
    scint::clear_error();
    return g_mode.exchange(mode);
}

int scint_batch_status(void* stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int* st = nullptr;
    {
        std::lock_guard<std::mutex> sl(g_status_mu);
        if ((int)g_last_status.size() > dev) st = g_last_status[dev];
    }
    if ((e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream))) != cudaSuccess)
        return cuda_fail(e, "cudaStreamSynchronize");
    if (!st) return scint::clear_error();
    int v = 0;
    if ((e = cudaMemcpy(&v, st, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    if (v == SCINT_ETIMEOUT) return set_error(SCINT_ETIMEOUT, "a dependency wait of the persistent batch kernel gave up");
    return scint::clear_error();
}

void scint_testing_persist(int withhold, int wait_limit) { scint::persist_testing(withhold, wait_limit); }

size_t scint_batch_workspace_bytes(const scint_batch_item* items, int n_items, int n_lambda, int n_lanes) {
    n_lanes = lanes_or_default(n_lanes);
    if (n_items <= 0 || !items || n_lambda < 1 || n_lanes > SCINT_MAX_LANES) return 0;
    for (int i = 0; i < n_items; ++i)
        if (scint::validate_params(&items[i].params)) return 0;
    const Sizes z = batch_sizes(items, n_items);
    size_t b = (size_t)std::min(n_lanes, n_items) * lane_bytes(z, std::min(n_lambda, SCINT_MAX_LAMBDA));
    if (persistent_ok(items, n_items))
        b = std::max(b, persistent_bytes(items, n_items, std::min(n_lambda, SCINT_MAX_LAMBDA),
                                         persist_slots(n_lanes, n_items)));
    return b;
}

int scint_run_batch(const scint_batch_item* items, int n_items, const double* lambdas_nm, const double* weights,
                    int n_lambda, int n_lanes, void* workspace, size_t workspace_bytes, void* stream) {
    n_lanes = lanes_or_default(n_lanes);
    int rc = check_batch(items, n_items, lambdas_nm, weights, n_lambda, n_lanes);
    if (rc) return rc;
    if (n_items == 0) return scint::clear_error();
    n_lanes = std::min(n_lanes, n_items);
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    const Sizes z = batch_sizes(items, n_items);

    // plans of grid sizes seen for the first time (scint_autotune), never while capturing
    if (scint::autotune_on()) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(caller, &cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
        if (cs == cudaStreamCaptureStatusNone) {
            for (int i = 0; i < n_items; ++i) {
                const int n = items[i].params.n;
                if (!scint::has_plan(n) && (rc = scint_tune(n, n_lambda, nullptr, caller))) return rc;
            }
        }
    }

    if (persistent_ok(items, n_items))
        return run_persistent(items, n_items, lambdas_nm, weights, n_lambda, n_lanes, workspace, workspace_bytes, caller);

    // lane slices: equal parts of the workspace; the largest group that fits
    size_t slice = 0;
    if (workspace) {
        if (reinterpret_cast<uintptr_t>(workspace) % 256)
            return set_error(SCINT_EINVAL, "workspace must be 256-byte aligned");
        slice = workspace_bytes / n_lanes / 256 * 256;
        if (slice < lane_bytes(z, 1)) {
            char msg[160];
            snprintf(msg, sizeof msg, "workspace of %zu bytes is smaller than the %zu bytes needed by %d lanes",
                     workspace_bytes, (size_t)n_lanes * lane_bytes(z, 1), n_lanes);
            return set_error(SCINT_ENOMEM, msg);
        }
    } else {
        slice = lane_bytes(z, std::min(n_lambda, SCINT_MAX_LAMBDA));
        if ((rc = scint::pool_workspace(slice * n_lanes, caller, &workspace))) return rc;
    }

    // longest-processing-time assignment
    std::vector<int> order(n_items);
    for (int i = 0; i < n_items; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return item_cost(items[a], n_lambda) > item_cost(items[b], n_lambda);
    });
    std::vector<std::vector<int>> queue(n_lanes);
    std::vector<double> load(n_lanes, 0.0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        queue[l].push_back(i);
        load[l] += item_cost(items[i], n_lambda);
    }

    std::lock_guard<std::mutex> lk(g_lanes_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Lanes* L = nullptr;
    if ((rc = lanes_of(dev, &L))) return rc;
    if ((e = cudaEventRecord(L->fork, caller)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    int first_rc = SCINT_OK;
    std::string first_msg;
    int forked = 0;
    for (int l = 0; l < n_lanes; ++l) {
        if (queue[l].empty()) continue;
        if ((e = cudaStreamWaitEvent(L->s[l], L->fork, 0)) != cudaSuccess) {
            first_rc = cuda_fail(e, "cudaStreamWaitEvent");
            first_msg = scint::last_error();
            break;
        }
        forked = l + 1;
        char* base = static_cast<char*>(workspace) + (size_t)l * slice;
        for (int i : queue[l]) {
            rc = run_item(items[i], lambdas_nm, weights, n_lambda, z, base, slice, L->s[l]);
            if (rc) {
                first_rc = rc;
                first_msg = std::string("item ") + std::to_string(i) + ": " + scint::last_error();
                break;
            }
        }
        if (first_rc) break;
    }
    // join every forked lane back into the caller's stream, also after an error,
    // so that a capture in progress stays consistent
    for (int l = 0; l < forked; ++l) {
        if (queue[l].empty()) continue;
        cudaError_t e1 = cudaEventRecord(L->join[l], L->s[l]);
        cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(caller, L->join[l], 0) : e1;
        if (e2 != cudaSuccess && !first_rc) {
            first_rc = cuda_fail(e2, "joining a lane");
            first_msg = scint::last_error();
        }
    }
    if (first_rc) return set_error(first_rc, first_msg.c_str());
    // the items' own calls each replaced the warning; report the first item that warns
    for (int i = 0; i < n_items; ++i) scint::sampling_warning(&items[i].params, lambdas_nm, n_lambda, i, i == 0);
    return scint::clear_error();
}

int scint_tune_batch(const scint_batch_item* items, int n_items, const double* lambdas_nm, const double* weights,
                     int n_lambda, void* workspace, size_t workspace_bytes, int* out_lanes, double* out_ms,
                     int* out_mode, void* stream) {
    int rc = check_batch(items, n_items, lambdas_nm, weights, n_lambda, 1);
    if (rc) return rc;
    if (n_items == 0 || !out_lanes) return set_error(SCINT_EINVAL, "scint_tune_batch needs items and out_lanes");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // lane counts tried: 4 and 8, or the item count when it is smaller
    std::vector<int> lane_opts;
    for (int l : {4, 8})
        if (std::find(lane_opts.begin(), lane_opts.end(), std::min(l, n_items)) == lane_opts.end())
            lane_opts.push_back(std::min(l, n_items));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return set_error(SCINT_EINVAL, "scint_tune_batch cannot run during capture");
    std::vector<int> sizes;
    for (int i = 0; i < n_items; ++i)
        if (std::find(sizes.begin(), sizes.end(), items[i].params.n) == sizes.end()) sizes.push_back(items[i].params.n);
    // plan sets: per-size winners alone, all one-wavelength, all packed
    std::vector<std::vector<scint_plan>> sets(3, std::vector<scint_plan>(sizes.size()));
    for (size_t k = 0; k < sizes.size(); ++k) {
        if ((rc = scint_tune(sizes[k], n_lambda, &sets[0][k], stream))) return rc;
        sets[1][k] = scint::one_wavelength_plan();
        sets[2][k] = scint::packed_default_plan(sizes[k]);
    }
    auto same = [&](const std::vector<scint_plan>& a, const std::vector<scint_plan>& b) {
        for (size_t k = 0; k < a.size(); ++k)
            if (a[k].packed != b[k].packed || (a[k].packed && (a[k].points != b[k].points ||
                a[k].row_twiddles != b[k].row_twiddles || a[k].col_twiddles != b[k].col_twiddles)))
                return false;
        return true;
    };
    // candidates: (plan set, form); the persistent form runs the one-wavelength plans
    std::vector<std::pair<int, int>> cand;
    for (int c = 0; c < 3; ++c) {
        bool dup = false;
        for (int d = 0; d < c; ++d) dup |= same(sets[c], sets[d]);
        if (!dup) cand.push_back({c, 0});
    }
    cand.push_back({1, 1});
    const Sizes z = batch_sizes(items, n_items);
    const int old_mode = g_mode.load();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    double best = 1e300;
    int best_c = -1, best_lanes = 0;
    for (size_t ci = 0; ci < cand.size() && !rc; ++ci) {
        const int set = cand[ci].first, mode = cand[ci].second;
        for (size_t k = 0; k < sizes.size() && !rc; ++k) rc = scint::set_tuned_plan(sizes[k], sets[set][k], 0.0);
        if (rc) break;
        g_mode = mode;
        if (mode == 1 && !persistent_ok(items, n_items)) continue;
        for (int lanes : lane_opts) {
            if (rc) break;
            if (workspace) {
                const size_t need = mode == 1 ? persistent_bytes(items, n_items, n_lambda, persist_slots(lanes, n_items))
                                              : (size_t)lanes * lane_bytes(z, 1);
                if (workspace_bytes < need) continue;
            }
            double t = 1e300;
            for (int rep = 0; rep < 3 && !rc; ++rep) {
                if ((e = cudaEventRecord(e0, s)) != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
                if (!rc) rc = scint_run_batch(items, n_items, lambdas_nm, weights, n_lambda, lanes, workspace,
                                              workspace_bytes, stream);
                if (!rc && ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess))
                    rc = cuda_fail(e, "timing the batch");
                if (!rc && mode == 1) rc = scint_batch_status(stream);
                float ms = 0.0f;
                if (!rc && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t = std::min(t, (double)ms);
            }
            if (!rc && t < best) {
                best = t;
                best_c = (int)ci;
                best_lanes = lanes;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_mode = old_mode;
    if (rc) return rc;
    if (best_c < 0) return set_error(SCINT_ENOMEM, "the workspace holds too few lanes of this batch");
    const int set = cand[best_c].first;
    for (size_t k = 0; k < sizes.size(); ++k)
        if ((rc = scint::set_tuned_plan(sizes[k], sets[set][k], best))) return rc;
    g_mode = cand[best_c].second;
    *out_lanes = best_lanes;
    if (out_ms) *out_ms = best;
    if (out_mode) *out_mode = cand[best_c].second;
    return scint::clear_error();
}

}  // extern "C"

// Called by scint_release: destroy the lanes of every device.
namespace scint {
void release_lanes() {
    std::lock_guard<std::mutex> lk(g_lanes_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_lanes.size(); ++d) {
        Lanes& L = g_lanes[d];
        if (!L.ready) continue;
        cudaSetDevice((int)d);
        for (int i = 0; i < SCINT_MAX_LANES; ++i) {
            cudaStreamSynchronize(L.s[i]);
            cudaStreamDestroy(L.s[i]);
            cudaEventDestroy(L.join[i]);
        }
        cudaEventDestroy(L.fork);
        L = Lanes{};
    }
    cudaSetDevice(cur);
}
}  // namespace scint
