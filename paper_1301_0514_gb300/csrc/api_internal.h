// Host-side helpers of csrc/api.cu used by the other host translation units
// (the batch executor): error reporting, parameter checks, workspace sizing and
// the per-device workspace pool.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "../../include/scint.h"

namespace scint {

// Set the calling thread's last-error message; returns code.
int set_error(int code, const char* msg);
// Clear the calling thread's last-error message; returns SCINT_OK.
int clear_error();
const char* last_error();
// The sampling warning of Sect. 3.2.2 (pixel >= R_diff(lambda)/2) for one screen,
// "item i: ..." for i >= 0; clear = start over, else keep the first warning.
void sampling_warning(const scint_params* p, const double* lambdas, int n_lambda, int item, bool clear);

// Host checks of one screen's parameters, and of a passband for it (the same
// checks, with the same messages, as the single-screen entry points).
int validate_params(const scint_params* p);
int validate_passband(const scint_params* p, const double* lambdas, const double* weights, int n_lambda);

// Bytes rounded up to the library's workspace alignment (256).
size_t aligned_bytes(size_t b);
// Workspace of the forward path of one N x N screen (synthesis, a passband
// group of g wavelengths, smoothing, moments): the maximum over its calls.
size_t forward_workspace_bytes(int n, int g);
// The per-device pool: at least `bytes`, grown outside stream capture only.
int pool_workspace(size_t bytes, cudaStream_t s, void** out);
// Destroy the batch executor's streams and events (csrc/batch.cu).
void release_lanes();
// Autotuning on first use (scint_autotune) is on; grid n has a plan on the current device.
bool autotune_on();
bool has_plan(int n);
// Plan of grid n on the current device (tuned or default), and setting it as measured (tuned = 1).
int plan_of(int n, scint_plan* out);
int set_tuned_plan(int n, scint_plan pl, double ms);
scint_plan one_wavelength_plan();
scint_plan packed_default_plan(int n);

// ---- persistent propagation of a batch (persist.cu; arguments built in api.cu) ----
// Workspace of the propagation of n screens (grid sizes `sizes`) in one persistent launch
// with n_slots field slots: counters, the argument table, taper tables, twiddles and the
// slots (each also large enough to serve as one lane's scratch for the other steps).
struct PersistLayout {
    size_t args = 0, tw = 0, sf = 0, slots = 0, slot_bytes = 0, total = 0;
};
PersistLayout persist_layout(const int* sizes, int n, int n_lambda, int n_slots);
bool persist_batch_supported(const int* sizes, int n);
constexpr int kPersistMaxScreensHost = 256;   // screens one persistent launch takes (kPersistMaxScreens)
// Run the propagation of every screen (phi in, intensity out; passband lambdas/weights)
// in one persistent launch on stream s; ws must hold persist_layout(...).total bytes.
// withhold / wait_limit: see scint_testing_persist.  The status word (0 or
// SCINT_ETIMEOUT once the launch has run) is at *status_out.
int persist_propagate(const scint_params* const* params, const double* const* phis, float* const* intensities,
                      int n, const double* lambdas, const double* weights, int n_lambda, char* ws, int n_slots,
                      int** status_out, cudaStream_t s);
void persist_testing(int withhold, int wait_limit);

}  // namespace scint
