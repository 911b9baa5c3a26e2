// Launch interface of the persistent batch propagation (persist.cu).
#pragma once

#include "kernels.cuh"

namespace scint {

constexpr int kPersistMaxScreens = 256;

struct PersistPlan {
    int n_phases;
    int withhold;          // testing: screen whose row count is one short (-1: none)
    int wait_limit;        // counter reads before a wait gives up
    const PropArgs* screens;   // device table, one entry per screen
    unsigned* counters;    // [0] next item, [1 + s] row items done, [1 + kPersistMaxScreens + s] column items done
    int* status;           // 0, or SCINT_ETIMEOUT
    int phase_first[2 * kPersistMaxScreens + 1];   // first item of each phase; [n_phases] = total
    short phase_screen[2 * kPersistMaxScreens];
    unsigned char phase_pass[2 * kPersistMaxScreens];   // 0 rows, 1 columns
    short slot_prev[kPersistMaxScreens];   // screen whose columns free this screen's field slot (-1: none)
    int row_items[kPersistMaxScreens];
    int col_items[kPersistMaxScreens];
};
constexpr size_t kPersistCounterBytes = sizeof(unsigned) * (1 + 2 * kPersistMaxScreens) + 256;

bool persist_supported(int n);          // grid sizes the persistent kernel runs
size_t persist_smem(int n);             // its shared memory for grid n
int persist_items(int n, int pass);     // work items of one screen's pass
cudaError_t launch_persist_args(const PropArgs& a, PropArgs* dst, cudaStream_t s);
cudaError_t launch_persist_prop(const PersistPlan& pl, size_t smem, cudaStream_t s);

}  // namespace scint
