// Persistent propagation of a whole batch: one launch of one block per SM walks a work
// list that holds, for every screen of the batch, its row-pass and column-pass work in
// blocks of lines, and runs each with the bodies of the ordinary passes (prop_body.cuh),
// so the results are those of the per-screen kernels bit for bit.
//
// Work list.  Phases in order: rows of screen 0, rows of screen 1, columns of screen 0,
// rows of screen 2, columns of screen 1, ... (a screen's columns are queued one phase
// after the next screen's rows, so their wait is usually over when they are reached).
// Screens are taken largest first (their tails are filled by the small ones).  Items are
// dispensed in list order by an atomic counter; a block runs its item to completion
// before it takes the next, and every block is resident (the grid is one block per SM),
// so every item a block waits for has been dispensed to a running block.
//
// Dependencies, with release/acquire counters: the columns of screen s wait until all
// its row items have finished; the rows of screen s wait until the columns of the screen
// that used its field slot before it have finished (the fields of a group live in one
// of a few slots of the workspace).  The fields are read through L2 only (the column
// body loads them with ld.global.cg), since L1 is not coherent across SMs.
//
// Bounded waits.  Thread 0 of a block spins on a counter with a pause between reads and
// gives up after wait_limit reads: it sets the status word to SCINT_ETIMEOUT (first
// writer wins) and the block returns.  Every block checks the status before it takes
// an item and returns once it is set, so a failed dependency ends the launch within
// one wait.  A test hook withholds one count to exercise this path.
//
// Block shape: 512 threads, one block per SM; an item is the work of one 512-thread
// block of the ordinary pass or of two 256-thread blocks, run side by side on the two
// halves of the block on disjoint shared memory, each half synchronising on its own
// named barrier (with one block-wide barrier the halves stalled together: 22 % slower).
#include <algorithm>
#include <vector>

#include "../../include/scint.h"
#include "dispatch.cuh"
#include "persist.cuh"
#include "prop_body.cuh"

namespace scint {

constexpr int kPersistThreads = 512;

template <int N> __host__ __device__ constexpr int rows_subs() { return kPersistThreads / prow_threads<N>(); }
template <int N> __host__ __device__ constexpr int cols_subs() { return kPersistThreads / pcol_threads<N>(); }
template <int N> constexpr size_t persist_smem_n() {
    return std::max((size_t)rows_subs<N>() * prow_smem<N>(), (size_t)cols_subs<N>() * pcol_smem<N>());
}
template <int N> constexpr bool persist_size() {
    return N >= 256 && N <= 4096 && prow_threads<N>() * rows_subs<N>() == kPersistThreads &&
           pcol_threads<N>() * cols_subs<N>() == kPersistThreads && persist_smem_n<N>() <= kMaxSmem;
}

bool persist_supported(int n) {
    bool ok = false;
    dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        ok = persist_size<N>();
        return cudaSuccess;
    });
    return ok;
}

size_t persist_smem(int n) {
    size_t b = 0;
    dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (persist_size<N>()) b = persist_smem_n<N>();
        return cudaSuccess;
    });
    return b;
}

int persist_items(int n, int pass) {
    int k = 0;
    dispatch_n(n, [&](auto nc) -> cudaError_t {
        constexpr int N = decltype(nc)::value;
        if constexpr (persist_size<N>())
            k = pass == 0 ? N / prow_lines<N>() / rows_subs<N>() : N / pcol_lines<N>() / cols_subs<N>();
        return cudaSuccess;
    });
    return k;
}

SCINT_DEV unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *c >= target; false (status set) after limit reads or when
// another block has failed.
SCINT_DEV bool wait_for(const unsigned* c, unsigned target, int limit, int* status) {
    for (int it = 0;; ++it) {
        if (ld_acquire(c) >= target) return true;
        if (*(volatile int*)status != 0) return false;
        if (it >= limit) {
            atomicCAS(status, 0, SCINT_ETIMEOUT);
            return false;
        }
        __nanosleep(200);
    }
}

template <int N>
SCINT_DEV void run_item(const PropArgs& a, int pass, int item, float2* smem) {
    const int tid = threadIdx.x;
    if constexpr (persist_size<N>()) {
        // two bodies side by side synchronise on their own named barriers
        if (pass == 0) {
            constexpr int SUB = prow_threads<N>();
            constexpr int BAR = rows_subs<N>() > 1 ? SUB : 0;
            prop_rows_body<N, false, BAR>(a, item * rows_subs<N>() + tid / SUB, tid % SUB,
                                          smem + (tid / SUB) * (prow_smem<N>() / sizeof(float2)));
        } else {
            constexpr int SUB = pcol_threads<N>();
            constexpr int BAR = cols_subs<N>() > 1 ? SUB : 0;
            prop_cols_body<N, false, BAR>(a, item * cols_subs<N>() + tid / SUB, tid % SUB,
                                          smem + (tid / SUB) * (pcol_smem<N>() / sizeof(float2)));
        }
    }
}

__global__ void __launch_bounds__(kPersistThreads, 1) persist_prop_kernel(PersistPlan pl) {
    extern __shared__ float2 psmem[];
    __shared__ int s_item, s_ok;
    // the current screen's arguments, staged in shared memory: the bodies read them many times
    // per wavelength, and from global memory those reads were the launch's main latency stall
    __shared__ PropArgs sa;
    int staged = -1;
    unsigned* next = pl.counters;
    unsigned* rows_done = pl.counters + 1;
    unsigned* cols_done = pl.counters + 1 + kPersistMaxScreens;
    const int total = pl.phase_first[pl.n_phases];
    int phase = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int g = -1;
            if (*(volatile int*)pl.status == 0) {
                g = (int)atomicAdd(next, 1u);
                if (g >= total) g = -1;
            }
            s_item = g;
        }
        __syncthreads();
        const int g = s_item;
        if (g < 0) return;
        while (pl.phase_first[phase + 1] <= g) ++phase;   // items are dispensed in increasing order
        const int s = pl.phase_screen[phase], pass = pl.phase_pass[phase];
        const int item = g - pl.phase_first[phase];
        if (threadIdx.x == 0) {
            bool ok = true;
            if (pass == 0) {
                const int prev = pl.slot_prev[s];
                if (prev >= 0) ok = wait_for(cols_done + prev, (unsigned)pl.col_items[prev], pl.wait_limit, pl.status);
            } else {
                const unsigned target = (unsigned)pl.row_items[s] + (s == pl.withhold ? 1u : 0u);
                ok = wait_for(rows_done + s, target, pl.wait_limit, pl.status);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        if (s != staged) {    // uniform across the block
            const int* src = reinterpret_cast<const int*>(pl.screens + s);
            int* dst = reinterpret_cast<int*>(&sa);
            for (int i = threadIdx.x; i < (int)(sizeof(PropArgs) / sizeof(int)); i += kPersistThreads) dst[i] = src[i];
            __syncthreads();
            staged = s;
        }
        const PropArgs& a = sa;
        switch (a.n) {
            case 256: run_item<256>(a, pass, item, psmem); break;
            case 512: run_item<512>(a, pass, item, psmem); break;
            case 1024: run_item<1024>(a, pass, item, psmem); break;
            case 2048: run_item<2048>(a, pass, item, psmem); break;
            case 4096: run_item<4096>(a, pass, item, psmem); break;
            default: break;
        }
        // the block barrier orders every thread's stores before thread 0's fence, which makes
        // them visible device-wide before the count (release, cumulative through the barrier)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(pass == 0 ? rows_done + s : cols_done + s, 1u);
        }
    }
}

// Copy one screen's arguments into the device table the persistent kernel reads.
__global__ void persist_args_kernel(PropArgs a, PropArgs* dst) {
    const int n = sizeof(PropArgs) / sizeof(int);
    const int* src = reinterpret_cast<const int*>(&a);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = src[i];
}

cudaError_t launch_persist_args(const PropArgs& a, PropArgs* dst, cudaStream_t s) {
    static_assert(sizeof(PropArgs) % sizeof(int) == 0, "PropArgs copied as ints");
    persist_args_kernel<<<1, 256, 0, s>>>(a, dst);
    return cudaGetLastError();
}

cudaError_t launch_persist_prop(const PersistPlan& pl, size_t smem, cudaStream_t s) {
    cudaError_t e = set_smem(persist_prop_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_prop_kernel, kPersistThreads, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // every block resident at once: the waits rely on it
    persist_prop_kernel<<<sms * per_sm, kPersistThreads, smem, s>>>(pl);
    return cudaGetLastError();
}

}  // namespace scint
