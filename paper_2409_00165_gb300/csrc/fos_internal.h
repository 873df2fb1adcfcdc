// Internal definitions shared by the libfos translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "fos.h"   // include/ is on the compiler include path

namespace fos {

// Bits of the per-device status word written by kernels (atomicOr).
enum : unsigned {
    DEV_INVALID = 1u,     // a value failed validation
    DEV_STEP_LIMIT = 2u,  // some photon reached max_events
    DEV_INJECTED = 4u,    // FOS_TEST_INJECT
    DEV_RANGE = 8u,       // input outside the kernel's supported range
    DEV_TIMEOUT = 16u,    // a bounded in-kernel wait ran out (the kernel returned early)
};

// status words on the device: [0] the current call, [1] accumulated FOS_ASYNC work,
// [2] first offending index of the current call (for diagnostics).  The buffer holds
// ST_REGIONS such groups: region 0 for the calls of the default path; regions 1.. for
// calls that may run concurrently on other streams (the surrogate's training slots),
// each with its own call word, all accumulating into region 0's async word.
enum { ST_CALL = 0, ST_ASYNC = 1, ST_INDEX = 2, ST_WORDS = 4, ST_REGIONS = 5 };

struct Workspace {
    int device = -1;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    unsigned* status = nullptr;             // device [ST_REGIONS * ST_WORDS]
    unsigned long long* cursor = nullptr;   // device work-queue counter(s) [4]
    void* mc_tables = nullptr;              // packed item tables + unit prefix
    size_t mc_bytes = 0;
    void* mie_scratch = nullptr;            // Mie recurrence scratch + per-species Q's
    size_t mie_bytes = 0;
    long long* tune_counts = nullptr;       // autotuner output
    size_t tune_bytes = 0;
    unsigned long long* walk_times = nullptr;  // per-block start/end of a recorded walk
    size_t walk_times_bytes = 0;
    cudaStream_t side = nullptr;            // private stream for graph capture
    unsigned long long generation = 0;      // bumps when a table is reallocated
};

// Per-device workspace of the current device (created on first use).
fos_status get_workspace(Workspace** ws);
// Grows a workspace buffer to at least `bytes` (synchronous cudaMalloc).
fos_status ensure_buffer(Workspace* ws, void** buf, size_t* cur, size_t bytes);

fos_status from_cuda(cudaError_t e);
fos_status status_from_bits(unsigned bits);

// Bounded wait: polls the stream until it is idle or timeout_ms passes.
fos_status wait_stream(cudaStream_t s, int timeout_ms);

// Enqueues work that moves the call status of `region` into the accumulated async status.
fos_status accumulate_async_status(Workspace* ws, cudaStream_t s, int region = 0);

// Ends a call: for synchronous calls waits (bounded) and converts the call word of
// `region`.
fos_status finish_call(Workspace* ws, cudaStream_t s, unsigned flags, int region = 0);

inline int default_timeout_ms() { return 600000; }

// NVTX range around a library entry point (visible in Nsight timelines; a no-op when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace fos

#define FOS_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return ::fos::from_cuda(_e);  \
    } while (0)
