// libfos runtime: status strings, per-device workspace, bounded waits.
#include <chrono>
#include <cstdio>
#include <mutex>
#include <thread>

#include "fos_internal.h"

namespace fos {

namespace {
std::mutex g_mutex;
Workspace g_ws[64];

__global__ void accumulate_status_kernel(const unsigned* call, unsigned* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned v = call[ST_CALL];
        if (v) atomicOr(&st[ST_ASYNC], v);
    }
}
}  // namespace

namespace {
thread_local char t_last_error[256] = "";
}

fos_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return FOS_OK;
    snprintf(t_last_error, sizeof(t_last_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return FOS_ERR_NOMEM;
    return FOS_ERR_CUDA;
}

fos_status status_from_bits(unsigned bits) {
    if (bits & DEV_INJECTED) return FOS_ERR_INJECTED;
    if (bits & DEV_INVALID) return FOS_ERR_INVALID_ARG;
    if (bits & DEV_TIMEOUT) return FOS_ERR_TIMEOUT;
    if (bits & DEV_RANGE) return FOS_ERR_OUT_OF_RANGE;
    if (bits & DEV_STEP_LIMIT) return FOS_ERR_STEP_LIMIT;
    return FOS_OK;
}

fos_status get_workspace(Workspace** out) {
    int dev = 0;
    FOS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FOS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    Workspace& ws = g_ws[dev];
    if (ws.device < 0) {
        cudaDeviceProp prop;
        FOS_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
        ws.num_sms = prop.multiProcessorCount;
        ws.cc_major = prop.major;
        ws.cc_minor = prop.minor;
        FOS_CUDA_TRY(cudaMalloc(&ws.status, ST_REGIONS * ST_WORDS * sizeof(unsigned)));
        FOS_CUDA_TRY(cudaMemset(ws.status, 0, ST_REGIONS * ST_WORDS * sizeof(unsigned)));
        FOS_CUDA_TRY(cudaMalloc(&ws.cursor, 4 * sizeof(unsigned long long)));
        FOS_CUDA_TRY(cudaMemset(ws.cursor, 0, 4 * sizeof(unsigned long long)));
        FOS_CUDA_TRY(cudaStreamCreateWithFlags(&ws.side, cudaStreamNonBlocking));
        ws.device = dev;
    }
    *out = &ws;
    return FOS_OK;
}

fos_status ensure_buffer(Workspace* ws, void** buf, size_t* cur, size_t bytes) {
    if (bytes <= *cur && *buf) return FOS_OK;
    // Nothing in flight may still use the old buffer.
    FOS_CUDA_TRY(cudaDeviceSynchronize());
    if (*buf) {
        cudaFree(*buf);
        *buf = nullptr;
        *cur = 0;
    }
    size_t want = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(buf, want);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return from_cuda(e);
    }
    *cur = want;
    ws->generation++;
    return FOS_OK;
}

fos_status wait_stream(cudaStream_t s, int timeout_ms) {
    if (timeout_ms <= 0) timeout_ms = default_timeout_ms();
    auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return FOS_OK;
        if (e != cudaErrorNotReady) return from_cuda(e);
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                      std::chrono::steady_clock::now() - t0).count();
        if (ms > timeout_ms) return FOS_ERR_TIMEOUT;
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

fos_status accumulate_async_status(Workspace* ws, cudaStream_t s, int region) {
    accumulate_status_kernel<<<1, 32, 0, s>>>(ws->status + region * ST_WORDS, ws->status);
    return from_cuda(cudaGetLastError());
}

fos_status finish_call(Workspace* ws, cudaStream_t s, unsigned flags, int region) {
    if (flags & FOS_ASYNC) return accumulate_async_status(ws, s, region);
    fos_status st = wait_stream(s, default_timeout_ms());
    if (st != FOS_OK) return st;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&bits, ws->status + region * ST_WORDS + ST_CALL, sizeof(unsigned),
                            cudaMemcpyDeviceToHost));
    return status_from_bits(bits);
}

}  // namespace fos

extern "C" {

const char* fos_status_string(fos_status s) {
    switch (s) {
        case FOS_OK: return "ok";
        case FOS_ERR_INVALID_ARG: return "invalid argument";
        case FOS_ERR_CUDA: return "CUDA runtime error";
        case FOS_ERR_NOMEM: return "out of device memory";
        case FOS_ERR_STEP_LIMIT: return "some photons reached max_events (counted as runaway)";
        case FOS_ERR_TIMEOUT: return "timed out waiting for the stream";
        case FOS_ERR_OUT_OF_RANGE: return "input outside the supported range";
        case FOS_ERR_INJECTED: return "injected test failure";
        case FOS_ERR_UNSUPPORTED: return "unsupported device or feature";
        default: return "unknown status";
    }
}

int fos_api_version(void) { return FOS_API_VERSION; }

const char* fos_last_cuda_error(void) { return fos::t_last_error; }

fos_status fos_sync_status(void* stream, int timeout_ms) {
    fos::Workspace* ws = nullptr;
    fos_status st = fos::get_workspace(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = fos::wait_stream(s, timeout_ms);
    if (st != FOS_OK) return st;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&bits, ws->status + fos::ST_ASYNC, sizeof(unsigned),
                            cudaMemcpyDeviceToHost));
    FOS_CUDA_TRY(cudaMemset(ws->status + fos::ST_ASYNC, 0, sizeof(unsigned)));
    return fos::status_from_bits(bits);
}

}  // extern "C"
