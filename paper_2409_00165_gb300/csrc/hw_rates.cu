// Hardware rates of the GPU that the kernels of this library are measured against
// (diagnostic; not on the path of the method): the FP64 FMA rate (the Mie kernel's
// bound), the MUFU tanh rate (the fused inference epilogue's), tcgen05.mma throughput by
// N with the A operand in shared or tensor memory (the inference MMAs'), and the L2 ->
// shared memory bulk-copy bandwidth (the inference weight stream's).  Each is one timed
// launch on a private stream after a warm-up; every wait is bounded.
#include <cstring>

#include "fos_internal.h"
#include "sm100_ptx.cuh"

namespace fos {
namespace hw {

using namespace fos::sm100;

// 8 independent DFMA chains per thread.
__global__ void fp64_kernel(int iters, double* out) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-9 * (threadIdx.x + j);
    const double b = 0.999999999, c = 1e-12;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent tanh.approx.f32 chains per thread.
__global__ void tanh_kernel(int iters, float* out) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.001f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("tanh.approx.f32 %0, %0;" : "+f"(a[j]));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same with the packed half-precision form (two values per instruction).
__global__ void tanh2_kernel(int iters, float* out) {
    uint32_t a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0x1c001c00u + threadIdx.x + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("tanh.approx.f16x2 %0, %0;" : "+r"(a[j]));
    }
    uint32_t s = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) s ^= a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// One thread per CTA issues iters x 4 MMAs (M = 128, N, K = 16) on zeroed operands: A from
// shared memory (TS = false) or tensor memory (TS = true).
constexpr int MMA_SMEM = 16384 + 32768 + 64 + 1024;
template <int N, bool TS>
__global__ void __launch_bounds__(128, 1) mma_kernel(int iters, unsigned* flag) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const uint32_t raw = smem_u32(sm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* basep = sm + (base - raw);
    const uint32_t A_s = base, B_s = base + 16384, bar = base + 16384 + 32768, slot = bar + 8;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (16384 + 32768) / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(basep)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(basep + 16384 + 32768 + 8);
    if (threadIdx.x == 0) {
        const uint64_t da = desc_sw128(A_s), db = desc_sw128(B_s);
        constexpr uint32_t ID = idesc_bf16(128, N);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                if (TS) mma_bf16_ts(tmem, tmem + 256 + 8 * kk, db + 2 * kk, ID, (i | kk) ? 1u : 0u);
                else mma_bf16(tmem, da + 2 * kk, db + 2 * kk, ID, (i | kk) ? 1u : 0u);
            }
        }
        mma_commit(bar);
        if (!mbar_wait(bar, 0, 2000000000LL)) atomicOr(flag, 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// One thread per CTA keeps 4 untiled bulk copies of 32 KB in flight from a 448 KB source
// (every CTA reads the same bytes, as the inference CTAs read the same weights).
constexpr int BULK_CHUNK = 32768, BULK_SLOTS = 4, BULK_SRC_CHUNKS = 14;
__global__ void bulk_kernel(const uint8_t* src, int iters, unsigned* flag) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const uint32_t base = smem_u32(sm);
    const uint32_t bars = base + BULK_SLOTS * BULK_CHUNK;
    if (threadIdx.x != 0) return;
    for (int i = 0; i < BULK_SLOTS; ++i) mbar_init(bars + 8 * i, 1);
    fence_barrier_init();
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < iters; ++i) {
        const int slot = i % BULK_SLOTS;
        if (i >= BULK_SLOTS &&
            !mbar_wait(bars + 8 * slot, (uint32_t)((i / BULK_SLOTS - 1) & 1), 100000000LL)) {
            ok = false;
            break;
        }
        mbar_arrive_expect_tx(bars + 8 * slot, BULK_CHUNK);
        const int c = (i + blockIdx.x) % BULK_SRC_CHUNKS;
        bulk_load(base + slot * BULK_CHUNK, src + (size_t)c * BULK_CHUNK, BULK_CHUNK,
                  bars + 8 * slot);
        ++issued;
    }
    const int first = issued > BULK_SLOTS ? issued - BULK_SLOTS : 0;
    for (int g = first; g < issued; ++g)
        if (!mbar_wait(bars + 8 * (g % BULK_SLOTS), (uint32_t)((g / BULK_SLOTS) & 1), 100000000LL))
            ok = false;
    if (!ok) atomicOr(flag, 1u);
}

// Milliseconds of one launch of `launch` on stream s (after one warm-up launch).
template <class F>
static fos_status time_ms(cudaStream_t s, F launch, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    FOS_CUDA_TRY(cudaEventCreate(&a));
    FOS_CUDA_TRY(cudaEventCreate(&b));
    launch(true);
    FOS_CUDA_TRY(cudaGetLastError());
    FOS_CUDA_TRY(cudaEventRecord(a, s));
    launch(false);
    FOS_CUDA_TRY(cudaGetLastError());
    FOS_CUDA_TRY(cudaEventRecord(b, s));
    fos_status st = wait_stream(s, default_timeout_ms());
    if (st == FOS_OK) FOS_CUDA_TRY(cudaEventElapsedTime(ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

template <int N, bool TS>
static fos_status mma_rate(int nsm, unsigned* flag, cudaStream_t s, double* tflops) {
    FOS_CUDA_TRY(cudaFuncSetAttribute(mma_kernel<N, TS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, MMA_SMEM));
    const int iters = 20000;
    float ms = 0.f;
    fos_status st = time_ms(s, [&](bool warm) {
        mma_kernel<N, TS><<<nsm, 128, MMA_SMEM, s>>>(warm ? 16 : iters, flag);
    }, &ms);
    if (st != FOS_OK) return st;
    *tflops = 2.0 * 128 * N * 16 * 4.0 * iters * nsm / (ms * 1e-3) / 1e12;
    return FOS_OK;
}

}  // namespace hw
}  // namespace fos

using namespace fos;

extern "C" {

fos_status fos_measure_hw_rates(fos_hw_rates* out) {
    if (!out) return FOS_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    if (ws->cc_major != 10) return FOS_ERR_UNSUPPORTED;
    const int nsm = ws->num_sms;
    cudaStream_t s = nullptr;
    FOS_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    void* scratch = nullptr;
    const size_t src_bytes = (size_t)hw::BULK_SRC_CHUNKS * hw::BULK_CHUNK;
    const size_t out_bytes = (size_t)nsm * 4 * 256 * sizeof(double);
    cudaError_t e = cudaMalloc(&scratch, src_bytes + out_bytes + 256);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return from_cuda(e);
    }
    uint8_t* src = (uint8_t*)scratch;
    double* dout = (double*)((uint8_t*)scratch + src_bytes);
    unsigned* flag = (unsigned*)((uint8_t*)scratch + src_bytes + out_bytes);
    auto run = [&]() -> fos_status {
        FOS_CUDA_TRY(cudaMemsetAsync(scratch, 0, src_bytes + out_bytes + 256, s));
        float ms = 0.f;
        const int blocks = nsm * 4, threads = 256, fiters = 20000, titers = 4096;
        fos_status r = hw::time_ms(s, [&](bool warm) {
            hw::fp64_kernel<<<blocks, threads, 0, s>>>(warm ? 100 : fiters, dout);
        }, &ms);
        if (r != FOS_OK) return r;
        out->fp64_tflops = 2.0 * 8 * fiters * (double)blocks * threads / (ms * 1e-3) / 1e12;
        r = hw::time_ms(s, [&](bool warm) {
            hw::tanh_kernel<<<blocks, threads * 2, 0, s>>>(warm ? 16 : titers, (float*)dout);
        }, &ms);
        if (r != FOS_OK) return r;
        out->tanh_per_s = 8.0 * titers * (double)blocks * threads * 2 / (ms * 1e-3);
        r = hw::time_ms(s, [&](bool warm) {
            hw::tanh2_kernel<<<blocks, threads * 2, 0, s>>>(warm ? 16 : titers, (float*)dout);
        }, &ms);
        if (r != FOS_OK) return r;
        out->tanh_f16x2_per_s = 2.0 * 8.0 * titers * (double)blocks * threads * 2 / (ms * 1e-3);
        r = hw::mma_rate<64, true>(nsm, flag, s, &out->mma_ts_tflops[0]);
        if (r == FOS_OK) r = hw::mma_rate<128, true>(nsm, flag, s, &out->mma_ts_tflops[1]);
        if (r == FOS_OK) r = hw::mma_rate<256, true>(nsm, flag, s, &out->mma_ts_tflops[2]);
        if (r == FOS_OK) r = hw::mma_rate<64, false>(nsm, flag, s, &out->mma_ss_tflops[0]);
        if (r == FOS_OK) r = hw::mma_rate<128, false>(nsm, flag, s, &out->mma_ss_tflops[1]);
        if (r == FOS_OK) r = hw::mma_rate<256, false>(nsm, flag, s, &out->mma_ss_tflops[2]);
        if (r != FOS_OK) return r;
        const int bsmem = hw::BULK_SLOTS * hw::BULK_CHUNK + 8 * hw::BULK_SLOTS;
        FOS_CUDA_TRY(cudaFuncSetAttribute(hw::bulk_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, bsmem));
        const int biters = 2048;
        r = hw::time_ms(s, [&](bool warm) {
            hw::bulk_kernel<<<nsm, 32, bsmem, s>>>(src, warm ? 64 : biters, flag);
        }, &ms);
        if (r != FOS_OK) return r;
        out->bulk_tbps = (double)nsm * biters * hw::BULK_CHUNK / (ms * 1e-3) / 1e12;
        unsigned h = 0;
        FOS_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        FOS_CUDA_TRY(cudaStreamSynchronize(s));
        return h ? FOS_ERR_TIMEOUT : FOS_OK;
    };
    st = run();
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    cudaStreamDestroy(s);
    return st;
}

}  // extern "C"
