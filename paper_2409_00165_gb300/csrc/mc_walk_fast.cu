// The fast photon walk (arxiv 2409.00165, section "Photon transport"): the kernel of
// walk_kernel.cuh with FAST = true, compiled with FMA contraction.  -ln u and cos 2 pi u
// run on the SFU (lg2.approx, cos.approx), the deflection's division and the
// direction update's square root are approximate; random numbers, decisions and the
// work distribution are those of the exact walk.  Its results are checked statistically
// (against the exact walk, the oracle's definition walk and the transfer equation),
// not bit for bit.
#include "walk_kernel.cuh"

namespace fos {
namespace mc {

const void* walk_kernel_fast(int block) { return walk_kernel_for<true>(block); }

namespace {
__global__ void walk_math_fast_kernel(const float* u, float* nl, float* cs, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (nl) nl[i] = walk_neg_log<true>(u[i]);
        if (cs) cs[i] = walk_cos_2pi<true>(u[i]);
    }
}
}  // namespace

}  // namespace mc
}  // namespace fos

extern "C" fos_status fos_walk_math_fast_f32(const float* u, float* neg_log, float* cos2pi,
                                             long long n, void* stream) {
    if (n < 0 || (n > 0 && !u)) return FOS_ERR_INVALID_ARG;
    if (n == 0) return FOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    fos::mc::walk_math_fast_kernel<<<(unsigned)blocks, 256, 0, s>>>(u, neg_log, cos2pi, n);
    FOS_CUDA_TRY(cudaGetLastError());
    return fos::from_cuda(cudaStreamSynchronize(s));
}
