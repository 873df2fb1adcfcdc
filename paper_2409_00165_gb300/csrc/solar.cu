// Solar-weighted totals of a spectrum (arxiv 2409.00165, section "Output", Eq. 21):
// R_s = integral(R_lambda G_lambda) / integral(G_lambda) over the simulated grid, and the
// same for A and T, by the trapezoidal rule on the grid points.  One block per stack
// reduces the counts of its n_wl items in FP64; nothing leaves the device.
#include "fos_internal.h"

namespace fos {
namespace solar {

constexpr int BLOCK = 256;

struct Args {
    int n_stacks, n_wl;
    const double* wl;
    const double* G;
    const long long* counts;
    double* out;
    unsigned* status;
    int inject;
};

__device__ __forceinline__ void fractions(const long long* c, double f[3]) {
    const double tot = (double)(c[0] + c[1] + c[2]);
    for (int k = 0; k < 3; ++k) f[k] = tot > 0.0 ? (double)c[k] / tot : 0.0;
}

__global__ void __launch_bounds__(BLOCK) solar_kernel(Args a) {
    __shared__ double red[4][BLOCK];
    const int s = blockIdx.x, t = threadIdx.x;
    if (a.inject && s == 0 && t == 0) atomicOr(&a.status[ST_CALL], DEV_INJECTED);
    const long long* c = a.counts + (long long)s * a.n_wl * FOS_NCOUNT;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // R, A, T numerators, G integral
    bool bad = false;
    if (a.n_wl == 1) {
        if (t == 0) {
            double f[3];
            fractions(c, f);
            const double g0 = a.G[0];
            bad = !(isfinite(g0) && g0 >= 0.0);
            for (int k = 0; k < 3; ++k) acc[k] = f[k];
            acc[3] = 1.0;
        }
    } else {
        // interval w-1 .. w: h (f_{w-1} G_{w-1} + f_w G_w) / 2
        for (int w = 1 + t; w < a.n_wl; w += BLOCK) {
            const double h = a.wl[w] - a.wl[w - 1];
            const double g0 = a.G[w - 1], g1 = a.G[w];
            bad = bad || !(h > 0.0) || !(isfinite(g0) && g0 >= 0.0) || !(isfinite(g1) && g1 >= 0.0);
            double f0[3], f1[3];
            fractions(c + (long long)(w - 1) * FOS_NCOUNT, f0);
            fractions(c + (long long)w * FOS_NCOUNT, f1);
            const double hh = 0.5 * h;
            for (int k = 0; k < 3; ++k) acc[k] += hh * (f0[k] * g0 + f1[k] * g1);
            acc[3] += hh * (g0 + g1);
        }
    }
    for (int k = 0; k < 4; ++k) red[k][t] = acc[k];
    __syncthreads();
    for (int off = BLOCK / 2; off > 0; off >>= 1) {   // fixed-order tree
        if (t < off)
            for (int k = 0; k < 4; ++k) red[k][t] += red[k][t + off];
        __syncthreads();
    }
    if (bad) {
        atomicOr(&a.status[ST_CALL], DEV_INVALID);
        atomicMin(&a.status[ST_INDEX], (unsigned)s);
    }
    if (t == 0) {
        const double den = red[3][0];
        if (!(den > 0.0) || !isfinite(den)) {
            atomicOr(&a.status[ST_CALL], DEV_INVALID);
            atomicMin(&a.status[ST_INDEX], (unsigned)s);
        }
        for (int k = 0; k < 3; ++k) a.out[(long long)s * 3 + k] = red[k][0] / den;
    }
}

}  // namespace solar
}  // namespace fos

using namespace fos;

extern "C" fos_status fos_solar_weighted(int n_stacks, int n_wl, const double* wl,
                                         const double* G, const long long* counts, double* out,
                                         unsigned flags, void* stream) {
    NvtxRange nvtx("fos_solar_weighted");
    if (n_stacks < 1 || n_wl < 1 || !wl || !G || !counts || !out) return FOS_ERR_INVALID_ARG;
    if ((long long)n_stacks * n_wl > 0x7fffffffLL) return FOS_ERR_INVALID_ARG;
    if (flags & ~(unsigned)(FOS_ASYNC | FOS_TEST_INJECT)) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    if (ws->cc_major != 10) return FOS_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_INDEX, 0xff, sizeof(unsigned), s));
    solar::Args a;
    a.n_stacks = n_stacks;
    a.n_wl = n_wl;
    a.wl = wl;
    a.G = G;
    a.counts = counts;
    a.out = out;
    a.status = ws->status;
    a.inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
    solar::solar_kernel<<<(unsigned)n_stacks, solar::BLOCK, 0, s>>>(a);
    FOS_CUDA_TRY(cudaGetLastError());
    return finish_call(ws, s, flags);
}
