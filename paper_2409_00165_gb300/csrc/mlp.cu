// Learned surrogate of the photon walk on GB300 (arxiv 2409.00165, section "Photon
// transport": a network trained on Monte Carlo spectra replaces the walk).
//
// Network: 9 features -> standardise -> [Linear 256, GELU (tanh form)] x 4 -> Linear 3 -> softmax
// (R, A, T).  BF16 weights and activations on the tensor cores, FP32 accumulation,
// FP32 master weights and Adam state.
//
// Inference runs in one fused persistent kernel (infer_kernel, below).  Every matrix
// product of training runs in gemm_kernel: a 128 x NT output
// tile per CTA; K-major BF16 operands are staged by TMA (128-byte swizzle) through a
// 4-stage mbarrier ring; one thread issues tcgen05.mma (M=128, N=NT, K=16) into FP32
// accumulators in tensor memory; the 4 warps read the accumulators back with tcgen05.ld
// and apply the fused epilogue of the layer (bias + GELU, softmax + cross-entropy
// gradient, GELU derivative, or a split-K weight-gradient partial).  Transposed copies of
// activations and gradients written by the epilogues make every product "A times B^T"
// with both operands K-major.
//
// Padded shapes (zero padding, never updated): layer 0 is 256 x 64 (9 real inputs),
// layers 1-3 are 256 x 256, layer 4 is 64 x 256 (3 real outputs).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "fos_internal.h"
#include "sm100_ptx.cuh"

namespace fos {
namespace mlp {

using namespace fos::sm100;
typedef __nv_bfloat16 bf16;

constexpr int N_LAYERS = 5;
constexpr int HID = 256;
constexpr int IN_PAD = 64;
constexpr int OUT_PAD = 64;
constexpr int N_FEAT = 9;
constexpr int N_OUT = 3;
// Pipeline stages of the training GEMM: 2 (a k block in flight while the previous one is
// multiplied) keep a CTA at 50-100 KB of shared memory, so that 2-4 CTAs share an SM and
// hide each other's TMA, epilogue and launch latency.
constexpr int STAGES = 2;
constexpr int BM = 128;
constexpr int BK = 64;

__host__ __device__ constexpr int lay_out(int l) { return l == 4 ? OUT_PAD : HID; }
__host__ __device__ constexpr int lay_in(int l) { return l == 0 ? IN_PAD : HID; }
__host__ __device__ constexpr int real_out(int l) { return l == 4 ? N_OUT : HID; }
__host__ __device__ constexpr int real_in(int l) { return l == 0 ? N_FEAT : HID; }

// ----------------------------------------------------------------------- model layout
// Per member (all offsets in elements of the named type, from the member base):
//   theta  fp32 [P]  : W_0 | b_0 | W_1 | b_1 | ... | W_4 | b_4  (W_l row-major [out][in])
//   adam_m fp32 [P], adam_v fp32 [P]
//   wb     bf16      : W_l in bf16, [out][in] per layer (forward B operands)
//   wt     bf16      : W_l^T in bf16, [in][out] for l = 1..4 (backward B operands)
//   stats  fp32 [64] : mean[16] | std[16] | lo[16] | hi[16] of the raw features
//   step   int32 [4]
//   wi     bf16      : the weights as shared-memory images for the fused inference
//                      kernel (see img_index), one contiguous block per pipeline stage
struct Layout {
    long long w_off[N_LAYERS], b_off[N_LAYERS], P;
    long long wb_off[N_LAYERS], wt_off[N_LAYERS], n_wb, n_wt;
    size_t theta_b, m_b, v_b, wb_b, wt_b, stats_b, step_b, wi_b, bytes;
};

// Weight image: the B operands of the fused inference kernel, already in the 128-byte-
// swizzled K-major layout a stage of shared memory holds, so that one untiled bulk copy
// fills a stage (32 KB).  Layer 0 is one stage: all 256 output rows x 64 inputs (9 real).
// Layers 1-3 are four stages each, (output half h, input pair j) in the order 2h + j:
// 128 output rows x inputs 128 j .. +127, as two k blocks of 128 x 64 (16 KB).  Layer 4
// keeps its first 16 output rows (3 real) as 4 blocks of 16 x 64 (2 KB), one per k
// block, copied as one stage.
constexpr long long IMG_BLK = 256 * 64;          // elements of a 32 KB stage
constexpr long long IMG_HALF_KB = 128 * 64;      // elements of a 16 KB k block of a half
constexpr long long IMG_L4_BLK = 16 * 64;        // elements of a 2 KB block
__host__ __device__ constexpr long long img_off(int l) {
    return l == 0 ? 0 : (l == 4 ? 13 * IMG_BLK : (1 + 4 * (l - 1)) * IMG_BLK);
}
constexpr long long IMG_ELEMS = 13 * IMG_BLK + 4 * IMG_L4_BLK;
constexpr int IMG_ROWS_L4 = 16;

// Element index in the image of weight (l, o, i), or -1 when the image leaves it out.
// Row n of a block starts at n * 64 elements; its 16-byte chunk j (inputs 8j..8j+7 of
// the k block) sits at chunk position j ^ (n mod 8).
__host__ __device__ inline long long img_index(int l, int o, int i) {
    const int kb = i >> 6, c = i & 63;
    const long long swz = (((c >> 3) ^ (o & 7)) << 3) | (c & 7);
    if (l == 4) {
        if (o >= IMG_ROWS_L4) return -1;
        return img_off(l) + (long long)kb * IMG_L4_BLK + o * 64 + swz;
    }
    if (l == 0) return img_off(l) + o * 64 + swz;
    return img_off(l) + (long long)((o >> 7) * 2 + (kb >> 1)) * IMG_BLK +
           (long long)(kb & 1) * IMG_HALF_KB + (o & 127) * 64 + swz;
}

static Layout make_layout() {
    Layout L;
    long long p = 0, q = 0, t = 0;
    for (int l = 0; l < N_LAYERS; ++l) {
        L.w_off[l] = p;
        p += (long long)lay_out(l) * lay_in(l);
        L.b_off[l] = p;
        p += lay_out(l);
        L.wb_off[l] = q;
        q += (long long)lay_out(l) * lay_in(l);
        L.wt_off[l] = t;
        if (l > 0) t += (long long)lay_out(l) * lay_in(l);
    }
    L.P = p;
    L.n_wb = q;
    L.n_wt = t;
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    size_t o = 0;
    L.theta_b = o; o = al(o + (size_t)p * 4);
    L.m_b = o;     o = al(o + (size_t)p * 4);
    L.v_b = o;     o = al(o + (size_t)p * 4);
    L.wb_b = o;    o = al(o + (size_t)q * 2);
    L.wt_b = o;    o = al(o + (size_t)t * 2);
    L.stats_b = o; o = al(o + 64 * 4);
    L.step_b = o;  o = al(o + 16);
    L.wi_b = o;    o = al(o + (size_t)IMG_ELEMS * 2);
    L.bytes = o;
    return L;
}
static const Layout LAY = make_layout();

struct MemberPtrs {
    float *theta, *m, *v, *stats;
    bf16 *wb, *wt, *wi;
    int* step;
};
static MemberPtrs member(void* model, int k) {
    char* base = (char*)model + (size_t)k * LAY.bytes;
    MemberPtrs p;
    p.theta = (float*)(base + LAY.theta_b);
    p.m = (float*)(base + LAY.m_b);
    p.v = (float*)(base + LAY.v_b);
    p.wb = (bf16*)(base + LAY.wb_b);
    p.wt = (bf16*)(base + LAY.wt_b);
    p.stats = (float*)(base + LAY.stats_b);
    p.step = (int*)(base + LAY.step_b);
    p.wi = (bf16*)(base + LAY.wi_b);
    return p;
}

// ----------------------------------------------------------------------- GEMM kernel
enum Mode {
    FWD_HIDDEN = 0,    // Z = acc + b; H = GELU(Z) (bf16) and H^T; GELU'(Z) (bf16)
    FWD_OUT = 2,       // softmax(acc + b) over 3 columns -> P; CE gradient G, G^T; loss
    BWD_HIDDEN = 4,    // dZ = acc * GELU'(Z_prev) (stored by FWD_HIDDEN) -> dZ (bf16), dZ^T
    DW_PARTIAL = 5,    // partial[split] = acc (fp32)
};

struct GemmArgs {
    int M, N;              // output rows / columns (unpadded extents to store)
    int k_per_split;       // multiple of BK
    const float* bias;     // [N]
    float* out_f;          // Z [M][ldf] | P [M][4] | partial [split][M][ldf]
    int ldf;
    bf16* out_h;           // H | G | dZ  [M][ldh]
    int ldh;
    bf16* out_t;           // H^T | G^T | dZ^T  [N][ldt]
    int ldt;
    const float* aux;      // targets [M][3] (FWD_OUT)
    int ld_aux;
    bf16* out_g;           // GELU'(Z) [M][ldh] (FWD_HIDDEN)
    const bf16* aux_g;     // GELU'(Z_prev) [M][ld_aux] (BWD_HIDDEN)
    float* loss_sum;
    float inv_batch;
    unsigned* status;
    int a_rows_box;        // rows of the A box (128, or fewer when A has fewer rows)
    unsigned tx_bytes;     // bytes one stage receives from the two TMA loads
    long long wait_limit;  // cycles an mbarrier wait may take before the kernel gives up
    int test_stall;        // test only: the producer never issues the load of chunk 0
};

// GELU in its tanh form, z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), with the
// hardware tanh approximation (relative error ~2^-11, below BF16 rounding).
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// GELU and its derivative from one tanh: d/dz [z/2 (1 + t)] = (1 + t)/2 + z/2 (1 - t^2) du/dz
// with t = tanh(u), u = sqrt(2/pi) (z + 0.044715 z^3).
__device__ __forceinline__ void gelu_and_grad(float z, float& gel, float& grad) {
    const float z2 = z * z;
    const float t = tanh_fast(z * fmaf(0.0356774081f, z2, 0.7978845608f));
    const float dudz = fmaf(0.1070322243f, z2, 0.7978845608f);   // d/dz of the tanh argument
    const float hz = 0.5f * z;
    gel = fmaf(hz, t, hz);
    grad = fmaf(0.5f, 1.0f + t, hz * (1.0f - t * t) * dudz);
}

template <int NT>
struct Smem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = NT * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int TOTAL = BAR_OFF + (2 * STAGES + 1) * 8 + 16;
    static constexpr int ALLOC = TOTAL + 1024;   // slack for 1024-byte alignment
};

template <int NT, int MODE>
__global__ void __launch_bounds__(128, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                GemmArgs args) {
    using S = Smem<NT>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar_full = base + S::BAR_OFF;
    const uint32_t bar_empty = bar_full + STAGES * 8;
    const uint32_t bar_done = bar_empty + STAGES * 8;
    const uint32_t tslot = bar_done + 8;
    uint32_t* tslot_ptr = (uint32_t*)(gbase + S::BAR_OFF + (2 * STAGES + 1) * 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * NT;
    const int k0 = blockIdx.z * args.k_per_split;
    const int n_k = args.k_per_split / BK;
    constexpr uint32_t NCOLS = NT < 32 ? 32 : NT;
    constexpr uint32_t IDESC = idesc_bf16(BM, NT);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_done, 1);
        fence_barrier_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(tslot, NCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_ptr;

    bool ok = true;
    if (threadIdx.x == 0) {
        int last_issued = -1, consumed = 0;
        auto load = [&](int j) {
            const int s = j % STAGES;
            const uint32_t a_s = base + s * S::STAGE, b_s = a_s + S::A_BYTES;
            last_issued = j;
            if (args.test_stall && j == 0) return;   // test: this stage never fills
            mbar_arrive_expect_tx(bar_full + 8 * s, args.tx_bytes);
            tma_load_2d(a_s, &tmA, bar_full + 8 * s, k0 + j * BK, m0);
            tma_load_2d(b_s, &tmB, bar_full + 8 * s, k0 + j * BK, n0);
        };
        for (int j = 0; j < n_k && j < STAGES; ++j) load(j);
        for (int j = 0; j < n_k; ++j) {
            const int s = j % STAGES;
            const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
            if (!mbar_wait(bar_full + 8 * s, ph, args.wait_limit)) {
                ok = false;
                break;
            }
            consumed++;
            tc_fence_after();
            const uint32_t a_s = base + s * S::STAGE, b_s = a_s + S::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                mma_bf16(tmem, desc_sw128(a_s + kk * 32), desc_sw128(b_s + kk * 32), IDESC,
                         (j > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(bar_empty + 8 * s);
            if (j + STAGES < n_k) {
                if (!mbar_wait(bar_empty + 8 * s, ph, args.wait_limit)) {
                    ok = false;
                    break;
                }
                load(j + STAGES);
            }
        }
        mma_commit(bar_done);
        if (!ok) {
            // let every load that was issued land before the CTA can exit
            for (int j = consumed; j <= last_issued; ++j) {
                if (args.test_stall && j == 0) continue;
                mbar_wait(bar_full + 8 * (j % STAGES), (uint32_t)(j / STAGES) & 1u,
                          1000000000LL);
            }
            atomicOr(&args.status[ST_CALL], DEV_TIMEOUT);
        }
    }
    __syncwarp();
    const bool done_ok = mbar_wait(bar_done, 0, args.wait_limit);
    __syncwarp();
    tc_fence_after();
    if (!done_ok && threadIdx.x == 0) atomicOr(&args.status[ST_CALL], DEV_TIMEOUT);

    // ------------------------------------------------------------------ epilogue
    const int r = warp * 32 + lane;           // tile row held by this thread
    const int m = m0 + r;
    const bool row_ok = m < args.M && done_ok;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float v[16];
    if (MODE == FWD_OUT) {
        tmem_ld16(trow, v);
        float li = 0.f;
        if (row_ok) {
            float lg[N_OUT], p[N_OUT];
            float mx = -3.0e38f;
#pragma unroll
            for (int c = 0; c < N_OUT; ++c) {
                lg[c] = v[c] + args.bias[c];
                mx = fmaxf(mx, lg[c]);
            }
            float sum = 0.f;
#pragma unroll
            for (int c = 0; c < N_OUT; ++c) {
                p[c] = expf(lg[c] - mx);
                sum += p[c];
            }
            const float inv = 1.0f / sum;
#pragma unroll
            for (int c = 0; c < N_OUT; ++c) p[c] *= inv;
            *reinterpret_cast<float4*>(args.out_f + (long long)m * 4) =
                make_float4(p[0], p[1], p[2], 0.f);
            if (MODE == FWD_OUT) {
#pragma unroll
                for (int c = 0; c < N_OUT; ++c) {
                    const float y = args.aux[(long long)m * 3 + c];
                    li -= y * logf(fmaxf(p[c], 1e-30f));
                    const bf16 gb = __float2bfloat16((p[c] - y) * args.inv_batch);
                    args.out_h[(long long)m * args.ldh + c] = gb;
                    args.out_t[(long long)c * args.ldt + m] = gb;
                }
            }
        }
        if (MODE == FWD_OUT) {   // batch-mean loss: warp sum, one atomic per warp
            li *= args.inv_batch;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) li += __shfl_xor_sync(0xffffffffu, li, off);
            if (lane == 0 && li != 0.f) atomicAdd(args.loss_sum, li);
        }
    } else {
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            __syncwarp();
            tmem_ld16(trow + c0, v);
            const int n = n0 + c0;
            if (!row_ok || n >= args.N) continue;
            if (MODE == DW_PARTIAL) {
                float* dst = args.out_f + (long long)blockIdx.z * args.M * args.ldf +
                             (long long)m * args.ldf + n;
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                continue;
            }
            __align__(16) bf16 hb[16];
            if (MODE == BWD_HIDDEN) {
                __align__(16) bf16 gp[16];
                const uint4* gs = reinterpret_cast<const uint4*>(args.aux_g + (long long)m * args.ld_aux + n);
                reinterpret_cast<uint4*>(gp)[0] = gs[0];
                reinterpret_cast<uint4*>(gp)[1] = gs[1];
#pragma unroll
                for (int i = 0; i < 16; ++i) hb[i] = __float2bfloat16(v[i] * __bfloat162float(gp[i]));
            } else {
                __align__(16) bf16 gd[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float gel, grad;
                    gelu_and_grad(v[i] + args.bias[n + i], gel, grad);
                    hb[i] = __float2bfloat16(gel);
                    gd[i] = __float2bfloat16(grad);
                }
                uint4* gdst = reinterpret_cast<uint4*>(args.out_g + (long long)m * args.ldh + n);
                gdst[0] = reinterpret_cast<const uint4*>(gd)[0];
                gdst[1] = reinterpret_cast<const uint4*>(gd)[1];
            }
            uint4* hd = reinterpret_cast<uint4*>(args.out_h + (long long)m * args.ldh + n);
            hd[0] = reinterpret_cast<const uint4*>(hb)[0];
            hd[1] = reinterpret_cast<const uint4*>(hb)[1];
#pragma unroll
            for (int i = 0; i < 16; ++i) args.out_t[(long long)(n + i) * args.ldt + m] = hb[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ----------------------------------------------------------------- fused inference
// The whole ensemble forward pass for 128-row tiles in one persistent kernel (one CTA
// per SM): raw features -> standardise -> 4 x (tcgen05 MMA, bias + GELU) -> MMA, softmax
// -> ensemble mean, spread and fallback flag.  Activations never leave the SM: they live
// in tensor memory, which holds the FP32 accumulator (columns 0-255) and two BF16
// activation buffers (columns 256-383 and 384-511, one 128 x 256 tile each, two elements
// per column).  A layer's MMAs read their A operand from one buffer while its epilogue
// writes the next layer's input into the other.
//
// Each layer's output is produced in two halves of 128 columns (MMAs with N = 128, the
// narrowest that keeps the tensor pipe at full rate; one commit per half), so that the
// epilogue of half 0 runs while the MMAs of half 1 do.  Half h of the epilogue is k
// blocks 2h, 2h + 1 of the next layer's input, and the next layer's first MMAs take
// those k blocks as soon as the half is written: only k blocks 2-3 wait for the
// epilogue of half 1.
//
// Weights stream from the model's weight image (L2-resident) through a ring of 32 KB
// stages filled by untiled bulk copies, in the order the MMAs use them: layer 0 whole,
// then per hidden layer (half 0, inputs 0-127), (half 0, inputs 128-255), (half 1, ...),
// then layer 4 (16 output rows).
//
// Roles: the epilogue warps 0-15; warp w reads and writes TMEM lanes 32 (w mod 4) .. +31
// (its tile rows), and in each half the 32 columns 32 (w / 4) .. +31.  The warps with
// w < 4 also build the layer-0 input and keep the ensemble sums of their rows.  Lane 0 of
// warp 16 issues the bulk copies; lane 0 of warp 17 issues the MMAs.  Barriers: full and
// empty per ring slot; `acc` h (an MMA commit: output half h of the layer is
// accumulated); `a_rdy` h (512 arrivals: k blocks 2h, 2h + 1 of the next layer's input are
// written and output half h read out); `par` (parameter staging).  Every wait is
// bounded; a wait that gives up sets DEV_TIMEOUT, and the kernel drains its copies and
// MMAs and returns.
constexpr int FI_STAGES = 6;
constexpr int FI_SLOT = 32768;
constexpr int FI_ITEMS = 1 + 4 * 3 + 1;                  // ring items per tile and member
// Per-member parameters staged in shared memory: biases of the 5 layers (256 each; the
// hidden layers' halved, see the epilogue) and the feature means and standard deviations
// (16 each); slots for up to 4 members.
constexpr int FI_PAR_FLOATS = N_LAYERS * 256 + 32;
constexpr int FI_PAR_SLOTS = 4;
constexpr int FI_PAR_BYTES = FI_PAR_SLOTS * FI_PAR_FLOATS * 4;
constexpr int FI_NBARS = 2 * FI_STAGES + 2 + 2 + 1;
constexpr int FI_BAR_BYTES = 8 * FI_NBARS + 16;
constexpr int FI_SMEM = FI_STAGES * FI_SLOT + FI_PAR_BYTES + FI_BAR_BYTES;
constexpr int FI_EPI_WARPS = 16;
constexpr int FI_THREADS = 32 * (FI_EPI_WARPS + 2);
constexpr uint32_t FI_TMEM_COLS = 512;
constexpr uint32_t FI_ACC = 0;      // accumulator columns 0-255
constexpr uint32_t FI_ABUF = 256;   // activation buffers: 256 + 128 b, b = 0, 1

struct InferArgs {
    const float* feat;          // raw features [n_rows][9]
    long long n_rows;
    int n_members;
    const uint8_t* model;
    size_t member_bytes, theta_b, stats_b, wi_b;
    long long b_off[N_LAYERS];  // bias offsets in theta (floats)
    float* rat;                 // [n_rows][3]
    float* spread;              // [n_rows] or NULL
    unsigned char* needs;       // [n_rows] or NULL
    float thr;
    unsigned* status;
    long long wait_limit;
    int test_stall;             // test only: the first weight copy is never issued
};

// Ring item q (0..13) of a tile-member: layer, stage index within the layer (2h + j for
// layers 1-3), source offset in the image (elements) and size.  Item 13 is layer 4 whole
// (its four 2 KB k blocks).
__device__ __forceinline__ void fi_item(int q, int& layer, int& blk, long long& src,
                                        uint32_t& bytes) {
    if (q == 0) {
        layer = 0; blk = 0;
    } else if (q < 13) {
        layer = 1 + (q - 1) / 4;
        blk = (q - 1) & 3;
    } else {
        layer = 4; blk = 0;
    }
    src = img_off(layer) + (long long)blk * IMG_BLK;
    bytes = (layer == 4) ? (uint32_t)(4 * IMG_L4_BLK * 2) : (uint32_t)FI_SLOT;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&p);
}
// Two-lane FP32 arithmetic (one instruction for both lanes, each lane rounded as the
// scalar operation would be).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// GELU (tanh form) of z = 2 hz from hz = z/2 = acc/2 + bias/2, for two columns: hz (1 +
// tanh(u)) with u = z (c0 + c1 z^2) = hz (2 c0 + 8 c1 hz^2), c0 = sqrt(2/pi), c1 =
// 0.044715 c0; returned as a packed BF16 pair.
__device__ __forceinline__ uint32_t gelu_half2(float acc0, float acc1, float hb0, float hb1) {
    const float2 hz = fma2(make_float2(0.5f, 0.5f), make_float2(acc0, acc1), make_float2(hb0, hb1));
    const float2 h2 = mul2(hz, hz);
    const float2 u = mul2(hz, fma2(make_float2(0.2854192648f, 0.2854192648f), h2,
                                   make_float2(1.5957691216f, 1.5957691216f)));
    const float2 g = fma2(hz, make_float2(tanh_fast(u.x), tanh_fast(u.y)), hz);
    return pack_bf16(g.x, g.y);
}

__global__ void __launch_bounds__(FI_THREADS, 1) infer_kernel(InferArgs A) {
    extern __shared__ __align__(1024) uint8_t fi_smem[];
    const uint32_t base = smem_u32(fi_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ring = base;
    float* par = reinterpret_cast<float*>(fi_smem + FI_STAGES * FI_SLOT);
    const uint32_t bars = ring + FI_STAGES * FI_SLOT + FI_PAR_BYTES;
    const uint32_t bar_full = bars, bar_empty = bars + 8 * FI_STAGES;
    const uint32_t bar_acc = bars + 16 * FI_STAGES;   // 2: output half h accumulated
    const uint32_t bar_a = bar_acc + 16;              // 2: input k blocks 2h, 2h+1 written
    const uint32_t bar_p = bar_a + 16;                // parameter staging done
    const uint32_t tslot = bar_p + 8;
    uint8_t* bars_g = fi_smem + FI_STAGES * FI_SLOT + FI_PAR_BYTES;
    volatile uint32_t* tslot_ptr = reinterpret_cast<volatile uint32_t*>(bars_g + 8 * FI_NBARS);
    volatile int& abort_flag = *reinterpret_cast<volatile int*>(bars_g + 8 * FI_NBARS + 4);

    if ((base & 1023u) != 0u) {   // the swizzled stages need 1024-byte alignment
        if (threadIdx.x == 0) atomicOr(&A.status[ST_CALL], DEV_RANGE);
        return;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < FI_STAGES; ++i) {
            mbar_init(bar_full + 8 * i, 1);
            mbar_init(bar_empty + 8 * i, 1);
        }
        for (int h = 0; h < 2; ++h) {
            mbar_init(bar_acc + 8 * h, 1);
            mbar_init(bar_a + 8 * h, 32 * FI_EPI_WARPS);
        }
        mbar_init(bar_p, 32 * FI_EPI_WARPS);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(tslot, FI_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_ptr;

    const long long n_tiles = (A.n_rows + 127) / 128;
    const int M = A.n_members;
    const long long my_tiles =
        n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = my_tiles * M * FI_ITEMS;

    if (warp == FI_EPI_WARPS) {
        // ------------------------------------------------------------ bulk copies
        if (lane == 0) {
            long long issued = 0;
            int slot = 0, item = 0, member = 0;
            uint32_t phase = 0;
            bool ok = true;
            const uint8_t* wi0 = A.model + A.wi_b;
            for (; issued < total && ok && !abort_flag; ++issued) {
                if (issued >= FI_STAGES &&
                    !mbar_wait_sleep(bar_empty + 8 * slot, phase ^ 1u, A.wait_limit)) {
                    ok = false;
                    break;
                }
                int layer, blk;
                long long src;
                uint32_t bytes;
                fi_item(item, layer, blk, src, bytes);
                if (!(A.test_stall && issued == 0)) {
                    mbar_arrive_expect_tx(bar_full + 8 * slot, bytes);
                    bulk_load(ring + slot * FI_SLOT,
                              wi0 + (size_t)member * A.member_bytes + (size_t)src * 2, bytes,
                              bar_full + 8 * slot);
                }
                if (++slot == FI_STAGES) {
                    slot = 0;
                    phase ^= 1u;
                }
                if (++item == FI_ITEMS) {
                    item = 0;
                    if (++member == M) member = 0;
                }
            }
            if (!ok) {
                atomicOr(&A.status[ST_CALL], DEV_TIMEOUT);
                abort_flag = 1;
            }
            // the last copy of each slot has landed before the CTA exits
            const long long first = issued > FI_STAGES ? issued - FI_STAGES : 0;
            for (long long g = first; g < issued; ++g) {
                if (A.test_stall && g == 0) continue;   // never issued
                mbar_wait(bar_full + 8 * (int)(g % FI_STAGES), (uint32_t)(g / FI_STAGES) & 1u,
                          1000000000LL);
            }
        }
        __syncwarp();
    } else if (warp == FI_EPI_WARPS + 1) {
        // ------------------------------------------------------------ MMAs
        if (lane == 0) {
            int slot = 0;
            uint32_t phase = 0, pa = 0;
            long long consumed = 0;
            bool ok = true;
            const uint64_t dring = desc_sw128(ring);
            constexpr uint32_t ID128 = idesc_bf16(128, 128), ID16 = idesc_bf16(128, 16);
            // next ring slot, once its copy has landed (bounded wait)
            auto take = [&](int& s) {
                if (!mbar_wait(bar_full + 8 * slot, phase, A.wait_limit)) return false;
                s = slot;
                ++consumed;
                if (++slot == FI_STAGES) {
                    slot = 0;
                    phase ^= 1u;
                }
                return true;
            };
            // k blocks 2h, 2h + 1 of the layer's input are written (bounded wait)
            auto wait_a = [&](int h) {
                if (!mbar_wait_sleep(bar_a + 8 * h, pa, A.wait_limit) || abort_flag) return false;
                tc_fence_after();
                return true;
            };
            auto bdesc = [&](int s) { return dring + (uint64_t)(s * (FI_SLOT >> 4)); };
            for (long long t = 0; t < my_tiles && ok; ++t) {
                for (int k = 0; k < M && ok; ++k) {
                    for (int l = 0; l < N_LAYERS && ok; ++l) {
                        const uint32_t ta = tmem + FI_ABUF + (uint32_t)((l & 1) * 128);
                        int s = 0;
                        if (l == 0) {
                            // K = 16 covers the 9 features; half h of the 256 output rows
                            // starts 128 rows (16 KB) into the stage
                            if (!(ok = take(s))) break;
                            ok = wait_a(0) && wait_a(1);
                            if (ok)
                                for (int h = 0; h < 2; ++h) {
                                    mma_bf16_ts(tmem + FI_ACC + (uint32_t)(h * 128), ta,
                                                bdesc(s) + (uint64_t)(h * (16384 >> 4)), ID128, 0u);
                                    mma_commit(bar_acc + 8 * h);
                                }
                            mma_commit(bar_empty + 8 * s);
                        } else if (l < 4) {
                            // stage (h, j): output rows 128 h .. +127 x k blocks 2j, 2j + 1
                            for (int h = 0; h < 2 && ok; ++h) {
                                for (int j = 0; j < 2 && ok; ++j) {
                                    if (!(ok = take(s))) break;
                                    if (h == 0 && !(ok = wait_a(j))) {
                                        mma_commit(bar_empty + 8 * s);
                                        break;
                                    }
#pragma unroll
                                    for (int x = 0; x < 2; ++x) {
                                        const int kb = 2 * j + x;
#pragma unroll
                                        for (int kk = 0; kk < 4; ++kk)
                                            mma_bf16_ts(tmem + FI_ACC + (uint32_t)(h * 128),
                                                        ta + (uint32_t)(kb * 32 + kk * 8),
                                                        bdesc(s) + (uint64_t)(x * (16384 >> 4) + 2 * kk),
                                                        ID128, (kb > 0 || kk > 0) ? 1u : 0u);
                                    }
                                    mma_commit(bar_empty + 8 * s);
                                }
                                if (ok) mma_commit(bar_acc + 8 * h);
                            }
                        } else {
                            // the 16 padded output columns (3 real), four 2 KB k blocks
                            if (!(ok = take(s))) break;
                            for (int kb = 0; kb < 4 && ok; ++kb) {
                                if ((kb & 1) == 0 && !(ok = wait_a(kb >> 1))) break;
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk)
                                    mma_bf16_ts(tmem + FI_ACC, ta + (uint32_t)(kb * 32 + kk * 8),
                                                bdesc(s) + (uint64_t)(kb * ((int)IMG_L4_BLK * 2 >> 4) + 2 * kk),
                                                ID16, (kb > 0 || kk > 0) ? 1u : 0u);
                            }
                            mma_commit(bar_empty + 8 * s);
                            if (ok)
                                for (int h = 0; h < 2; ++h) mma_commit(bar_acc + 8 * h);
                        }
                        pa ^= 1u;
                    }
                }
            }
            if (!ok) {
                atomicOr(&A.status[ST_CALL], DEV_TIMEOUT);
                abort_flag = 1;
            }
            // every MMA has finished before the CTA exits (commits complete in order)
            if (consumed > 0) {
                const long long g = consumed - 1;
                mbar_wait(bar_empty + 8 * (int)(g % FI_STAGES), (uint32_t)(g / FI_STAGES) & 1u,
                          1000000000LL);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue warps
        const int lq = warp & 3, cg = warp >> 2;            // TMEM lane quarter, column group
        const int r = lq * 32 + lane;                       // tile row = TMEM lane
        const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16);
        const bool lead = cg == 0;                          // builds X0, keeps the ensemble
        const int et = threadIdx.x;                         // 0 .. 32 * FI_EPI_WARPS - 1
        uint32_t pp = 0;
        bool ok = true;
        // stages member k's biases (hidden layers halved, for gelu_half) and feature
        // statistics into parameter slot k mod 4, then waits (bounded) until every
        // epilogue thread has written its share
        auto stage = [&](int k) {
            const uint8_t* mb = A.model + (size_t)k * A.member_bytes;
            const float* th = reinterpret_cast<const float*>(mb + A.theta_b);
            const float* st = reinterpret_cast<const float*>(mb + A.stats_b);
            float* dst = par + (k % FI_PAR_SLOTS) * FI_PAR_FLOATS;
            for (int i = et; i < FI_PAR_FLOATS; i += 32 * FI_EPI_WARPS) {
                float v;
                if (i < N_LAYERS * 256) {
                    const int l = i >> 8, c = i & 255;
                    v = (c < real_out(l)) ? __ldg(th + A.b_off[l] + c) : 0.f;
                    if (l < 4) v *= 0.5f;
                } else {
                    v = __ldg(st + (i - N_LAYERS * 256));   // mean[16] | std[16]
                }
                dst[i] = v;
            }
            mbar_arrive(bar_p);
            if (!mbar_wait_sleep(bar_p, pp, A.wait_limit)) ok = false;
            pp ^= 1u;
        };
        const bool staged_once = M <= FI_PAR_SLOTS;
        if (staged_once)
            for (int k = 0; k < M && ok; ++k) stage(k);
        uint32_t pacc = 0;
        for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const long long row = t * 128 + r;
            const bool live = row < A.n_rows;
            float x[N_FEAT];
#pragma unroll
            for (int f = 0; f < N_FEAT; ++f)
                x[f] = (lead && live) ? A.feat[row * N_FEAT + f] : 0.f;
            float mean[3] = {0.f, 0.f, 0.f}, lo[3] = {3.f, 3.f, 3.f}, hi[3] = {-3.f, -3.f, -3.f};
            for (int k = 0; k < M && ok; ++k) {
                if (!staged_once) {
                    stage(k);
                    if (!ok) break;
                }
                const float* pk_par = par + (k % FI_PAR_SLOTS) * FI_PAR_FLOATS;
                if (lead) {   // layer-0 input: standardised features in k 0-8, zeros to 15
                    const float* st = pk_par + N_LAYERS * 256;
                    float z[N_FEAT];
#pragma unroll
                    for (int f = 0; f < N_FEAT; ++f) z[f] = (x[f] - st[f]) / st[16 + f];
                    const uint32_t pk[8] = {pack_bf16(z[0], z[1]), pack_bf16(z[2], z[3]),
                                            pack_bf16(z[4], z[5]), pack_bf16(z[6], z[7]),
                                            pack_bf16(z[8], 0.f), 0u, 0u, 0u};
                    tmem_st8(trow + FI_ABUF, pk);
                    tmem_wait_st();
                }
                tc_fence_before();
                mbar_arrive(bar_a);
                mbar_arrive(bar_a + 8);
                for (int l = 0; l < N_LAYERS && ok; ++l) {
                    // pacc: parity of this layer's phase of the acc barriers; every thread
                    // waits for both halves of every layer (a parity wait that fell two
                    // phases behind its barrier would return at once)
                    const float* bias = pk_par + l * 256;
                    const uint32_t dst = trow + FI_ABUF + (uint32_t)(((l + 1) & 1) * 128);
                    for (int h = 0; h < 2; ++h) {
                        if (!mbar_wait_sleep(bar_acc + 8 * h, pacc, A.wait_limit)) {
                            ok = false;
                            break;
                        }
                        if (l == 4) continue;
                        tc_fence_after();
                        uint32_t v[32];
                        tmem_ld32_async(trow + FI_ACC + (uint32_t)(h * 128 + cg * 32), v);
                        tmem_wait_ld(v);
                        // output columns 128 h + 32 cg .. +31 = next-layer inputs, two per
                        // TMEM column, stored 16 at a time
#pragma unroll
                        for (int c16 = 0; c16 < 32; c16 += 16) {
                            const float* b = bias + h * 128 + cg * 32 + c16;
                            uint32_t pk[8];
#pragma unroll
                            for (int i = 0; i < 16; i += 4) {
                                const float4 b4 = *reinterpret_cast<const float4*>(b + i);
                                pk[i / 2] = gelu_half2(__uint_as_float(v[c16 + i]),
                                                       __uint_as_float(v[c16 + i + 1]), b4.x, b4.y);
                                pk[i / 2 + 1] = gelu_half2(__uint_as_float(v[c16 + i + 2]),
                                                           __uint_as_float(v[c16 + i + 3]), b4.z,
                                                           b4.w);
                            }
                            tmem_st8(dst + (uint32_t)(h * 64 + cg * 16 + c16 / 2), pk);
                        }
                        tmem_wait_st();
                        tc_fence_before();
                        mbar_arrive(bar_a + 8 * h);
                    }
                    if (ok && l == 4 && lead) {
                        tc_fence_after();
                        float v[16];
                        tmem_ld16(trow + FI_ACC, v);
                        float lg[N_OUT], mx = -3.0e38f;
#pragma unroll
                        for (int c = 0; c < N_OUT; ++c) {
                            lg[c] = v[c] + bias[c];
                            mx = fmaxf(mx, lg[c]);
                        }
                        float p[N_OUT], sum = 0.f;
#pragma unroll
                        for (int c = 0; c < N_OUT; ++c) {
                            p[c] = expf(lg[c] - mx);
                            sum += p[c];
                        }
                        const float inv = 1.0f / sum;
#pragma unroll
                        for (int c = 0; c < N_OUT; ++c) {
                            const float q = p[c] * inv;
                            mean[c] += q;
                            lo[c] = fminf(lo[c], q);
                            hi[c] = fmaxf(hi[c], q);
                        }
                    }
                    pacc ^= 1u;
                }
                if (abort_flag) ok = false;
            }
            if (ok && lead && live) {
                float spr = 0.f;
#pragma unroll
                for (int c = 0; c < N_OUT; ++c) {
                    A.rat[row * 3 + c] = mean[c] / (float)M;
                    spr = fmaxf(spr, hi[c] - lo[c]);
                }
                if (A.spread) A.spread[row] = spr;
                if (A.needs) {
                    const float* st0 = reinterpret_cast<const float*>(A.model + A.stats_b);
                    bool out = spr > A.thr;
#pragma unroll
                    for (int f = 0; f < N_FEAT; ++f)
                        out = out || !(x[f] >= __ldg(st0 + 32 + f) && x[f] <= __ldg(st0 + 48 + f));
                    A.needs[row] = out ? 1 : 0;
                }
            }
        }
        if (!ok) atomicOr(&A.status[ST_CALL], DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, FI_TMEM_COLS);
}

// ----------------------------------------------------------------------- small kernels
// Raw features of row (d, w): wavelength, n_p, log10 k_p, radius, volume fraction,
// log10 thickness, g, log10(mu_s d + 1e-6), log10(mu_a d + 1e-6).
__global__ void features_kernel(int n_designs, int n_wl, const double* wl, const double* np_re,
                                const double* np_im, const double* radius, const double* vf,
                                const double* thick, const double* g, const double* mu_s,
                                const double* mu_a, float* out, unsigned* status) {
    const long long n = (long long)n_designs * n_wl;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int d, w;
        if (n <= 0xffffffffLL) {   // 32-bit division where the row count allows it
            d = (int)((unsigned)i / (unsigned)n_wl);
            w = (int)((unsigned)i - (unsigned)d * (unsigned)n_wl);
        } else {
            d = (int)(i / n_wl);
            w = (int)(i % n_wl);
        }
        const double t = thick[d];
        float* o = out + i * N_FEAT;
        // the logarithms in FP32: the features are FP32, and an FP64 log10 costs tens of
        // instructions on GB300's narrow FP64 pipe
        o[0] = (float)wl[w];
        o[1] = (float)np_re[i];
        o[2] = log10f((float)fmax(np_im[i], 1e-12));
        o[3] = (float)radius[d];
        o[4] = (float)vf[d];
        o[5] = log10f((float)t);
        o[6] = (float)g[i];
        o[7] = log10f((float)(mu_s[i] * t + 1e-6));
        o[8] = log10f((float)(mu_a[i] * t + 1e-6));
        if (!(t > 0.0) || !isfinite(mu_s[i]) || !isfinite(mu_a[i]))
            atomicOr(&status[ST_CALL], DEV_INVALID);
    }
}

// Features of a homogeneous slab given by its optical properties (the inputs of the
// paper's network, Table 1: matrix index, mu_s, mu_a, g, thickness):
// [n, log10(mu_s + 1e-4), log10(mu_a + 1e-4), g, log10 d, log10(mu_s d + 1e-6),
//  log10(mu_a d + 1e-6), log10(1 - g + 1e-3), log10(mu_s (1 - g) d + 1e-6)].  Each raw
// input maps monotonically to one of the first five features, so a box in feature space
// holds the box of Table 1; the optical depths, 1 - g and the reduced scattering depth
// help the fit (transport near g = 1 depends on mu_s (1 - g)).
__global__ void features_slab_kernel(long long n, const double* nl, const double* mu_s,
                                     const double* mu_a, const double* g, const double* d,
                                     float* out, unsigned* status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double t = d[i], ms = mu_s[i], ma = mu_a[i];
        float* o = out + i * N_FEAT;
        o[0] = (float)nl[i];
        o[1] = (float)log10(ms + 1e-4);
        o[2] = (float)log10(ma + 1e-4);
        o[3] = (float)g[i];
        o[4] = (float)log10(t);
        o[5] = (float)log10(ms * t + 1e-6);
        o[6] = (float)log10(ma * t + 1e-6);
        o[7] = (float)log10(1.0 - g[i] + 1e-3);
        o[8] = (float)log10(ms * (1.0 - g[i]) * t + 1e-6);
        if (!(t > 0.0) || !(ms >= 0.0) || !(ma >= 0.0) || !isfinite(ms * t) ||
            !isfinite(ma * t) || !(nl[i] > 0.0) || !isfinite(g[i]))
            atomicOr(&status[ST_CALL], DEV_INVALID);
    }
}

__global__ void fractions_kernel(const long long* counts, long long n, const int* rows,
                                 float* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long* c = counts + i * FOS_NCOUNT;
        const double tot = (double)(c[0] + c[1] + c[2]);
        const double inv = tot > 0 ? 1.0 / tot : 0.0;
        const long long o = rows ? (long long)rows[i] : i;
        out[o * 3 + 0] = (float)(c[0] * inv);
        out[o * 3 + 1] = (float)(c[1] * inv);
        out[o * 3 + 2] = (float)(c[2] * inv);
    }
}

// Indices of the nonzero bytes of mask [n] -> rows (ascending within each block of 1024,
// blocks in any order) and their number in *count (which must start at 0).
__global__ void mask_rows_kernel(const unsigned char* mask, long long n, int* rows,
                                 unsigned long long* count) {
    __shared__ unsigned wsum[32];
    __shared__ unsigned long long base;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool on = i < n && mask[i] != 0;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (unsigned w = 0; w < blockDim.x / 32; ++w) {
            const unsigned v = wsum[w];
            wsum[w] = tot;
            tot += v;
        }
        base = tot ? atomicAdd(count, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    if (on) rows[base + wsum[warp] + __popc(bal & ((1u << lane) - 1u))] = (int)i;
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {   // a 32-bit integer hash (murmur3 finaliser)
    x ^= x >> 16; x *= 0x85ebca6bu; x ^= x >> 13; x *= 0xc2b2ae35u; x ^= x >> 16;
    return x;
}

// Training batch: rows given, or drawn uniformly (with replacement) by hashing (seed,
// step, slot);
// standardised features -> X0 [B][64] and X0^T [64][B] (pads stay 0); targets -> Y.
// Step schedule of one member's training step, computed on the device from the member's
// step counter (graph-captured training, where the host does not see each step).
struct SchedOut {
    unsigned step;        // the member's global step g (Adam's t = g + 1)
    float lr, c1, c2;     // learning rate; 1 - b1^t, 1 - b2^t
};

// Device schedule of graph-captured training: the member's step counter g, the table of
// the call's steps (entry g - *base, written by the host with the same arithmetic as the
// per-step entry point), and where the step's entry goes for Adam.
struct DevSched {
    int* step_ctr;
    const SchedOut* table;
    const int* base;
    SchedOut* out;
};

__global__ void set_step_kernel(int* step_ctr, int value) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *step_ctr = value;
}

// With a device schedule (ds.step_ctr non-NULL) the step is the member's step counter, and
// thread 0 also writes the step's schedule for Adam (the counter advances in the bias
// gradient kernel, after every thread here has read it).
__global__ void gather_kernel(const float* feat, const float* targets, long long n_rows, int B,
                              unsigned seed, unsigned step, const int* rows, const float* stats,
                              bf16* X0, bf16* X0T, float* Y, DevSched ds) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (ds.step_ctr) {
        const int g = *ds.step_ctr;
        step = (unsigned)g;
        if (b == 0) *ds.out = ds.table[g - *ds.base];
    }
    if (b >= B) return;
    long long src;
    if (rows) {
        src = rows[b];
    } else {
        const uint32_t h = mix32(mix32(seed ^ 0x9E3779B9u) ^ mix32(step * 0x85ebca6bu + (uint32_t)b));
        src = (long long)(((unsigned long long)h * (unsigned long long)n_rows) >> 32);
    }
    for (int f = 0; f < N_FEAT; ++f) {
        const float x = (feat[src * N_FEAT + f] - stats[f]) / stats[16 + f];
        const bf16 xb = __float2bfloat16(x);
        X0[(long long)b * IN_PAD + f] = xb;
        X0T[(long long)f * B + b] = xb;
    }
    for (int c = 0; c < N_OUT; ++c) Y[(long long)b * 3 + c] = targets[src * 3 + c];
}

// Column sums of a bf16 [rows][ld] matrix (bias gradients), in two deterministic
// passes.  Pass 1: block (x, y) sums rows y*chunk .. +chunk of columns 64x .. +63 (4 row
// phases, then a fixed combine) into part[y][c].  Pass 2 sums the COLSUM_SPLITS partials
// of each column in order.
constexpr int COLSUM_SPLITS = 64;
// Bias gradients of all layers in one launch (blockIdx.z = layer): per-split column sums
// part[l][split][c] of layer l's output gradient G_l [rows][ld]; Adam adds the splits in
// a fixed order, so the result does not depend on scheduling.
struct ColsumArgs {
    const bf16* G[N_LAYERS];
    int ld[N_LAYERS];
    float* part[N_LAYERS];
    int rows;
    int* step_ctr;   // device schedule: advanced here (NULL: none)
};
__global__ void colsum_layers_kernel(ColsumArgs A) {
    __shared__ float ph[4][64];
    if (A.step_ctr && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
        *A.step_ctr += 1;
    const int l = blockIdx.z;
    const int ncols = real_out(l), rows = A.rows, ld = A.ld[l];
    if ((int)blockIdx.x * 64 >= ncols) return;   // the whole block: no column of this layer
    const bf16* G = A.G[l];
    float* part = A.part[l];
    const int c = blockIdx.x * 64 + (threadIdx.x & 63);
    const int q = threadIdx.x >> 6;   // 4 row phases
    const int chunk = (rows + COLSUM_SPLITS - 1) / COLSUM_SPLITS;
    const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float a0 = 0.f, a1 = 0.f;   // two running sums, loads in flight together
    if (c < ncols) {
        int r = r0 + q;
        for (; r + 4 < r1; r += 8) {
            a0 += __bfloat162float(G[(long long)r * ld + c]);
            a1 += __bfloat162float(G[(long long)(r + 4) * ld + c]);
        }
        if (r < r1) a0 += __bfloat162float(G[(long long)r * ld + c]);
    }
    const float acc = a0 + a1;
    ph[q][threadIdx.x & 63] = acc;
    __syncthreads();
    if (q == 0 && c < ncols)
        part[blockIdx.y * ncols + c] =
            ph[0][threadIdx.x] + ph[1][threadIdx.x] + ph[2][threadIdx.x] + ph[3][threadIdx.x];
}
// Sum of n values v[k * stride + e], k = 0..n-1, in a fixed order: four running sums over
// k mod 4 (their loads independent, so they are in flight together), then added in order.
__device__ __forceinline__ float split_sum(const float* v, long long stride, int n, long long e) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        a0 += v[(k + 0) * stride + e];
        a1 += v[(k + 1) * stride + e];
        a2 += v[(k + 2) * stride + e];
        a3 += v[(k + 3) * stride + e];
    }
    for (; k < n; ++k) a0 += v[k * stride + e];
    return (a0 + a1) + (a2 + a3);
}
// Bias gradient of output o of layer l from its per-split column sums.
__device__ __forceinline__ float bias_grad(const float* part, int ncols, int o) {
    return split_sum(part, ncols, COLSUM_SPLITS, o);
}

struct AdamArgs {
    float *theta, *m, *v;
    bf16 *wb, *wt, *wi;
    long long w_off[N_LAYERS], b_off[N_LAYERS], wb_off[N_LAYERS], wt_off[N_LAYERS];
    const float* part[N_LAYERS];   // split-K partials of dW_l [splits][out][in]
    const float* bpart[N_LAYERS];  // per-split column sums of G_l [COLSUM_SPLITS][real out]
    int splits;
    float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
    const SchedOut* sched;          // non-NULL: lr, c1, c2 from the device schedule
};

// Adam (Kingma & Ba) on every real parameter, then the bf16 copies W (and W^T for
// layers >= 1).  Padding stays zero.
__global__ void adam_kernel(AdamArgs A, long long P) {
    if (A.sched) {
        A.lr = A.sched->lr;
        A.c1 = A.sched->c1;
        A.c2 = A.sched->c2;
    }
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < N_LAYERS && idx >= A.w_off[l + 1]) ++l;
        const int in_p = lay_in(l), out_p = lay_out(l);
        float g;
        long long e = -1;
        int o, i = 0;
        if (idx < A.b_off[l]) {
            e = idx - A.w_off[l];
            o = (int)(e / in_p);
            i = (int)(e % in_p);
            if (o >= real_out(l) || i >= real_in(l)) continue;
            g = split_sum(A.part[l], (long long)out_p * in_p, A.splits, e);
        } else {
            o = (int)(idx - A.b_off[l]);
            if (o >= real_out(l)) continue;
            g = bias_grad(A.bpart[l], real_out(l), o);
        }
        const float mm = A.b1 * A.m[idx] + (1.f - A.b1) * g;
        const float vv = A.b2 * A.v[idx] + (1.f - A.b2) * g * g;
        A.m[idx] = mm;
        A.v[idx] = vv;
        const float th = A.theta[idx] - A.lr * (mm / A.c1) / (sqrtf(vv / A.c2) + A.eps);
        A.theta[idx] = th;
        if (e >= 0) {
            const bf16 tb = __float2bfloat16(th);
            A.wb[A.wb_off[l] + e] = tb;
            if (l > 0) A.wt[A.wt_off[l] + (long long)i * out_p + o] = tb;
            const long long ii = img_index(l, o, i);
            if (ii >= 0) A.wi[ii] = tb;
        }
    }
}

// The gradient vector in the layout of theta (padding 0): what adam_kernel consumes.
__global__ void grad_kernel(AdamArgs A, long long P, float* grad) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < N_LAYERS && idx >= A.w_off[l + 1]) ++l;
        const int in_p = lay_in(l), out_p = lay_out(l);
        float g = 0.f;
        if (idx < A.b_off[l]) {
            const long long e = idx - A.w_off[l];
            const int o = (int)(e / in_p), i = (int)(e % in_p);
            if (o < real_out(l) && i < real_in(l))
                g = split_sum(A.part[l], (long long)out_p * in_p, A.splits, e);
        } else {
            const int o = (int)(idx - A.b_off[l]);
            if (o < real_out(l)) g = bias_grad(A.bpart[l], real_out(l), o);
        }
        grad[idx] = g;
    }
}

// He-uniform initial weights (hash of seed, member, index -> uniform), zero biases,
// zero Adam state, bf16 copies, step 0.
__global__ void init_kernel(float* theta, float* m, float* v, bf16* wb, bf16* wt, bf16* wi,
                            int* step, unsigned seed, unsigned member, AdamArgs lay,
                            long long P) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < N_LAYERS && idx >= lay.w_off[l + 1]) ++l;
        const int in_p = lay_in(l), out_p = lay_out(l);
        float th = 0.f;
        long long e = -1;
        int o = 0, i = 0;
        if (idx < lay.b_off[l]) {
            e = idx - lay.w_off[l];
            o = (int)(e / in_p);
            i = (int)(e % in_p);
            if (o < real_out(l) && i < real_in(l)) {
                const uint32_t h = mix32(mix32(seed) ^ mix32(member * 0x27d4eb2du + 0x165667b1u) ^
                                         mix32((uint32_t)idx));
                const float u = ((float)(h >> 8) + 0.5f) * 0x1p-24f;   // (0,1)
                const float lim = sqrtf(6.0f / (float)real_in(l));
                th = (2.f * u - 1.f) * lim;
            }
        }
        theta[idx] = th;
        m[idx] = 0.f;
        v[idx] = 0.f;
        if (e >= 0) {
            const bf16 tb = __float2bfloat16(th);
            wb[lay.wb_off[l] + e] = tb;
            if (l > 0) wt[lay.wt_off[l] + (long long)i * out_p + o] = tb;
            const long long ii = img_index(l, o, i);
            if (ii >= 0) wi[ii] = tb;
        }
        if (idx == 0) step[0] = 0;
    }
}

// Parameters given by the caller (device theta in the padded layout): entries outside
// the real rows and columns are stored as 0; Adam state and step are reset and the bf16
// copies rebuilt.
__global__ void load_kernel(const float* src, float* theta, float* m, float* v, bf16* wb,
                            bf16* wt, bf16* wi, int* step, AdamArgs lay, long long P) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < N_LAYERS && idx >= lay.w_off[l + 1]) ++l;
        const int in_p = lay_in(l), out_p = lay_out(l);
        float th = 0.f;
        long long e = -1;
        int o = 0, i = 0;
        if (idx < lay.b_off[l]) {
            e = idx - lay.w_off[l];
            o = (int)(e / in_p);
            i = (int)(e % in_p);
            if (o < real_out(l) && i < real_in(l)) th = src[idx];
        } else if ((int)(idx - lay.b_off[l]) < real_out(l)) {
            th = src[idx];
        }
        theta[idx] = th;
        m[idx] = 0.f;
        v[idx] = 0.f;
        if (e >= 0) {
            const bf16 tb = __float2bfloat16(th);
            wb[lay.wb_off[l] + e] = tb;
            if (l > 0) wt[lay.wt_off[l] + (long long)i * out_p + o] = tb;
            const long long ii = img_index(l, o, i);
            if (ii >= 0) wi[ii] = tb;
        }
        if (idx == 0) step[0] = 0;
    }
}

// Feature statistics: per feature mean, standard deviation (floored at 1e-3 so that a
// feature constant over the training set cannot blow up), and the range [min, max]
// over n rows widened by 1 % of its span on each side (the trusted input range).
// One block per feature; FP64 accumulation; writes stats[f], [16+f], [32+f], [48+f].
__global__ void stats_kernel(const float* feat, long long n, float* stats) {
    __shared__ double s1[256], s2[256];
    __shared__ float mn[256], mx[256];
    const int f = blockIdx.x;
    double a = 0.0, b = 0.0;
    float lo = 3.0e38f, hi = -3.0e38f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float x = feat[i * N_FEAT + f];
        a += x;
        b += (double)x * x;
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    mn[threadIdx.x] = lo;
    mx[threadIdx.x] = hi;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            s1[threadIdx.x] += s1[threadIdx.x + off];
            s2[threadIdx.x] += s2[threadIdx.x + off];
            mn[threadIdx.x] = fminf(mn[threadIdx.x], mn[threadIdx.x + off]);
            mx[threadIdx.x] = fmaxf(mx[threadIdx.x], mx[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)n;
        const double var = s2[0] / (double)n - mean * mean;
        stats[f] = (float)mean;
        stats[16 + f] = fmaxf((float)sqrt(var > 0.0 ? var : 0.0), 1e-3f);
        const float span = fmaxf(mx[0] - mn[0], 1e-3f);
        stats[32 + f] = mn[0] - 0.01f * span;   // training range, widened by 1 % of its span
        stats[48 + f] = mx[0] + 0.01f * span;
    }
}

// ----------------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_mu;

static fos_status get_encoder() {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_encode) return FOS_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return FOS_ERR_CUDA;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return FOS_OK;
}

// 2-D BF16 row-major matrix [rows][ld] (K = cols used), box of box_rows x 64, 128B swizzle.
static fos_status make_map(CUtensorMap* map, const void* ptr, long long rows, long long cols,
                           long long ld, int box_rows) {
    if (((uintptr_t)ptr & 15u) != 0 || (ld * 2) % 16 != 0 || cols % BK != 0) return FOS_ERR_INVALID_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FOS_OK : FOS_ERR_CUDA;
}

struct Operand {
    const bf16* ptr;
    long long rows, cols, ld;   // cols = K extent (multiple of 64)
};

template <int NT, int MODE>
static fos_status gemm(const Operand& A, const Operand& B, int splits, GemmArgs g,
                       cudaStream_t s) {
    static bool attr_set[64] = {false};
    int dev = 0;
    FOS_CUDA_TRY(cudaGetDevice(&dev));
    if (!attr_set[dev]) {
        FOS_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel<NT, MODE>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          Smem<NT>::ALLOC));
        attr_set[dev] = true;
    }
    if (A.cols != B.cols || A.cols % ((long long)splits * BK) != 0) return FOS_ERR_INVALID_ARG;
    if (B.rows < NT) return FOS_ERR_INVALID_ARG;
    const int a_box = A.rows < BM ? (int)A.rows : BM;
    CUtensorMap ta, tb;
    fos_status st = make_map(&ta, A.ptr, A.rows, A.cols, A.ld, a_box);
    if (st != FOS_OK) return st;
    st = make_map(&tb, B.ptr, B.rows, B.cols, B.ld, NT);
    if (st != FOS_OK) return st;
    g.k_per_split = (int)(A.cols / splits);
    g.a_rows_box = a_box;
    g.tx_bytes = (unsigned)(a_box * BK * 2 + NT * BK * 2);
    dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + NT - 1) / NT), (unsigned)splits);
    gemm_kernel<NT, MODE><<<grid, 128, Smem<NT>::ALLOC, s>>>(ta, tb, g);
    return from_cuda(cudaGetLastError());
}

// Training workspace for batch B (library-owned, per device).
struct TrainWs {
    int B = 0;
    int splits = 0;
    void* mem = nullptr;
    size_t bytes = 0;
    bf16 *X0, *X0T, *H[4], *HT[4], *G4, *G4T, *dZ[4], *dZT[4];
    bf16* Gp[4];   // GELU'(Z_l) of the hidden layers
    float *P, *Y, *part[N_LAYERS], *colpart[N_LAYERS], *loss;
    SchedOut* sched;
    // the weight gradients and bias column sums run on a side stream, off the chain of
    // backward products: fork after each gradient G_l is written, join before Adam
    cudaStream_t side = nullptr;
    cudaEvent_t ev_g[N_LAYERS] = {}, ev_join = nullptr;
};
// One training workspace per device and member slot (member mod TRAIN_SLOTS), so that
// the steps of up to TRAIN_SLOTS members can run concurrently on separate streams.
constexpr int TRAIN_SLOTS = 4;
static_assert(TRAIN_SLOTS + 1 <= ST_REGIONS, "a status region per training slot");
static TrainWs g_tws[64][TRAIN_SLOTS];

static fos_status ensure_train_ws(int dev, int slot, int B, Workspace* ws = nullptr) {
    TrainWs& w = g_tws[dev][slot];
    if (w.mem && w.B == B) return FOS_OK;
    if (ws) ws->generation++;   // captured training graphs hold the old buffers
    if (w.mem) {
        FOS_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(w.mem);
        w.mem = nullptr;
    }
    // split-K of the weight gradients: K = B / splits rows each (>= 512 for B >= 4096),
    // fewer partials for Adam to read
    const int splits = B >= 8192 ? 16 : (B / 256 > 0 ? (B / 256 < 16 ? B / 256 : 16) : 1);
    size_t o = 0;
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    struct Item { void** p; size_t bytes; };
    std::vector<Item> items;
    auto add = [&](void** p, size_t bytes) { items.push_back({p, bytes}); };
    add((void**)&w.X0, (size_t)B * IN_PAD * 2);
    add((void**)&w.X0T, (size_t)IN_PAD * B * 2);
    for (int l = 0; l < 4; ++l) {
        add((void**)&w.Gp[l], (size_t)B * HID * 2);
        add((void**)&w.H[l], (size_t)B * HID * 2);
        add((void**)&w.HT[l], (size_t)HID * B * 2);
    }
    add((void**)&w.P, (size_t)B * 4 * 4);
    add((void**)&w.Y, (size_t)B * 3 * 4);
    add((void**)&w.G4, (size_t)B * OUT_PAD * 2);
    add((void**)&w.G4T, (size_t)OUT_PAD * B * 2);
    for (int k = 0; k < 4; ++k) {   // the output gradient of hidden layer k
        add((void**)&w.dZ[k], (size_t)B * HID * 2);
        add((void**)&w.dZT[k], (size_t)HID * B * 2);
    }
    for (int l = 0; l < N_LAYERS; ++l) {
        add((void**)&w.part[l], (size_t)splits * lay_out(l) * lay_in(l) * 4);
        add((void**)&w.colpart[l], (size_t)COLSUM_SPLITS * real_out(l) * 4);
    }
    add((void**)&w.loss, 16);
    add((void**)&w.sched, sizeof(SchedOut));
    for (auto& it : items) o = al(o + it.bytes);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, o);
    if (e != cudaSuccess) return from_cuda(e);
    FOS_CUDA_TRY(cudaMemset(mem, 0, o));   // padding columns stay zero for good
    size_t q = 0;
    for (auto& it : items) {
        *it.p = (char*)mem + q;
        q = al(q + it.bytes);
    }
    w.mem = mem;
    w.bytes = o;
    w.B = B;
    w.splits = splits;
    if (!w.side) {
        FOS_CUDA_TRY(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
        for (int l = 0; l < N_LAYERS; ++l)
            FOS_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_g[l], cudaEventDisableTiming));
        FOS_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_join, cudaEventDisableTiming));
    }
    return FOS_OK;
}

static AdamArgs layout_args(const MemberPtrs& mp) {
    AdamArgs a;
    std::memset(&a, 0, sizeof(a));
    a.theta = mp.theta;
    a.m = mp.m;
    a.v = mp.v;
    a.wb = mp.wb;
    a.wt = mp.wt;
    a.wi = mp.wi;
    for (int l = 0; l < N_LAYERS; ++l) {
        a.w_off[l] = LAY.w_off[l];
        a.b_off[l] = LAY.b_off[l];
        a.wb_off[l] = LAY.wb_off[l];
        a.wt_off[l] = LAY.wt_off[l];
    }
    return a;
}

static GemmArgs gargs(unsigned* status) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.status = status;
    g.wait_limit = 4000000000LL;   // ~2 s at 2 GHz
    return g;
}

// Forward + backward + Adam for one member on one batch (all on stream s).
// One Adam step of one member on stream s.  sched = NULL: step and lr as given; else the
// step, lr and bias corrections come from the device schedule (graph-captured training).
static fos_status train_step(Workspace* ws, int slot, const MemberPtrs& mp, const float* feat,
                             const float* targets, long long n_rows, int B, unsigned seed,
                             unsigned step, const int* rows, float lr, float* grad_out,
                             cudaStream_t s, const DevSched* ds = nullptr) {
    TrainWs& w = g_tws[ws->device][slot];
    unsigned* status = ws->status + ST_WORDS * (1 + slot);   // this slot's status region
    const int splits = w.splits;
    DevSched dsv;
    std::memset(&dsv, 0, sizeof(dsv));
    if (ds) dsv = *ds;
    FOS_CUDA_TRY(cudaMemsetAsync(w.loss, 0, 4, s));
    gather_kernel<<<(B + 255) / 256, 256, 0, s>>>(feat, targets, n_rows, B, seed, step, rows,
                                                  mp.stats, w.X0, w.X0T, w.Y, dsv);
    FOS_CUDA_TRY(cudaGetLastError());
    const float* bias[N_LAYERS];
    const bf16* wb[N_LAYERS];
    const bf16* wt[N_LAYERS];
    for (int l = 0; l < N_LAYERS; ++l) {
        bias[l] = mp.theta + LAY.b_off[l];
        wb[l] = mp.wb + LAY.wb_off[l];
        wt[l] = mp.wt + LAY.wt_off[l];
    }
    fos_status st;
    // forward
    for (int l = 0; l < 4; ++l) {
        Operand A = (l == 0) ? Operand{w.X0, B, IN_PAD, IN_PAD} : Operand{w.H[l - 1], B, HID, HID};
        Operand Bm{wb[l], HID, lay_in(l), lay_in(l)};
        GemmArgs g = gargs(status);
        g.M = B; g.N = HID; g.bias = bias[l];
        g.out_g = w.Gp[l]; g.out_h = w.H[l]; g.ldh = HID; g.out_t = w.HT[l]; g.ldt = B;
        st = gemm<128, FWD_HIDDEN>(A, Bm, 1, g, s);
        if (st != FOS_OK) return st;
    }
    {
        GemmArgs g = gargs(status);
        g.M = B; g.N = OUT_PAD; g.bias = bias[4];
        g.out_f = w.P; g.out_h = w.G4; g.ldh = OUT_PAD; g.out_t = w.G4T; g.ldt = B;
        g.aux = w.Y; g.loss_sum = w.loss; g.inv_batch = 1.0f / (float)B;
        st = gemm<64, FWD_OUT>(Operand{w.H[3], B, HID, HID}, Operand{wb[4], OUT_PAD, HID, HID}, 1, g, s);
        if (st != FOS_OK) return st;
    }
    // backward: layer 4 gradients, then down through the hidden layers
    const bf16* Gcur = w.G4;
    const bf16* GcurT = w.G4T;
    int gcols = OUT_PAD;
    ColsumArgs ca;
    ca.rows = B;
    ca.step_ctr = dsv.step_ctr;
    for (int l = 4; l >= 0; --l) {
        // the bias gradient's column sums wait for one launch after the loop
        ca.G[l] = Gcur;
        ca.ld[l] = gcols;
        ca.part[l] = w.colpart[l];
        // weight gradient dW_l = G^T · H_{l-1}  (A = G^T [out][B], B = H_{l-1}^T [in][B]),
        // on the side stream once G is written
        {
            FOS_CUDA_TRY(cudaEventRecord(w.ev_g[l], s));
            FOS_CUDA_TRY(cudaStreamWaitEvent(w.side, w.ev_g[l], 0));
            Operand A{GcurT, lay_out(l), B, B};
            Operand Bm = (l == 0) ? Operand{w.X0T, IN_PAD, B, B} : Operand{w.HT[l - 1], HID, B, B};
            GemmArgs g = gargs(status);
            g.M = lay_out(l); g.N = lay_in(l); g.out_f = w.part[l]; g.ldf = lay_in(l);
            if (l == 0) st = gemm<64, DW_PARTIAL>(A, Bm, splits, g, w.side);
            else st = gemm<256, DW_PARTIAL>(A, Bm, splits, g, w.side);
            if (st != FOS_OK) return st;
        }
        if (l == 0) break;
        // dZ_{l-1} = (G · W_l) * GELU'(Z_{l-1})  (A = G [B][out], B = W_l^T [in][out])
        {
            bf16* dz = w.dZ[l - 1];
            bf16* dzt = w.dZT[l - 1];
            Operand A{Gcur, B, lay_out(l), gcols};
            Operand Bm{wt[l], HID, lay_out(l), lay_out(l)};
            GemmArgs g = gargs(status);
            g.M = B; g.N = HID; g.aux_g = w.Gp[l - 1]; g.ld_aux = HID;
            g.out_h = dz; g.ldh = HID; g.out_t = dzt; g.ldt = B;
            st = gemm<128, BWD_HIDDEN>(A, Bm, 1, g, s);
            if (st != FOS_OK) return st;
            Gcur = dz;
            GcurT = dzt;
            gcols = HID;
        }
    }
    colsum_layers_kernel<<<dim3(HID / 64, COLSUM_SPLITS, N_LAYERS), 256, 0, w.side>>>(ca);
    FOS_CUDA_TRY(cudaGetLastError());
    FOS_CUDA_TRY(cudaEventRecord(w.ev_join, w.side));
    FOS_CUDA_TRY(cudaStreamWaitEvent(s, w.ev_join, 0));
    // Adam
    AdamArgs a = layout_args(mp);
    for (int l = 0; l < N_LAYERS; ++l) {
        a.part[l] = w.part[l];
        a.bpart[l] = w.colpart[l];
    }
    a.splits = splits;
    if (grad_out) {   // diagnostic: export the gradient instead of updating
        grad_kernel<<<(unsigned)((LAY.P + 255) / 256), 256, 0, s>>>(a, LAY.P, grad_out);
        return from_cuda(cudaGetLastError());
    }
    a.lr = lr;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    const double t = (double)step + 1.0;
    a.c1 = (float)(1.0 - pow(0.9, t));
    a.c2 = (float)(1.0 - pow(0.999, t));
    a.sched = dsv.out;
    adam_kernel<<<(unsigned)((LAY.P + 255) / 256), 256, 0, s>>>(a, LAY.P);
    return from_cuda(cudaGetLastError());
}

// ----------------------------------------------------------------------- graph training
// Many steps of every member with no host work per step: one ensemble step (for each
// member: its schedule from its device step counter, the Adam step of train_step, its
// loss, the status of its slot folded into the accumulated word) is captured once into a
// CUDA graph, the members of different slots on parallel branches, and the graph is
// launched once per step.
struct FitKey {
    void* model;
    int n_members, B, device;
    const float *feat, *targets;
    long long n_rows;
    unsigned long long seed;
    float* loss_out;
    const SchedOut* table;   // [n_members][table_cap]
    long long table_cap;
    unsigned long long generation;
    bool operator==(const FitKey& o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};
struct FitGraph {
    FitKey key;
    cudaGraphExec_t exec = nullptr;
};
struct FitDev {
    bool ready = false;
    cudaStream_t slot_stream[TRAIN_SLOTS] = {};
    cudaEvent_t fork = nullptr, join[TRAIN_SLOTS] = {};
    std::vector<FitGraph> graphs;
    SchedOut* table = nullptr;   // [members][cap] schedule entries, then [members] bases
    long long table_cap = 0;
    int table_members = 0;
};
static FitDev g_fit[64];

static fos_status fit_resources(int dev) {
    FitDev& f = g_fit[dev];
    if (f.ready) return FOS_OK;
    for (int i = 0; i < TRAIN_SLOTS; ++i) {
        FOS_CUDA_TRY(cudaStreamCreateWithFlags(&f.slot_stream[i], cudaStreamNonBlocking));
        FOS_CUDA_TRY(cudaEventCreateWithFlags(&f.join[i], cudaEventDisableTiming));
    }
    FOS_CUDA_TRY(cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming));
    f.ready = true;
    return FOS_OK;
}

// Enqueues one ensemble step on the capture stream cs (forked to the slot streams).
static fos_status enqueue_fit_step(Workspace* ws, const FitKey& k, cudaStream_t cs) {
    FitDev& f = g_fit[ws->device];
    const int slots = k.n_members < TRAIN_SLOTS ? k.n_members : TRAIN_SLOTS;
    FOS_CUDA_TRY(cudaEventRecord(f.fork, cs));
    for (int i = 0; i < slots; ++i) FOS_CUDA_TRY(cudaStreamWaitEvent(f.slot_stream[i], f.fork, 0));
    for (int m = 0; m < k.n_members; ++m) {
        const int slot = m % TRAIN_SLOTS;
        cudaStream_t s = f.slot_stream[slot];
        TrainWs& w = g_tws[ws->device][slot];
        const int region = 1 + slot;
        FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_WORDS * region + ST_CALL, 0,
                                     sizeof(unsigned), s));
        MemberPtrs mp = member(k.model, m);
        const int* bases = reinterpret_cast<const int*>(k.table + (long long)k.n_members * k.table_cap);
        const DevSched ds{mp.step, k.table + (long long)m * k.table_cap, bases + m, w.sched};
        const unsigned seed = (unsigned)(k.seed ^ (k.seed >> 32)) ^ (unsigned)(m * 0x9E3779B9u);
        fos_status st = train_step(ws, slot, mp, k.feat, k.targets, k.n_rows, k.B, seed, 0,
                                   nullptr, 1.0f, nullptr, s, &ds);
        if (st != FOS_OK) return st;
        if (k.loss_out)
            FOS_CUDA_TRY(cudaMemcpyAsync(k.loss_out + m, w.loss, sizeof(float),
                                         cudaMemcpyDeviceToDevice, s));
        st = accumulate_async_status(ws, s, region);
        if (st != FOS_OK) return st;
    }
    for (int i = 0; i < slots; ++i) {
        FOS_CUDA_TRY(cudaEventRecord(f.join[i], f.slot_stream[i]));
        FOS_CUDA_TRY(cudaStreamWaitEvent(cs, f.join[i], 0));
    }
    return FOS_OK;
}

static fos_status fit_graph(Workspace* ws, const FitKey& k, cudaGraphExec_t* out) {
    FitDev& f = g_fit[ws->device];
    for (auto& g : f.graphs)
        if (g.key == k) {
            *out = g.exec;
            return FOS_OK;
        }
    cudaGraph_t graph = nullptr;
    FOS_CUDA_TRY(cudaStreamBeginCapture(ws->side, cudaStreamCaptureModeThreadLocal));
    fos_status st = enqueue_fit_step(ws, k, ws->side);
    cudaError_t ce = cudaStreamEndCapture(ws->side, &graph);
    if (st != FOS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    FOS_CUDA_TRY(ce);
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    FOS_CUDA_TRY(ce);
    if (f.graphs.size() >= 8) {
        cudaGraphExecDestroy(f.graphs.front().exec);
        f.graphs.erase(f.graphs.begin());
    }
    f.graphs.push_back(FitGraph{k, exec});
    *out = exec;
    return FOS_OK;
}

// Inference workspace: rows per chunk.
static fos_status predict(Workspace* ws, void* model, int n_members, const float* feat,
                          long long n_rows, float* rat, float* spread, unsigned char* needs,
                          float thr, bool stall, cudaStream_t s) {
    static bool attr_set[64] = {};
    if (!attr_set[ws->device]) {
        FOS_CUDA_TRY(cudaFuncSetAttribute(infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          FI_SMEM));
        attr_set[ws->device] = true;
    }
    InferArgs a;
    std::memset(&a, 0, sizeof(a));
    a.feat = feat;
    a.n_rows = n_rows;
    a.n_members = n_members;
    a.model = (const uint8_t*)model;
    a.member_bytes = LAY.bytes;
    a.theta_b = LAY.theta_b;
    a.stats_b = LAY.stats_b;
    a.wi_b = LAY.wi_b;
    for (int l = 0; l < N_LAYERS; ++l) a.b_off[l] = LAY.b_off[l];
    a.rat = rat;
    a.spread = spread;
    a.needs = needs;
    a.thr = thr;
    a.status = ws->status;
    a.wait_limit = stall ? 2000000LL : 4000000000LL;
    a.test_stall = stall ? 1 : 0;
    const long long tiles = (n_rows + 127) / 128;
    long long grid = (long long)ws->num_sms;
    if (grid > tiles) grid = tiles;
    infer_kernel<<<(unsigned)grid, FI_THREADS, FI_SMEM, s>>>(a);
    FOS_CUDA_TRY(cudaGetLastError());
    return FOS_OK;
}

static fos_status prep(Workspace** ws) {
    fos_status st = get_workspace(ws);
    if (st != FOS_OK) return st;
    if ((*ws)->cc_major != 10) return FOS_ERR_UNSUPPORTED;
    return get_encoder();
}

}  // namespace mlp
}  // namespace fos

using namespace fos;

extern "C" {

size_t fos_surrogate_model_bytes(void) { return mlp::LAY.bytes; }

long long fos_surrogate_param_count(void) { return mlp::LAY.P; }

fos_status fos_surrogate_param_offsets(long long* w_off, long long* b_off) {
    if (!w_off || !b_off) return FOS_ERR_INVALID_ARG;
    for (int l = 0; l < mlp::N_LAYERS; ++l) {
        w_off[l] = mlp::LAY.w_off[l];
        b_off[l] = mlp::LAY.b_off[l];
    }
    return FOS_OK;
}

fos_status fos_surrogate_init(void* model, int n_members, unsigned long long seed,
                              const float* feat_stats, void* stream) {
    if (!model || n_members < 1 || !feat_stats) return FOS_ERR_INVALID_ARG;
    for (int f = 0; f < mlp::N_FEAT; ++f)
        if (!(feat_stats[16 + f] > 0.f) || !(feat_stats[32 + f] <= feat_stats[48 + f]))
            return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = mlp::prep(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < n_members; ++k) {
        mlp::MemberPtrs mp = mlp::member(model, k);
        mlp::AdamArgs lay = mlp::layout_args(mp);
        FOS_CUDA_TRY(cudaMemsetAsync((char*)model + (size_t)k * mlp::LAY.bytes, 0, mlp::LAY.bytes, s));
        mlp::init_kernel<<<(unsigned)((mlp::LAY.P + 255) / 256), 256, 0, s>>>(
            mp.theta, mp.m, mp.v, mp.wb, mp.wt, mp.wi, mp.step, (unsigned)(seed ^ (seed >> 32)),
            (unsigned)k, lay, mlp::LAY.P);
        FOS_CUDA_TRY(cudaGetLastError());
        FOS_CUDA_TRY(cudaMemcpyAsync(mp.stats, feat_stats, 64 * sizeof(float),
                                     cudaMemcpyHostToDevice, s));
    }
    FOS_CUDA_TRY(cudaStreamSynchronize(s));
    return FOS_OK;
}

fos_status fos_surrogate_load(void* model, int member, const float* theta,
                              const float* feat_stats, void* stream) {
    if (!model || member < 0 || !theta || !feat_stats) return FOS_ERR_INVALID_ARG;
    for (int f = 0; f < mlp::N_FEAT; ++f)
        if (!(feat_stats[16 + f] > 0.f) || !(feat_stats[32 + f] <= feat_stats[48 + f]))
            return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = mlp::prep(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    mlp::MemberPtrs mp = mlp::member(model, member);
    mlp::AdamArgs lay = mlp::layout_args(mp);
    FOS_CUDA_TRY(cudaMemsetAsync((char*)model + (size_t)member * mlp::LAY.bytes, 0,
                                 mlp::LAY.bytes, s));
    mlp::load_kernel<<<(unsigned)((mlp::LAY.P + 255) / 256), 256, 0, s>>>(
        theta, mp.theta, mp.m, mp.v, mp.wb, mp.wt, mp.wi, mp.step, lay, mlp::LAY.P);
    FOS_CUDA_TRY(cudaGetLastError());
    FOS_CUDA_TRY(cudaMemcpyAsync(mp.stats, feat_stats, 64 * sizeof(float),
                                 cudaMemcpyHostToDevice, s));
    FOS_CUDA_TRY(cudaStreamSynchronize(s));
    return FOS_OK;
}

fos_status fos_surrogate_features(int n_designs, int n_wl, const double* wl, const double* np_re,
                                  const double* np_im, const double* radius,
                                  const double* vol_frac, const double* thickness, const double* g,
                                  const double* mu_s, const double* mu_a, float* features,
                                  unsigned flags, void* stream) {
    if (n_designs < 0 || n_wl < 1) return FOS_ERR_INVALID_ARG;
    if (!wl || !np_re || !np_im || !radius || !vol_frac || !thickness || !g || !mu_s || !mu_a ||
        !features)
        return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    const long long n = (long long)n_designs * n_wl;
    if (n > 0) {
        long long blocks = (n + 255) / 256;
        if (blocks > (long long)ws->num_sms * 16) blocks = (long long)ws->num_sms * 16;
        mlp::features_kernel<<<(unsigned)blocks, 256, 0, s>>>(n_designs, n_wl, wl, np_re, np_im,
                                                              radius, vol_frac, thickness, g, mu_s,
                                                              mu_a, features, ws->status);
        FOS_CUDA_TRY(cudaGetLastError());
    }
    return finish_call(ws, s, flags);
}

fos_status fos_surrogate_features_slab(long long n_rows, const double* n_layer,
                                       const double* mu_s, const double* mu_a, const double* g,
                                       const double* thickness, float* features,
                                       unsigned flags, void* stream) {
    if (n_rows < 0) return FOS_ERR_INVALID_ARG;
    if (n_rows > 0 && (!n_layer || !mu_s || !mu_a || !g || !thickness || !features))
        return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    if (n_rows > 0) {
        long long blocks = (n_rows + 255) / 256;
        if (blocks > (long long)ws->num_sms * 16) blocks = (long long)ws->num_sms * 16;
        mlp::features_slab_kernel<<<(unsigned)blocks, 256, 0, s>>>(
            n_rows, n_layer, mu_s, mu_a, g, thickness, features, ws->status);
        FOS_CUDA_TRY(cudaGetLastError());
    }
    return finish_call(ws, s, flags);
}

fos_status fos_surrogate_feature_stats(const float* features, long long n_rows, float* stats,
                                       void* stream) {
    if (!features || !stats || n_rows < 1) return FOS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(stats, 0, 64 * sizeof(float), s));
    mlp::stats_kernel<<<mlp::N_FEAT, 256, 0, s>>>(features, n_rows, stats);
    FOS_CUDA_TRY(cudaGetLastError());
    return from_cuda(cudaStreamSynchronize(s));
}

fos_status fos_counts_to_fractions(const long long* counts, long long n_rows, const int* rows,
                                   float* fractions, void* stream) {
    if (n_rows < 0 || (n_rows > 0 && (!counts || !fractions))) return FOS_ERR_INVALID_ARG;
    if (n_rows == 0) return FOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long blocks = (n_rows + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    mlp::fractions_kernel<<<(unsigned)blocks, 256, 0, s>>>(counts, n_rows, rows, fractions);
    return from_cuda(cudaGetLastError());
}

fos_status fos_mask_to_rows(const unsigned char* mask, long long n, int* rows, long long* count,
                            void* stream) {
    if (n < 0 || n > 0x7fffffffLL || (n > 0 && (!mask || !rows)) || !count)
        return FOS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(long long), s));
    if (n == 0) return FOS_OK;
    mlp::mask_rows_kernel<<<(unsigned)((n + 1023) / 1024), 1024, 0, s>>>(
        mask, n, rows, (unsigned long long*)count);
    return from_cuda(cudaGetLastError());
}

fos_status fos_surrogate_train_step(void* model, int member, const float* features,
                                    const float* targets, long long n_rows, int batch,
                                    const int* batch_rows, unsigned long long seed, int step,
                                    float lr, float* loss_out, float* grad_out, unsigned flags,
                                    void* stream) {
    NvtxRange nvtx("fos_surrogate_train_step");
    if (!model || member < 0 || !features || !targets || n_rows < 1 || step < 0) return FOS_ERR_INVALID_ARG;
    if (batch < 256 || batch % 256 != 0 || batch > 65536) return FOS_ERR_INVALID_ARG;
    if (!(lr > 0.f)) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = mlp::prep(&ws);
    if (st != FOS_OK) return st;
    const int slot = member % mlp::TRAIN_SLOTS;
    st = mlp::ensure_train_ws(ws->device, slot, batch, ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int region = 1 + slot;   // concurrent slots keep separate call words
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_WORDS * region + ST_CALL, 0, sizeof(unsigned), s));
    mlp::MemberPtrs mp = mlp::member(model, member);
    st = mlp::train_step(ws, slot, mp, features, targets, n_rows, batch,
                         (unsigned)(seed ^ (seed >> 32)) ^ (unsigned)(member * 0x9E3779B9u),
                         (unsigned)step, batch_rows, lr, grad_out, s);
    if (st != FOS_OK) return st;
    if (loss_out) {
        mlp::TrainWs& w = mlp::g_tws[ws->device][slot];
        FOS_CUDA_TRY(cudaMemcpyAsync(loss_out, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    if (!grad_out) {   // the member's step count in the model (read by fos_surrogate_fit)
        mlp::set_step_kernel<<<1, 32, 0, s>>>(mp.step, step + 1);
        FOS_CUDA_TRY(cudaGetLastError());
    }
    return finish_call(ws, s, flags, region);
}

fos_status fos_surrogate_fit(void* model, int n_members, const float* features,
                             const float* targets, long long n_rows, int batch,
                             unsigned long long seed, int n_steps, float lr_max, float lr_min,
                             int schedule_origin, int schedule_total, float* loss_out,
                             unsigned flags, void* stream) {
    NvtxRange nvtx("fos_surrogate_fit");
    if (!model || n_members < 1 || !features || !targets || n_rows < 1 || n_steps < 0)
        return FOS_ERR_INVALID_ARG;
    if (batch < 256 || batch % 256 != 0 || batch > 65536) return FOS_ERR_INVALID_ARG;
    if (!(lr_max > 0.f) || !(lr_min >= 0.f) || schedule_total < 1 || schedule_origin < 0)
        return FOS_ERR_INVALID_ARG;
    if (flags & ~(unsigned)FOS_ASYNC) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = mlp::prep(&ws);
    if (st != FOS_OK) return st;
    const int slots = n_members < mlp::TRAIN_SLOTS ? n_members : mlp::TRAIN_SLOTS;
    for (int i = 0; i < slots; ++i) {
        st = mlp::ensure_train_ws(ws->device, i, batch, ws);
        if (st != FOS_OK) return st;
    }
    st = mlp::fit_resources(ws->device);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_steps > 0) {
        // the schedule of this call's steps, per member from its step count, computed here
        // as the per-step entry point's callers and train_step compute it
        mlp::FitDev& fd = mlp::g_fit[ws->device];
        if (fd.table_cap < n_steps || fd.table_members < n_members) {
            FOS_CUDA_TRY(cudaStreamSynchronize(s));
            FOS_CUDA_TRY(cudaDeviceSynchronize());
            if (fd.table) cudaFree(fd.table);
            fd.table = nullptr;
            const long long cap = n_steps > fd.table_cap ? n_steps : fd.table_cap;
            const int mem = n_members > fd.table_members ? n_members : fd.table_members;
            FOS_CUDA_TRY(cudaMalloc(&fd.table, (size_t)mem * cap * sizeof(mlp::SchedOut) +
                                                   (size_t)mem * sizeof(int) + 256));
            fd.table_cap = cap;
            fd.table_members = mem;
        }
        std::vector<mlp::SchedOut> tab((size_t)n_members * fd.table_cap);
        std::vector<int> base(n_members);
        // earlier steps (of any stream) must be done: they read the table rewritten here
        // and advance the step counts read here
        FOS_CUDA_TRY(cudaDeviceSynchronize());
        for (int m = 0; m < n_members; ++m) {
            mlp::MemberPtrs mp = mlp::member(model, m);
            FOS_CUDA_TRY(cudaMemcpy(&base[m], mp.step, sizeof(int), cudaMemcpyDeviceToHost));
            for (int i = 0; i < n_steps; ++i) {
                const int g = base[m] + i;
                double gs = (double)(g - schedule_origin > 0 ? g - schedule_origin : 0);
                if (gs > (double)schedule_total) gs = (double)schedule_total;
                const double lr = (double)lr_min + 0.5 * ((double)lr_max - (double)lr_min) *
                                                       (1.0 + cos(M_PI * gs / (double)schedule_total));
                const double t = (double)g + 1.0;
                mlp::SchedOut& o = tab[(size_t)m * fd.table_cap + i];
                o.step = (unsigned)g;
                o.lr = (float)lr;
                o.c1 = (float)(1.0 - pow(0.9, t));
                o.c2 = (float)(1.0 - pow(0.999, t));
            }
        }
        FOS_CUDA_TRY(cudaMemcpy(fd.table, tab.data(), tab.size() * sizeof(mlp::SchedOut),
                                cudaMemcpyHostToDevice));
        FOS_CUDA_TRY(cudaMemcpy(fd.table + (size_t)n_members * fd.table_cap, base.data(),
                                (size_t)n_members * sizeof(int), cudaMemcpyHostToDevice));
        mlp::FitKey k;
        std::memset(&k, 0, sizeof(k));
        k.model = model;
        k.n_members = n_members;
        k.B = batch;
        k.device = ws->device;
        k.feat = features;
        k.targets = targets;
        k.n_rows = n_rows;
        k.seed = seed;
        k.loss_out = loss_out;
        k.table = fd.table;
        k.table_cap = fd.table_cap;
        k.generation = ws->generation;
        cudaGraphExec_t exec = nullptr;
        st = mlp::fit_graph(ws, k, &exec);
        if (st != FOS_OK) return st;
        for (int i = 0; i < n_steps; ++i) FOS_CUDA_TRY(cudaGraphLaunch(exec, s));
    }
    if (flags & FOS_ASYNC) return FOS_OK;
    st = wait_stream(s, default_timeout_ms());
    if (st != FOS_OK) return st;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&bits, ws->status + ST_ASYNC, sizeof(unsigned), cudaMemcpyDeviceToHost));
    FOS_CUDA_TRY(cudaMemset(ws->status + ST_ASYNC, 0, sizeof(unsigned)));
    return status_from_bits(bits);
}

fos_status fos_surrogate_predict(void* model, int n_members, const float* features,
                                 long long n_rows, float* rat, float* spread,
                                 unsigned char* needs_mc, float threshold, unsigned flags,
                                 void* stream) {
    NvtxRange nvtx("fos_surrogate_predict");
    if (!model || n_members < 1 || n_members > 16 || n_rows < 0) return FOS_ERR_INVALID_ARG;
    if (n_rows > 0 && (!features || !rat)) return FOS_ERR_INVALID_ARG;
    if (n_rows == 0) return FOS_OK;
    Workspace* ws = nullptr;
    fos_status st = mlp::prep(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    st = mlp::predict(ws, model, n_members, features, n_rows, rat, spread, needs_mc, threshold,
                      (flags & FOS_TEST_STALL) != 0, s);
    if (st != FOS_OK) return st;
    return finish_call(ws, s, flags);
}

// Plain GEMM through the same kernel (diagnostic): C[M][N] fp32 = A[M][K] * B[N][K]^T,
// A and B bf16 row-major with K a multiple of 64.
fos_status fos_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, int splits,
                         unsigned flags, void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 64 || K % 64 != 0 || splits < 1 ||
        K % (64 * splits) != 0 || N % 64 != 0)
        return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = mlp::prep(&ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    mlp::GemmArgs g = mlp::gargs(ws->status);
    g.M = M;
    g.N = N;
    g.out_f = C;
    g.ldf = N;
    if (flags & FOS_TEST_STALL) {   // test: one stage never fills; the wait gives up fast
        g.test_stall = 1;
        g.wait_limit = 2000000LL;
    }
    mlp::Operand a{(const mlp::bf16*)A, M, K, K}, b{(const mlp::bf16*)B, N, K, K};
    if (N % 256 == 0) st = mlp::gemm<256, mlp::DW_PARTIAL>(a, b, splits, g, s);
    else st = mlp::gemm<64, mlp::DW_PARTIAL>(a, b, splits, g, s);
    if (st != FOS_OK) return st;
    return finish_call(ws, s, flags & FOS_ASYNC);
}

}  // extern "C"
