// Learned surrogate of the photon walk on GB300 (arxiv 2409.00165, section "Photon
// transport": a network trained on Monte Carlo spectra replaces the walk).
//
// Network: 9 features -> standardise -> [Linear 256, GELU (tanh form)] x 4 -> Linear 3 -> softmax
// (R, A, T).  BF16 weights and activations on the tensor cores, FP32 accumulation,
// FP32 master weights and Adam state.
//
// Inference runs in one fused persistent kernel (infer_kernel): per 128-row tile the
// activations stay in tensor memory from the features to the softmax.  Training runs the
// same way: train_kernel takes a (member, 128-row tile) of the batch through the forward
// pass, the softmax cross-entropy gradient and the backward pass down to the output
// gradient of layer 0, with every activation and gradient on chip; it writes to global
// memory only what the weight gradients need (each layer's input and output gradient) and
// GELU'(Z), which it reads back itself.  Those arrays are row-blocked and chunk-major,
// X[row/64][c/8][row%64][c%8]: one 16-byte store per thread and 8 columns, 512 contiguous
// bytes per warp; each 8-row x 8-column block is a 128-byte core matrix of the tensor
// cores' MN-major operand layout, and the 64 rows x 128 columns a product stage needs are
// 16 contiguous KB.  dw_kernel then forms every weight gradient dW_l = dZ_l^T H_{l-1} as a
// split-K tcgen05 product over the batch with both operands MN-major (one bulk copy per
// operand and stage), and the bias gradients as the same product with a column of ones.
// Adam sums the split partials in a fixed order and rewrites the BF16 weight images.
//
// gemm_kernel is a plain C = A B^T product (K-major BF16 operands staged by TMA with
// 128-byte swizzle through an mbarrier ring, FP32 accumulators in tensor memory), kept
// as a diagnostic entry point.
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
//   stats  fp32 [64] : mean[16] | std[16] | lo[16] | hi[16] of the raw features
//   step   int32 [4]
//   wi     bf16      : the weights as shared-memory images for the fused kernels (see
//                      img_index), one contiguous block per pipeline stage
struct Layout {
    long long w_off[N_LAYERS], b_off[N_LAYERS], P;
    size_t theta_b, m_b, v_b, stats_b, step_b, wi_b, bytes;
};

// Weight image: the B operands of the fused kernels, already in the 128-byte-swizzled
// K-major layout a stage of shared memory holds, so that one untiled bulk copy fills a
// stage (32 KB).  Layer 0 is one stage: all 256 output rows x 64 inputs
// (9 real).  Layers 1-3 are four stages each, (output half h, input pair j) in the order
// 2h + j: 128 output rows x inputs 128 j .. +127, as two k blocks of 128 x 64 (16 KB).
// Layer 4 keeps its first 16 output rows (3 real) as 4 blocks of 16 x 64 (2 KB), one per k
// block, copied as one stage.
constexpr long long IMG_BLK = 256 * 64;          // elements of a 32 KB stage
constexpr long long IMG_HALF_KB = 128 * 64;      // elements of a 16 KB k block of a half
constexpr long long IMG_L4_BLK = 16 * 64;        // elements of a 2 KB block
__host__ __device__ constexpr long long img_off(int l) {
    return l == 0 ? 0 : (l == 4 ? 13 * IMG_BLK : (1 + 4 * (l - 1)) * IMG_BLK);
}
constexpr long long IMG_ELEMS = 13 * IMG_BLK + 4 * IMG_L4_BLK;
constexpr int IMG_ROWS_L4 = 16;

// Position of element (n, c) of a 64-column k block in the 128-byte swizzle: row n starts
// at n * 64 elements; its 16-byte chunk j (columns 8j..8j+7) sits at chunk j ^ (n mod 8).
__host__ __device__ constexpr long long swz64(int n, int c) {
    return (long long)n * 64 + ((((c >> 3) ^ (n & 7)) << 3) | (c & 7));
}

// The backward pass multiplies an output gradient dZ_l [rows][out] by W_l: its B operand
// is W_l^T [in][out] with K = out, and the image, whose rows are outputs and whose 128-byte
// rows hold 64 consecutive inputs, is exactly that operand in the MN-major 128-byte-
// swizzled layout (8-row groups 1024 bytes apart along K, 64-input blocks along N).
//
// Element index in the image of weight (l, o, i), or -1 when the image leaves it out.
__host__ __device__ inline long long img_index(int l, int o, int i) {
    const int kb = i >> 6, c = i & 63;
    if (l == 4) {
        if (o >= IMG_ROWS_L4) return -1;
        return img_off(l) + (long long)kb * IMG_L4_BLK + swz64(o, c);
    }
    if (l == 0) return img_off(l) + swz64(o, c);
    return img_off(l) + (long long)((o >> 7) * 2 + (kb >> 1)) * IMG_BLK +
           (long long)(kb & 1) * IMG_HALF_KB + swz64(o & 127, c);
}

static Layout make_layout() {
    Layout L;
    long long p = 0;
    for (int l = 0; l < N_LAYERS; ++l) {
        L.w_off[l] = p;
        p += (long long)lay_out(l) * lay_in(l);
        L.b_off[l] = p;
        p += lay_out(l);
    }
    L.P = p;
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    size_t o = 0;
    L.theta_b = o; o = al(o + (size_t)p * 4);
    L.m_b = o;     o = al(o + (size_t)p * 4);
    L.v_b = o;     o = al(o + (size_t)p * 4);
    L.stats_b = o; o = al(o + 64 * 4);
    L.step_b = o;  o = al(o + 16);
    L.wi_b = o;    o = al(o + (size_t)IMG_ELEMS * 2);
    L.bytes = o;
    return L;
}
static const Layout LAY = make_layout();

struct MemberPtrs {
    float *theta, *m, *v, *stats;
    bf16* wi;
    int* step;
};
static MemberPtrs member(void* model, int k) {
    char* base = (char*)model + (size_t)k * LAY.bytes;
    MemberPtrs p;
    p.theta = (float*)(base + LAY.theta_b);
    p.m = (float*)(base + LAY.m_b);
    p.v = (float*)(base + LAY.v_b);
    p.stats = (float*)(base + LAY.stats_b);
    p.step = (int*)(base + LAY.step_b);
    p.wi = (bf16*)(base + LAY.wi_b);
    return p;
}

// ----------------------------------------------------------------------- GEMM kernel
// C[split] = A B^T over one K range per split: a 128 x NT output tile per CTA, FP32
// partials [split][M][ldf].
struct GemmArgs {
    int M, N;              // output rows / columns (unpadded extents to store)
    int k_per_split;       // multiple of BK
    float* out_f;          // partial [split][M][ldf]
    int ldf;
    unsigned* status;
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

template <int NT>
struct Smem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = NT * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int TOTAL = BAR_OFF + (2 * STAGES + 1) * 8 + 16;
    static constexpr int ALLOC = TOTAL + 1024;   // slack for 1024-byte alignment
};

template <int NT>
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
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
        __syncwarp();
        tmem_ld16(trow + c0, v);
        const int n = n0 + c0;
        if (!row_ok || n >= args.N) continue;
        float* dst = args.out_f + (long long)blockIdx.z * args.M * args.ldf +
                     (long long)m * args.ldf + n;
#pragma unroll
        for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
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

// Step schedule of one member's training step (graph-captured training, where the host
// does not see each step): the member's global step g (Adam's t = g + 1), the learning
// rate and Adam's bias corrections 1 - b1^t, 1 - b2^t.
struct SchedOut {
    unsigned step;
    float lr, c1, c2;
};

// ----------------------------------------------------------------- fused training
// The products of one Adam step for 128-row tiles of every member's batch in one
// persistent kernel, with infer_kernel's roles, tensor-memory plan and weight ring.  A
// work item is (member k, tile t).  Its layer sequence s = 0..8 reads activation buffer
// s mod 2 and writes the next layer's input into the other:
//   s = 0..3  hidden layer s forward: Z = X W_s^T + b_s; H_s = GELU(Z) is the next
//             input; H_s and GELU'(Z) go to global memory (chunk-major);
//   s = 4     output layer: P = softmax(X W_4^T + b_4); the batch-mean cross-entropy
//             -sum y log P into the member's loss; its gradient G = (P - y) / B (3 real
//             columns of 16) is the next input and goes to global memory, with its
//             column sums per tile and warp (the bias gradient of layer 4);
//   s = 5..8  backward through layer j + 1, j = 8 - s: dZ_j = (G_{j+1} W_{j+1}) *
//             GELU'(Z_j), where G_4 = G and G_{j+1} = dZ_{j+1} is the previous output;
//             dZ_j goes to global memory and, except for j = 0, is the next input.
// s = 0 and 5 multiply K = 16 (the features; the output gradient) by a 256 x 64 stage,
// s = 4 gives N = 16 outputs, the others are 256 x 256 products in four stages, as in
// infer_kernel.  The weight ring carries the forward image (14 items) and then the
// backward image (13 items) of the item's member.  The batch rows are drawn in the
// kernel: the caller's rows, or a hash of (seed, step, row) scaled to the data set.
constexpr int FT_ITEMS = FI_ITEMS + 13;   // ring items per work item
// Raw feature rows of the next work item (9 features and 3 targets per row), staged in
// shared memory while the current item runs its backward pass: two buffers after the
// barriers.
constexpr int FT_ROW_FLOATS = 12;
constexpr int FT_XBUF_BYTES = 128 * FT_ROW_FLOATS * 4;
constexpr int FT_XBUF_OFF = (FI_SMEM + 32 + 15) & ~15;   // after 4 more barriers
constexpr int FT_SMEM = FT_XBUF_OFF + 2 * FT_XBUF_BYTES;
static_assert(FT_SMEM <= 227 * 1024, "shared memory of the fused training kernel");
// Roles: infer_kernel's 16 epilogue warps, copy warp and MMA warp, and a staging warp
// that stages each work item's parameters and rows ahead of it.  19 warps keep the
// register cap of 18 (five warps on a sub-partition: 96 registers a thread).
constexpr int FT_STAGE_WARP = FI_EPI_WARPS + 2;
constexpr int FT_THREADS = 32 * (FI_EPI_WARPS + 3);
// The staged-item barriers (full and empty per buffer) follow infer_kernel's shared
// memory, whose barrier area ends with the tensor-memory slot and the abort flag.
static_assert(FI_BAR_BYTES >= 8 * FI_NBARS + 8, "tmem slot and abort flag after the barriers");

struct TrainArgs {
    const float* feat;            // raw features [n_rows][9]
    const float* targets;         // [n_rows][3]
    long long n_rows;
    const int* rows;              // the batch's rows [B] (one member), or NULL: hashed
    int B, n_tiles, n_members;
    unsigned seed, seed_mul;      // member k draws with seed ^ ((member0 + k) * seed_mul)
    int member0;
    unsigned step;                // the draw's step without a device schedule
    const uint8_t* model;
    size_t member_bytes, theta_b, stats_b, wi_b, step_b;
    long long b_off[N_LAYERS];
    // device schedule (graph-captured training): member k's step is its step counter,
    // and table[k * table_cap + step - table_base[k]] is copied to the member's slot
    int dev_step;
    const SchedOut* table;
    long long table_cap;
    const int* table_base;
    // workspace: member k's arrays at ws + k * region_bytes (byte offsets below)
    uint8_t* ws;
    size_t region_bytes;
    size_t x0_b, h_b[4], g4_b, dz_b[4], gp_b[4], bp4_b, sched_b;
    float* loss;                  // [n_members], zeroed by the caller
    unsigned* status;
    long long wait_limit;
    int test_stall;               // test only: the first weight copy is never issued
};

// GELU (tanh form) and its derivative for two columns, from hz = z/2 = acc/2 + bias/2:
// GELU = hz (1 + t), t = tanh(u), u = hz (2 c0 + 8 c1 hz^2); d GELU / dz = (1 + t)/2 +
// hz (1 - t^2) (c0 + 12 c1 hz^2), with c0 = sqrt(2/pi), c1 = 0.044715 c0.  Both as packed
// BF16 pairs.
__device__ __forceinline__ void gelu_grad_half2(float acc0, float acc1, float hb0, float hb1,
                                                uint32_t& gel, uint32_t& grad) {
    const float2 hz = fma2(make_float2(0.5f, 0.5f), make_float2(acc0, acc1), make_float2(hb0, hb1));
    const float2 h2 = mul2(hz, hz);
    const float2 u = mul2(hz, fma2(make_float2(0.2854192648f, 0.2854192648f), h2,
                                   make_float2(1.5957691216f, 1.5957691216f)));
    const float2 t = make_float2(tanh_fast(u.x), tanh_fast(u.y));
    const float2 g = fma2(hz, t, hz);
    gel = pack_bf16(g.x, g.y);
    const float2 du = fma2(make_float2(0.4281288972f, 0.4281288972f), h2,
                           make_float2(0.7978845608f, 0.7978845608f));
    const float2 om = fma2(make_float2(-t.x, -t.y), t, make_float2(1.0f, 1.0f));
    const float2 half1 = fma2(make_float2(0.5f, 0.5f), t, make_float2(0.5f, 0.5f));
    const float2 d = fma2(mul2(hz, om), du, half1);
    grad = pack_bf16(d.x, d.y);
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {   // a 32-bit integer hash (murmur3 finaliser)
    x ^= x >> 16; x *= 0x85ebca6bu; x ^= x >> 13; x *= 0xc2b2ae35u; x ^= x >> 16;
    return x;
}

// Data-set row of batch row b at a step: drawn uniformly (with replacement) by hashing
// (seed, step, b).
__device__ __forceinline__ long long draw_row(unsigned seed, unsigned step, int b, long long n_rows) {
    const uint32_t h = mix32(mix32(seed ^ 0x9E3779B9u) ^ mix32(step * 0x85ebca6bu + (uint32_t)b));
    return (long long)(((unsigned long long)h * (unsigned long long)n_rows) >> 32);
}

__global__ void __launch_bounds__(FT_THREADS, 1) train_kernel(TrainArgs A) {
    extern __shared__ __align__(1024) uint8_t ft_smem[];
    const uint32_t base = smem_u32(ft_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ring = base;
    float* par = reinterpret_cast<float*>(ft_smem + FI_STAGES * FI_SLOT);
    const uint32_t bars = ring + FI_STAGES * FI_SLOT + FI_PAR_BYTES;
    const uint32_t bar_full = bars, bar_empty = bars + 8 * FI_STAGES;
    const uint32_t bar_acc = bars + 16 * FI_STAGES;   // 2: output half h accumulated
    const uint32_t bar_a = bar_acc + 16;              // 2: input k blocks 2h, 2h+1 written
    const uint32_t bar_p = bar_a + 16;                // parameter staging done
    const uint32_t tslot = bar_p + 8;
    uint8_t* bars_g = ft_smem + FI_STAGES * FI_SLOT + FI_PAR_BYTES;
    volatile uint32_t* tslot_ptr = reinterpret_cast<volatile uint32_t*>(bars_g + 8 * FI_NBARS);
    volatile int& abort_flag = *reinterpret_cast<volatile int*>(bars_g + 8 * FI_NBARS + 4);
    const uint32_t bar_sf = base + FI_SMEM;     // 2: staged item in buffer b (32 arrivals)
    const uint32_t bar_se = bar_sf + 16;        // 2: buffer b read (one arrival per epilogue warp)
    float* xbuf = reinterpret_cast<float*>(ft_smem + FT_XBUF_OFF);

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
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_sf + 8 * b, 32);
            mbar_init(bar_se + 8 * b, FI_EPI_WARPS);
        }
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(tslot, FI_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_ptr;

    const long long n_items = (long long)A.n_members * A.n_tiles;
    const long long my_items =
        n_items > blockIdx.x ? (n_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == FI_EPI_WARPS) {
        // ------------------------------------------------------------ bulk copies
        if (lane == 0) {
            const long long total = my_items * FT_ITEMS;
            long long issued = 0, it = blockIdx.x;
            int slot = 0, q = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (; issued < total && ok && !abort_flag; ++issued) {
                if (issued >= FI_STAGES &&
                    !mbar_wait_sleep(bar_empty + 8 * slot, phase ^ 1u, A.wait_limit)) {
                    ok = false;
                    break;
                }
                const int k = (int)(it / A.n_tiles);
                const uint8_t* mb = A.model + (size_t)k * A.member_bytes;
                const uint8_t* src;
                uint32_t bytes;
                if (q < FI_ITEMS) {
                    int layer, blk;
                    long long off;
                    fi_item(q, layer, blk, off, bytes);
                    src = mb + A.wi_b + (size_t)off * 2;
                } else {
                    // backward: layer 4 whole (8 KB), then layers 3, 2, 1, four stages each
                    // in the order (output rows 0-127, inputs 0-127), (128-255, 0-127),
                    // (0-127, 128-255), (128-255, 128-255): input half h of the product
                    // takes the two stages that hold inputs 128 h .. +127
                    const int qb = q - FI_ITEMS;
                    if (qb == 0) {
                        src = mb + A.wi_b + (size_t)img_off(4) * 2;
                        bytes = (uint32_t)(4 * IMG_L4_BLK * 2);
                    } else {
                        const int l = 3 - (qb - 1) / 4, p = (qb - 1) & 3;
                        src = mb + A.wi_b + (size_t)(img_off(l) + (long long)((p >> 1) | ((p & 1) << 1)) * IMG_BLK) * 2;
                        bytes = FI_SLOT;
                    }
                }
                if (!(A.test_stall && issued == 0)) {
                    mbar_arrive_expect_tx(bar_full + 8 * slot, bytes);
                    bulk_load(ring + slot * FI_SLOT, src, bytes, bar_full + 8 * slot);
                }
                if (++slot == FI_STAGES) {
                    slot = 0;
                    phase ^= 1u;
                }
                if (++q == FT_ITEMS) {
                    q = 0;
                    it += gridDim.x;
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
            constexpr uint32_t ID128_BMN = idesc_bf16_major(128, 128, false, true);
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
            auto wait_a = [&](int h) {
                if (!mbar_wait_sleep(bar_a + 8 * h, pa, A.wait_limit) || abort_flag) return false;
                tc_fence_after();
                return true;
            };
            auto bdesc = [&](int s) { return dring + (uint64_t)(s * (FI_SLOT >> 4)); };
            for (long long i = 0; i < my_items && ok; ++i) {
                for (int s = 0; s < 9 && ok; ++s) {
                    const uint32_t ta = tmem + FI_ABUF + (uint32_t)((s & 1) * 128);
                    int st = 0;
                    if (s == 0) {
                        // K = 16 (the features) x 256 outputs: half h of the stage's 256 rows
                        // starts 16 KB into it
                        if (!(ok = take(st))) break;
                        ok = wait_a(0) && wait_a(1);
                        if (ok)
                            for (int h = 0; h < 2; ++h) {
                                mma_bf16_ts(tmem + FI_ACC + (uint32_t)(h * 128), ta,
                                            bdesc(st) + (uint64_t)(h * (16384 >> 4)), ID128, 0u);
                                mma_commit(bar_acc + 8 * h);
                            }
                        mma_commit(bar_empty + 8 * st);
                    } else if (s == 4) {
                        // the 16 padded output columns (3 real), four 2 KB k blocks
                        if (!(ok = take(st))) break;
                        for (int kb = 0; kb < 4 && ok; ++kb) {
                            if ((kb & 1) == 0 && !(ok = wait_a(kb >> 1))) break;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                mma_bf16_ts(tmem + FI_ACC, ta + (uint32_t)(kb * 32 + kk * 8),
                                            bdesc(st) + (uint64_t)(kb * ((int)IMG_L4_BLK * 2 >> 4) + 2 * kk),
                                            ID16, (kb > 0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(bar_empty + 8 * st);
                        if (ok)
                            for (int h = 0; h < 2; ++h) mma_commit(bar_acc + 8 * h);
                    } else if (s == 5) {
                        // G (K = 16 outputs) x W_4 -> 256 inputs: the layer-4 stage read
                        // MN-major, input half h = its 2 KB blocks 2h, 2h + 1 (8-output-row
                        // groups 1 KB apart, 64-input blocks 2 KB apart)
                        if (!(ok = take(st))) break;
                        ok = wait_a(0) && wait_a(1);
                        if (ok)
                            for (int h = 0; h < 2; ++h) {
                                mma_bf16_ts(tmem + FI_ACC + (uint32_t)(h * 128), ta,
                                            desc_sw128_mn(ring + st * FI_SLOT + h * 4096, 2048, 1024),
                                            ID128_BMN, 0u);
                                mma_commit(bar_acc + 8 * h);
                            }
                        mma_commit(bar_empty + 8 * st);
                    } else if (s > 5) {
                        // dZ (K = 256 outputs) x W_l -> 256 inputs, input half h from the
                        // stages (outputs 128 g .. +127, inputs 128 h .. +127), g = 0, 1,
                        // read MN-major: 16 output rows (2048 bytes) per MMA, the two 64-input
                        // k blocks of the stage 16 KB apart
                        for (int h = 0; h < 2 && ok; ++h) {
                            for (int g = 0; g < 2 && ok; ++g) {
                                if (!(ok = take(st))) break;
                                if (h == 0 && !(ok = wait_a(g))) {
                                    mma_commit(bar_empty + 8 * st);
                                    break;
                                }
#pragma unroll
                                for (int kk = 0; kk < 8; ++kk)
                                    mma_bf16_ts(tmem + FI_ACC + (uint32_t)(h * 128),
                                                ta + (uint32_t)(g * 64 + kk * 8),
                                                desc_sw128_mn(ring + st * FI_SLOT + kk * 2048, 16384, 1024),
                                                ID128_BMN, (g > 0 || kk > 0) ? 1u : 0u);
                                mma_commit(bar_empty + 8 * st);
                            }
                            if (ok) mma_commit(bar_acc + 8 * h);
                        }
                    } else {
                        // stage (h, j): output rows 128 h .. +127 x k blocks 2j, 2j + 1
                        for (int h = 0; h < 2 && ok; ++h) {
                            for (int j = 0; j < 2 && ok; ++j) {
                                if (!(ok = take(st))) break;
                                if (h == 0 && !(ok = wait_a(j))) {
                                    mma_commit(bar_empty + 8 * st);
                                    break;
                                }
#pragma unroll
                                for (int x = 0; x < 2; ++x) {
                                    const int kb = 2 * j + x;
#pragma unroll
                                    for (int kk = 0; kk < 4; ++kk)
                                        mma_bf16_ts(tmem + FI_ACC + (uint32_t)(h * 128),
                                                    ta + (uint32_t)(kb * 32 + kk * 8),
                                                    bdesc(st) + (uint64_t)(x * (16384 >> 4) + 2 * kk),
                                                    ID128, (kb > 0 || kk > 0) ? 1u : 0u);
                                }
                                mma_commit(bar_empty + 8 * st);
                            }
                            if (ok) mma_commit(bar_acc + 8 * h);
                        }
                    }
                    pa ^= 1u;
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
    } else if (warp == FT_STAGE_WARP) {
        // ------------------------------------------------------------ staging
        // Work item n into buffer n mod 2 once the epilogue warps have read the item two
        // before it: member k's biases (hidden layers halved, for the GELU in z/2) and
        // feature statistics into parameter slot b, the raw features and targets of the
        // item's 128 rows into row buffer b.
        bool ok = true;
        long long n = 0;
        for (long long it = blockIdx.x; it < n_items && ok && !abort_flag; it += gridDim.x, ++n) {
            const int b = (int)(n & 1);
            if (n >= 2 && !__all_sync(0xffffffffu, mbar_wait_sleep(bar_se + 8 * b,
                                                                    (uint32_t)((n - 2) >> 1) & 1u,
                                                                    A.wait_limit))) {
                ok = false;
                break;
            }
            const int kn = (int)(it / A.n_tiles);
            const int tn = (int)(it - (long long)kn * A.n_tiles);
            const uint8_t* mbn = A.model + (size_t)kn * A.member_bytes;
            const float* th = reinterpret_cast<const float*>(mbn + A.theta_b);
            const float* stt = reinterpret_cast<const float*>(mbn + A.stats_b);
            float* dst = par + b * FI_PAR_FLOATS;
            {   // all 41 loads of a lane in flight together, then the stores
                static_assert(FI_PAR_FLOATS % 32 == 0, "parameter staging: whole lanes");
                float v[FI_PAR_FLOATS / 32];
#pragma unroll
                for (int q = 0; q < FI_PAR_FLOATS / 32; ++q) {
                    const int i = q * 32 + lane;
                    v[q] = 0.f;
                    if (i < N_LAYERS * 256) {
                        const int l = i >> 8, c = i & 255;
                        if (c < real_out(l)) v[q] = __ldg(th + A.b_off[l] + c) * (l < 4 ? 0.5f : 1.0f);
                    } else {
                        v[q] = __ldg(stt + (i - N_LAYERS * 256));   // mean[16] | std[16]
                    }
                }
#pragma unroll
                for (int q = 0; q < FI_PAR_FLOATS / 32; ++q) dst[q * 32 + lane] = v[q];
            }
            {   // rows q * 32 + lane: the 48 loads of a lane in flight together
                const unsigned stepn =
                    A.dev_step ? (unsigned)*reinterpret_cast<const int*>(mbn + A.step_b) : A.step;
                long long src[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long rown = (long long)tn * 128 + q * 32 + lane;
                    src[q] = A.rows ? (long long)A.rows[rown]
                                    : draw_row(A.seed ^ ((unsigned)(A.member0 + kn) * A.seed_mul), stepn, (int)rown,
                                               A.n_rows);
                }
                float xv[4][FT_ROW_FLOATS];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int f = 0; f < N_FEAT; ++f) xv[q][f] = A.feat[src[q] * N_FEAT + f];
#pragma unroll
                    for (int c = 0; c < N_OUT; ++c) xv[q][N_FEAT + c] = A.targets[src[q] * 3 + c];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float* xr = xbuf + (b * 128 + q * 32 + lane) * FT_ROW_FLOATS;
#pragma unroll
                    for (int c = 0; c < FT_ROW_FLOATS; c += 4)
                        *reinterpret_cast<float4*>(xr + c) =
                            make_float4(xv[q][c], xv[q][c + 1], xv[q][c + 2], xv[q][c + 3]);
                }
            }
            mbar_arrive(bar_sf + 8 * b);
            if (n == 0 && A.dev_step && blockIdx.x == 0) {
                // the schedule entry of each member's step, for Adam
                for (int km = lane; km < A.n_members; km += 32) {
                    const int g = *reinterpret_cast<const int*>(A.model + (size_t)km * A.member_bytes +
                                                                A.step_b);
                    *reinterpret_cast<SchedOut*>(A.ws + (size_t)km * A.region_bytes + A.sched_b) =
                        A.table[(long long)km * A.table_cap + (g - A.table_base[km])];
                }
            }
        }
        if (!ok) {
            atomicOr(&A.status[ST_CALL], DEV_TIMEOUT);
            abort_flag = 1;
        }
    } else {
        // ------------------------------------------------------------ epilogue warps
        const int lq = warp & 3, cg = warp >> 2;            // TMEM lane quarter, column group
        const int r = lq * 32 + lane;                       // tile row = TMEM lane
        const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16);
        const bool lead = cg == 0;                          // builds X0, the output layer
        const float inv_b = 1.0f / (float)A.B;
        uint32_t pacc = 0;
        bool ok = true;
        long long n_done = 0;
        for (long long it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++n_done) {
            const int k = (int)(it / A.n_tiles);
            const int t = (int)(it - (long long)k * A.n_tiles);
            uint8_t* reg = A.ws + (size_t)k * A.region_bytes;
            const long long row = (long long)t * 128 + r;   // batch row (B is a multiple of 128)
            // 16-byte block (chunk, this row) of a row-blocked chunk-major array of nc
            // chunks at byte offset off
            auto cm = [&](size_t off, int nc, int chunk) {
                return reinterpret_cast<uint4*>(
                    reg + off + (((size_t)(row >> 6) * nc + chunk) * 64 + (row & 63)) * 16);
            };
            const int slot = (int)(n_done & 1);
            const float* pk_par = par + slot * FI_PAR_FLOATS;
            if (!__all_sync(0xffffffffu, mbar_wait_sleep(bar_sf + 8 * slot, (uint32_t)(n_done >> 1) & 1u,
                                                         A.wait_limit))) {
                ok = false;
                break;
            }
            float y[N_OUT] = {0.f, 0.f, 0.f};
            if (lead) {   // layer-0 input: standardised features in k 0-8, zeros to 15
                const float* st = pk_par + N_LAYERS * 256;
                const float* xr = xbuf + (slot * 128 + r) * FT_ROW_FLOATS;
                float z[N_FEAT];
#pragma unroll
                for (int f = 0; f < N_FEAT; ++f) z[f] = (xr[f] - st[f]) / st[16 + f];
#pragma unroll
                for (int c = 0; c < N_OUT; ++c) y[c] = xr[N_FEAT + c];
                const uint32_t pk[8] = {pack_bf16(z[0], z[1]), pack_bf16(z[2], z[3]),
                                        pack_bf16(z[4], z[5]), pack_bf16(z[6], z[7]),
                                        pack_bf16(z[8], 0.f), 0u, 0u, 0u};
                tmem_st8(trow + FI_ABUF, pk);
                *cm(A.x0_b, 2, 0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *cm(A.x0_b, 2, 1) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                tmem_wait_st();
            }
            tc_fence_before();
            mbar_arrive(bar_a);
            mbar_arrive(bar_a + 8);
            for (int s = 0; s < 9 && ok; ++s) {
                // every thread waits for both halves of every layer (a parity wait that fell
                // two phases behind its barrier would return at once); a wait's outcome is
                // made uniform over the warp, whose TMEM accesses and shuffles are collective
                const uint32_t dst = trow + FI_ABUF + (uint32_t)(((s + 1) & 1) * 128);
                if (s < 4) {
                    const float* bias = pk_par + s * 256;
                    for (int h = 0; h < 2; ++h) {
                        if (!__all_sync(0xffffffffu, mbar_wait_sleep(bar_acc + 8 * h, pacc, A.wait_limit))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        uint32_t v[32];
                        tmem_ld32_async(trow + FI_ACC + (uint32_t)(h * 128 + cg * 32), v);
                        tmem_wait_ld(v);
#pragma unroll
                        for (int c16 = 0; c16 < 32; c16 += 16) {
                            const float* b = bias + h * 128 + cg * 32 + c16;
                            uint32_t pk[8], gk[8];
#pragma unroll
                            for (int i = 0; i < 16; i += 4) {
                                const float4 b4 = *reinterpret_cast<const float4*>(b + i);
                                gelu_grad_half2(__uint_as_float(v[c16 + i]), __uint_as_float(v[c16 + i + 1]),
                                                b4.x, b4.y, pk[i / 2], gk[i / 2]);
                                gelu_grad_half2(__uint_as_float(v[c16 + i + 2]),
                                                __uint_as_float(v[c16 + i + 3]), b4.z, b4.w,
                                                pk[i / 2 + 1], gk[i / 2 + 1]);
                            }
                            tmem_st8(dst + (uint32_t)(h * 64 + cg * 16 + c16 / 2), pk);
                            const int ch = (h * 128 + cg * 32 + c16) >> 3;
                            *cm(A.h_b[s], 32, ch) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            *cm(A.h_b[s], 32, ch + 1) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                            *cm(A.gp_b[s], 32, ch) = make_uint4(gk[0], gk[1], gk[2], gk[3]);
                            *cm(A.gp_b[s], 32, ch + 1) = make_uint4(gk[4], gk[5], gk[6], gk[7]);
                        }
                        tmem_wait_st();
                        tc_fence_before();
                        mbar_arrive(bar_a + 8 * h);
                    }
                } else if (s == 4) {
                    for (int h = 0; h < 2; ++h)
                        if (!__all_sync(0xffffffffu, mbar_wait_sleep(bar_acc + 8 * h, pacc, A.wait_limit)))
                            ok = false;
                    if (ok && lead) {
                        tc_fence_after();
                        float v[16];
                        tmem_ld16(trow + FI_ACC, v);
                        const float* b4 = pk_par + 4 * 256;
                        float lg[N_OUT], mx = -3.0e38f;
#pragma unroll
                        for (int c = 0; c < N_OUT; ++c) {
                            lg[c] = v[c] + b4[c];
                            mx = fmaxf(mx, lg[c]);
                        }
                        float p[N_OUT], sum = 0.f;
#pragma unroll
                        for (int c = 0; c < N_OUT; ++c) {
                            p[c] = expf(lg[c] - mx);
                            sum += p[c];
                        }
                        const float inv = 1.0f / sum;
                        float li = 0.f, gq[N_OUT];
#pragma unroll
                        for (int c = 0; c < N_OUT; ++c) {
                            p[c] *= inv;
                            li -= y[c] * logf(fmaxf(p[c], 1e-30f));
                            // the gradient as the products will see it (BF16)
                            gq[c] = __bfloat162float(__float2bfloat16((p[c] - y[c]) * inv_b));
                        }
                        const uint32_t pk[8] = {pack_bf16(gq[0], gq[1]), pack_bf16(gq[2], 0.f),
                                                0u, 0u, 0u, 0u, 0u, 0u};
                        tmem_st8(dst, pk);
                        *cm(A.g4_b, 2, 0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *cm(A.g4_b, 2, 1) = make_uint4(0u, 0u, 0u, 0u);
                        // per-warp sums: the bias gradient of layer 4 (column sums of G over
                        // the warp's 32 rows) and the loss
                        li *= inv_b;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            li += __shfl_xor_sync(0xffffffffu, li, off);
#pragma unroll
                            for (int c = 0; c < N_OUT; ++c) gq[c] += __shfl_xor_sync(0xffffffffu, gq[c], off);
                        }
                        if (lane == 0) {
                            float* bp = reinterpret_cast<float*>(reg + A.bp4_b) + ((long long)t * 4 + lq) * 4;
                            *reinterpret_cast<float4*>(bp) = make_float4(gq[0], gq[1], gq[2], 0.f);
                            if (li != 0.f) atomicAdd(A.loss + k, li);
                        }
                        tmem_wait_st();
                    }
                    tc_fence_before();
                    mbar_arrive(bar_a);
                    mbar_arrive(bar_a + 8);
                    // this item's parameters and rows are no longer read: buffer free
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_se + 8 * slot);
                } else {
                    const int j = 8 - s;   // this step's output gradient dZ_j
                    for (int h = 0; h < 2; ++h) {
                        const int ch = (h * 128 + cg * 32) >> 3;   // this thread's 4 chunks
                        uint4 gp[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) gp[q] = *cm(A.gp_b[j], 32, ch + q);
                        if (!__all_sync(0xffffffffu, mbar_wait_sleep(bar_acc + 8 * h, pacc, A.wait_limit))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        uint32_t v[32];
                        tmem_ld32_async(trow + FI_ACC + (uint32_t)(h * 128 + cg * 32), v);
                        tmem_wait_ld(v);
#pragma unroll
                        for (int c16 = 0; c16 < 32; c16 += 16) {
                            uint32_t pk[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const uint4 g4 = gp[c16 / 8 + e / 4];
                                const uint32_t w = (e & 3) == 0 ? g4.x : (e & 3) == 1 ? g4.y
                                                 : (e & 3) == 2 ? g4.z : g4.w;
                                const float2 d = mul2(make_float2(__uint_as_float(v[c16 + 2 * e]),
                                                                  __uint_as_float(v[c16 + 2 * e + 1])),
                                                      make_float2(__uint_as_float(w << 16),
                                                                  __uint_as_float(w & 0xffff0000u)));
                                pk[e] = pack_bf16(d.x, d.y);
                            }
                            if (s < 8) tmem_st8(dst + (uint32_t)(h * 64 + cg * 16 + c16 / 2), pk);
                            *cm(A.dz_b[j], 32, ch + c16 / 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            *cm(A.dz_b[j], 32, ch + c16 / 8 + 1) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        }
                        // GELU'(Z_j) of these rows and columns is dead: its 16 L2 lines (the
                        // warp's 4 chunks x 512 bytes) go without a write-back
                        __syncwarp();
                        if (lane < 16) {
                            const long long row0 = row - lane + (lane & 3) * 8;
                            l2_discard(reg + A.gp_b[j] +
                                       (((size_t)(row0 >> 6) * 32 + ch + (lane >> 2)) * 64 + (row0 & 63)) * 16);
                        }
                        if (s < 8) {
                            tmem_wait_st();
                            tc_fence_before();
                            mbar_arrive(bar_a + 8 * h);
                        }
                    }
                }
                pacc ^= 1u;
            }
            if (abort_flag) ok = false;
        }
        if (!ok) atomicOr(&A.status[ST_CALL], DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, FI_TMEM_COLS);
    // the weight-gradient launch that follows may start (programmatic dependent launch;
    // it waits in griddepcontrol.wait until this grid has completed)
    asm volatile("griddepcontrol.launch_dependents;");
}

// ----------------------------------------------------------------- weight gradients
// Split-K partials of the weight gradients, C[split][m][n] = sum over the split's batch
// rows b of A[b][m] B[b][n], where A and B are train_kernel's row-blocked chunk-major
// arrays: dW_l = dZ_l^T H_{l-1} (H_{-1} = the features) for l = 0..3, and dW_4^T = H_3^T G.
// Both operands are MN-major without swizzle: a core matrix is 8 batch rows x 8 columns
// (16 bytes per row), core matrices consecutive in b lie 128 bytes apart (the descriptor's
// leading byte offset) and those consecutive in m or n DW_BK * 16 bytes apart (its stride
// byte offset), which is the order a 64-row block of the arrays already has: a stage is
// one bulk copy per operand.  A CTA computes the 128 x NT tile (m tile, column block) of
// one (member, layer, split); with a bias partial, the CTAs of column block 0 also form
// sum_b A[b][m] (the bias gradient) as the product with a K-major tile whose row 0 is
// ones, in 16 more accumulator columns.
constexpr int DW_BK = 64;
constexpr int DW_STAGES = 3;
constexpr int DW_LAYS = 3;

struct DwArgs {
    int n_lay;                  // layers in this launch; blockIdx.y = member * n_lay + lay
    int k_per_split;            // multiple of DW_BK; blockIdx.z = split
    const uint8_t* ws;          // member k's region at ws + k * region_bytes
    size_t region_bytes;
    size_t a_b[DW_LAYS], b_b[DW_LAYS];  // the operands' arrays (byte offsets in the region)
    int a_chunks[DW_LAYS], b_chunks[DW_LAYS];
    size_t part_b[DW_LAYS];     // partial [split][256][part_ld] FP32
    int part_ld[DW_LAYS];
    size_t bias_b[DW_LAYS];     // bias partial [split][256] FP32, or 0: none
    unsigned* status;
    long long wait_limit;
};

template <int NT>
struct DwSmem {
    static constexpr int A_BYTES = 128 * DW_BK * 2;
    static constexpr int B_BYTES = NT * DW_BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;     // a multiple of 1024
    static constexpr int ONES_OFF = DW_STAGES * STAGE;  // 1024-aligned (128-byte swizzle)
    static constexpr int BAR_OFF = ONES_OFF + 16 * 128;
    static constexpr int TOTAL = BAR_OFF + (2 * DW_STAGES + 1) * 8 + 16;
    static constexpr int ALLOC = TOTAL + 1024;          // slack for 1024-byte alignment
    static constexpr uint32_t TCOLS = NT + 16 <= 32 ? 32 : (NT + 16 <= 64 ? 64 : (NT + 16 <= 128 ? 128 : 256));
};

template <int NT>
__global__ void __launch_bounds__(128, 1) dw_kernel(const __grid_constant__ DwArgs args) {
    using S = DwSmem<NT>;
    static_assert(S::STAGE % 1024 == 0 && NT + 16 <= 256, "stage alignment, tensor memory");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t ones = base + S::ONES_OFF;
    const uint32_t bar_full = base + S::BAR_OFF;
    const uint32_t bar_empty = bar_full + DW_STAGES * 8;
    const uint32_t bar_done = bar_empty + DW_STAGES * 8;
    const uint32_t tslot = bar_done + 8;
    volatile uint32_t* tslot_ptr = (volatile uint32_t*)(gbase + S::BAR_OFF + (2 * DW_STAGES + 1) * 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x & 1, nb = blockIdx.x >> 1;
    const int lay = blockIdx.y % args.n_lay, k = blockIdx.y / args.n_lay;
    const int split = blockIdx.z;
    const int k0 = split * args.k_per_split, n_k = args.k_per_split / DW_BK;
    const bool bias = args.bias_b[lay] != 0 && nb == 0;
    const uint8_t* reg = args.ws + (size_t)k * args.region_bytes;
    const uint8_t* ga = reg + args.a_b[lay] + (size_t)(mt * 16) * 1024;
    const uint8_t* gb = reg + args.b_b[lay] + (size_t)(nb * (NT / 8)) * 1024;
    const size_t a_blk = (size_t)args.a_chunks[lay] * 1024, b_blk = (size_t)args.b_chunks[lay] * 1024;
    constexpr uint32_t ID_W = idesc_bf16_major(128, NT, true, true);
    constexpr uint32_t ID_B = idesc_bf16_major(128, 16, true, false);

    {   // the ones tile: row 0 of a K-major 16 x 64 BF16 tile is 1.0 (0x3F80), the rest 0
        uint32_t* o = reinterpret_cast<uint32_t*>(gbase + S::ONES_OFF);
        for (int i = threadIdx.x; i < 16 * 64 / 2; i += blockDim.x) o[i] = i < 32 ? 0x3F803F80u : 0u;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the MMAs
    if (threadIdx.x == 0) {
        for (int s = 0; s < DW_STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_done, 1);
        fence_barrier_init();
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(tslot, S::TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_ptr;
    // launched as a programmatic dependent of train_kernel: its outputs are complete and
    // visible after this (at once without such a launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (threadIdx.x == 0) {
        bool ok = true;
        int last_issued = -1, consumed = 0;
        auto load = [&](int j) {
            const int s = j % DW_STAGES;
            const uint32_t a_s = base + s * S::STAGE, b_s = a_s + S::A_BYTES;
            last_issued = j;
            const size_t rb = (size_t)(k0 / DW_BK + j);   // 64-row block of the batch
            mbar_arrive_expect_tx(bar_full + 8 * s, (uint32_t)S::STAGE);
            bulk_load(a_s, ga + rb * a_blk, (uint32_t)S::A_BYTES, bar_full + 8 * s);
            bulk_load(b_s, gb + rb * b_blk, (uint32_t)S::B_BYTES, bar_full + 8 * s);
        };
        for (int j = 0; j < n_k && j < DW_STAGES; ++j) load(j);
        for (int j = 0; j < n_k; ++j) {
            const int s = j % DW_STAGES;
            const uint32_t ph = (uint32_t)(j / DW_STAGES) & 1u;
            if (!mbar_wait(bar_full + 8 * s, ph, args.wait_limit)) {
                ok = false;
                break;
            }
            consumed++;
            tc_fence_after();
            const uint32_t a_s = base + s * S::STAGE, b_s = a_s + S::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < DW_BK / 16; ++kk) {   // 16 batch rows = 2 core matrices = 256 B
                const uint64_t da = desc_mn_plain(a_s + kk * 256, 128, DW_BK * 16);
                const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
                mma_bf16(tmem, da, desc_mn_plain(b_s + kk * 256, 128, DW_BK * 16), ID_W, acc);
                if (bias) mma_bf16(tmem + NT, da, desc_sw128(ones + kk * 32), ID_B, acc);
            }
            mma_commit(bar_empty + 8 * s);
            if (j + DW_STAGES < n_k) {
                if (!mbar_wait(bar_empty + 8 * s, ph, args.wait_limit)) {
                    ok = false;
                    break;
                }
                load(j + DW_STAGES);
            }
        }
        mma_commit(bar_done);
        if (!ok) {
            // let every load that was issued land before the CTA can exit
            for (int j = consumed; j <= last_issued; ++j)
                mbar_wait(bar_full + 8 * (j % DW_STAGES), (uint32_t)(j / DW_STAGES) & 1u,
                          1000000000LL);
            atomicOr(&args.status[ST_CALL], DEV_TIMEOUT);
        }
    }
    __syncwarp();
    const bool done_ok = __all_sync(0xffffffffu, mbar_wait(bar_done, 0, args.wait_limit));
    tc_fence_after();
    if (!done_ok && lane == 0) atomicOr(&args.status[ST_CALL], DEV_TIMEOUT);

    const int r = warp * 32 + lane;
    const int m = mt * 128 + r;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    uint8_t* wreg = const_cast<uint8_t*>(reg);
    const int ld = args.part_ld[lay];
    if (done_ok) {
        float* out = reinterpret_cast<float*>(wreg + args.part_b[lay]) +
                     ((long long)split * 256 + m) * ld + nb * NT;
        float v[16];
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4*>(out + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
        if (bias) {
            tmem_ld16(trow + NT, v);
            reinterpret_cast<float*>(wreg + args.bias_b[lay])[(long long)split * 256 + m] = v[0];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, S::TCOLS);
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

// Offsets of each layer's weights and biases in theta (floats).
struct ParamOffsets {
    long long w_off[N_LAYERS], b_off[N_LAYERS];
};

// Layer l and the weight (o, i) or bias o that parameter idx of theta is; false for
// padding (never updated, always 0).
__device__ __forceinline__ bool param_locate(const ParamOffsets& po, long long idx, int& l,
                                             int& o, int& i, bool& is_w) {
    l = 0;
    while (l + 1 < N_LAYERS && idx >= po.w_off[l + 1]) ++l;
    if (idx < po.b_off[l]) {
        const long long e = idx - po.w_off[l];
        const int sh = l == 0 ? 6 : 8;   // log2 of the padded input width (64 or 256)
        o = (int)(e >> sh);
        i = (int)(e & ((1 << sh) - 1));
        is_w = true;
        return o < real_out(l) && i < real_in(l);
    }
    o = (int)(idx - po.b_off[l]);
    i = 0;
    is_w = false;
    return o < real_out(l);
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

struct AdamArgs {
    ParamOffsets po;
    uint8_t* model;                 // member k = blockIdx.y at model + k * member_bytes
    size_t member_bytes, theta_b, m_b, v_b, wi_b, step_b;
    const uint8_t* ws;              // member k's training arrays at ws + k * region_bytes
    size_t region_bytes;
    size_t part_b[N_LAYERS];        // dW_l split partials [split][rows][ld]; l = 4 transposed
    int part_ld[N_LAYERS];
    long long part_plane[N_LAYERS]; // floats per split
    int splits;
    size_t bias_b[N_LAYERS];        // bias partials: bias_n[l] partials bias_ld[l] floats apart
    int bias_n[N_LAYERS], bias_ld[N_LAYERS];
    float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
    int dev_sched;                  // lr, c1, c2 from the member's schedule slot; step += 1
    size_t sched_b;
    int host_step;                  // without a device schedule: the step count becomes this + 1
    // graph-captured training: the step's call status word folded into the accumulated
    // word by the last kernel of the step (NULL: the caller does it)
    const unsigned* fold_call;
    unsigned* fold_acc;
};

// Gradient of weight (o, i) or bias o of layer l from the member's partials, each summed
// in a fixed order (so the result does not depend on scheduling).
__device__ __forceinline__ float param_grad(const AdamArgs& A, const uint8_t* reg, int l, int o,
                                            int i, bool is_w) {
    if (is_w) {
        const float* part = reinterpret_cast<const float*>(reg + A.part_b[l]);
        const long long e = (l == 4) ? (long long)i * A.part_ld[l] + o : (long long)o * A.part_ld[l] + i;
        return split_sum(part, A.part_plane[l], A.splits, e);
    }
    const float* bp = reinterpret_cast<const float*>(reg + A.bias_b[l]);
    return split_sum(bp, A.bias_ld[l], A.bias_n[l], o);
}

// Weight (l, o, i) = th into the BF16 weight image of a member.
__device__ __forceinline__ void write_image(bf16* wi, int l, int o, int i, float th) {
    const long long ii = img_index(l, o, i);
    if (ii >= 0) wi[ii] = __float2bfloat16(th);
}

// The same sum for four consecutive elements e .. e + 3 (e and stride multiples of 4).
__device__ __forceinline__ float4 split_sum4(const float* v, long long stride, int n, long long e) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a, d = a;
    auto add = [](float4& x, const float4 y) {
        x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
    };
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        add(a, *reinterpret_cast<const float4*>(v + (k + 0) * stride + e));
        add(b, *reinterpret_cast<const float4*>(v + (k + 1) * stride + e));
        add(c, *reinterpret_cast<const float4*>(v + (k + 2) * stride + e));
        add(d, *reinterpret_cast<const float4*>(v + (k + 3) * stride + e));
    }
    for (; k < n; ++k) add(a, *reinterpret_cast<const float4*>(v + k * stride + e));
    return make_float4((a.x + b.x) + (c.x + d.x), (a.y + b.y) + (c.y + d.y),
                       (a.z + b.z) + (c.z + d.z), (a.w + b.w) + (c.w + d.w));
}

// Adam (Kingma & Ba) on every real parameter of member blockIdx.y, four consecutive
// parameters per thread (one weight row or the biases of a layer: every layer's block
// of theta and every row are multiples of 4 long), then its BF16 weight image; the
// member's step count advances.  Padding stays zero.  The parameters' moments and values
// are loaded before the gradient partials, so that all of a thread's loads are in flight
// together; four real weights of a row sit in one 8-byte piece of the image (a 16-byte
// chunk of 8 inputs, i a multiple of 4), stored at once.
__global__ void __launch_bounds__(256) adam_kernel(AdamArgs A, long long P) {
    const int k = blockIdx.y;
    uint8_t* mb = A.model + (size_t)k * A.member_bytes;
    const uint8_t* reg = A.ws + (size_t)k * A.region_bytes;
    float lr = A.lr, c1 = A.c1, c2 = A.c2;
    if (A.dev_sched) {
        const SchedOut* so = reinterpret_cast<const SchedOut*>(reg + A.sched_b);
        lr = so->lr;
        c1 = so->c1;
        c2 = so->c2;
    }
    const float lr_c1 = lr / c1, ic2 = 1.0f / c2;
    float* theta = reinterpret_cast<float*>(mb + A.theta_b);
    float* am = reinterpret_cast<float*>(mb + A.m_b);
    float* av = reinterpret_cast<float*>(mb + A.v_b);
    bf16* wi = reinterpret_cast<bf16*>(mb + A.wi_b);
    // The output layer's biases are updated by an extra last block: their gradient is a sum
    // of bias_n[4] per-tile, per-warp partials, which its first warp adds (lane j adds
    // partials j, j + 32, ... in order, then a shuffle tree, which leaves the same value in
    // every lane), so that no block of the parameter loop waits for that sum.
    if (blockIdx.x == gridDim.x - 1) {
        if (threadIdx.x >= 32) return;
        const long long b4 = A.po.b_off[4];
        float mo = 0.f, vo = 0.f, to = 0.f;
        if (threadIdx.x < N_OUT) {
            mo = am[b4 + threadIdx.x];
            vo = av[b4 + threadIdx.x];
            to = theta[b4 + threadIdx.x];
        }
        const float* bp = reinterpret_cast<const float*>(reg + A.bias_b[4]);
        float acc[N_OUT] = {};
#pragma unroll 8
        for (int j = threadIdx.x; j < A.bias_n[4]; j += 32)
#pragma unroll
            for (int c = 0; c < N_OUT; ++c) acc[c] += bp[(long long)j * A.bias_ld[4] + c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < N_OUT; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
        if (threadIdx.x < N_OUT) {
            float gg = acc[0];
#pragma unroll
            for (int c = 1; c < N_OUT; ++c)
                if (threadIdx.x == c) gg = acc[c];
            mo = A.b1 * mo + (1.f - A.b1) * gg;
            vo = A.b2 * vo + (1.f - A.b2) * gg * gg;
            to = to - __fdividef(lr_c1 * mo, sqrtf(vo * ic2) + A.eps);
            am[b4 + threadIdx.x] = mo;
            av[b4 + threadIdx.x] = vo;
            theta[b4 + threadIdx.x] = to;
        }
        return;
    }
    const long long span = (long long)(gridDim.x - 1) * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < P / 4; q += span) {
        const long long idx = q * 4;
        int l, o, i;
        bool is_w;
        param_locate(A.po, idx, l, o, i, is_w);
        // the four parameters: weights (o, i .. i + 3) or biases o .. o + 3 of layer l
        const int n_real = is_w ? (o < real_out(l) ? min(4, max(0, real_in(l) - i)) : 0)
                                : min(4, max(0, real_out(l) - o));
        if (n_real == 0 || (l == 4 && !is_w)) continue;   // output biases: the last block
        const float4 m0 = *reinterpret_cast<const float4*>(am + idx);
        const float4 v0 = *reinterpret_cast<const float4*>(av + idx);
        const float4 t0 = *reinterpret_cast<const float4*>(theta + idx);
        float g[4];
        if (n_real == 4 && l != 4) {
            const float4 g4 = is_w ? split_sum4(reinterpret_cast<const float*>(reg + A.part_b[l]),
                                                A.part_plane[l], A.splits,
                                                (long long)o * A.part_ld[l] + i)
                                   : split_sum4(reinterpret_cast<const float*>(reg + A.bias_b[l]),
                                                A.bias_ld[l], A.bias_n[l], o);
            g[0] = g4.x; g[1] = g4.y; g[2] = g4.z; g[3] = g4.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                g[e] = e < n_real ? param_grad(A, reg, l, is_w ? o : o + e, is_w ? i + e : 0, is_w) : 0.f;
        }
        float mm[4] = {m0.x, m0.y, m0.z, m0.w}, vv[4] = {v0.x, v0.y, v0.z, v0.w};
        float th[4] = {t0.x, t0.y, t0.z, t0.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= n_real) continue;   // padding: stays 0
            mm[e] = A.b1 * mm[e] + (1.f - A.b1) * g[e];
            vv[e] = A.b2 * vv[e] + (1.f - A.b2) * g[e] * g[e];
            // lr m_hat / (sqrt(v_hat) + eps) with the bias corrections as reciprocals and
            // the quotient by the SFU reciprocal (a few ulp; Adam needs no more)
            th[e] = th[e] - __fdividef(lr_c1 * mm[e], sqrtf(vv[e] * ic2) + A.eps);
        }
        *reinterpret_cast<float4*>(am + idx) = make_float4(mm[0], mm[1], mm[2], mm[3]);
        *reinterpret_cast<float4*>(av + idx) = make_float4(vv[0], vv[1], vv[2], vv[3]);
        *reinterpret_cast<float4*>(theta + idx) = make_float4(th[0], th[1], th[2], th[3]);
        if (is_w) {
            const long long ii = n_real == 4 ? img_index(l, o, i) : -1;
            if (ii >= 0) {
                const uint32_t lo = pack_bf16(th[0], th[1]), hi = pack_bf16(th[2], th[3]);
                *reinterpret_cast<uint2*>(wi + ii) = make_uint2(lo, hi);
            } else {
                for (int e = 0; e < n_real; ++e) write_image(wi, l, o, i + e, th[e]);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int* st = reinterpret_cast<int*>(mb + A.step_b);
        *st = A.dev_sched ? *st + 1 : A.host_step + 1;
        // every other kernel of the step has finished (stream order; Adam sets no status)
        if (A.fold_acc && k == 0) {
            const unsigned v = A.fold_call[ST_CALL];
            if (v) atomicOr(&A.fold_acc[ST_ASYNC], v);
        }
    }
}

// The gradient vector of member 0 in the layout of theta (padding 0): what adam_kernel
// consumes.
__global__ void grad_kernel(AdamArgs A, long long P, float* grad) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l, o, i;
        bool is_w;
        grad[idx] = param_locate(A.po, idx, l, o, i, is_w) ? param_grad(A, A.ws, l, o, i, is_w) : 0.f;
    }
}

// He-uniform initial weights (hash of seed, member, index -> uniform), zero biases,
// zero Adam state, BF16 weight image, step 0.
__global__ void init_kernel(float* theta, float* m, float* v, bf16* wi, int* step,
                            unsigned seed, unsigned member, ParamOffsets po, long long P) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l, o, i;
        bool is_w;
        const bool real = param_locate(po, idx, l, o, i, is_w);
        float th = 0.f;
        if (real && is_w) {
            const uint32_t h = mix32(mix32(seed) ^ mix32(member * 0x27d4eb2du + 0x165667b1u) ^
                                     mix32((uint32_t)idx));
            const float u = ((float)(h >> 8) + 0.5f) * 0x1p-24f;   // (0,1)
            const float lim = sqrtf(6.0f / (float)real_in(l));
            th = (2.f * u - 1.f) * lim;
        }
        theta[idx] = th;
        m[idx] = 0.f;
        v[idx] = 0.f;
        if (is_w) write_image(wi, l, o, i, th);
        if (idx == 0) step[0] = 0;
    }
}

// Parameters given by the caller (device theta in the padded layout): entries outside
// the real rows and columns are stored as 0; Adam state and step are reset and the BF16
// weight image rebuilt.
__global__ void load_kernel(const float* src, float* theta, float* m, float* v, bf16* wi,
                            int* step, ParamOffsets po, long long P) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
         idx += (long long)gridDim.x * blockDim.x) {
        int l, o, i;
        bool is_w;
        const float th = param_locate(po, idx, l, o, i, is_w) ? src[idx] : 0.f;
        theta[idx] = th;
        m[idx] = 0.f;
        v[idx] = 0.f;
        if (is_w) write_image(wi, l, o, i, th);
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

template <int NT>
static fos_status gemm(const Operand& A, const Operand& B, int splits, GemmArgs g,
                       cudaStream_t s) {
    static bool attr_set[64] = {false};
    int dev = 0;
    FOS_CUDA_TRY(cudaGetDevice(&dev));
    if (!attr_set[dev]) {
        FOS_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    g.tx_bytes = (unsigned)(a_box * BK * 2 + NT * BK * 2);
    dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + NT - 1) / NT), (unsigned)splits);
    gemm_kernel<NT><<<grid, 128, Smem<NT>::ALLOC, s>>>(ta, tb, g);
    return from_cuda(cudaGetLastError());
}

// Training workspace (library-owned, per device), in member regions of region_bytes: a
// per-step call for member m uses region m mod TRAIN_SLOTS (so that the steps of up to
// TRAIN_SLOTS members can run concurrently on separate streams), graph-captured training
// region k for member k.  A region holds train_kernel's chunk-major arrays (the features
// X0 and output gradient G: 2 chunks; H_l, dZ_l, GELU'(Z_l): 32 chunks), the split-K
// partials of the weight and bias gradients, the layer-4 bias partials per tile and warp,
// and the schedule slot; the members' losses sit in one array after the regions.
constexpr int TRAIN_SLOTS = 4;
static_assert(TRAIN_SLOTS + 1 <= ST_REGIONS, "a status region per training slot");
struct TrainWs {
    int B = 0, splits = 0, regions = 0;
    uint8_t* mem = nullptr;
    size_t region_bytes = 0;
    float* loss = nullptr;   // [regions]
    size_t x0_b, h_b[4], g4_b, dz_b[4], gp_b[4], part_b[N_LAYERS], bias_b[4], bp4_b, sched_b;
    // the weight gradients of layers 0 and 4 run on a side stream beside those of 1-3
    cudaStream_t side[TRAIN_SLOTS] = {};
    cudaEvent_t ev_fork[TRAIN_SLOTS] = {}, ev_join[TRAIN_SLOTS] = {};
    // graph-captured training: the branches of the member groups after the first
    cudaStream_t branch[TRAIN_SLOTS] = {};
    cudaEvent_t ev_bfork[TRAIN_SLOTS] = {}, ev_bjoin[TRAIN_SLOTS] = {};
};
static TrainWs g_tws[64];

// Split-K count of the weight gradients: at most 4 (at batch 8192, 4 splits of 2048 rows
// measured 0.126 ms per 4-member step against 0.131 ms with 8: half the partials to sum,
// and the hidden layers' 192 CTAs in one wave), each split at least 1024 batch rows (or 1
// split), and dividing the batch's 64-row blocks.
static int dw_splits(int B) {
    int s = 4;
    while (s > 1 && ((B / 64) % s != 0 || B / s < 1024)) s >>= 1;
    return s;
}

static fos_status ensure_train_ws(int dev, int B, int regions, Workspace* ws) {
    TrainWs& w = g_tws[dev];
    if (w.mem && w.B == B && w.regions >= regions) return FOS_OK;
    if (regions < TRAIN_SLOTS) regions = TRAIN_SLOTS;
    if (w.mem && w.B == B && regions < w.regions) regions = w.regions;
    ws->generation++;   // captured training graphs hold the old buffers
    if (w.mem) {
        FOS_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(w.mem);
        w.mem = nullptr;
    }
    const int splits = dw_splits(B);
    const size_t Bp = (size_t)B;
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = al(o + bytes);
        return at;
    };
    w.x0_b = take(2 * Bp * 16);
    for (int l = 0; l < 4; ++l) w.h_b[l] = take(32 * Bp * 16);
    w.g4_b = take(2 * Bp * 16);
    for (int l = 0; l < 4; ++l) w.dz_b[l] = take(32 * Bp * 16);
    for (int l = 0; l < 4; ++l) w.gp_b[l] = take(32 * Bp * 16);
    for (int l = 0; l < N_LAYERS; ++l)
        w.part_b[l] = take((size_t)splits * 256 * ((l == 0 || l == 4) ? 16 : 256) * 4);
    for (int l = 0; l < 4; ++l) w.bias_b[l] = take((size_t)splits * 256 * 4);
    w.bp4_b = take((Bp / 128) * 4 * 4 * 4);
    w.sched_b = take(sizeof(SchedOut));
    w.region_bytes = o;
    const size_t total = o * (size_t)regions + al((size_t)regions * 4);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) return from_cuda(e);
    FOS_CUDA_TRY(cudaMemset(mem, 0, total));
    w.mem = (uint8_t*)mem;
    w.loss = (float*)(w.mem + o * (size_t)regions);
    w.B = B;
    w.splits = splits;
    w.regions = regions;
    if (!w.side[0]) {
        for (int i = 0; i < TRAIN_SLOTS; ++i) {
            FOS_CUDA_TRY(cudaStreamCreateWithFlags(&w.side[i], cudaStreamNonBlocking));
            FOS_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_fork[i], cudaEventDisableTiming));
            FOS_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_join[i], cudaEventDisableTiming));
            FOS_CUDA_TRY(cudaStreamCreateWithFlags(&w.branch[i], cudaStreamNonBlocking));
            FOS_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_bfork[i], cudaEventDisableTiming));
            FOS_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_bjoin[i], cudaEventDisableTiming));
        }
    }
    return FOS_OK;
}

static ParamOffsets param_offsets() {
    ParamOffsets po;
    for (int l = 0; l < N_LAYERS; ++l) {
        po.w_off[l] = LAY.w_off[l];
        po.b_off[l] = LAY.b_off[l];
    }
    return po;
}

static GemmArgs gargs(unsigned* status) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.status = status;
    g.wait_limit = 4000000000LL;   // ~2 s at 2 GHz
    return g;
}

// Device schedule of graph-captured training: member k's entries at table[k * cap + i],
// its first step at base[k].
struct DevSched {
    const SchedOut* table;
    long long cap;
    const int* base;
};

// One Adam step of n_members consecutive members (model at their first member) whose
// workspace regions start at region0, on stream s: train_kernel, the weight gradients
// (layers 1-3 on s, layers 0 and 4 on the slot's side stream), then Adam, or with
// grad_out the gradient of one member.  Without a device schedule the step, learning rate
// and bias corrections are the given ones.
static fos_status train_step(Workspace* ws, int slot, uint8_t* model, int n_members, int region0,
                             const float* feat, const float* targets, long long n_rows, int B,
                             unsigned seed, unsigned seed_mul, unsigned step, const int* rows,
                             float lr, float* grad_out, unsigned* status, cudaStream_t s,
                             const DevSched* ds = nullptr, bool fold_status = false,
                             int member0 = 0) {
    static bool attr_set[64] = {};
    if (!attr_set[ws->device]) {
        FOS_CUDA_TRY(cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          FT_SMEM));
        FOS_CUDA_TRY(cudaFuncSetAttribute(dw_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          DwSmem<128>::ALLOC));
        FOS_CUDA_TRY(cudaFuncSetAttribute(dw_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          DwSmem<16>::ALLOC));
        attr_set[ws->device] = true;
    }
    TrainWs& w = g_tws[ws->device];
    uint8_t* reg0 = w.mem + (size_t)region0 * w.region_bytes;
    const int n_tiles = B / 128;
    FOS_CUDA_TRY(cudaMemsetAsync(w.loss + region0, 0, (size_t)n_members * sizeof(float), s));

    TrainArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.feat = feat;
    ta.targets = targets;
    ta.n_rows = n_rows;
    ta.rows = rows;
    ta.B = B;
    ta.n_tiles = n_tiles;
    ta.n_members = n_members;
    ta.seed = seed;
    ta.seed_mul = seed_mul;
    ta.member0 = member0;
    ta.step = step;
    ta.model = model;
    ta.member_bytes = LAY.bytes;
    ta.theta_b = LAY.theta_b;
    ta.stats_b = LAY.stats_b;
    ta.wi_b = LAY.wi_b;
    ta.step_b = LAY.step_b;
    for (int l = 0; l < N_LAYERS; ++l) ta.b_off[l] = LAY.b_off[l];
    if (ds) {
        ta.dev_step = 1;
        ta.table = ds->table;
        ta.table_cap = ds->cap;
        ta.table_base = ds->base;
    }
    ta.ws = reg0;
    ta.region_bytes = w.region_bytes;
    ta.x0_b = w.x0_b;
    ta.g4_b = w.g4_b;
    for (int l = 0; l < 4; ++l) {
        ta.h_b[l] = w.h_b[l];
        ta.dz_b[l] = w.dz_b[l];
        ta.gp_b[l] = w.gp_b[l];
    }
    ta.bp4_b = w.bp4_b;
    ta.sched_b = w.sched_b;
    ta.loss = w.loss + region0;
    ta.status = status;
    ta.wait_limit = 4000000000LL;   // ~2 s at 2 GHz
    const long long items = (long long)n_members * n_tiles;
    const long long grid = items < ws->num_sms ? items : ws->num_sms;
    train_kernel<<<(unsigned)grid, FT_THREADS, FT_SMEM, s>>>(ta);
    FOS_CUDA_TRY(cudaGetLastError());

    // weight gradients
    const int splits = w.splits;
    DwArgs da;
    std::memset(&da, 0, sizeof(da));
    da.k_per_split = B / splits;
    da.ws = reg0;
    da.region_bytes = w.region_bytes;
    da.status = status;
    da.wait_limit = 4000000000LL;
    {   // layers 0 and 4 (16 columns) on the side stream
        DwArgs d = da;
        d.n_lay = 2;
        d.a_b[0] = w.dz_b[0];
        d.a_chunks[0] = 32;
        d.b_b[0] = w.x0_b;
        d.b_chunks[0] = 2;
        d.part_b[0] = w.part_b[0];
        d.part_ld[0] = 16;
        d.bias_b[0] = w.bias_b[0];
        d.a_b[1] = w.h_b[3];
        d.a_chunks[1] = 32;
        d.b_b[1] = w.g4_b;
        d.b_chunks[1] = 2;
        d.part_b[1] = w.part_b[4];
        d.part_ld[1] = 16;
        d.bias_b[1] = 0;
        FOS_CUDA_TRY(cudaEventRecord(w.ev_fork[slot], s));
        FOS_CUDA_TRY(cudaStreamWaitEvent(w.side[slot], w.ev_fork[slot], 0));
        dw_kernel<16><<<dim3(2, 2 * n_members, splits), 128, DwSmem<16>::ALLOC, w.side[slot]>>>(d);
        FOS_CUDA_TRY(cudaGetLastError());
        FOS_CUDA_TRY(cudaEventRecord(w.ev_join[slot], w.side[slot]));
    }
    {   // layers 1-3: dW_l = dZ_l^T H_{l-1}, two column blocks of 128
        DwArgs d = da;
        d.n_lay = 3;
        for (int l = 1; l <= 3; ++l) {
            d.a_b[l - 1] = w.dz_b[l];
            d.a_chunks[l - 1] = 32;
            d.b_b[l - 1] = w.h_b[l - 1];
            d.b_chunks[l - 1] = 32;
            d.part_b[l - 1] = w.part_b[l];
            d.part_ld[l - 1] = 256;
            d.bias_b[l - 1] = w.bias_b[l];
        }
        // a programmatic dependent of train_kernel: its prologue overlaps that grid's end
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(4, 3 * n_members, splits);
        cfg.blockDim = dim3(128, 1, 1);
        cfg.dynamicSmemBytes = DwSmem<128>::ALLOC;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        FOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, dw_kernel<128>, d));
    }
    FOS_CUDA_TRY(cudaStreamWaitEvent(s, w.ev_join[slot], 0));

    AdamArgs a;
    std::memset(&a, 0, sizeof(a));
    a.po = param_offsets();
    a.model = model;
    a.member_bytes = LAY.bytes;
    a.theta_b = LAY.theta_b;
    a.m_b = LAY.m_b;
    a.v_b = LAY.v_b;
    a.wi_b = LAY.wi_b;
    a.step_b = LAY.step_b;
    a.ws = reg0;
    a.region_bytes = w.region_bytes;
    for (int l = 0; l < N_LAYERS; ++l) {
        a.part_b[l] = w.part_b[l];
        a.part_ld[l] = (l == 0 || l == 4) ? 16 : 256;
        a.part_plane[l] = 256LL * a.part_ld[l];
        if (l < 4) {
            a.bias_b[l] = w.bias_b[l];
            a.bias_n[l] = splits;
            a.bias_ld[l] = 256;
        } else {
            a.bias_b[l] = w.bp4_b;
            a.bias_n[l] = n_tiles * 4;
            a.bias_ld[l] = 4;
        }
    }
    a.splits = splits;
    const unsigned pblocks = (unsigned)((LAY.P + 255) / 256);
    const unsigned qblocks = (unsigned)((LAY.P / 4 + 255) / 256);
    if (grad_out) {   // diagnostic: export the gradient instead of updating
        grad_kernel<<<pblocks, 256, 0, s>>>(a, LAY.P, grad_out);
        return from_cuda(cudaGetLastError());
    }
    a.lr = lr;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    const double t = (double)step + 1.0;
    a.c1 = (float)(1.0 - pow(0.9, t));
    a.c2 = (float)(1.0 - pow(0.999, t));
    a.dev_sched = ds ? 1 : 0;
    a.sched_b = w.sched_b;
    a.host_step = (int)step;
    if (fold_status) {
        a.fold_call = status;
        a.fold_acc = ws->status;
    }
    adam_kernel<<<dim3(qblocks + 1, (unsigned)n_members), 256, 0, s>>>(a, LAY.P);
    return from_cuda(cudaGetLastError());
}

// ----------------------------------------------------------------------- graph training
// Many steps of every member with no host work per step: one ensemble step (every
// member's schedule entry from its device step counter, train_step over all members, the
// losses, the status folded into the accumulated word) is captured into CUDA graphs of
// FIT_REPS steps and of one step, and a call launches as many of each as its steps need.
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
    long long reps;          // ensemble steps per graph launch
    bool operator==(const FitKey& o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};
struct FitGraph {
    FitKey key;
    cudaGraphExec_t exec = nullptr;
};
struct FitDev {
    std::vector<FitGraph> graphs;
    SchedOut* table = nullptr;   // [members][cap] schedule entries, then [members] bases
    long long table_cap = 0;
    int table_members = 0;
};
static FitDev g_fit[64];
constexpr int FIT_REPS = 8;
// member groups on parallel branches of a step (3 or 4 groups of a 4-member ensemble
// measured no faster than 2)
constexpr int FIT_GROUPS = 2;

// Enqueues one ensemble step on stream cs (status region 1).
static fos_status enqueue_fit_step(Workspace* ws, const FitKey& k, cudaStream_t cs) {
    TrainWs& w = g_tws[ws->device];
    const int region = 1;
    unsigned* status = ws->status + ST_WORDS * region;
    FOS_CUDA_TRY(cudaMemsetAsync(status + ST_CALL, 0, sizeof(unsigned), cs));
    const int* bases = reinterpret_cast<const int*>(k.table + (long long)k.n_members * k.table_cap);
    const unsigned seed = (unsigned)(k.seed ^ (k.seed >> 32));
    // The members in FIT_GROUPS groups on parallel branches, each its own train_kernel,
    // weight gradients and Adam: the weight gradients and Adam of one group run beside the
    // other groups' tiles instead of after every member's (the members are independent).
    const int G = k.n_members < FIT_GROUPS ? k.n_members : FIT_GROUPS;
    for (int g = 1; g < G; ++g) {
        FOS_CUDA_TRY(cudaEventRecord(w.ev_bfork[g], cs));
        FOS_CUDA_TRY(cudaStreamWaitEvent(w.branch[g], w.ev_bfork[g], 0));
    }
    for (int g = 0; g < G; ++g) {
        const int m0 = g * k.n_members / G, m1 = (g + 1) * k.n_members / G;
        const DevSched dsg{k.table + (long long)m0 * k.table_cap, k.table_cap, bases + m0};
        cudaStream_t sg = g == 0 ? cs : w.branch[g];
        const fos_status st = train_step(ws, g, (uint8_t*)k.model + (size_t)m0 * LAY.bytes,
                                         m1 - m0, m0, k.feat, k.targets, k.n_rows, k.B, seed,
                                         0x9E3779B9u, 0, nullptr, 1.0f, nullptr, status, sg, &dsg,
                                         true, m0);   // Adam folds the status word
        if (st != FOS_OK) return st;
    }
    for (int g = 1; g < G; ++g) {
        FOS_CUDA_TRY(cudaEventRecord(w.ev_bjoin[g], w.branch[g]));
        FOS_CUDA_TRY(cudaStreamWaitEvent(cs, w.ev_bjoin[g], 0));
    }
    if (k.loss_out)
        FOS_CUDA_TRY(cudaMemcpyAsync(k.loss_out, w.loss, (size_t)k.n_members * sizeof(float),
                                     cudaMemcpyDeviceToDevice, cs));
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
    fos_status st = FOS_OK;
    for (long long r = 0; r < k.reps && st == FOS_OK; ++r) st = enqueue_fit_step(ws, k, ws->side);
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
        FOS_CUDA_TRY(cudaMemsetAsync((char*)model + (size_t)k * mlp::LAY.bytes, 0, mlp::LAY.bytes, s));
        mlp::init_kernel<<<(unsigned)((mlp::LAY.P + 255) / 256), 256, 0, s>>>(
            mp.theta, mp.m, mp.v, mp.wi, mp.step, (unsigned)(seed ^ (seed >> 32)),
            (unsigned)k, mlp::param_offsets(), mlp::LAY.P);
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
    FOS_CUDA_TRY(cudaMemsetAsync((char*)model + (size_t)member * mlp::LAY.bytes, 0,
                                 mlp::LAY.bytes, s));
    mlp::load_kernel<<<(unsigned)((mlp::LAY.P + 255) / 256), 256, 0, s>>>(
        theta, mp.theta, mp.m, mp.v, mp.wi, mp.step, mlp::param_offsets(), mlp::LAY.P);
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
    st = mlp::ensure_train_ws(ws->device, batch, mlp::TRAIN_SLOTS, ws);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int region = 1 + slot;   // concurrent slots keep separate call words
    unsigned* status = ws->status + ST_WORDS * region;
    FOS_CUDA_TRY(cudaMemsetAsync(status + ST_CALL, 0, sizeof(unsigned), s));
    st = mlp::train_step(ws, slot, (uint8_t*)model + (size_t)member * mlp::LAY.bytes, 1, slot,
                         features, targets, n_rows, batch,
                         (unsigned)(seed ^ (seed >> 32)) ^ (unsigned)(member * 0x9E3779B9u), 0u,
                         (unsigned)step, batch_rows, lr, grad_out, status, s);
    if (st != FOS_OK) return st;
    if (loss_out)
        FOS_CUDA_TRY(cudaMemcpyAsync(loss_out, mlp::g_tws[ws->device].loss + slot, sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
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
    st = mlp::ensure_train_ws(ws->device, batch, n_members, ws);
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
        // graphs of FIT_REPS steps (fewer gaps between graph launches), then single steps
        for (const long long reps : {(long long)mlp::FIT_REPS, 1LL}) {
            const long long n = reps > 1 ? n_steps / reps : n_steps % mlp::FIT_REPS;
            if (n == 0) continue;
            k.reps = reps;
            cudaGraphExec_t exec = nullptr;
            st = mlp::fit_graph(ws, k, &exec);
            if (st != FOS_OK) return st;
            for (long long i = 0; i < n; ++i) FOS_CUDA_TRY(cudaGraphLaunch(exec, s));
        }
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
    if (N % 256 == 0) st = mlp::gemm<256>(a, b, splits, g, s);
    else st = mlp::gemm<64>(a, b, splits, g, s);
    if (st != FOS_OK) return st;
    return finish_call(ws, s, flags & FOS_ASYNC);
}

}  // extern "C"
