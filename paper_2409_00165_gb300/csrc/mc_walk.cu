// Monte Carlo photon transport on GB300 (arxiv 2409.00165, section "Photon transport"):
// validation and packing of the item tables, the work-unit prefix, the exact walk's
// kernels (walk_kernel.cuh, compiled here with -fmad=false so that the FP32 operation
// order is exactly the one written), the launch sequence, its CUDA-graph cache and the
// launch-shape autotuner.  mc_walk_fast.cu compiles the fast (SFU) walk.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <curand_philox4x32_x.h>

#include "walk_kernel.cuh"

namespace fos {
namespace mc {

// ---------------------------------------------------------------------------------
// Packed per-row tables (row = position in the run list).
// ---------------------------------------------------------------------------------
static size_t tables_bytes(long long n_run, int max_layers) {
    size_t b = 0;
    b += (size_t)n_run * sizeof(int4) * 2;
    b += (size_t)n_run * sizeof(float4);
    b += (size_t)n_run * max_layers * sizeof(float4) * 3;
    b += (size_t)(n_run + 1) * sizeof(long long);
    return b + 8 * 256;   // each of the 7 regions is rounded up to 256 bytes
}

static Tables carve(void* base, long long n_run, int max_layers) {
    Tables t;
    char* p = (char*)base;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    t.head = (int4*)take((size_t)n_run * sizeof(int4));
    t.info = (int4*)take((size_t)n_run * sizeof(int4));
    t.edge = (float4*)take((size_t)n_run * sizeof(float4));
    t.layA = (float4*)take((size_t)n_run * max_layers * sizeof(float4));
    t.layB = (float4*)take((size_t)n_run * max_layers * sizeof(float4));
    t.layC = (float4*)take((size_t)n_run * max_layers * sizeof(float4));
    t.prefix = (long long*)take((size_t)(n_run + 1) * sizeof(long long));
    return t;
}

struct PackArgs {
    fos_mc_batch b;
    int n_run;
    long long log_stride;  // 0: no photon log
    int inject;
    Tables t;
    unsigned* status;
};

__device__ __forceinline__ void flag_invalid(unsigned* status, int row) {
    atomicOr(&status[ST_CALL], DEV_INVALID);
    atomicMin(&status[ST_INDEX], (unsigned)row);
}

__device__ __forceinline__ bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Validates one row and writes its packed tables (one thread per row).
__global__ void pack_kernel(PackArgs A) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (A.inject && r == 0) atomicOr(&A.status[ST_CALL], DEV_INJECTED);
    if (r >= A.n_run) return;
    const fos_mc_batch& b = A.b;
    const long long n_items = (long long)b.n_stacks * b.n_wl;
    long long it = b.item_list ? (long long)b.item_list[r] : (long long)r;
    bool ok = it >= 0 && it < n_items;
    if (!ok) {
        flag_invalid(A.status, r);
        it = 0;
    }
    const int s = (int)(it / b.n_wl), w = (int)(it % b.n_wl);
    int nl = b.n_layers ? b.n_layers[s] : b.max_layers;
    if (nl < 1 || nl > b.max_layers) {
        ok = false;
        nl = 1;
    }
    for (int j = 0; j < b.max_layers; ++j) {
        float4 la = make_float4(0.f, 0.f, 0.f, 1.f), lb = make_float4(1.f, 1.f, 1.f, 1.f);
        float4 lc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < nl) {
            const long long pi = ((long long)s * b.max_layers + j) * b.n_wl + w;
            const double ms = b.mu_s[pi], ma = b.mu_a[pi], gg = b.g[pi], nn = b.n_layer[pi];
            const double dd = b.thickness[(long long)s * b.max_layers + j];
            if (!(isfinite(ms) && ms >= 0.0) || !(isfinite(ma) && ma >= 0.0) ||
                !(gg > -1.0 && gg < 1.0) || !finite_pos(nn) || !finite_pos(dd))
                ok = false;
            const float msf = (float)ms, maf = (float)ma, gf = (float)gg;
            const float mt = msf + maf;
            const float pabs = (mt > 0.0f) ? maf / mt : 0.0f;
            if (!isfinite(mt) || !isfinite((float)dd) || (float)dd <= 0.0f || (float)nn <= 0.0f)
                ok = false;
            // absorption test on the word itself: uni(w) = (2k+1) 2^-24 with k = w >> 9,
            // and (2k+1) 2^-24 < pabs exactly when k < ceil((pabs 2^24 - 1) / 2)
            const double kab = fmin(fmax(ceil(((double)pabs * 16777216.0 - 1.0) * 0.5), 0.0),
                                    8388608.0);
            la = make_float4(mt, __uint_as_float((unsigned)kab), gf, (float)nn);
            lb = make_float4((float)dd, 1.0f - gf * gf, 1.0f + gf * gf, 1.0f - gf);
            lc = make_float4((mt > 0.0f) ? 1.0f / mt : 0.0f,
                             (fabsf(gf) < 0x1.0c6f7ap-20f) ? 0.0f : 1.0f / (gf + gf), 0.f, 0.f);
        }
        A.t.layA[(long long)r * b.max_layers + j] = la;
        A.t.layB[(long long)r * b.max_layers + j] = lb;
        A.t.layC[(long long)r * b.max_layers + j] = lc;
    }
    const double na = b.n_above ? b.n_above[it] : 1.0;
    const double nb = b.n_below ? b.n_below[it] : 1.0;
    if (!finite_pos(na) || !finite_pos(nb)) ok = false;
    // index quotients of each layer's faces (the walk's Fresnel step at boundary events)
    for (int j = 0; j < nl; ++j) {
        float4* lc = &A.t.layC[(long long)r * b.max_layers + j];
        const float nj = A.t.layA[(long long)r * b.max_layers + j].w;
        const float n_up = (j == 0) ? (float)na : A.t.layA[(long long)r * b.max_layers + j - 1].w;
        const float n_dn = (j == nl - 1) ? (float)nb : A.t.layA[(long long)r * b.max_layers + j + 1].w;
        lc->z = nj / n_up;
        lc->w = nj / n_dn;
    }
    float rsub = -1.0f;
    if (b.substrate_R) {
        const double v = b.substrate_R[it];
        if (!(v >= 0.0 && v <= 1.0)) ok = false;
        rsub = (float)v;
    }
    const double cin = b.cos_incidence ? b.cos_incidence[it] : 1.0;
    const double kb = b.k_below ? b.k_below[it] : 0.0;
    if (!(cin > 0.0 && cin <= 1.0) || !(kb >= 0.0 && isfinite(kb))) ok = false;
    if (kb > 0.0 && b.substrate_R) ok = false;
    const float cin_f = (float)cin, kb_f = (float)kb;
    if (!(cin_f > 0.0f)) ok = false;
    if (kb_f > 0.0f && !b.substrate_R) rsub = -2.0f;
    const long long N = b.n_photons ? b.n_photons[it] : b.photons_per_item;
    const long long first = b.photon_first ? b.photon_first[it] : 0;
    if (N < 0 || N > 0xffffffffLL || first < 0 || first + N > 4294967296LL) ok = false;
    if (A.log_stride > 0 && N > A.log_stride) ok = false;
    if (!ok) flag_invalid(A.status, r);
    A.t.head[r] = make_int4(nl, __float_as_int((float)na), __float_as_int((float)nb),
                            __float_as_int(rsub));
    float r_entry = 0.0f, mu_in = cin_f;
    {
        const float na_f = (float)na, n0 = A.t.layA[(long long)r * b.max_layers].w;
        if (na_f != n0) {
            float ct;
            bool tir;
            r_entry = fresnel(na_f, n0, cin_f, ct, tir);   // 1 under total reflection
            if (!tir) mu_in = ct;
        }
    }
    A.t.edge[r] = make_float4(mu_in, cin_f, kb_f, 0.0f);
    A.t.info[r] = make_int4((int)(b.item_id_base + (unsigned)it), (int)(unsigned)first,
                            ok ? (int)(unsigned)N : 0, __float_as_int(r_entry));
}

// Exclusive prefix of work units per row, one block: each thread sums a contiguous
// slice, the block scans the slice sums, each thread writes its slice.
__global__ void unit_scan_kernel(const int4* info, int n_run, unsigned unit,
                                 unsigned long long scale, long long* prefix) {
    __shared__ long long sums[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (n_run + T - 1) / T;
    const int lo = min(n_run, t * per), hi = min(n_run, lo + per);
    long long acc = 0;
    for (int r = lo; r < hi; ++r) {
        const unsigned long long n = scaled_count((unsigned)info[r].z, scale);
        acc += (long long)((n + unit - 1) / unit);
    }
    sums[t] = acc;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        long long v = (t >= off) ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    long long run = sums[t] - acc;
    for (int r = lo; r < hi; ++r) {
        prefix[r] = run;
        const unsigned long long n = scaled_count((unsigned)info[r].z, scale);
        run += (long long)((n + unit - 1) / unit);
    }
    if (t == T - 1) prefix[n_run] = sums[T - 1];
}

// ---------------------------------------------------------------------------------
// Diagnostics.
// ---------------------------------------------------------------------------------

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with its key schedule: 10 rounds of
// two 32x32->64 products; high halves XOR the other counter words and the key; the key
// advances by the Weyl increments before each round after the first.
__device__ __forceinline__ uint4 philox(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__global__ void philox_fill_kernel(const uint4* ctr, unsigned k0, unsigned k1, uint4* out,
                                   long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = philox(ctr[i], k0, k1);
}

// The same generator as computed by cuRAND's device Philox4x32-10 (a library routine,
// called, for the parity tests).
__global__ void philox_curand_kernel(const uint4* ctr, unsigned k0, unsigned k1, uint4* out,
                                     long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = curand_Philox4x32_10(ctr[i], make_uint2(k0, k1));
}

__global__ void walk_math_kernel(const float* u, float* nl, float* cs, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (nl) nl[i] = neg_log_u(u[i]);
        if (cs) cs[i] = cos_2pi_u(u[i]);
    }
}

// ---------------------------------------------------------------------------------
// Host side: launch sequence, CUDA graph cache, tuning.
// ---------------------------------------------------------------------------------
const void* walk_kernel_exact(int block) { return walk_kernel_for<false>(block); }

static const void* walk_fn(bool fast, int block) {
    return fast ? walk_kernel_fast(block) : walk_kernel_exact(block);
}

struct Tuning {
    int block = 128;
    int ppt = 8;
    int epr = WALK_EVENTS_PER_REFILL;   // events per live photon between refill votes
};

struct GraphKey {
    fos_mc_batch b;
    long long* counts;
    int* log;
    long long log_stride;
    int block, ppt, epr, inject, device, fast;
    unsigned long long* times;
    unsigned long long generation;
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
};

struct ShapeKey {
    int device, n_stacks, n_wl, max_layers, n_list, per_item_array, fast;
    long long photons_per_item;
    bool operator==(const ShapeKey& o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct State {
    std::mutex mu;
    Tuning override_t;
    bool has_override = false;
    std::vector<std::pair<ShapeKey, Tuning>> tuned;
    std::vector<GraphEntry> graphs;
    unsigned long long clock = 0;
    int times_blocks[64] = {};   // blocks of the last launch that recorded its times
};
static State g_state;

static ShapeKey shape_of(const fos_mc_batch* b, int dev, bool fast) {
    ShapeKey k;
    std::memset(&k, 0, sizeof(k));
    k.device = dev;
    k.n_stacks = b->n_stacks;
    k.n_wl = b->n_wl;
    k.max_layers = b->max_layers;
    k.n_list = b->item_list ? b->n_list : -1;
    k.per_item_array = b->n_photons != nullptr;
    k.fast = fast ? 1 : 0;
    k.photons_per_item = b->n_photons ? 0 : b->photons_per_item;
    return k;
}

static fos_status validate_host(const fos_mc_batch* b, const long long* counts,
                                const int* log, long long log_stride, long long* n_run) {
    if (!b) return FOS_ERR_INVALID_ARG;
    if (b->n_stacks < 1 || b->n_wl < 1) return FOS_ERR_INVALID_ARG;
    if (b->max_layers < 1 || b->max_layers > FOS_MAX_LAYERS) return FOS_ERR_INVALID_ARG;
    const long long n_items = (long long)b->n_stacks * b->n_wl;
    if (n_items > 0x7fffffffLL) return FOS_ERR_INVALID_ARG;
    if (!b->mu_s || !b->mu_a || !b->g || !b->n_layer || !b->thickness)
        return FOS_ERR_INVALID_ARG;
    if (!b->n_photons && (b->photons_per_item < 0 || b->photons_per_item > 0xffffffffLL))
        return FOS_ERR_INVALID_ARG;
    if (b->max_events < 0 || b->max_events > 0xffffffffLL) return FOS_ERR_INVALID_ARG;
    if (b->item_list && b->n_list < 0) return FOS_ERR_INVALID_ARG;
    *n_run = b->item_list ? b->n_list : n_items;
    if (*n_run > 0 && !counts) return FOS_ERR_INVALID_ARG;
    if (log && log_stride <= 0) return FOS_ERR_INVALID_ARG;
    return FOS_OK;
}

static Tuning pick_tuning(const fos_mc_batch* b, int dev, bool fast) {
    std::lock_guard<std::mutex> lock(g_state.mu);
    if (g_state.has_override) return g_state.override_t;
    ShapeKey k = shape_of(b, dev, fast);
    for (auto& e : g_state.tuned)
        if (e.first == k) return e.second;
    return Tuning();
}

// Persistent grid: SMs x resident blocks of the variant.
static int grid_for(const Workspace* ws, bool fast, int block) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_fn(fast, block), block, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    return ws->num_sms * per_sm;
}

constexpr unsigned long long SCALE_ALL = 1ull << 32;

// Enqueues the status and counter resets and the validation + packing of the tables.
static fos_status enqueue_pack(Workspace* ws, const fos_mc_batch* b, long long n_run,
                               long long* counts, int* log, long long log_stride, int inject,
                               cudaStream_t s) {
    Tables t = carve(ws->mc_tables, n_run, b->max_layers);
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_INDEX, 0xff, sizeof(unsigned), s));
    FOS_CUDA_TRY(cudaMemsetAsync(ws->cursor, 0, sizeof(unsigned long long), s));
    if (counts)
        FOS_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)n_run * FOS_NCOUNT * sizeof(long long), s));
    PackArgs pa;
    pa.b = *b;
    pa.n_run = (int)n_run;
    pa.log_stride = log ? log_stride : 0;
    pa.inject = inject;
    pa.t = t;
    pa.status = ws->status;
    const int pb = 256;
    pack_kernel<<<(unsigned)((n_run + pb - 1) / pb), pb, 0, s>>>(pa);
    FOS_CUDA_TRY(cudaGetLastError());
    return FOS_OK;
}

// Enqueues the unit prefix and the walk on tables already packed.
static fos_status enqueue_walk(Workspace* ws, const fos_mc_batch* b, long long n_run,
                               long long* counts, int* log, long long log_stride, Tuning tu,
                               unsigned long long scale, bool fast,
                               unsigned long long* times, cudaStream_t s) {
    Tables t = carve(ws->mc_tables, n_run, b->max_layers);
    const unsigned unit = 32u * (unsigned)tu.ppt;
    unit_scan_kernel<<<1, 1024, 0, s>>>(t.info, (int)n_run, unit, scale, t.prefix);
    FOS_CUDA_TRY(cudaGetLastError());
    WalkArgs wa;
    wa.t = t;
    wa.n_run = (int)n_run;
    wa.max_layers = b->max_layers;
    wa.unit = unit;
    wa.scale = scale;
    wa.events_per_refill = tu.epr;
    {
        unsigned k0 = (unsigned)(b->seed & 0xffffffffull), k1 = (unsigned)(b->seed >> 32);
        for (int r = 0; r < 10; ++r) {
            wa.rk.k0[r] = k0;
            wa.rk.k1[r] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    wa.max_events = b->max_events > 0 ? (unsigned)b->max_events : 100000000u;
    wa.cursor = ws->cursor;
    wa.counts = (unsigned long long*)counts;
    wa.photon_log = log;
    wa.log_stride = log ? log_stride : 0;
    wa.status = ws->status;
    wa.cta_times = times;
    void* args[] = {&wa};
    FOS_CUDA_TRY(cudaLaunchKernel(walk_fn(fast, tu.block), dim3(grid_for(ws, fast, tu.block)),
                                  dim3(tu.block), args, 0, s));
    return FOS_OK;
}

// Enqueues the whole call on `s`.
static fos_status enqueue(Workspace* ws, const fos_mc_batch* b, long long n_run,
                          long long* counts, int* log, long long log_stride, Tuning tu,
                          unsigned long long scale, int inject, bool fast,
                          unsigned long long* times, cudaStream_t s) {
    fos_status st = enqueue_pack(ws, b, n_run, counts, log, log_stride, inject, s);
    if (st != FOS_OK) return st;
    return enqueue_walk(ws, b, n_run, counts, log, log_stride, tu, scale, fast, times, s);
}

static fos_status launch(Workspace* ws, const fos_mc_batch* b, long long n_run,
                         long long* counts, int* log, long long log_stride, Tuning tu,
                         unsigned flags, cudaStream_t s) {
    const int inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
    const bool fast = (flags & FOS_FAST_WALK) != 0;
    unsigned long long* times = nullptr;
    if (flags & FOS_RECORD_TIMES) {
        const int grid = grid_for(ws, fast, tu.block);
        fos_status st = ensure_buffer(ws, (void**)&ws->walk_times, &ws->walk_times_bytes,
                                      (size_t)grid * 2 * sizeof(unsigned long long));
        if (st != FOS_OK) return st;
        times = ws->walk_times;
        std::lock_guard<std::mutex> lock(g_state.mu);
        g_state.times_blocks[ws->device] = grid;
    }
    if (flags & FOS_NO_GRAPH)
        return enqueue(ws, b, n_run, counts, log, log_stride, tu, SCALE_ALL, inject, fast, times,
                       s);
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.b = *b;
    key.counts = counts;
    key.log = log;
    key.log_stride = log_stride;
    key.block = tu.block;
    key.ppt = tu.ppt;
    key.epr = tu.epr;
    key.inject = inject;
    key.device = ws->device;
    key.fast = fast ? 1 : 0;
    key.times = times;
    key.generation = ws->generation;
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_state.mu);
        for (auto& g : g_state.graphs) {
            if (std::memcmp(&g.key, &key, sizeof(key)) == 0) {
                exec = g.exec;
                g.last_use = ++g_state.clock;
                break;
            }
        }
    }
    if (!exec) {
        cudaGraph_t graph = nullptr;
        FOS_CUDA_TRY(cudaStreamBeginCapture(ws->side, cudaStreamCaptureModeThreadLocal));
        fos_status st = enqueue(ws, b, n_run, counts, log, log_stride, tu, SCALE_ALL, inject,
                                fast, times, ws->side);
        cudaError_t ce = cudaStreamEndCapture(ws->side, &graph);
        if (st != FOS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        FOS_CUDA_TRY(ce);
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        FOS_CUDA_TRY(ce);
        std::lock_guard<std::mutex> lock(g_state.mu);
        if (g_state.graphs.size() >= 16) {
            size_t oldest = 0;
            for (size_t i = 1; i < g_state.graphs.size(); ++i)
                if (g_state.graphs[i].last_use < g_state.graphs[oldest].last_use) oldest = i;
            cudaGraphExecDestroy(g_state.graphs[oldest].exec);
            g_state.graphs.erase(g_state.graphs.begin() + oldest);
        }
        GraphEntry ge;
        ge.key = key;
        ge.exec = exec;
        ge.last_use = ++g_state.clock;
        g_state.graphs.push_back(ge);
    }
    FOS_CUDA_TRY(cudaGraphLaunch(exec, s));
    return FOS_OK;
}

// Photons the autotuner's probe runs: enough for tens of work units per resident warp,
// so that the probe measures the steady state rather than the tail of its last units.
constexpr double PROBE_PHOTONS = 67108864.0;   // 2^26

// Times every (block, ppt) candidate, then the other refill cadences at the best of those,
// on a copy of the batch whose photon budgets are all scaled by one factor (so the probe
// keeps the batch's budget distribution; rows keep at least one photon), and caches the
// fastest per batch shape.
static fos_status autotune(Workspace* ws, const fos_mc_batch* b, long long n_run, bool fast,
                           cudaStream_t s, Tuning* best) {
    const size_t cbytes = (size_t)n_run * FOS_NCOUNT * sizeof(long long);
    fos_status st = ensure_buffer(ws, (void**)&ws->tune_counts, &ws->tune_bytes, cbytes);
    if (st != FOS_OK) return st;
    // total photons of the batch: the unit prefix with one photon per unit
    st = enqueue_pack(ws, b, n_run, ws->tune_counts, nullptr, 0, 0, s);
    if (st != FOS_OK) return st;
    Tables t = carve(ws->mc_tables, n_run, b->max_layers);
    unit_scan_kernel<<<1, 1024, 0, s>>>(t.info, (int)n_run, 1u, SCALE_ALL, t.prefix);
    FOS_CUDA_TRY(cudaGetLastError());
    st = wait_stream(s, default_timeout_ms());
    if (st != FOS_OK) return st;
    long long total = 0;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&total, t.prefix + n_run, sizeof(long long), cudaMemcpyDeviceToHost));
    FOS_CUDA_TRY(cudaMemcpy(&bits, ws->status + ST_CALL, sizeof(unsigned),
                            cudaMemcpyDeviceToHost));
    if (bits & (DEV_INVALID | DEV_INJECTED | DEV_RANGE)) return status_from_bits(bits);
    if (total <= 0) return FOS_ERR_INVALID_ARG;
    unsigned long long scale = SCALE_ALL;
    if ((double)total > PROBE_PHOTONS)
        scale = (unsigned long long)(PROBE_PHOTONS / (double)total * 4294967296.0);
    if (scale < 1) scale = 1;
    const int ppts[] = {4, 8, 16};
    const bool verbose = getenv("FOS_AUTOTUNE_VERBOSE") != nullptr;
    cudaEvent_t e0, e1;
    FOS_CUDA_TRY(cudaEventCreate(&e0));
    FOS_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    Tuning bt;
    bool first = true;
    // the fastest of two or three timed runs of one shape (the very first run is a warm-up)
    auto probe = [&](const Tuning& tu, float* out_ms) -> fos_status {
        float ms_min = 1e30f;
        for (int rep = 0; rep < (first ? 3 : 2); ++rep) {
            fos_status r = enqueue_pack(ws, b, n_run, ws->tune_counts, nullptr, 0, 0, s);
            if (r != FOS_OK) return r;
            cudaEventRecord(e0, s);
            r = enqueue_walk(ws, b, n_run, ws->tune_counts, nullptr, 0, tu, scale, fast, nullptr, s);
            if (r != FOS_OK) return r;
            cudaEventRecord(e1, s);
            r = wait_stream(s, default_timeout_ms());
            if (r != FOS_OK) return r;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if ((rep > 0 || !first) && ms < ms_min) ms_min = ms;
        }
        first = false;
        if (verbose)
            fprintf(stderr, "fos autotune: %s block %d ppt %d events per refill %d: %.3f ms\n",
                    fast ? "fast" : "exact", tu.block, tu.ppt, tu.epr, ms_min);
        *out_ms = ms_min;
        return FOS_OK;
    };
    // (block, photons per thread) at the default refill cadence, then the other cadences at
    // the best of those
    for (int bl : WALK_BLOCKS) {
        for (int pp : ppts) {
            Tuning tu;
            tu.block = bl;
            tu.ppt = pp;
            float ms = 0.f;
            st = probe(tu, &ms);
            if (st != FOS_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                bt = tu;
            }
        }
        if (st != FOS_OK) break;
    }
    for (int epr : WALK_EVENTS_PER_REFILL_ALT) {
        if (st != FOS_OK) break;
        Tuning tu = bt;
        tu.epr = epr;
        float ms = 0.f;
        st = probe(tu, &ms);
        if (st == FOS_OK && ms < best_ms) {
            best_ms = ms;
            bt = tu;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FOS_OK) return st;
    FOS_CUDA_TRY(cudaMemcpy(&bits, ws->status + ST_CALL, sizeof(unsigned),
                            cudaMemcpyDeviceToHost));
    if (bits & (DEV_INVALID | DEV_INJECTED | DEV_RANGE)) return status_from_bits(bits);
    *best = bt;
    std::lock_guard<std::mutex> lock(g_state.mu);
    ShapeKey k = shape_of(b, ws->device, fast);
    for (auto& e : g_state.tuned)
        if (e.first == k) {
            e.second = bt;
            return FOS_OK;
        }
    g_state.tuned.push_back({k, bt});
    return FOS_OK;
}

static fos_status prepare(const fos_mc_batch* b, Workspace** ws, long long n_run) {
    fos_status st = get_workspace(ws);
    if (st != FOS_OK) return st;
    if ((*ws)->cc_major != 10) return FOS_ERR_UNSUPPORTED;
    return ensure_buffer(*ws, &(*ws)->mc_tables, &(*ws)->mc_bytes,
                         tables_bytes(n_run, b->max_layers));
}

}  // namespace mc
}  // namespace fos

using namespace fos;

extern "C" {

fos_status fos_mc_spectrum(const fos_mc_batch* batch, long long* counts, int* photon_log,
                           long long log_stride, unsigned flags, void* stream) {
    NvtxRange nvtx("fos_mc_spectrum");
    long long n_run = 0;
    fos_status st = mc::validate_host(batch, counts, photon_log, log_stride, &n_run);
    if (st != FOS_OK) return st;
    if (n_run == 0) return FOS_OK;
    Workspace* ws = nullptr;
    st = mc::prepare(batch, &ws, n_run);
    if (st != FOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool fast = (flags & FOS_FAST_WALK) != 0;
    mc::Tuning tu = mc::pick_tuning(batch, ws->device, fast);
    if (flags & FOS_AUTOTUNE) {
        st = mc::autotune(ws, batch, n_run, fast, s, &tu);
        if (st != FOS_OK) return st;
        std::lock_guard<std::mutex> lock(mc::g_state.mu);
        if (mc::g_state.has_override) tu = mc::g_state.override_t;
    }
    st = mc::launch(ws, batch, n_run, counts, photon_log, log_stride, tu, flags, s);
    if (st != FOS_OK) return st;
    return finish_call(ws, s, flags);
}

fos_status fos_mc_set_tuning(int block, int ppt) {
    std::lock_guard<std::mutex> lock(mc::g_state.mu);
    if (block == 0 && ppt == 0) {
        mc::g_state.has_override = false;
        return FOS_OK;
    }
    if (block < 32 || block > mc::WALK_MAX_BLOCK || (block % 32) != 0 || ppt < 1 || ppt > 1024)
        return FOS_ERR_INVALID_ARG;
    mc::g_state.override_t.block = block;
    mc::g_state.override_t.ppt = ppt;
    mc::g_state.has_override = true;
    return FOS_OK;
}

fos_status fos_mc_get_tuning(const fos_mc_batch* batch, unsigned flags, int* block, int* ppt) {
    if (!batch || !block || !ppt) return FOS_ERR_INVALID_ARG;
    int dev = 0;
    FOS_CUDA_TRY(cudaGetDevice(&dev));
    mc::Tuning tu = mc::pick_tuning(batch, dev, (flags & FOS_FAST_WALK) != 0);
    *block = tu.block;
    *ppt = tu.ppt;
    return FOS_OK;
}

fos_status fos_mc_autotune(const fos_mc_batch* batch, unsigned flags, void* stream, int* block,
                           int* ppt) {
    long long n_run = 0;
    long long dummy = 0;
    fos_status st = mc::validate_host(batch, &dummy, nullptr, 0, &n_run);
    if (st != FOS_OK) return st;
    if (n_run == 0) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    st = mc::prepare(batch, &ws, n_run);
    if (st != FOS_OK) return st;
    mc::Tuning tu;
    st = mc::autotune(ws, batch, n_run, (flags & FOS_FAST_WALK) != 0, (cudaStream_t)stream, &tu);
    if (st != FOS_OK) return st;
    if (block) *block = tu.block;
    if (ppt) *ppt = tu.ppt;
    return FOS_OK;
}

fos_status fos_mc_walk_times(long long* start_end_ns, int capacity, int* n_blocks) {
    if (!n_blocks || capacity < 0 || (capacity > 0 && !start_end_ns)) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    int n = 0;
    {
        std::lock_guard<std::mutex> lock(mc::g_state.mu);
        n = mc::g_state.times_blocks[ws->device];
    }
    *n_blocks = n;
    if (n == 0 || !ws->walk_times || !start_end_ns) return FOS_OK;   // size query
    if (capacity < n) return FOS_ERR_INVALID_ARG;
    FOS_CUDA_TRY(cudaMemcpy(start_end_ns, ws->walk_times, (size_t)n * 2 * sizeof(long long),
                            cudaMemcpyDeviceToHost));
    return FOS_OK;
}

fos_status fos_philox4x32_10(const unsigned* ctr, unsigned k0, unsigned k1, unsigned* out,
                             long long n, void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return FOS_ERR_INVALID_ARG;
    if (n == 0) return FOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    mc::philox_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>((const uint4*)ctr, k0, k1,
                                                            (uint4*)out, n);
    FOS_CUDA_TRY(cudaGetLastError());
    return from_cuda(cudaStreamSynchronize(s));
}

fos_status fos_philox4x32_10_curand(const unsigned* ctr, unsigned k0, unsigned k1,
                                    unsigned* out, long long n, void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return FOS_ERR_INVALID_ARG;
    if (n == 0) return FOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    mc::philox_curand_kernel<<<(unsigned)blocks, 256, 0, s>>>((const uint4*)ctr, k0, k1,
                                                              (uint4*)out, n);
    FOS_CUDA_TRY(cudaGetLastError());
    return from_cuda(cudaStreamSynchronize(s));
}

fos_status fos_walk_math_f32(const float* u, float* neg_log, float* cos2pi, long long n,
                             void* stream) {
    if (n < 0 || (n > 0 && !u)) return FOS_ERR_INVALID_ARG;
    if (n == 0) return FOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    mc::walk_math_kernel<<<(unsigned)blocks, 256, 0, s>>>(u, neg_log, cos2pi, n);
    FOS_CUDA_TRY(cudaGetLastError());
    return from_cuda(cudaStreamSynchronize(s));
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// fos_mc_spectrum_noalloc: the photon walk without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is wholly
// reserved by another allocator (a framework's caching pool that took the GPU), or a
// host under a fixed memory budget where an allocation could fail or stall at the
// wrong moment.  This entry point runs the same kernels as fos_mc_spectrum, but its
// scratch (work-queue counter, status words, packed item tables and unit prefix) lives
// in the file-scope array below.  Host code only sees a stand-in for that array, so the
// device address is looked up with cudaGetSymbolAddress on each device's first call.
//
// CUDA loads modules and kernels lazily (on first use) by default, and loading one
// takes device memory: the array itself and the kernels' code.  So the first call on a
// device sets everything up at once: it looks up the array (which loads this module)
// and loads every kernel the entry point launches (cudaFuncGetAttributes).  Later calls
// need nothing more.  A call with an empty batch does only this set-up.
// ---------------------------------------------------------------------------------
namespace fos {
namespace mc {

constexpr long long NOALLOC_ROWS = FOS_NOALLOC_MAX_ITEMS;
constexpr size_t NOALLOC_HDR = 512;   // status words at 0, work-queue counter at 256
constexpr size_t NOALLOC_BYTES =
    NOALLOC_HDR + (size_t)NOALLOC_ROWS * sizeof(int4) * 2 +
    (size_t)NOALLOC_ROWS * sizeof(float4) +
    (size_t)NOALLOC_ROWS * FOS_MAX_LAYERS * sizeof(float4) * 3 +
    (size_t)(NOALLOC_ROWS + 1) * sizeof(long long) + 8 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];             // device address of g_noalloc_scratch per device
static cudaStream_t g_noalloc_pending[64];  // stream of a call whose wait ran out
static bool g_noalloc_has_pending[64];

// Per-device set-up, with the device current (caller holds g_noalloc_mu).
static fos_status noalloc_setup(int dev) {
    if (g_noalloc_ptr[dev]) return FOS_OK;
    void* p = nullptr;
    FOS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    cudaFuncAttributes fa;
    FOS_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)pack_kernel));
    FOS_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)unit_scan_kernel));
    for (int bl : WALK_BLOCKS) FOS_CUDA_TRY(cudaFuncGetAttributes(&fa, walk_kernel_exact(bl)));
    g_noalloc_ptr[dev] = p;
    return FOS_OK;
}

}  // namespace mc
}  // namespace fos

extern "C" fos_status fos_mc_spectrum_noalloc(const fos_mc_batch* batch, long long* counts,
                                              unsigned flags, void* stream) {
    if (flags & ~(unsigned)FOS_TEST_INJECT) return FOS_ERR_INVALID_ARG;
    long long n_run = 0;
    fos_status st = mc::validate_host(batch, counts, nullptr, 0, &n_run);
    if (st != FOS_OK) return st;
    if (n_run > mc::NOALLOC_ROWS) return FOS_ERR_OUT_OF_RANGE;
    int dev = 0;
    FOS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FOS_ERR_UNSUPPORTED;
    int major = 0, sms = 0;
    FOS_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    FOS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (major != 10) return FOS_ERR_UNSUPPORTED;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(mc::g_noalloc_mu);
        st = mc::noalloc_setup(dev);
        if (st != FOS_OK) return st;
        // A call whose bounded wait ran out may still be running on the array: refuse
        // until its stream has drained.
        if (mc::g_noalloc_has_pending[dev]) {
            const cudaError_t q = cudaStreamQuery(mc::g_noalloc_pending[dev]);
            if (q == cudaErrorNotReady) return FOS_ERR_TIMEOUT;
            mc::g_noalloc_has_pending[dev] = false;
            if (q != cudaSuccess) return from_cuda(q);
        }
        base = mc::g_noalloc_ptr[dev];
    }
    if (n_run == 0) return FOS_OK;
    Workspace w;   // views into the static array; nothing is allocated
    w.device = dev;
    w.num_sms = sms;
    w.cc_major = major;
    w.status = (unsigned*)base;
    w.cursor = (unsigned long long*)((char*)base + 256);
    w.mc_tables = (char*)base + mc::NOALLOC_HDR;
    w.mc_bytes = mc::NOALLOC_BYTES - mc::NOALLOC_HDR;
    cudaStream_t s = (cudaStream_t)stream;
    mc::Tuning tu = mc::pick_tuning(batch, dev, false);
    const int inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
    st = mc::enqueue(&w, batch, n_run, counts, nullptr, 0, tu, mc::SCALE_ALL, inject, false,
                     nullptr, s);
    if (st != FOS_OK) return st;
    st = wait_stream(s, default_timeout_ms());
    if (st == FOS_ERR_TIMEOUT) {
        std::lock_guard<std::mutex> lock(mc::g_noalloc_mu);
        mc::g_noalloc_pending[dev] = s;
        mc::g_noalloc_has_pending[dev] = true;
    }
    if (st != FOS_OK) return st;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&bits, w.status + ST_CALL, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return status_from_bits(bits);
}
