// Monte Carlo photon transport on GB300 (arxiv 2409.00165, section "Photon transport").
//
// One photon per thread, persistent grid, warp-level work units:
//   * a warp claims a unit of 32*ppt photons of one item from a global atomic
//     counter over the units of all items (prefix sums built on the device), and
//     hands photons to its lanes as they become free, so a lane whose photon ends
//     starts the next one at once (live photons stay packed in full warps);
//   * each lane walks its photon event by event (collision or boundary arrival);
//   * counts accumulate in registers per lane, tagged by item, and are reduced
//     across the warp (shuffles/REDUX) before one int64 atomicAdd per counter.
//
// Arithmetic: IEEE FP32, compiled with -fmad=false so that a*b+c is never fused;
// fused multiply-adds appear only where fmaf is written.  The natural log and
// cos(2 pi u) are self-contained series (see neg_log_u / cos_2pi_u) so that the walk
// is a fixed sequence of IEEE operations: the same operation order on any machine
// gives the same photons bit for bit.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "fos_internal.h"

namespace fos {
namespace mc {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
// products; high halves XOR the other counter words and the key; the key advances by
// the Weyl increments before each round after the first.
// ---------------------------------------------------------------------------------
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

// The same generator with the 10 round keys computed on the host (the key is the
// seed, identical for every photon): key words of round r are k + r * Weyl increment.
struct RoundKeys {
    unsigned k0[10], k1[10];
};
__device__ __forceinline__ uint4 philox_rk(uint4 c, const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
    }
    return c;
}

// Top 23 bits k of a word -> (2k+1) 2^-24, exactly representable, in (0,1): the float
// 1 + k 2^-23 (k as mantissa) minus (1 - 2^-24), an exact subtraction.
__device__ __forceinline__ float uni(unsigned x) {
    return __uint_as_float((x >> 9) | 0x3f800000u) - 0x1.fffffep-1f;
}

__device__ __forceinline__ unsigned word(uint4 b, unsigned i) {
    return i == 0 ? b.x : (i == 1 ? b.y : (i == 2 ? b.z : b.w));
}

// -ln(u), u in (0,1): u = m 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s),
// s = (m-1)/(m+1), atanh by its Taylor series to s^9; e ln 2 with ln 2 split into an
// exactly-multipliable head (0x1.62e4p-1) and a tail.
__device__ __forceinline__ float neg_log_u(float u) {
    const unsigned bits = __float_as_uint(u);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float f = m - 1.0f;
    const float s = f / (2.0f + f);
    const float z = s * s;
    float p = fmaf(z, 0x1.c71c72p-4f, 0x1.24924ap-3f);   // 1/9, 1/7
    p = fmaf(z, p, 0x1.99999ap-3f);                       // 1/5
    p = fmaf(z, p, 0x1.555556p-2f);                       // 1/3
    p = p * z;
    const float two_s = s + s;
    const float lnm = fmaf(two_s, p, two_s);
    const float ef = (float)e;
    const float r = fmaf(ef, 0x1.62e4p-1f, fmaf(ef, 0x1.7f7d1cp-20f, lnm));
    return -r;
}

// cos(2 pi u), u in (0,1): exact reductions u -> min(u, 1-u) -> [0,1/4] (sign flip
// past 1/4) -> b in [0, 1/8] (the complement past 1/8 turns cos into sin); then one
// Horner chain in w = x^2, x = 2 pi b, with per-branch Taylor coefficients:
// cos x = 1 + w P_c(w), sin x = x + (x w) P_s(w).  No divergent branch.
__device__ __forceinline__ float cos_2pi_u(float u) {
    float a = (u > 0.5f) ? (1.0f - u) : u;
    float sign = 1.0f;
    if (a > 0.25f) {
        a = 0.5f - a;
        sign = -1.0f;
    }
    const bool use_sin = a > 0.125f;
    const float b = use_sin ? (0.25f - a) : a;
    const float x = b * 0x1.921fb6p+2f;
    const float w = x * x;
    const float k4 = use_sin ? 0.0f : -0x1.27e4fcp-22f;            // 0 | -1/10!
    const float k3 = use_sin ? 0x1.71de3ap-19f : 0x1.a01a02p-16f;   // 1/9! | 1/8!
    const float k2 = use_sin ? -0x1.a01a02p-13f : -0x1.6c16c2p-10f; // -1/7! | -1/6!
    const float k1 = use_sin ? 0x1.111112p-7f : 0x1.555556p-5f;     // 1/5! | 1/4!
    const float k0 = use_sin ? -0x1.555556p-3f : -0.5f;             // -1/3! | -1/2!
    float p = fmaf(w, k4, k3);
    p = fmaf(w, p, k2);
    p = fmaf(w, p, k1);
    p = fmaf(w, p, k0);
    const float m = use_sin ? x * w : w;
    const float base = use_sin ? x : 1.0f;
    return sign * fmaf(m, p, base);
}

// Unpolarised Fresnel reflectance (mean of s and p) from index ni into nt at
// incidence cosine ci.  tir = total internal reflection; ct = refraction cosine.
__device__ __forceinline__ float fresnel(float ni, float nt, float ci, float& ct, bool& tir) {
    const float ratio = ni / nt;
    const float r2 = ratio * ratio;
    const float st2 = r2 * fmaf(-ci, ci, 1.0f);
    if (st2 >= 1.0f) {
        tir = true;
        ct = 0.0f;
        return 1.0f;
    }
    tir = false;
    ct = sqrtf(1.0f - st2);
    const float a = ni * ci, b = nt * ct;
    const float rs = (a - b) / (a + b);
    const float c = ni * ct, d = nt * ci;
    const float rp = (c - d) / (c + d);
    return (rs * rs + rp * rp) * 0.5f;
}

// Unpolarised Fresnel reflectance from real index ni into a conductor n2 + i k2 (k2 > 0)
// at incidence cosine ci.  w = (n2 + i k2)^2 - ni^2 (1 - ci^2), u + i v = sqrt(w) with
// Re >= 0 (the larger of u, v from the modulus, the other by division, so that neither
// cancels); r_s = (ni ci - sqrt w)/(ni ci + sqrt w), r_p = ((n2+ik2)^2 ci - ni sqrt w) /
// ((n2+ik2)^2 ci + ni sqrt w).
__device__ __noinline__ float fresnel_conductor(float ni, float n2, float k2, float ci) {
    const float s2 = fmaf(-ci, ci, 1.0f);
    const float e_re = n2 * n2 - k2 * k2;
    const float e_im = (n2 + n2) * k2;
    const float w_re = e_re - (ni * ni) * s2;
    const float w_im = e_im;
    const float mod = sqrtf(w_re * w_re + w_im * w_im);
    float u, v;
    if (w_re >= 0.0f) {
        u = sqrtf((mod + w_re) * 0.5f);
        v = w_im / (u + u);
    } else {
        v = sqrtf((mod - w_re) * 0.5f);
        u = w_im / (v + v);
    }
    const float a = ni * ci;
    const float rs_n = (a - u) * (a - u) + v * v;
    const float rs_d = (a + u) * (a + u) + v * v;
    const float c1 = e_re * ci, c2 = e_im * ci, q1 = ni * u, q2 = ni * v;
    const float rp_n = (c1 - q1) * (c1 - q1) + (c2 - q2) * (c2 - q2);
    const float rp_d = (c1 + q1) * (c1 + q1) + (c2 + q2) * (c2 + q2);
    return (rs_n / rs_d + rp_n / rp_d) * 0.5f;
}

// Henyey-Greenstein deflection cosine by inversion of its distribution function.
// {1-g^2, 1+g^2, 1-g, 1/(2g)} are precomputed per layer by pack_kernel.
__device__ __forceinline__ float hg_cos(float g, float omg2, float opg2, float omg,
                                        float inv2g, float u) {
    float cost;
    if (fabsf(g) < 0x1.0c6f7ap-20f) {   // |g| < 1e-6: isotropic
        cost = (u + u) - 1.0f;
    } else {
        const float two_g = g + g;
        const float den = fmaf(two_g, u, omg);
        const float t = omg2 / den;
        const float num = fmaf(-t, t, opg2);
        cost = num * inv2g;
    }
    cost = fminf(fmaxf(cost, -1.0f), 1.0f);
    return cost;
}

// ---------------------------------------------------------------------------------
// Packed per-row tables (row = position in the run list).
// ---------------------------------------------------------------------------------
struct Tables {
    int4* head;       // {n_layers, n_above bits, n_below bits, substrate R bits: >= 0
                      //  reflector, -1 none, -2 conductor}
    int4* info;       // {rng item id, first photon id, photon count, entry reflectance bits}
    float4* edge;     // {entry mu_z (refraction cosine), cos incidence, k below, 0}
    float4* layA;     // [row*max_layers + j] {mu_t, absorption threshold (uint bits), g, n}
    float4* layB;     // [row*max_layers + j] {d, 1-g^2, 1+g^2, 1-g}
    float4* layC;     // [row*max_layers + j] {1/mu_t, 1/(2g), 0, 0}
    long long* prefix;  // [n_run + 1] exclusive prefix of work units
};

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
    if (N < 0 || first < 0 || first + N > 4294967296LL) ok = false;
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
__global__ void unit_scan_kernel(const int4* info, int n_run, unsigned unit, unsigned cap,
                                 long long* prefix) {
    __shared__ long long sums[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (n_run + T - 1) / T;
    const int lo = min(n_run, t * per), hi = min(n_run, lo + per);
    long long acc = 0;
    for (int r = lo; r < hi; ++r) {
        const unsigned long long n = min((unsigned)info[r].z, cap);
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
        const unsigned long long n = min((unsigned)info[r].z, cap);
        run += (long long)((n + unit - 1) / unit);
    }
    if (t == T - 1) prefix[n_run] = sums[T - 1];
}

struct WalkArgs {
    Tables t;
    int n_run, max_layers;
    unsigned unit;        // photons per warp work unit
    unsigned cap;         // photon cap per row (autotuner), 0xffffffff otherwise
    RoundKeys rk;
    unsigned max_events;
    unsigned long long* cursor;
    unsigned long long* counts;
    int* photon_log;
    long long log_stride;
    unsigned* status;
};

// Sums the tallies of the lanes in `want` per tag and adds them with one atomic per
// counter and tag.  Must be called by all 32 lanes together.
__device__ __forceinline__ void warp_flush(bool want, int tag, unsigned c0, unsigned c1,
                                           unsigned c2, unsigned c3,
                                           unsigned long long c4, unsigned long long c5,
                                           unsigned long long* counts, unsigned* status) {
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(FULL, want);
    while (m) {
        const int leader = __ffs(m) - 1;
        const int t = __shfl_sync(FULL, tag, leader);
        const bool in = want && tag == t;
        const unsigned grp = __ballot_sync(FULL, in);
        const unsigned s0 = __reduce_add_sync(FULL, in ? c0 : 0u);
        const unsigned s1 = __reduce_add_sync(FULL, in ? c1 : 0u);
        const unsigned s2 = __reduce_add_sync(FULL, in ? c2 : 0u);
        const unsigned s3 = __reduce_add_sync(FULL, in ? c3 : 0u);
        unsigned long long s4 = in ? c4 : 0ull, s5 = in ? c5 : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s4 += __shfl_xor_sync(FULL, s4, off);
            s5 += __shfl_xor_sync(FULL, s5, off);
        }
        if (lane == leader) {
            unsigned long long* c = counts + (long long)t * FOS_NCOUNT;
            if (s0) atomicAdd(c + 0, (unsigned long long)s0);
            if (s1) atomicAdd(c + 1, (unsigned long long)s1);
            if (s2) atomicAdd(c + 2, (unsigned long long)s2);
            if (s3) {
                atomicAdd(c + 3, (unsigned long long)s3);
                atomicOr(&status[ST_CALL], DEV_STEP_LIMIT);
            }
            if (s4) atomicAdd(c + 4, s4);
            if (s5) atomicAdd(c + 5, s5);
        }
        m &= ~grp;
        want = want && !in;
    }
}

enum { O_R = 0, O_A = 1, O_T = 2, O_X = 3 };
constexpr int WALK_MAX_BLOCK = 128;

// 128-thread blocks, 7 per SM: the register budget (72 per thread) that gives 28
// resident warps, which hide the latency of the dependent Philox and float chains better
// than 24 warps at 80 registers.
__global__ void __launch_bounds__(WALK_MAX_BLOCK, 7) walk_kernel(WalkArgs A) {
    if (A.status[ST_CALL] & (DEV_INVALID | DEV_INJECTED | DEV_RANGE)) return;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long total_units = A.t.prefix[A.n_run];

    // warp work unit (uniform across the warp)
    int u_row = 0;
    unsigned u_next = 0, u_end = 0;
    bool exhausted = false;

    // photon state
    bool alive = false;
    int row = 0, j = 0, nl = 1;
    unsigned item_rng = 0, p = 0, p_first = 0, e = 0, kif = 0, ev = 0;
    float z = 0.f, mu = 1.f, tau = 0.f, u2 = 0.f, u3 = 0.f;
    unsigned w1 = 0u;   // the absorption draw's Philox word
    unsigned l_kabs = 0u;
    float l_mut = 0.f, l_g = 0.f, l_n = 1.f, l_d = 1.f, l_omg2 = 1.f,
          l_opg2 = 1.f, l_omg = 1.f, l_imt = 0.f, l_i2g = 0.f;

    // tallies of the current tag (row)
    int tag = -1;
    unsigned cR = 0, cA = 0, cT = 0, cX = 0;
    unsigned long long cC = 0, cI = 0;

    auto load_layer = [&](int jj) {
        const long long li = (long long)row * A.max_layers + jj;
        const float4 a = A.t.layA[li];
        const float4 b = A.t.layB[li];
        const float2 c = *reinterpret_cast<const float2*>(&A.t.layC[li]);
        l_mut = a.x; l_kabs = __float_as_uint(a.y); l_g = a.z; l_n = a.w;
        l_d = b.x; l_omg2 = b.y; l_opg2 = b.z; l_omg = b.w;
        l_imt = c.x; l_i2g = c.y;
    };
    // The photon's collisions are its scatterings e (+ 1 if the last one absorbed it) and
    // its boundary events the rest of its ev events: tallied here, once per photon.
    auto finish = [&](int out) {
        if (out == O_R) cR++;
        else if (out == O_A) cA++;
        else if (out == O_T) cT++;
        else cX++;
        const unsigned long long coll = (unsigned long long)e + (out == O_A ? 1ull : 0ull);
        cC += coll;
        cI += (unsigned long long)ev - coll;
        if (A.photon_log) {
            unsigned long long rec = (coll << 2) | (unsigned long long)out;
            if (rec > 0x7fffffffull) rec = 0x7fffffffull;
            A.photon_log[(long long)row * A.log_stride + (p - p_first)] = (int)rec;
        }
        alive = false;
    };

    for (;;) {
        // ---------------- refill free lanes (warp-uniform control flow)
        for (;;) {
            const unsigned need = __ballot_sync(FULL, !alive);
            if (need == 0u || exhausted) break;
            if (u_next >= u_end) {
                unsigned long long uidx = 0;
                int r = 0;
                if (lane == 0) {
                    uidx = atomicAdd(A.cursor, 1ull);
                    if ((long long)uidx < total_units) {
                        int lo = 0, hi = A.n_run - 1;   // largest r with prefix[r] <= uidx
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (A.t.prefix[mid] <= (long long)uidx) lo = mid;
                            else hi = mid - 1;
                        }
                        r = lo;
                    }
                }
                uidx = __shfl_sync(FULL, uidx, 0);
                r = __shfl_sync(FULL, r, 0);
                if ((long long)uidx >= total_units) {
                    exhausted = true;
                    break;
                }
                const unsigned q = (unsigned)(uidx - (unsigned long long)A.t.prefix[r]);
                const unsigned n_eff = min((unsigned)A.t.info[r].z, A.cap);
                u_row = r;
                u_next = q * A.unit;
                u_end = (unsigned)min((unsigned long long)u_next + A.unit,
                                      (unsigned long long)n_eff);
                continue;
            }
            const unsigned avail = u_end - u_next;
            const unsigned rank = __popc(need & lt_mask);
            const bool mine = ((need >> lane) & 1u) && rank < avail;
            const unsigned taken = __ballot_sync(FULL, mine);
            const bool switching = mine && tag >= 0 && tag != u_row;
            warp_flush(switching, tag, cR, cA, cT, cX, cC, cI, A.counts, A.status);
            if (mine) {
                if (tag != u_row) {
                    tag = u_row;
                    cR = cA = cT = cX = 0u;
                    cC = cI = 0ull;
                }
                row = u_row;
                const int4 inf = A.t.info[row];
                const int4 hd = A.t.head[row];
                item_rng = (unsigned)inf.x;
                p_first = (unsigned)inf.y;
                p = p_first + u_next + rank;
                nl = hd.x;
                j = 0;
                load_layer(0);
                e = 0u;
                kif = 0u;
                ev = 0u;
                const uint4 blk0 = philox_rk(make_uint4(p, item_rng, 0u, 0u), A.rk);
                const float2 ed = *reinterpret_cast<const float2*>(&A.t.edge[row]);
                unsigned w_entry = blk0.w;   // normal incidence: azimuth word of block 0
                if (ed.y != 1.0f && __int_as_float(inf.w) > 0.0f)   // oblique
                    w_entry = philox_rk(make_uint4(p, item_rng, 0u, 2u), A.rk).x;
                if (uni(w_entry) < __int_as_float(inf.w)) {
                    finish(O_R);
                } else {
                    z = 0.0f;
                    mu = ed.x;
                    tau = neg_log_u(uni(blk0.x));
                    w1 = blk0.y;
                    u2 = uni(blk0.z);
                    u3 = uni(blk0.w);
                    alive = true;
                }
            }
            u_next += __popc(taken);
        }
        if (!__any_sync(FULL, alive)) break;   // refill ended: queue exhausted

        // ---------------- one event per live photon
        if (alive) {
            if (ev >= A.max_events) {
                finish(O_X);
                continue;
            }
            // collides first iff tau |mu| < mu_t dist (no division on this path)
            const float am = fabsf(mu);
            const float dist = (mu > 0.0f) ? (l_d - z) : z;
            const bool collide = (mu != 0.0f) ? (tau * am < l_mut * dist) : (l_mut > 0.0f);
            // one Philox block per event at a common point (no divergence around it):
            // collision -> next collision block; boundary -> interface block of draw kif
            const uint4 blk = philox_rk(make_uint4(p, item_rng, collide ? e + 1u : (kif >> 2),
                                                   collide ? 0u : 1u), A.rk);
            if (collide) {
                // collision inside the layer
                const float s = tau * l_imt;
                z = fmaf(mu, s, z);
                ev++;
                if ((w1 >> 9) < l_kabs) {   // uni(w1) < mu_a / mu_t
                    finish(O_A);
                    continue;
                }
                const float cost = hg_cos(l_g, l_omg2, l_opg2, l_omg, l_i2g, u2);
                if (am > 0x1.fffeb0p-1f) {
                    mu = (mu > 0.0f) ? cost : -cost;
                } else {
                    const float q = sqrtf(fmaf(-mu, mu, 1.0f) * fmaf(-cost, cost, 1.0f));
                    const float cp = cos_2pi_u(u3);
                    mu = fmaf(q, cp, mu * cost);
                    mu = fminf(fmaxf(mu, -1.0f), 1.0f);
                }
                e++;
                tau = neg_log_u(uni(blk.x));
                w1 = blk.y;
                u2 = uni(blk.z);
                u3 = uni(blk.w);
            } else {
                // boundary of the layer reached first; carry the rest of tau (>= 0)
                const float tb = (mu != 0.0f) ? l_mut * (dist / am) : 0.0f;
                tau = fmaxf(tau - tb, 0.0f);
                const bool down = mu > 0.0f;
                z = down ? l_d : 0.0f;
                ev++;
                const int nb = down ? j + 1 : j - 1;
                const bool outside = (nb < 0) || (nb >= nl);
                // media and substrate of the row, read at boundary events only (L1-resident)
                const int4 hd2 = A.t.head[row];
                const float n_above = __int_as_float(hd2.y), n_below = __int_as_float(hd2.z),
                            r_sub = __int_as_float(hd2.w);
                if (down && outside && r_sub != -1.0f) {
                    // opaque below: reflector (R_sub) or conductor (Fresnel with n + ik)
                    const float Rb = (r_sub >= 0.0f)
                        ? r_sub : fresnel_conductor(l_n, n_below, A.t.edge[row].z, am);
                    const float u = uni(word(blk, kif & 3u));
                    kif++;
                    if (u < Rb) mu = -mu;
                    else finish(O_T);
                    continue;
                }
                const float ni = l_n;
                const float nt = outside ? (down ? n_below : n_above)
                                         : A.t.layA[(long long)row * A.max_layers + nb].w;
                bool transmit;
                float mu_t_dir = mu;
                if (ni == nt) {
                    transmit = true;
                } else {
                    float ct;
                    bool tir;
                    const float Rf = fresnel(ni, nt, fabsf(mu), ct, tir);
                    if (tir) {
                        transmit = false;
                    } else {
                        const float u = uni(word(blk, kif & 3u));
                        kif++;
                        transmit = !(u < Rf);
                        mu_t_dir = down ? ct : -ct;
                    }
                }
                if (!transmit) {
                    mu = -mu;
                } else if (outside) {
                    finish(down ? O_T : O_R);
                } else {
                    j = nb;
                    load_layer(nb);
                    mu = mu_t_dir;
                    z = down ? 0.0f : l_d;
                }
            }
        }
    }
    const bool have = tag >= 0 && (cR | cA | cT | cX) != 0u;
    warp_flush(have, tag, cR, cA, cT, cX, cC, cI, A.counts, A.status);
}

// ---------------------------------------------------------------------------------
// Diagnostics.
// ---------------------------------------------------------------------------------
__global__ void philox_fill_kernel(const uint4* ctr, unsigned k0, unsigned k1, uint4* out,
                                   long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = philox(ctr[i], k0, k1);
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
struct Tuning {
    int block = 128;
    int ppt = 8;
};

struct GraphKey {
    fos_mc_batch b;
    long long* counts;
    int* log;
    long long log_stride;
    int block, ppt, inject, device;
    unsigned long long generation;
    cudaStream_t stream_unused;
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
};

struct ShapeKey {
    int device, n_stacks, n_wl, max_layers, n_list, per_item_array;
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
};
static State g_state;

static ShapeKey shape_of(const fos_mc_batch* b, int dev) {
    ShapeKey k;
    std::memset(&k, 0, sizeof(k));
    k.device = dev;
    k.n_stacks = b->n_stacks;
    k.n_wl = b->n_wl;
    k.max_layers = b->max_layers;
    k.n_list = b->item_list ? b->n_list : -1;
    k.per_item_array = b->n_photons != nullptr;
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
    if (!b->n_photons && b->photons_per_item < 0) return FOS_ERR_INVALID_ARG;
    if (b->max_events < 0 || b->max_events > 0xffffffffLL) return FOS_ERR_INVALID_ARG;
    if (b->item_list && b->n_list < 0) return FOS_ERR_INVALID_ARG;
    *n_run = b->item_list ? b->n_list : n_items;
    if (*n_run > 0 && !counts) return FOS_ERR_INVALID_ARG;
    if (log && log_stride <= 0) return FOS_ERR_INVALID_ARG;
    return FOS_OK;
}

static Tuning pick_tuning(const fos_mc_batch* b, int dev) {
    std::lock_guard<std::mutex> lock(g_state.mu);
    if (g_state.has_override) return g_state.override_t;
    ShapeKey k = shape_of(b, dev);
    for (auto& e : g_state.tuned)
        if (e.first == k) return e.second;
    return Tuning();
}

static int grid_for(Workspace* ws, int block) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel, block, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    return ws->num_sms * per_sm;
}

// Enqueues the whole call on `s`.
static fos_status enqueue(Workspace* ws, const fos_mc_batch* b, long long n_run,
                          long long* counts, int* log, long long log_stride, Tuning tu,
                          unsigned cap, int inject, cudaStream_t s) {
    Tables t = carve(ws->mc_tables, n_run, b->max_layers);
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_INDEX, 0xff, sizeof(unsigned), s));
    FOS_CUDA_TRY(cudaMemsetAsync(ws->cursor, 0, sizeof(unsigned long long), s));
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
    const unsigned unit = 32u * (unsigned)tu.ppt;
    unit_scan_kernel<<<1, 1024, 0, s>>>(t.info, (int)n_run, unit, cap, t.prefix);
    FOS_CUDA_TRY(cudaGetLastError());
    WalkArgs wa;
    wa.t = t;
    wa.n_run = (int)n_run;
    wa.max_layers = b->max_layers;
    wa.unit = unit;
    wa.cap = cap;
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
    walk_kernel<<<grid_for(ws, tu.block), tu.block, 0, s>>>(wa);
    FOS_CUDA_TRY(cudaGetLastError());
    return FOS_OK;
}

static fos_status launch(Workspace* ws, const fos_mc_batch* b, long long n_run,
                         long long* counts, int* log, long long log_stride, Tuning tu,
                         unsigned flags, cudaStream_t s) {
    const int inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
    if (flags & FOS_NO_GRAPH)
        return enqueue(ws, b, n_run, counts, log, log_stride, tu, 0xffffffffu, inject, s);
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.b = *b;
    key.counts = counts;
    key.log = log;
    key.log_stride = log_stride;
    key.block = tu.block;
    key.ppt = tu.ppt;
    key.inject = inject;
    key.device = ws->device;
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
        fos_status st = enqueue(ws, b, n_run, counts, log, log_stride, tu, 0xffffffffu, inject,
                                ws->side);
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

static fos_status autotune(Workspace* ws, const fos_mc_batch* b, long long n_run,
                           cudaStream_t s, Tuning* best) {
    const size_t cbytes = (size_t)n_run * FOS_NCOUNT * sizeof(long long);
    fos_status st = ensure_buffer(ws, (void**)&ws->tune_counts, &ws->tune_bytes, cbytes);
    if (st != FOS_OK) return st;
    // cap each row so that the probe runs about 2^24 photons in total: enough photons per
    // warp that the probe measures the steady state, not the tail of the last units
    long long cap = (1LL << 24) / (n_run > 0 ? n_run : 1);
    if (cap < 4096) cap = 4096;
    // Candidate shapes: the kernel's 128-thread blocks (7 resident per SM) with 4 to 32
    // photons per thread per work unit.
    const int blocks[] = {128};
    const int ppts[] = {4, 8, 16, 32};
    const bool verbose = getenv("FOS_AUTOTUNE_VERBOSE") != nullptr;
    cudaEvent_t e0, e1;
    FOS_CUDA_TRY(cudaEventCreate(&e0));
    FOS_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    Tuning bt;
    for (int bl : blocks) {
        for (int pp : ppts) {
            Tuning tu;
            tu.block = bl;
            tu.ppt = pp;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                st = enqueue(ws, b, n_run, ws->tune_counts, nullptr, 0, tu, (unsigned)cap, 0, s);
                if (st != FOS_OK) break;
                cudaEventRecord(e1, s);
                st = wait_stream(s, default_timeout_ms());
                if (st != FOS_OK) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < ms_min) ms_min = ms;
            }
            if (st != FOS_OK) break;
            if (verbose) fprintf(stderr, "fos autotune: block %d ppt %d: %.3f ms\n", bl, pp, ms_min);
            if (ms_min < best_ms) {
                best_ms = ms_min;
                bt = tu;
            }
        }
        if (st != FOS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FOS_OK) return st;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&bits, ws->status + ST_CALL, sizeof(unsigned),
                            cudaMemcpyDeviceToHost));
    if (bits & (DEV_INVALID | DEV_INJECTED | DEV_RANGE)) return status_from_bits(bits);
    *best = bt;
    std::lock_guard<std::mutex> lock(g_state.mu);
    ShapeKey k = shape_of(b, ws->device);
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
    mc::Tuning tu = mc::pick_tuning(batch, ws->device);
    if (flags & FOS_AUTOTUNE) {
        st = mc::autotune(ws, batch, n_run, s, &tu);
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

fos_status fos_mc_get_tuning(const fos_mc_batch* batch, int* block, int* ppt) {
    if (!batch || !block || !ppt) return FOS_ERR_INVALID_ARG;
    int dev = 0;
    FOS_CUDA_TRY(cudaGetDevice(&dev));
    mc::Tuning tu = mc::pick_tuning(batch, dev);
    *block = tu.block;
    *ppt = tu.ppt;
    return FOS_OK;
}

fos_status fos_mc_autotune(const fos_mc_batch* batch, void* stream, int* block, int* ppt) {
    long long n_run = 0;
    long long dummy = 0;
    fos_status st = mc::validate_host(batch, &dummy, nullptr, 0, &n_run);
    if (st != FOS_OK) return st;
    if (n_run == 0) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    st = mc::prepare(batch, &ws, n_run);
    if (st != FOS_OK) return st;
    mc::Tuning tu;
    st = mc::autotune(ws, batch, n_run, (cudaStream_t)stream, &tu);
    if (st != FOS_OK) return st;
    if (block) *block = tu.block;
    if (ppt) *ppt = tu.ppt;
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
// in the file-scope array below, which every GPU that loads the library holds until
// the process exits.  Host code only sees a stand-in for that array, so the device
// address is looked up with cudaGetSymbolAddress on each device's first call.
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
static void* g_noalloc_ptr[64];   // device address of g_noalloc_scratch per device

}  // namespace mc
}  // namespace fos

extern "C" fos_status fos_mc_spectrum_noalloc(const fos_mc_batch* batch, long long* counts,
                                              unsigned flags, void* stream) {
    if (flags & ~(unsigned)FOS_TEST_INJECT) return FOS_ERR_INVALID_ARG;
    long long n_run = 0;
    fos_status st = mc::validate_host(batch, counts, nullptr, 0, &n_run);
    if (st != FOS_OK) return st;
    if (n_run > mc::NOALLOC_ROWS) return FOS_ERR_OUT_OF_RANGE;
    if (n_run == 0) return FOS_OK;
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
        if (!mc::g_noalloc_ptr[dev]) {
            void* p = nullptr;
            FOS_CUDA_TRY(cudaGetSymbolAddress(&p, mc::g_noalloc_scratch));
            mc::g_noalloc_ptr[dev] = p;
        }
        base = mc::g_noalloc_ptr[dev];
    }
    Workspace w;   // views into the static array; nothing is allocated
    w.device = dev;
    w.num_sms = sms;
    w.cc_major = major;
    w.status = (unsigned*)base;
    w.cursor = (unsigned long long*)((char*)base + 256);
    w.mc_tables = (char*)base + mc::NOALLOC_HDR;
    w.mc_bytes = mc::NOALLOC_BYTES - mc::NOALLOC_HDR;
    cudaStream_t s = (cudaStream_t)stream;
    mc::Tuning tu = mc::pick_tuning(batch, dev);
    const int inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
    st = mc::enqueue(&w, batch, n_run, counts, nullptr, 0, tu, 0xffffffffu, inject, s);
    if (st != FOS_OK) return st;
    st = wait_stream(s, default_timeout_ms());
    if (st != FOS_OK) return st;
    unsigned bits = 0;
    FOS_CUDA_TRY(cudaMemcpy(&bits, w.status + ST_CALL, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return status_from_bits(bits);
}
