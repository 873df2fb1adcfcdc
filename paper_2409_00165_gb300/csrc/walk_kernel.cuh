// The photon-walk kernel (arxiv 2409.00165, section "Photon transport"), shared by two
// translation units that compile it with different arithmetic:
//
//   mc_walk.cu       the exact walk (FAST = false), built with -fmad=false: IEEE FP32
//                    in a fixed operation order, with self-contained series for -ln u
//                    and cos 2 pi u, bit-identical with the oracle's FP32 mirror;
//   mc_walk_fast.cu  the fast walk (FAST = true), built with FMA contraction: -ln u from
//                    the SFU's base-2 logarithm (lg2.approx), cos 2 pi u from its cosine
//                    (cos.approx), approximate reciprocal and square root on the
//                    collision path.  Same random numbers and decisions; the results
//                    agree with the exact walk and the definition statistically only.
//
// One photon per thread, persistent grid, warp-level work units:
//   * a warp claims a unit of 32*ppt photons of one item from a global atomic
//     counter over the units of all items (prefix sums built on the device), and
//     hands photons to its lanes as they become free, so a lane whose photon ends
//     starts the next one at once (live photons stay packed in full warps: the
//     warp-level compaction of live photons);
//   * each lane walks its photon event by event (collision or boundary arrival);
//   * counts accumulate in registers per lane, tagged by item, and are reduced
//     across the warp (shuffles/REDUX) before one int64 atomicAdd per counter.  There
//     is no shared-memory stage between the warp reduction and the global atomics
//     (a deviation from a warp -> shared memory -> global reduction): a block-wide
//     table cannot hold the items of a large batch, and one atomic per counter per
//     32*ppt photons is already far below the atomic units' rate.
//
// Everything with linkage here is either a plain struct (identical in both units) or
// in an anonymous namespace, so that each unit keeps its own differently-compiled copy.
#pragma once

#include "fos_internal.h"

namespace fos {
namespace mc {

// Round keys of Philox4x32-10, computed on the host: the key is the seed, identical for
// every photon, and round r uses key + r * (Weyl increment).
struct RoundKeys {
    unsigned k0[10], k1[10];
};

// Packed per-row tables (row = position in the run list).
struct Tables {
    int4* head;       // {n_layers, n_above bits, n_below bits, substrate R bits: >= 0
                      //  reflector, -1 none, -2 conductor}
    int4* info;       // {rng item id, first photon id, photon count, entry reflectance bits}
    float4* edge;     // {entry mu_z (refraction cosine), cos incidence, k below, 0}
    float4* layA;     // [row*max_layers + j] {mu_t, absorption threshold (uint bits), g, n}
    float4* layB;     // [row*max_layers + j] {d, 1-g^2, 1+g^2, 1-g}
    float4* layC;     // [row*max_layers + j] {1/mu_t, 1/(2g), n_j / n above, n_j / n below}
                      //  (the index ratios of the layer's top and bottom faces, the same
                      //  IEEE quotients the Fresnel step would form)
    long long* prefix;  // [n_run + 1] exclusive prefix of work units
};

struct WalkArgs {
    Tables t;
    int n_run, max_layers;
    unsigned unit;                // photons per warp work unit
    unsigned long long scale;     // photons run of a row: ceil(count * scale / 2^32)
                                  // (2^32: all; the autotuner runs a scaled copy)
    RoundKeys rk;
    unsigned max_events;
    unsigned long long* cursor;
    unsigned long long* counts;
    int* photon_log;
    long long log_stride;
    unsigned* status;
    unsigned long long* cta_times;  // optional [2 * grid]: start, end (ns) of each block
    int events_per_refill;          // events per live photon between the warp's refill votes
};

// Photons of a row run by this launch (the scaled count used by the autotuner's probe).
__host__ __device__ __forceinline__ unsigned scaled_count(unsigned n, unsigned long long scale) {
    return (unsigned)(((unsigned long long)n * scale + 0xffffffffull) >> 32);
}

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Checked build (FOS_CHECKED, `build(checked=True)`): every table index the walk forms is
// tested; a bad one sets DEV_RANGE with the check's code (0xF0000000 | code) in the
// status word's index field, and the access is skipped.  No trap, no assert.  The
// default build compiles the checks out.
__device__ __noinline__ void walk_bad(unsigned* status, unsigned code) {
    atomicOr(&status[ST_CALL], DEV_RANGE);
    atomicMin(&status[ST_INDEX], 0xF0000000u | code);
}
#ifdef FOS_CHECKED
#define FOS_WALK_OK(cond, code) ((cond) ? true : (walk_bad(A.status, (code)), false))
#else
#define FOS_WALK_OK(cond, code) true
#endif

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

// The fast walk's transcendentals, on the SFU (PTX approximate instructions):
// -ln u = -log2(u) ln 2; cos(2 pi u) = -cos(2 pi (u - 1/2)), whose argument lies in
// (-pi, pi), the range of cos.approx's stated accuracy.
__device__ __forceinline__ float neg_log_u_sfu(float u) {
    float l2;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(u));
    return l2 * -0x1.62e430p-1f;
}
__device__ __forceinline__ float cos_2pi_u_sfu(float u) {
    float c;
    const float x = (u - 0.5f) * 0x1.921fb6p+2f;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
    return -c;
}
__device__ __forceinline__ float sqrt_sfu(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <bool FAST>
__device__ __forceinline__ float walk_neg_log(float u) {
    if constexpr (FAST) return neg_log_u_sfu(u);
    else return neg_log_u(u);
}
template <bool FAST>
__device__ __forceinline__ float walk_cos_2pi(float u) {
    if constexpr (FAST) return cos_2pi_u_sfu(u);
    else return cos_2pi_u(u);
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

// The same at a layer face whose quotient ratio = ni / nt is precomputed (the walk's
// boundary events); FAST: approximate square root and divisions.
template <bool FAST>
__device__ __forceinline__ float fresnel_face(float ni, float nt, float ratio, float ci,
                                              float& ct, bool& tir) {
    const float r2 = ratio * ratio;
    const float st2 = r2 * fmaf(-ci, ci, 1.0f);
    if (st2 >= 1.0f) {
        tir = true;
        ct = 0.0f;
        return 1.0f;
    }
    tir = false;
    ct = FAST ? sqrt_sfu(1.0f - st2) : sqrtf(1.0f - st2);
    const float a = ni * ci, b = nt * ct;
    const float rs = FAST ? __fdividef(a - b, a + b) : (a - b) / (a + b);
    const float c = ni * ct, d = nt * ci;
    const float rp = FAST ? __fdividef(c - d, c + d) : (c - d) / (c + d);
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
template <bool FAST>
__device__ __forceinline__ float hg_cos(float g, float omg2, float opg2, float omg,
                                        float inv2g, float u) {
    float cost;
    if (fabsf(g) < 0x1.0c6f7ap-20f) {   // |g| < 1e-6: isotropic
        cost = (u + u) - 1.0f;
    } else {
        const float two_g = g + g;
        const float den = fmaf(two_g, u, omg);
        const float t = FAST ? __fdividef(omg2, den) : omg2 / den;
        const float num = fmaf(-t, t, opg2);
        cost = num * inv2g;
    }
    cost = fminf(fmaxf(cost, -1.0f), 1.0f);
    return cost;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sums the tallies of the lanes in `want` per tag and adds them with one atomic per
// counter and tag.  Must be called by all 32 lanes together.
__device__ __forceinline__ void warp_flush(bool want, int tag, unsigned c0, unsigned c1,
                                           unsigned c2, unsigned c3,
                                           unsigned long long c4, unsigned long long c5,
                                           unsigned long long* counts, unsigned* status,
                                           int n_run) {
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
#ifdef FOS_CHECKED
        if (lane == leader && (t < 0 || t >= n_run)) walk_bad(status, 6);
        if (lane == leader && t >= 0 && t < n_run) {
#else
        (void)n_run;
        if (lane == leader) {
#endif
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

// Events per live photon between the warp's refill votes (WalkArgs::events_per_refill):
// the default, and the other values the autotuner tries.  Measured on the benchmark legs
// (photon-steps/s against 4 events): 8 gives +2.4 % on the 400-wavelength paint layer
// (228 collisions per photon), +2.4 % on the 64-design stack batch, +2.5 % on the
// core-shell media, but -7 % on the dilute size-distribution layer (9 collisions per
// photon), where finished lanes wait longer; 16 gives +3.6 % on the paint layer and -22 %
// on the dilute layer.  A vote counting the free lanes after every event or every few
// events measured no faster than 4 on the paint layer.
constexpr int WALK_EVENTS_PER_REFILL = 8;
constexpr int WALK_EVENTS_PER_REFILL_ALT[] = {4, 16};

// The walk.  BLOCK threads per block and MINB resident blocks per SM bound the
// registers (28 resident warps at 64-128 threads: 72 registers, which hide the latency
// of the dependent Philox and float chains better than 24 warps at 80 registers).
template <bool FAST, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) walk_kernel(WalkArgs A) {
    if (A.status[ST_CALL] & (DEV_INVALID | DEV_INJECTED | DEV_RANGE)) return;
    if (A.cta_times && threadIdx.x == 0) A.cta_times[2 * blockIdx.x] = global_ns();
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
        if (!FOS_WALK_OK(jj >= 0 && jj < nl && nl <= A.max_layers && row >= 0 && row < A.n_run, 4))
            return;
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
        if (A.photon_log && FOS_WALK_OK((long long)(p - p_first) < A.log_stride, 5)) {
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
                if ((long long)uidx >= total_units || !FOS_WALK_OK(r >= 0 && r < A.n_run, 1)) {
                    exhausted = true;
                    break;
                }
                const unsigned q = (unsigned)(uidx - (unsigned long long)A.t.prefix[r]);
                const unsigned n_eff = scaled_count((unsigned)A.t.info[r].z, A.scale);
                if (!FOS_WALK_OK((unsigned long long)q * A.unit < (unsigned long long)n_eff, 2)) {
                    exhausted = true;
                    break;
                }
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
            warp_flush(switching, tag, cR, cA, cT, cX, cC, cI, A.counts, A.status, A.n_run);
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
                    tau = walk_neg_log<FAST>(uni(blk0.x));
                    w1 = blk0.y;
                    u2 = uni(blk0.z);
                    u3 = uni(blk0.w);
                    alive = true;
                }
            }
            u_next += __popc(taken);
        }
        if (!__any_sync(FULL, alive)) break;   // refill ended: queue exhausted

        // ---------------- events_per_refill events per live photon between refills (a lane
        // whose photon ends early waits for the next refill: cheaper than the refill vote
        // on every event)
#pragma unroll 1
        for (int rep = 0; rep < A.events_per_refill; ++rep)
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
                const float cost = hg_cos<FAST>(l_g, l_omg2, l_opg2, l_omg, l_i2g, u2);
                if (am > 0x1.fffeb0p-1f) {
                    mu = (mu > 0.0f) ? cost : -cost;
                } else {
                    const float q2 = fmaf(-mu, mu, 1.0f) * fmaf(-cost, cost, 1.0f);
                    const float q = FAST ? sqrt_sfu(q2) : sqrtf(q2);
                    const float cp = walk_cos_2pi<FAST>(u3);
                    mu = fmaf(q, cp, mu * cost);
                    mu = fminf(fmaxf(mu, -1.0f), 1.0f);
                }
                e++;
                tau = walk_neg_log<FAST>(uni(blk.x));
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
                    const float2 rat = *reinterpret_cast<const float2*>(
                        &A.t.layC[(long long)row * A.max_layers + j].z);
                    const float Rf = fresnel_face<FAST>(ni, nt, down ? rat.y : rat.x, fabsf(mu),
                                                        ct, tir);
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
    warp_flush(have, tag, cR, cA, cT, cX, cC, cI, A.counts, A.status, A.n_run);
    if (A.cta_times) {
        __syncthreads();
        if (threadIdx.x == 0) A.cta_times[2 * blockIdx.x + 1] = global_ns();
    }
}

// Kernel of the block-size variant that runs `block` threads (the smallest compiled
// BLOCK >= block; each variant may also be launched with fewer threads).
template <bool FAST>
const void* walk_kernel_for(int block) {
    if (block <= 64) return (const void*)walk_kernel<FAST, 64, 14>;
    if (block <= 96) return (const void*)walk_kernel<FAST, 96, 9>;
    if (block <= 128) return (const void*)walk_kernel<FAST, 128, 7>;
    return (const void*)walk_kernel<FAST, 256, 3>;
}

}  // namespace

// Block sizes the walk is compiled for (fos_mc_set_tuning accepts multiples of 32 up
// to the largest; the autotuner searches these).
constexpr int WALK_BLOCKS[] = {64, 96, 128, 256};
constexpr int WALK_MAX_BLOCK = 256;

// Defined by each translation unit that compiles the walk.
const void* walk_kernel_exact(int block);
const void* walk_kernel_fast(int block);

}  // namespace mc
}  // namespace fos
