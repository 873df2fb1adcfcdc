// FOS oracle: plain, slow, single-thread CPU reference for the FOS hot path.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may load this file or the
// library built from it; only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline (and its reference arm) call it. It shares no code with the CUDA path.
//
// Contents (each function cites the passage of arxiv 2409.00165 "FOS" it follows):
//   * Philox4x32-10 counter-based generator (Salmon et al., SC'11), used to draw
//     the random numbers of the photon walk.
//   * Monte Carlo photon walk (section "Photon transport": MCML-style walk that
//     tracks only depth z and the direction cosine mu_z; step size from the
//     extinction coefficient, absorb-or-scatter from mu_a/mu_t, new direction from
//     Henyey-Greenstein with g; Fresnel reflection at boundaries with the matrix
//     index).  Three forms:
//       - definition (walk_photon_definition): the walk in plain double arithmetic
//         in the order the section describes it, with a sequential random stream
//         of its own; the statistical judge of the other two.
//       - FP32 mirror: the GPU walk's operation order and random-number layout in
//         IEEE single precision (no contraction; fma only where written) with
//         self-contained series for -ln(u) and cos(2 pi u) built from +,*,/,fma,
//         so that any other implementation of the same operation order reproduces
//         it bit for bit: the photon-for-photon judge of the GPU walk.
//       - the same order and layout in double precision with libm (walk_photon
//         with MathF64), which separates the effect of FP32 from that of the order.
//   * Mie theory for a sphere in an absorbing host (Eqs. 1-5, 10-12, 15), with the
//     Riccati-Bessel logarithmic derivative D_n evaluated per order by Lentz's
//     continued fraction for j_{n-1}/j_n, psi_n by upward recurrence below |x| and
//     from D_n above it, and xi_n by upward recurrence of its values.
//   * Effective-medium step (Eqs. 13, 14, 16), clamp of negative coefficients,
//     dependent-scattering correction (Eqs. 17-19) and matrix absorption (Eq. 20).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fno-fast-math -shared -fPIC
// (no contraction, so that the FP32 mirror performs exactly the operations written).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>

typedef std::complex<double> cd;

// --------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11).  One round: two 32x32->64 products of counter words 0 and 2
// with the multipliers, the high halves XORed with the other counter words and the
// key; the key is advanced by the Weyl constants before every round but the first.
// --------------------------------------------------------------------------------
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// A 32-bit word to a uniform in the open interval (0,1): keep the top 23 bits k
// and return (2k+1) * 2^-24.  The value has at most 24 significant bits, so it is
// exact in both float and double.
static double uniform_of(uint32_t x) {
    return (double)(((x >> 9) << 1) | 1u) * 0x1p-24;
}

// --------------------------------------------------------------------------------
// FP32 mirror: -ln(u) and cos(2 pi u) for u in (0,1) from textbook series.
//   ln m = 2 atanh(s), s = (m-1)/(m+1), after splitting u = m 2^e with m in
//   [sqrt(1/2), sqrt(2)); ln 2 is split into a short head (exact products e*hi)
//   and a tail.  cos(2 pi u) uses the symmetries of cosine to reduce u exactly to
//   [0, 1/8] (cos Taylor series) or (1/8, 1/4] (sin Taylor series of the
//   complement), both evaluated by one Horner chain.  Constants are the float
//   roundings of 1/(2j+1), 1/k!, 2 pi, ln 2.
// --------------------------------------------------------------------------------
static inline uint32_t f2u(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
static inline float u2f(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }

static float neg_log_f32(float u) {
    uint32_t bits = f2u(u);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    float m = u2f((bits & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e = e + 1; }
    float f = m - 1.0f;
    float s = f / (2.0f + f);
    float z = s * s;
    float p = std::fmaf(z, 0x1.c71c72p-4f, 0x1.24924ap-3f);
    p = std::fmaf(z, p, 0x1.99999ap-3f);
    p = std::fmaf(z, p, 0x1.555556p-2f);
    p = p * z;
    float two_s = s + s;
    float lnm = std::fmaf(two_s, p, two_s);
    float ef = (float)e;
    float r = std::fmaf(ef, 0x1.62e4p-1f, std::fmaf(ef, 0x1.7f7d1cp-20f, lnm));
    return -r;
}

// cos(2 pi u): after the exact reductions, b in [0, 1/8] and x = 2 pi b; the cosine
// branch evaluates cos x = 1 + w P_c(w) and the sine branch (complement past 1/8)
// sin x = x + (x w) P_s(w), with w = x^2 and P_c, P_s degree-4 Taylor polynomials
// (coefficients 1/k!, with the unused top sine coefficient 0) evaluated by one Horner
// chain whose coefficients are selected per branch.
static float cos2pi_f32(float u) {
    float a = (u > 0.5f) ? (1.0f - u) : u;   // cos(2 pi u) = cos(2 pi (1-u)); exact
    float sign = 1.0f;
    if (a > 0.25f) { a = 0.5f - a; sign = -1.0f; }  // cos(2 pi a) = -cos(2 pi (1/2 - a)); exact
    const bool use_sin = a > 0.125f;            // cos(2 pi a) = sin(2 pi (1/4 - a))
    const float b = use_sin ? (0.25f - a) : a;  // exact
    const float x = b * 0x1.921fb6p+2f;
    const float w = x * x;
    const float k4 = use_sin ? 0.0f : -0x1.27e4fcp-22f;           // 0 | -1/10!
    const float k3 = use_sin ? 0x1.71de3ap-19f : 0x1.a01a02p-16f;  // 1/9! | 1/8!
    const float k2 = use_sin ? -0x1.a01a02p-13f : -0x1.6c16c2p-10f;  // -1/7! | -1/6!
    const float k1 = use_sin ? 0x1.111112p-7f : 0x1.555556p-5f;    // 1/5! | 1/4!
    const float k0 = use_sin ? -0x1.555556p-3f : -0.5f;            // -1/3! | -1/2!
    float p = std::fmaf(w, k4, k3);
    p = std::fmaf(w, p, k2);
    p = std::fmaf(w, p, k1);
    p = std::fmaf(w, p, k0);
    const float m = use_sin ? x * w : w;
    const float base = use_sin ? x : 1.0f;
    return sign * std::fmaf(m, p, base);
}

// --------------------------------------------------------------------------------
// Arithmetic policies for the walk.
// --------------------------------------------------------------------------------
struct MathF64 {
    typedef double R;
    static R neg_log(R u) { return -std::log(u); }
    static R cos2pi(R u) { return std::cos(2.0 * M_PI * u); }
    static R sqrt_(R x) { return std::sqrt(x); }
    static R fma_(R a, R b, R c) { return std::fma(a, b, c); }
    static R abs_(R x) { return std::fabs(x); }
    static R uni(uint32_t x) { return uniform_of(x); }
    static R g_iso() { return 1e-6; }
    static R mu_vert() { return 1.0 - 1e-5; }
};
struct MathF32 {
    typedef float R;
    static R neg_log(R u) { return neg_log_f32(u); }
    static R cos2pi(R u) { return cos2pi_f32(u); }
    static R sqrt_(R x) { return std::sqrt(x); }
    static R fma_(R a, R b, R c) { return std::fmaf(a, b, c); }
    static R abs_(R x) { return std::fabs(x); }
    static R uni(uint32_t x) { return (float)uniform_of(x); }
    static R g_iso() { return 0x1.0c6f7ap-20f; }       // 1e-6 rounded to float
    static R mu_vert() { return 0x1.fffeb0p-1f; }      // 1 - 1e-5 rounded to float
};

// Henyey-Greenstein deflection cosine by inversion of its cumulative distribution
// (the "new direction angle" drawn from g, section "Photon transport").
template <class M>
static typename M::R hg_cos(typename M::R g, typename M::R u) {
    typedef typename M::R R;
    R cost;
    if (M::abs_(g) < M::g_iso()) {
        cost = (u + u) - (R)1;
    } else {
        R one_m_g2 = (R)1 - g * g;
        R one_p_g2 = (R)1 + g * g;
        R one_m_g = (R)1 - g;
        R two_g = g + g;
        R inv_two_g = (R)1 / two_g;
        R den = M::fma_(two_g, u, one_m_g);
        R t = one_m_g2 / den;
        R num = M::fma_(-t, t, one_p_g2);
        cost = num * inv_two_g;
    }
    if (cost < (R)-1) cost = (R)-1;
    if (cost > (R)1) cost = (R)1;
    return cost;
}

// Unpolarised Fresnel reflectance from medium ni to medium nt at incidence cosine
// ci (mean of the s and p intensity reflectances).  Returns 1 for total internal
// reflection and writes the refraction cosine to *ct otherwise.
template <class M>
static typename M::R fresnel(typename M::R ni, typename M::R nt, typename M::R ci,
                             typename M::R* ct, bool* tir) {
    typedef typename M::R R;
    R ratio = ni / nt;
    R r2 = ratio * ratio;
    R st2 = r2 * M::fma_(-ci, ci, (R)1);
    if (st2 >= (R)1) { *tir = true; *ct = (R)0; return (R)1; }
    *tir = false;
    R c_t = M::sqrt_((R)1 - st2);
    *ct = c_t;
    R a = ni * ci, b = nt * c_t;
    R rs = (a - b) / (a + b);
    R c = ni * c_t, d = nt * ci;
    R rp = (c - d) / (c + d);
    return (rs * rs + rp * rp) * (R)0.5;
}

// Unpolarised Fresnel reflectance from a medium of real index ni into an absorbing
// medium n2 + i k2 (k2 > 0, a conductor below the stack) at incidence cosine ci: with
// w = (n2 + i k2)^2 - ni^2 (1 - ci^2) and u + i v = sqrt(w) (the refracted wave's
// normal component times its index, Re >= 0), r_s = (ni ci - sqrt w)/(ni ci + sqrt w)
// and r_p = ((n2 + i k2)^2 ci - ni sqrt w)/((n2 + i k2)^2 ci + ni sqrt w).  The square
// root takes whichever of u, v is the larger from the modulus and the other by
// division, which avoids cancellation for either sign of Re w.
template <class M>
static typename M::R fresnel_conductor(typename M::R ni, typename M::R n2, typename M::R k2,
                                       typename M::R ci) {
    typedef typename M::R R;
    const R s2 = M::fma_(-ci, ci, (R)1);
    const R e_re = n2 * n2 - k2 * k2;          // (n2 + i k2)^2
    const R e_im = (n2 + n2) * k2;
    const R w_re = e_re - (ni * ni) * s2;
    const R w_im = e_im;
    const R mod = M::sqrt_(w_re * w_re + w_im * w_im);
    R u, v;
    if (w_re >= (R)0) {
        u = M::sqrt_((mod + w_re) * (R)0.5);
        v = w_im / (u + u);
    } else {
        v = M::sqrt_((mod - w_re) * (R)0.5);
        u = w_im / (v + v);
    }
    const R a = ni * ci;
    const R rs_n = (a - u) * (a - u) + v * v;
    const R rs_d = (a + u) * (a + u) + v * v;
    const R c1 = e_re * ci, c2 = e_im * ci, q1 = ni * u, q2 = ni * v;
    const R rp_n = (c1 - q1) * (c1 - q1) + (c2 - q2) * (c2 - q2);
    const R rp_d = (c1 + q1) * (c1 + q1) + (c2 + q2) * (c2 + q2);
    return (rs_n / rs_d + rp_n / rp_d) * (R)0.5;
}

// --------------------------------------------------------------------------------
// Monte Carlo photon walk.
// --------------------------------------------------------------------------------
enum { ORC_MAX_LAYERS = 8 };
enum { OUT_R = 0, OUT_A = 1, OUT_T = 2, OUT_RUNAWAY = 3 };

extern "C" {
typedef struct orc_batch {
    int n_stacks, n_wl, max_layers;
    const int* n_layers;          // [n_stacks] or NULL (all max_layers)
    const double* mu_s;           // [(n_stacks*max_layers)*n_wl]
    const double* mu_a;
    const double* g;
    const double* n_layer;
    const double* thickness;      // [n_stacks*max_layers]
    const double* n_above;        // [n_items] or NULL -> 1
    const double* n_below;        // [n_items] or NULL -> 1
    const double* substrate_R;    // [n_items] or NULL -> no substrate
    const long long* n_photons;   // [n_items] or NULL -> photons_per_item
    long long photons_per_item;
    const long long* photon_first;// [n_items] or NULL -> 0
    const int* item_list;         // [n_list] or NULL -> every item
    int n_list;
    unsigned long long seed;
    unsigned int item_id_base;
    long long max_events;         // 0 -> 100000000
    const double* cos_incidence;  // [n_items] in (0, 1] or NULL -> 1 (normal incidence)
    const double* k_below;        // [n_items] >= 0 or NULL -> 0 (k > 0: conductor below)
} orc_batch;
}

template <class M>
struct LayerP {
    typedef typename M::R R;
    R mu_t, inv_mu_t, p_abs, g, n, d;
};

// Random numbers of one photon.  Collision event e reads the block at counter
// (p, item, e, 0): u0 free path, u1 absorb test, u2 HG deflection, u3 azimuth (in
// block 0, u3 is the entry Fresnel test instead).  Interface draw k (boundary
// crossings after entry) reads word k mod 4 of the block at counter (p, item, k/4, 1).
struct PhotonRng {
    uint32_t key[2];
    uint32_t p, item;
    void block(uint32_t idx, uint32_t tag, uint32_t out[4]) const {
        uint32_t c[4] = {p, item, idx, tag};
        philox4x32_10(c, key, out);
    }
};

template <class M>
static int walk_photon(const LayerP<M>* L, int nl, typename M::R n_above, typename M::R n_below,
                       bool has_sub, typename M::R r_sub, typename M::R cos_in,
                       typename M::R k_below, const PhotonRng& rng,
                       unsigned long long max_events, unsigned long long* n_coll,
                       unsigned long long* n_iface) {
    typedef typename M::R R;
    uint32_t k_if = 0;          // interface draws so far
    uint32_t e = 0;             // collision events so far
    unsigned long long events = 0, coll = 0, iface = 0;
    uint32_t blk[4];
    int outcome = -1;

    // Launch at the top surface (z = 0) from the medium above, at incidence cosine cos_in.
    // Normal incidence: the entry Fresnel test reads word 3 of collision block 0, the
    // azimuth of the first collision, which is never used because mu_z stays exactly
    // +-1 until the first scattering.  Oblique incidence: the first collision needs its
    // azimuth, so the entry test reads word 0 of the block at counter (p, item, 0, 2).
    // Entry under total internal reflection (medium above denser) reflects the photon.
    rng.block(e, 0u, blk);
    R mu_in = cos_in;
    {
        R ni = n_above, nt = L[0].n;
        if (ni != nt) {
            R ct; bool tir;
            R Rf = fresnel<M>(ni, nt, cos_in, &ct, &tir);
            if (tir) { *n_coll = 0; *n_iface = 0; return OUT_R; }
            R u_entry;
            if (cos_in == (R)1) {
                u_entry = M::uni(blk[3]);
            } else {
                uint32_t eb[4];
                rng.block(0u, 2u, eb);
                u_entry = M::uni(eb[0]);
            }
            if (u_entry < Rf) { *n_coll = 0; *n_iface = 0; return OUT_R; }
            mu_in = ct;
        }
    }
    int j = 0;
    R z = (R)0, mu = mu_in;
    R tau = M::neg_log(M::uni(blk[0]));
    R u1 = M::uni(blk[1]), u2 = M::uni(blk[2]), u3 = M::uni(blk[3]);

    for (;;) {
        if (events >= max_events) { outcome = OUT_RUNAWAY; break; }
        const LayerP<M>& Lj = L[j];
        // Distance to the boundary ahead along z; the photon collides first iff
        // tau |mu_z| < mu_t dist (tau < mu_t dist / |mu_z| without the division).
        const R am = M::abs_(mu);
        const R dist = (mu > (R)0) ? (Lj.d - z) : z;
        bool collide;
        if (mu != (R)0) collide = tau * am < Lj.mu_t * dist;
        else collide = Lj.mu_t > (R)0;

        if (collide) {
            // Collision inside layer j.
            R s = tau * Lj.inv_mu_t;
            z = M::fma_(mu, s, z);
            events++; coll++;
            if (u1 < Lj.p_abs) { outcome = OUT_A; break; }
            R cost = hg_cos<M>(Lj.g, u2);
            if (M::abs_(mu) > M::mu_vert()) {
                mu = (mu > (R)0) ? cost : -cost;
            } else {
                R q = M::sqrt_(M::fma_(-mu, mu, (R)1) * M::fma_(-cost, cost, (R)1));
                R cp = M::cos2pi(u3);
                mu = M::fma_(q, cp, mu * cost);
                if (mu < (R)-1) mu = (R)-1;
                if (mu > (R)1) mu = (R)1;
            }
            e++;
            rng.block(e, 0u, blk);
            tau = M::neg_log(M::uni(blk[0]));
            u1 = M::uni(blk[1]); u2 = M::uni(blk[2]); u3 = M::uni(blk[3]);
            continue;
        }
        // Optical depth to the boundary (0 when mu_z = 0); the remainder of tau is
        // carried on, never below 0.
        const R tb = (mu != (R)0) ? Lj.mu_t * (dist / am) : (R)0;

        // The free path reaches the boundary of layer j first.
        tau = tau - tb;
        if (tau < (R)0) tau = (R)0;
        bool down = mu > (R)0;
        z = down ? Lj.d : (R)0;
        events++; iface++;
        int nb = down ? j + 1 : j - 1;
        bool outside = (nb < 0) || (nb >= nl);
        if (down && outside && (has_sub || k_below > (R)0)) {
            // Opaque specular reflector below the stack, or a conductor n + ik (k > 0)
            // reflecting with its Fresnel reflectance; what is not reflected enters the
            // substrate and is counted as transmitted.
            const R Rb = has_sub ? r_sub : fresnel_conductor<M>(Lj.n, n_below, k_below, am);
            rng.block(k_if >> 2, 1u, blk);
            R u = M::uni(blk[k_if & 3u]);
            k_if++;
            if (u < Rb) { mu = -mu; continue; }
            outcome = OUT_T; break;
        }
        R ni = Lj.n;
        R nt = outside ? (down ? n_below : n_above) : L[nb].n;
        bool transmit;
        R mu_t_dir = mu;
        if (ni == nt) {
            transmit = true;
        } else {
            R ci = M::abs_(mu);
            R ct; bool tir;
            R Rf = fresnel<M>(ni, nt, ci, &ct, &tir);
            if (tir) {
                transmit = false;
            } else {
                rng.block(k_if >> 2, 1u, blk);
                R u = M::uni(blk[k_if & 3u]);
                k_if++;
                transmit = !(u < Rf);
                mu_t_dir = down ? ct : -ct;
            }
        }
        if (!transmit) { mu = -mu; continue; }
        if (outside) { outcome = down ? OUT_T : OUT_R; break; }
        j = nb;
        mu = mu_t_dir;
        z = down ? (R)0 : L[nb].d;
    }
    *n_coll = coll;
    *n_iface = iface;
    return outcome;
}

// --------------------------------------------------------------------------------
// The walk as the paper states it, in double precision: the definition that both
// fast walks (the FP32 mirror above and the GPU kernel) are judged against
// statistically.  Section "Photon transport": a photon enters through the top
// surface (specular Fresnel reflection there), travels a step drawn from the
// extinction coefficient, is absorbed with probability mu_a/mu_t at a collision or
// else scattered into a new direction drawn from Henyey-Greenstein with g; at a
// boundary it is reflected or refracted by Fresnel's equations with the matrix
// indices, and it leaves the stack through the top (R) or the bottom (T).
//
// Written straight from that description, with none of the fast walks' choices:
//   * the step is a length, s = -ln(u) / mu_t, compared with the distance to the
//     boundary along the direction, s_b = (d - z)/mu_z or -z/mu_z (divisions, no
//     reciprocals); at a boundary the unused part of the step is kept as optical
//     depth, (s - s_b) mu_t, and becomes a length in the next layer (MCML's
//     carry-over, the reading of the paper taken throughout);
//   * the deflection is the closed-form inverse of the HG distribution function,
//     (1 + g^2 - ((1 - g^2)/(1 - g + 2 g u))^2) / (2 g), and the azimuth
//     phi = 2 pi u with libm's cos; sin(theta) from sqrt(1 - cos^2(theta));
//   * uniforms are drawn one at a time, in the order the walk needs them, from a
//     sequential stream of its own: the words of the Philox4x32-10 blocks at
//     counter (photon, item, k, 3), k = 0, 1, 2, ..., each word x mapped to
//     (x + 1/2) 2^-32 (a finer grid than the fast walks' 2^-23).
// So it shares neither operation order nor random-number layout with the fast walks;
// agreement with them is statistical (binomial), and its own pins are closed forms
// and the discrete-ordinates solution of the transfer equation.
// --------------------------------------------------------------------------------
struct SeqStream {
    uint32_t key[2];
    uint32_t p, item;
    uint32_t k;
    int i;
    uint32_t w[4];
    void start(uint32_t photon) { p = photon; k = 0; i = 4; }
    double next() {
        if (i == 4) {
            uint32_t c[4] = {p, item, k, 3u};
            philox4x32_10(c, key, w);
            ++k;
            i = 0;
        }
        return ((double)w[i++] + 0.5) * 0x1p-32;
    }
};

struct DefLayer {
    double mu_s, mu_a, g, n, d;
};

static double hg_cos_definition(double g, double u) {
    if (std::fabs(g) < 1e-6) return 2.0 * u - 1.0;
    const double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    double c = (1.0 + g * g - t * t) / (2.0 * g);
    if (c < -1.0) c = -1.0;
    if (c > 1.0) c = 1.0;
    return c;
}

static int walk_photon_definition(const DefLayer* L, int nl, double n_above, double n_below,
                                  bool has_sub, double r_sub, double cos_in, double k_below,
                                  SeqStream& rs, unsigned long long max_events,
                                  unsigned long long* n_coll, unsigned long long* n_iface) {
    unsigned long long events = 0, coll = 0, iface = 0;
    *n_coll = 0;
    *n_iface = 0;
    // Entry through the top surface at incidence cosine cos_in.
    double mu = cos_in;
    if (n_above != L[0].n) {
        double ct;
        bool tir;
        const double Rf = fresnel<MathF64>(n_above, L[0].n, cos_in, &ct, &tir);
        if (tir) return OUT_R;
        if (rs.next() < Rf) return OUT_R;
        mu = ct;
    }
    int j = 0;
    double z = 0.0;
    double tau = -std::log(rs.next());   // optical depth still to travel before colliding
    for (;;) {
        if (events >= max_events) {
            *n_coll = coll;
            *n_iface = iface;
            return OUT_RUNAWAY;
        }
        const DefLayer& Lj = L[j];
        const double mu_t = Lj.mu_s + Lj.mu_a;
        const double inf = std::numeric_limits<double>::infinity();
        const double s = (mu_t > 0.0) ? tau / mu_t : inf;                  // step length
        const double s_b = (mu > 0.0) ? (Lj.d - z) / mu : (mu < 0.0) ? -z / mu : inf;
        if (s < s_b) {
            // Collision inside layer j.
            z = z + mu * s;
            events++;
            coll++;
            if (rs.next() < Lj.mu_a / mu_t) {
                *n_coll = coll;
                *n_iface = iface;
                return OUT_A;
            }
            const double cost = hg_cos_definition(Lj.g, rs.next());
            const double phi = 2.0 * M_PI * rs.next();
            if (std::fabs(mu) > 1.0 - 1e-5) {
                mu = (mu > 0.0) ? cost : -cost;
            } else {
                const double sint = std::sqrt(1.0 - cost * cost);
                mu = mu * cost + std::sqrt(1.0 - mu * mu) * sint * std::cos(phi);
                if (mu < -1.0) mu = -1.0;
                if (mu > 1.0) mu = 1.0;
            }
            tau = -std::log(rs.next());
            continue;
        }
        // The boundary of layer j comes first (a photon travelling parallel to the
        // layers in a transparent layer is sent to the top one).
        const bool down = mu > 0.0;
        if (s_b < inf) tau = tau - mu_t * s_b;
        if (tau < 0.0) tau = 0.0;   // rounding only
        z = down ? Lj.d : 0.0;
        events++;
        iface++;
        const int nb = down ? j + 1 : j - 1;
        const bool outside = (nb < 0) || (nb >= nl);
        if (down && outside && (has_sub || k_below > 0.0)) {
            const double Rb = has_sub ? r_sub
                                      : fresnel_conductor<MathF64>(Lj.n, n_below, k_below,
                                                                   std::fabs(mu));
            if (rs.next() < Rb) {
                mu = -mu;
                continue;
            }
            *n_coll = coll;
            *n_iface = iface;
            return OUT_T;
        }
        const double ni = Lj.n;
        const double nt = outside ? (down ? n_below : n_above) : L[nb].n;
        double mu_next = mu;
        bool transmit = true;
        if (ni != nt) {
            double ct;
            bool tir;
            const double Rf = fresnel<MathF64>(ni, nt, std::fabs(mu), &ct, &tir);
            if (tir || rs.next() < Rf) transmit = false;
            else mu_next = down ? ct : -ct;
        }
        if (!transmit) {
            mu = -mu;
            continue;
        }
        if (outside) {
            *n_coll = coll;
            *n_iface = iface;
            return down ? OUT_T : OUT_R;
        }
        j = nb;
        mu = mu_next;
        z = down ? 0.0 : L[nb].d;
    }
}

static int run_batch_definition(const orc_batch* b, long long* counts, int* photon_log,
                                long long log_stride) {
    const long long n_items = (long long)b->n_stacks * b->n_wl;
    const int n_run = b->item_list ? b->n_list : (int)n_items;
    const unsigned long long max_ev = b->max_events > 0 ? (unsigned long long)b->max_events
                                                        : 100000000ull;
    for (int r = 0; r < n_run; ++r) {
        const long long it = b->item_list ? b->item_list[r] : r;
        const int s = (int)(it / b->n_wl), w = (int)(it % b->n_wl);
        const int nl = b->n_layers ? b->n_layers[s] : b->max_layers;
        DefLayer L[ORC_MAX_LAYERS];
        for (int j = 0; j < nl; ++j) {
            const long long pi = ((long long)s * b->max_layers + j) * b->n_wl + w;
            L[j].mu_s = b->mu_s[pi];
            L[j].mu_a = b->mu_a[pi];
            L[j].g = b->g[pi];
            L[j].n = b->n_layer[pi];
            L[j].d = b->thickness[(long long)s * b->max_layers + j];
        }
        const double na = b->n_above ? b->n_above[it] : 1.0;
        const double nbw = b->n_below ? b->n_below[it] : 1.0;
        const bool has_sub = b->substrate_R != nullptr;
        const double rsub = has_sub ? b->substrate_R[it] : 0.0;
        const double cin = b->cos_incidence ? b->cos_incidence[it] : 1.0;
        const double kbw = (b->k_below && !has_sub) ? b->k_below[it] : 0.0;
        const long long N = b->n_photons ? b->n_photons[it] : b->photons_per_item;
        const long long first = b->photon_first ? b->photon_first[it] : 0;
        SeqStream rs;
        rs.key[0] = (uint32_t)(b->seed & 0xffffffffull);
        rs.key[1] = (uint32_t)(b->seed >> 32);
        rs.item = b->item_id_base + (uint32_t)it;
        long long* c = counts + (long long)r * 6;
        for (int q = 0; q < 6; ++q) c[q] = 0;
        for (long long i = 0; i < N; ++i) {
            rs.start((uint32_t)(first + i));
            unsigned long long nc, ni;
            const int out = walk_photon_definition(L, nl, na, nbw, has_sub, rsub, cin, kbw, rs,
                                                   max_ev, &nc, &ni);
            c[out] += 1;
            c[4] += (long long)nc;
            c[5] += (long long)ni;
            if (photon_log) {
                const unsigned long long rec = (nc << 2) | (unsigned long long)out;
                photon_log[(long long)r * log_stride + i] =
                    (int)(rec > 0x7fffffffull ? 0x7fffffffull : rec);
            }
        }
    }
    return 0;
}

template <class M>
static int run_batch(const orc_batch* b, long long* counts, int* photon_log, long long log_stride) {
    typedef typename M::R R;
    const long long n_items = (long long)b->n_stacks * b->n_wl;
    const int n_run = b->item_list ? b->n_list : (int)n_items;
    const unsigned long long max_ev = b->max_events > 0 ? (unsigned long long)b->max_events
                                                        : 100000000ull;
    for (int r = 0; r < n_run; ++r) {
        long long it = b->item_list ? b->item_list[r] : r;
        int s = (int)(it / b->n_wl), w = (int)(it % b->n_wl);
        int nl = b->n_layers ? b->n_layers[s] : b->max_layers;
        LayerP<M> L[ORC_MAX_LAYERS];
        for (int j = 0; j < nl; ++j) {
            long long pi = ((long long)s * b->max_layers + j) * b->n_wl + w;
            R ms = (R)b->mu_s[pi], ma = (R)b->mu_a[pi];
            L[j].mu_t = ms + ma;
            L[j].inv_mu_t = (L[j].mu_t > (R)0) ? (R)1 / L[j].mu_t : (R)0;
            L[j].p_abs = (L[j].mu_t > (R)0) ? ma / L[j].mu_t : (R)0;
            L[j].g = (R)b->g[pi];
            L[j].n = (R)b->n_layer[pi];
            L[j].d = (R)b->thickness[(long long)s * b->max_layers + j];
        }
        R na = b->n_above ? (R)b->n_above[it] : (R)1;
        R nbw = b->n_below ? (R)b->n_below[it] : (R)1;
        bool has_sub = b->substrate_R != nullptr;
        R rsub = has_sub ? (R)b->substrate_R[it] : (R)0;
        R cin = b->cos_incidence ? (R)b->cos_incidence[it] : (R)1;
        R kbw = (b->k_below && !has_sub) ? (R)b->k_below[it] : (R)0;
        long long N = b->n_photons ? b->n_photons[it] : b->photons_per_item;
        long long first = b->photon_first ? b->photon_first[it] : 0;
        PhotonRng rng;
        rng.key[0] = (uint32_t)(b->seed & 0xffffffffull);
        rng.key[1] = (uint32_t)(b->seed >> 32);
        rng.item = b->item_id_base + (uint32_t)it;
        long long* c = counts + (long long)r * 6;
        for (int q = 0; q < 6; ++q) c[q] = 0;
        for (long long i = 0; i < N; ++i) {
            rng.p = (uint32_t)(first + i);
            unsigned long long nc, ni;
            int out = walk_photon<M>(L, nl, na, nbw, has_sub, rsub, cin, kbw, rng, max_ev, &nc, &ni);
            c[out] += 1;
            c[4] += (long long)nc;
            c[5] += (long long)ni;
            if (photon_log) {
                unsigned long long rec = (nc << 2) | (unsigned long long)out;
                photon_log[(long long)r * log_stride + i] =
                    (int)(rec > 0x7fffffffull ? 0x7fffffffull : rec);
            }
        }
    }
    return 0;
}

// --------------------------------------------------------------------------------
// Mie theory for a homogeneous sphere in an absorbing host (section "Scattering
// properties", Eqs. 1-5, 10-12, 15).
// --------------------------------------------------------------------------------

// j_{n-1}(z)/j_n(z) by the modified Lentz method (Lentz 1976; Thompson & Barnett
// 1986) on the continued fraction r_n = (2n+1)/z - 1/r_{n+1}, which follows from
// the three-term recurrence j_{n-1} + j_{n+1} = (2n+1)/z j_n.
static cd ratio_j(int n, cd z) {
    const double tiny = 1e-300;
    cd f = (double)(2 * n + 1) / z;
    if (std::abs(f) == 0.0) f = tiny;
    cd C = f, D = 0.0;
    for (int k = 1; k < 100000; ++k) {
        cd bk = (double)(2 * (n + k) + 1) / z;
        D = bk - D;
        if (std::abs(D) == 0.0) D = tiny;
        D = 1.0 / D;
        C = bk - 1.0 / C;
        if (std::abs(C) == 0.0) C = tiny;
        cd delta = C * D;
        f *= delta;
        if (std::abs(delta - 1.0) < 1e-16) break;
    }
    return f;
}

// Riccati-Bessel logarithmic derivative D_n(z) = psi_n'(z)/psi_n(z), psi_n = z j_n
// (A_n of Eq. 4): D_n = j_{n-1}/j_n - n/z.
static cd log_deriv_psi(int n, cd z) { return ratio_j(n, z) - (double)n / z; }

// Geometric term of Eq. 10 with alpha = 4 pi r k_m / lambda (the printed alpha is
// garbled; this is the reading in which gamma -> 1 as the host absorption -> 0).
// For small alpha the bracket cancels, so the Taylor series
// gamma = 2 sum_{k>=2} (k-1)/k! alpha^(k-2) is summed instead.
static double gamma_term(double alpha) {
    if (alpha < 0.5) {
        double sum = 0.0, fact = 2.0, pw = 1.0;  // k = 2: (k-1)/k! = 1/2
        for (int k = 2; k < 60; ++k) {
            if (k > 2) { fact *= k; pw *= alpha; }
            double term = 2.0 * (double)(k - 1) / fact * pw;
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        return sum;
    }
    return 2.0 * (1.0 + (alpha - 1.0) * std::exp(alpha)) / (alpha * alpha);
}

extern "C" int orc_mie_sphere(double wl, double npr, double npi, double nmr, double nmi, double r,
                              double* q_ext, double* q_sca, double* g_out, int* nmax_out,
                              double* an_out, double* bn_out, int an_cap) {
    const cd n_p(npr, npi), n_m(nmr, nmi);
    const cd x = 2.0 * M_PI * r * n_m / wl;   // Eq. 1
    const cd y = 2.0 * M_PI * r * n_p / wl;
    const double ay = std::abs(y);
    const int nmax = (int)std::ceil(2.0 + ay + 4.3 * std::cbrt(ay));  // below Eq. 12
    const int nt = nmax + 1;   // a_{n+1}, b_{n+1} are needed by Eq. 15 at n = nmax
    cd* a = new cd[nt + 1];
    cd* bb = new cd[nt + 1];
    // psi_n(x) = x j_n(x): upward recurrence of its values while n <= |x| (where
    // psi_n and the second solution have the same size), and psi_{n-1}/(D_n + n/x)
    // above |x| (where psi_n decreases monotonically).  xi_n(x) = x h_n^(1)(x) by
    // upward recurrence of its values from xi_{-1} = e^{ix}, xi_0 = sin x - i cos x.
    // Eqs. 2-3 are evaluated multiplied through by psi_n(x) and xi_n(x):
    //   a_n = (n_m A_n(y) psi_n - n_p psi_n') / (n_m A_n(y) xi_n - n_p xi_n'),
    // the same quotient, without the 0 * infinity of A_n(x) at zeros of psi_n(x).
    const double ax = std::abs(x);
    cd psi_m1 = std::cos(x);
    cd psi_prev = std::sin(x);
    cd xi_m1 = std::exp(cd(0.0, 1.0) * x);
    cd xi_prev = std::sin(x) - cd(0.0, 1.0) * std::cos(x);
    for (int n = 1; n <= nt; ++n) {
        cd psi_n;
        if ((double)n <= ax) psi_n = (double)(2 * n - 1) / x * psi_prev - psi_m1;
        else psi_n = psi_prev / (log_deriv_psi(n, x) + (double)n / x);
        cd xi_n = (double)(2 * n - 1) / x * xi_prev - xi_m1;
        cd dpsi = psi_prev - (double)n * psi_n / x;   // psi_n'(x)
        cd dxi = xi_prev - (double)n * xi_n / x;      // xi_n'(x)
        cd Dy = log_deriv_psi(n, y);                  // A_n(y), Eq. 4
        a[n] = (n_m * Dy * psi_n - n_p * dpsi) / (n_m * Dy * xi_n - n_p * dxi);   // Eq. 2
        bb[n] = (n_p * Dy * psi_n - n_m * dpsi) / (n_p * Dy * xi_n - n_m * dxi);  // Eq. 3
        psi_m1 = psi_prev;
        psi_prev = psi_n;
        xi_m1 = xi_prev;
        xi_prev = xi_n;
    }
    double s_ext = 0.0, s_sca = 0.0, s_g = 0.0;
    for (int n = 1; n <= nmax; ++n) {
        double w = 2.0 * n + 1.0;
        s_ext += w * std::real((a[n] + bb[n]) / (n_m * n_m));             // Eq. 11
        s_sca += w * (std::norm(a[n]) + std::norm(bb[n]));               // Eq. 12
        s_g += (double)n * (n + 2.0) / (n + 1.0) *
                   std::real(a[n] * std::conj(a[n + 1]) + bb[n] * std::conj(bb[n + 1])) +
               w / ((double)n * (n + 1.0)) * std::real(a[n] * std::conj(bb[n]));  // Eq. 15
    }
    const double alpha = 4.0 * M_PI * r * nmi / wl;
    const double gam = gamma_term(alpha);
    const double c_ext = wl * wl / (2.0 * M_PI) * s_ext;
    const double c_sca = wl * wl * std::exp(-alpha) / (2.0 * M_PI * gam * std::norm(n_m)) * s_sca;
    const double area = M_PI * r * r;
    *q_ext = c_ext / area;
    *q_sca = c_sca / area;
    *g_out = (s_sca > 0.0) ? 2.0 * s_g / s_sca : 0.0;
    if (nmax_out) *nmax_out = nmax;
    if (an_out && bn_out) {
        for (int n = 1; n <= nt && n <= an_cap; ++n) {
            an_out[2 * (n - 1)] = a[n].real(); an_out[2 * (n - 1) + 1] = a[n].imag();
            bn_out[2 * (n - 1)] = bb[n].real(); bn_out[2 * (n - 1) + 1] = bb[n].imag();
        }
    }
    delete[] a;
    delete[] bb;
    return 0;
}


// --------------------------------------------------------------------------------
// Core-shell sphere (supplement section 3, Eqs. S1-S9, Bohren & Huffman 8.1): core
// radius a with index n_c, shell out to radius b with index n_s, host n_m.
// m1 = n_c/n_m, m2 = n_s/n_m, x = k a, y = k b with k = 2 pi n_m / lambda.
// A_n, B_n (S3, S4) are evaluated divided through by psi_n(m1 x), i.e. with the
// logarithmic derivative D_n(m1 x) (continued fraction); psi_n, chi_n of the shell
// arguments by upward recurrence of values (psi_n from D_n above |z|); chi_n = z y_n(z)
// (S8), xi_n = psi_n + i chi_n (S9).
// --------------------------------------------------------------------------------
static void riccati_psi_chi(int nt, cd z, cd* psi, cd* chi) {
    // psi[0..nt], chi[0..nt]
    const double az = std::abs(z);
    cd psi_m1 = std::cos(z), chi_m1 = std::sin(z);       // n = -1
    psi[0] = std::sin(z);
    chi[0] = -std::cos(z);
    for (int n = 1; n <= nt; ++n) {
        const cd prev_psi = (n == 1) ? psi_m1 : psi[n - 2];
        const cd prev_chi = (n == 1) ? chi_m1 : chi[n - 2];
        if ((double)n <= az) psi[n] = (double)(2 * n - 1) / z * psi[n - 1] - prev_psi;
        else psi[n] = psi[n - 1] / (log_deriv_psi(n, z) + (double)n / z);
        chi[n] = (double)(2 * n - 1) / z * chi[n - 1] - prev_chi;
    }
}

extern "C" int orc_mie_coated(double wl, double ncr, double nci, double nsr, double nsi,
                              double nmr, double nmi, double a, double b, double* q_ext,
                              double* q_sca, double* g_out, int* nmax_out, double* an_out,
                              double* bn_out, int an_cap) {
    const cd n_c(ncr, nci), n_s(nsr, nsi), n_m(nmr, nmi);
    const cd m1 = n_c / n_m, m2 = n_s / n_m;
    const double kv = 2.0 * M_PI / wl;
    const cd x = kv * a * n_m, y = kv * b * n_m;
    const double ymax = kv * b * std::max(std::abs(n_c), std::abs(n_s));
    const int nmax = (int)std::ceil(2.0 + ymax + 4.3 * std::cbrt(ymax));
    const int nt = nmax + 1;
    cd *ps2x = new cd[nt + 1], *ch2x = new cd[nt + 1], *ps2y = new cd[nt + 1], *ch2y = new cd[nt + 1];
    cd *psy = new cd[nt + 1], *chy = new cd[nt + 1];
    riccati_psi_chi(nt, m2 * x, ps2x, ch2x);
    riccati_psi_chi(nt, m2 * y, ps2y, ch2y);
    riccati_psi_chi(nt, y, psy, chy);
    cd* an = new cd[nt + 1];
    cd* bn = new cd[nt + 1];
    const cd I(0.0, 1.0);
    for (int n = 1; n <= nt; ++n) {
        const double dn = n;
        const cd z2x = m2 * x, z2y = m2 * y;
        const cd D1 = log_deriv_psi(n, m1 * x);                         // psi'/psi at m1 x
        const cd d_ps2x = ps2x[n - 1] - dn * ps2x[n] / z2x, d_ch2x = ch2x[n - 1] - dn * ch2x[n] / z2x;
        const cd D2x = d_ps2x / ps2x[n];
        const cd An = ps2x[n] * (m2 * D1 - m1 * D2x) / (m2 * D1 * ch2x[n] - m1 * d_ch2x);       // S3
        const cd Bn = ps2x[n] * (m2 * D2x - m1 * D1) / (m2 * d_ch2x - m1 * D1 * ch2x[n]);       // S4
        const cd d_ps2y = ps2y[n - 1] - dn * ps2y[n] / z2y, d_ch2y = ch2y[n - 1] - dn * ch2y[n] / z2y;
        const cd xi = psy[n] + I * chy[n];                                   // S9
        const cd d_psy = psy[n - 1] - dn * psy[n] / y;
        const cd d_xi = (psy[n - 1] + I * chy[n - 1]) - dn * xi / y;
        const cd Ua = d_ps2y - An * d_ch2y, Va = ps2y[n] - An * ch2y[n];
        const cd Ub = d_ps2y - Bn * d_ch2y, Vb = ps2y[n] - Bn * ch2y[n];
        an[n] = (psy[n] * Ua - m2 * d_psy * Va) / (xi * Ua - m2 * d_xi * Va);                    // S1
        bn[n] = (m2 * psy[n] * Ub - d_psy * Vb) / (m2 * xi * Ub - d_xi * Vb);                    // S2
    }
    double s_ext = 0.0, s_sca = 0.0, s_g = 0.0;
    for (int n = 1; n <= nmax; ++n) {
        double w = 2.0 * n + 1.0;
        s_ext += w * std::real((an[n] + bn[n]) / (n_m * n_m));
        s_sca += w * (std::norm(an[n]) + std::norm(bn[n]));
        s_g += (double)n * (n + 2.0) / (n + 1.0) *
                   std::real(an[n] * std::conj(an[n + 1]) + bn[n] * std::conj(bn[n + 1])) +
               w / ((double)n * (n + 1.0)) * std::real(an[n] * std::conj(bn[n]));
    }
    const double alpha = 4.0 * M_PI * b * nmi / wl;
    const double gam = gamma_term(alpha);
    const double area = M_PI * b * b;
    *q_ext = wl * wl / (2.0 * M_PI) * s_ext / area;
    *q_sca = wl * wl * std::exp(-alpha) / (2.0 * M_PI * gam * std::norm(n_m)) * s_sca / area;
    *g_out = (s_sca > 0.0) ? 2.0 * s_g / s_sca : 0.0;
    if (nmax_out) *nmax_out = nmax;
    if (an_out && bn_out) {
        for (int n = 1; n <= nt && n <= an_cap; ++n) {
            an_out[2 * (n - 1)] = an[n].real(); an_out[2 * (n - 1) + 1] = an[n].imag();
            bn_out[2 * (n - 1)] = bn[n].real(); bn_out[2 * (n - 1) + 1] = bn[n].imag();
        }
    }
    delete[] ps2x; delete[] ch2x; delete[] ps2y; delete[] ch2y; delete[] psy; delete[] chy;
    delete[] an; delete[] bn;
    return 0;
}

extern "C" double orc_gamma_term(double alpha) { return gamma_term(alpha); }

extern "C" int orc_mie_properties_cs(int n_wl, const double* wl, int n_groups,
                                     const double* nm_re, const double* nm_im, int n_species,
                                     const int* species_group, const double* np_re,
                                     const double* np_im, const double* nc_re,
                                     const double* nc_im, const double* radius,
                                     const double* core_radius, const double* vol_frac,
                                     double* mu_s, double* mu_a, double* g, double* q_ext,
                                     double* q_sca, double* g_sp);

extern "C" int orc_mie_properties(int n_wl, const double* wl, int n_groups, const double* nm_re,
                                  const double* nm_im, int n_species, const int* species_group,
                                  const double* np_re, const double* np_im, const double* radius,
                                  const double* vol_frac, double* mu_s, double* mu_a, double* g,
                                  double* q_ext, double* q_sca, double* g_sp) {
    return orc_mie_properties_cs(n_wl, wl, n_groups, nm_re, nm_im, n_species, species_group,
                                 np_re, np_im, nullptr, nullptr, radius, nullptr, vol_frac, mu_s,
                                 mu_a, g, q_ext, q_sca, g_sp);
}
extern "C" void orc_log_deriv_psi(int n, double zr, double zi, double* out) {
    cd d = log_deriv_psi(n, cd(zr, zi));
    out[0] = d.real(); out[1] = d.imag();
}

// Effective medium of one (group, wavelength): Eqs. 13, 14 and 16, the clamp of
// negative coefficients to zero, the dependent-scattering correction of Eqs. 17-19
// when the summed volume fraction exceeds 0.08, and the matrix absorption of Eq. 20.
//   species s belongs to group species_group[s]; particle index [n_species*n_wl];
//   matrix index [n_groups*n_wl]; outputs [n_groups*n_wl].
extern "C" int orc_mie_coated(double wl, double ncr, double nci, double nsr, double nsi,
                              double nmr, double nmi, double a, double b, double* q_ext,
                              double* q_sca, double* g_out, int* nmax_out, double* an_out,
                              double* bn_out, int an_cap);

// With core arrays (nc_re, nc_im [n_species*n_wl], core_radius [n_species]), species with
// core_radius > 0 are core-shell spheres (shell index np, outer radius radius).
extern "C" int orc_mie_properties_cs(int n_wl, const double* wl, int n_groups,
                                     const double* nm_re, const double* nm_im, int n_species,
                                     const int* species_group, const double* np_re,
                                     const double* np_im, const double* nc_re,
                                     const double* nc_im, const double* radius,
                                     const double* core_radius, const double* vol_frac,
                                     double* mu_s, double* mu_a, double* g, double* q_ext,
                                     double* q_sca, double* g_sp) {
    for (int gi = 0; gi < n_groups; ++gi) {
        for (int w = 0; w < n_wl; ++w) {
            const long long gw = (long long)gi * n_wl + w;
            double sum_f = 0.0, ms = 0.0, ma = 0.0, mg = 0.0;
            for (int s = 0; s < n_species; ++s) {
                if (species_group[s] != gi) continue;
                const long long sw = (long long)s * n_wl + w;
                double qe, qs, gg;
                if (core_radius && core_radius[s] > 0.0)
                    orc_mie_coated(wl[w], nc_re[sw], nc_im[sw], np_re[sw], np_im[sw], nm_re[gw],
                                   nm_im[gw], core_radius[s], radius[s], &qe, &qs, &gg, nullptr,
                                   nullptr, nullptr, 0);
                else
                    orc_mie_sphere(wl[w], np_re[sw], np_im[sw], nm_re[gw], nm_im[gw], radius[s],
                                   &qe, &qs, &gg, nullptr, nullptr, nullptr, 0);
                if (q_ext) q_ext[sw] = qe;
                if (q_sca) q_sca[sw] = qs;
                if (g_sp) g_sp[sw] = gg;
                const double f = vol_frac[s], rr = radius[s];
                sum_f += f;
                ms += 1.5 * qs * f / (2.0 * rr);           // Eq. 13
                ma += 1.5 * (qe - qs) * f / (2.0 * rr);    // Eq. 14
                mg += 1.5 * qs * f * gg / (2.0 * rr);      // numerator of Eq. 16
            }
            double gv = (ms > 0.0) ? mg / ms : 0.0;        // Eq. 16
            if (ms < 0.0) ms = 0.0;
            if (ma < 0.0) ma = 0.0;
            if (sum_f > 0.08) {                             // Eqs. 17-19
                const double C = 1.0 + 1.5 * sum_f - 0.75 * sum_f * sum_f;
                ms *= C;
                ma *= C;
            }
            ma += 4.0 * M_PI * nm_im[gw] * (1.0 - sum_f) / wl[w];  // Eq. 20
            mu_s[gw] = ms;
            mu_a[gw] = ma;
            g[gw] = gv;
        }
    }
    return 0;
}

// --------------------------------------------------------------------------------
// Exported entry points for tests.
// --------------------------------------------------------------------------------
extern "C" void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    philox4x32_10(ctr, key, out);
}
extern "C" double orc_uniform(uint32_t x) { return uniform_of(x); }
extern "C" float orc_neg_log_f32(float u) { return neg_log_f32(u); }
extern "C" float orc_cos2pi_f32(float u) { return cos2pi_f32(u); }
extern "C" void orc_neg_log_f32_many(const float* u, float* out, long long n) {
    for (long long i = 0; i < n; ++i) out[i] = neg_log_f32(u[i]);
}
extern "C" void orc_cos2pi_f32_many(const float* u, float* out, long long n) {
    for (long long i = 0; i < n; ++i) out[i] = cos2pi_f32(u[i]);
}
extern "C" double orc_hg_cos_f64(double g, double u) { return hg_cos<MathF64>(g, u); }
extern "C" float orc_hg_cos_f32(float g, float u) { return hg_cos<MathF32>(g, u); }
extern "C" double orc_fresnel_f64(double ni, double nt, double ci, double* ct) {
    bool tir;
    double c;
    double R = fresnel<MathF64>(ni, nt, ci, &c, &tir);
    if (ct) *ct = c;
    return R;
}
extern "C" double orc_fresnel_conductor_f64(double ni, double n2, double k2, double ci) {
    return fresnel_conductor<MathF64>(ni, n2, k2, ci);
}

extern "C" float orc_fresnel_conductor_f32(float ni, float n2, float k2, float ci) {
    return fresnel_conductor<MathF32>(ni, n2, k2, ci);
}

// Solar-weighted totals (section "Output", Eq. 21): for each stack s and each of R, A,
// T, the integral of the spectral fraction times G over the wavelength grid divided by
// the integral of G, both by the trapezoidal rule on the grid points.  The spectral
// fraction at a wavelength is the count over R + A + T of that item (counts rows
// item = s * n_wl + w, FOS_NCOUNT = 6 columns).  One wavelength: the fractions there.
extern "C" int orc_solar_weighted(int n_stacks, int n_wl, const double* wl, const double* G,
                                  const long long* counts, double* out) {
    for (int s = 0; s < n_stacks; ++s) {
        double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
        double frac[2][3];
        double gw[2];
        for (int w = 0; w < n_wl; ++w) {
            const long long* c = counts + ((long long)s * n_wl + w) * 6;
            const double tot = (double)(c[0] + c[1] + c[2]);
            for (int k = 0; k < 3; ++k) frac[w & 1][k] = tot > 0.0 ? (double)c[k] / tot : 0.0;
            gw[w & 1] = G[w];
            if (n_wl == 1) {
                for (int k = 0; k < 3; ++k) num[k] = frac[0][k];
                den = 1.0;
                break;
            }
            if (w == 0) continue;
            const double h = wl[w] - wl[w - 1];
            const int a = (w - 1) & 1, b = w & 1;
            for (int k = 0; k < 3; ++k)
                num[k] += 0.5 * h * (frac[a][k] * gw[a] + frac[b][k] * gw[b]);
            den += 0.5 * h * (gw[a] + gw[b]);
        }
        for (int k = 0; k < 3; ++k) out[(long long)s * 3 + k] = num[k] / den;
    }
    return 0;
}

// mode 0: the fast walk's operation order and random-number layout in FP64 (libm);
// mode 1: the FP32 mirror of the GPU walk; mode 2: the definition walk above.
extern "C" int orc_mc_run(const orc_batch* b, int mode, long long* counts, int* photon_log,
                          long long log_stride) {
    if (b->max_layers < 1 || b->max_layers > ORC_MAX_LAYERS) return 1;
    if (mode == 1) return run_batch<MathF32>(b, counts, photon_log, log_stride);
    if (mode == 2) return run_batch_definition(b, counts, photon_log, log_stride);
    return run_batch<MathF64>(b, counts, photon_log, log_stride);
}
