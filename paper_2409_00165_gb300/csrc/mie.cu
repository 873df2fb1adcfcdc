// Mie theory + effective medium on GB300, FP64 (arxiv 2409.00165, section
// "Scattering properties", Eqs. 1-20).
//
// mie_kernel: one thread per (species, wavelength), grid-stride; homogeneous spheres
//   (sphere_eval) and core-shell spheres (coated_eval, supplement Eqs. S1-S9).  The logarithmic
//   derivative D_n(z) = psi_n'(z)/psi_n(z) of psi_n(z) = z j_n(z) (A_n of Eq. 4) comes
//   from the downward recurrence D_{n-1} = n/z - 1/(D_n + n/z) started at
//   N* = n_max + 17 with D = 0, for the particle argument y (and, for |x| < 1.5, the
//   host argument x).  The values are kept in a scratch laid out [order][thread] so
//   that a warp's accesses coalesce.  An upward sweep then builds psi_n(x) (upward
//   recurrence; for |x| < 1.5 only while n <= |x|, psi_{n-1}/(D_n(x) + n/x) above)
//   and xi_n(x) = x h^(1)_n(x)
//   (upward recurrence), forms a_n, b_n of Eqs. 2-3 multiplied through by psi_n(x)
//   and xi_n(x) (well conditioned at zeros of psi_n(x)), and accumulates the sums of
//   Eqs. 11, 12 and 15.
// emt_kernel: one thread per (group, wavelength): Eqs. 13, 14, 16, clamp to 0,
//   Eqs. 17-19 when the summed volume fraction exceeds 0.08, Eq. 20.
#include <cmath>

#include "fos_internal.h"

namespace fos {
namespace mie {

struct cx {
    double re, im;
};
__device__ __forceinline__ cx mk(double r, double i) { return cx{r, i}; }
__device__ __forceinline__ cx operator+(cx a, cx b) { return cx{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cx operator-(cx a, cx b) { return cx{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cx operator*(cx a, cx b) {
    return cx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cx operator*(double s, cx a) { return cx{s * a.re, s * a.im}; }
// Complex division a/b = a conj(b) / |b|^2 with one real division; Smith's algorithm
// (no intermediate overflow) when the larger part of b is outside [2^-490, 2^491).  The
// range test reads the exponent fields with integer instructions, which keeps it off the
// FP64 pipe that bounds this kernel.
__device__ __forceinline__ cx div_smith(cx a, cx b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return cx{(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    } else {
        const double r = b.re / b.im, d = b.re * r + b.im;
        return cx{(a.re * r + a.im) / d, (a.im * r - a.re) / d};
    }
}
__device__ __forceinline__ int exponent_field(double v) {
    return (__double2hiint(v) >> 20) & 0x7ff;
}
__device__ __forceinline__ cx operator/(cx a, cx b) {
    const int e = max(exponent_field(b.re), exponent_field(b.im));
    if (e > 1023 + 490 || e < 1023 - 490) return div_smith(a, b);
    const double inv = 1.0 / (b.re * b.re + b.im * b.im);
    return cx{(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}
// 1/b = conj(b) / |b|^2 (the quotient above with a = 1, without its products by 0).
__device__ __forceinline__ cx crcp(cx b) {
    const int e = max(exponent_field(b.re), exponent_field(b.im));
    if (e > 1023 + 490 || e < 1023 - 490) return div_smith(cx{1.0, 0.0}, b);
    const double inv = 1.0 / (b.re * b.re + b.im * b.im);
    return cx{b.re * inv, -b.im * inv};
}
__device__ __forceinline__ double norm2(cx a) { return a.re * a.re + a.im * a.im; }
// Two quotients na/da, nb/db with one real division: 1/|da|^2 = |db|^2 / (|da|^2 |db|^2)
// and the same for db, when both denominators' larger parts lie within 2^(+-240) (the
// product of the squared moduli then neither overflows nor underflows); otherwise two
// divisions.
__device__ __forceinline__ void div_pair(cx na, cx da, cx nb, cx db, cx& qa, cx& qb) {
    const int ea = max(exponent_field(da.re), exponent_field(da.im));
    const int eb = max(exponent_field(db.re), exponent_field(db.im));
    if (ea > 1023 + 240 || ea < 1023 - 240 || eb > 1023 + 240 || eb < 1023 - 240) {
        qa = na / da;
        qb = nb / db;
        return;
    }
    const double pa = da.re * da.re + da.im * da.im, pb = db.re * db.re + db.im * db.im;
    const double inv = 1.0 / (pa * pb);
    const double ia = pb * inv, ib = pa * inv;
    qa = cx{(na.re * da.re + na.im * da.im) * ia, (na.im * da.re - na.re * da.im) * ia};
    qb = cx{(nb.re * db.re + nb.im * db.im) * ib, (nb.im * db.re - nb.re * db.im) * ib};
}
// a b - c, a b + c and c - a b with the addition folded into the fused multiply-adds (two
// FP64 instructions per part instead of three).
__device__ __forceinline__ cx mul_sub(cx a, cx b, cx c) {
    return cx{fma(a.re, b.re, fma(-a.im, b.im, -c.re)), fma(a.re, b.im, fma(a.im, b.re, -c.im))};
}
__device__ __forceinline__ cx mul_add(cx a, cx b, cx c) {
    return cx{fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
__device__ __forceinline__ cx sub_mul(cx c, cx a, cx b) {
    return cx{fma(-a.re, b.re, fma(a.im, b.im, c.re)), fma(-a.re, b.im, fma(-a.im, b.re, c.im))};
}
__device__ __forceinline__ double cabs_(cx a) { return hypot(a.re, a.im); }
// |z| of a size parameter (far from overflow: no hypot scaling needed).
__device__ __forceinline__ double size_abs(cx a) { return sqrt(fma(a.re, a.re, a.im * a.im)); }
// Order counts that only bound a sum or a recurrence: in FP32, off the narrow FP64 pipe.
// n_max of Eq. 12's criterion, 2 + |y| + 4.3 |y|^(1/3), and Wiscombe's count for the host
// argument, |x| + 4.05 |x|^(1/3) + 2, rounded up.
__device__ __forceinline__ int nmax_of(double ay) {
    const float a = (float)ay;
    return (int)ceilf(2.0f + a + 4.3f * cbrtf(a));
}
__device__ __forceinline__ int wiscombe_of(double ax) {
    const float a = (float)ax;
    return (int)ceilf(a + 4.05f * cbrtf(a) + 2.0f);
}
__device__ __forceinline__ cx csin(cx z) {
    return cx{sin(z.re) * cosh(z.im), cos(z.re) * sinh(z.im)};
}
__device__ __forceinline__ cx ccos(cx z) {
    return cx{cos(z.re) * cosh(z.im), -sin(z.re) * sinh(z.im)};
}

// Geometric term of Eq. 10 with alpha = 4 pi r k_m / lambda.  Below alpha = 0.5 the
// bracket cancels, so its Taylor series 2 sum_{k>=2} (k-1)/k! alpha^(k-2) is used, by
// Horner's rule over a table of its coefficients: 19 terms (the next one is < 1e-18 at
// alpha = 0.5), or 6 below alpha = 2^-10 (the next one is < 1e-21 there).
struct GammaSeries {
    double c[19];   // c[i] = 2 (i + 1) / (i + 2)!
    constexpr GammaSeries() : c() {
        double fact = 2.0;
        for (int i = 0; i < 19; ++i) {
            if (i > 0) fact *= (double)(i + 2);
            c[i] = 2.0 * (double)(i + 1) / fact;
        }
    }
};
__constant__ GammaSeries g_gamma = GammaSeries();
__device__ __forceinline__ double gamma_term(double a) {
    if (a < 0x1p-10) {
        double p = g_gamma.c[5];
#pragma unroll
        for (int i = 4; i >= 0; --i) p = fma(p, a, g_gamma.c[i]);
        return p;
    }
    if (a < 0.5) {
        double p = g_gamma.c[18];
#pragma unroll
        for (int i = 17; i >= 0; --i) p = fma(p, a, g_gamma.c[i]);
        return p;
    }
    return 2.0 * (1.0 + (a - 1.0) * exp(a)) / (a * a);
}

// psi_{-1}(x) = cos x, psi_0(x) = sin x and xi_{-1}(x) = e^{ix} for x = a + ib, with the
// hyperbolic functions of b from one expm1: E = e^b, cosh b = (E + 1/E)/2,
// sinh b = (e^b - 1)(1 + 1/E)/2 (no cancellation for small b), e^{-b} = 1/E.
__device__ __forceinline__ void start_values(cx x, cx& psi_m1, cx& psi_0, cx& xi_m1) {
    double sa, ca;
    sincos(x.re, &sa, &ca);
    const double em1 = expm1(x.im);
    const double ie = 1.0 / (1.0 + em1);
    const double ch = 0.5 * (1.0 + em1 + ie), sh = 0.5 * em1 * (1.0 + ie);
    psi_m1 = mk(ca * ch, -sa * sh);
    psi_0 = mk(sa * ch, ca * sh);
    xi_m1 = mk(ie * ca, ie * sa);
}

// psi_n(x) comes from its upward recurrence at every order when |x| >= this (as in Bohren
// and Huffman's BHMIE and Wiscombe's Mie algorithm).  Above n = |x| the recurrence's
// rounding errors grow like the increasing solution chi_n, so psi_n carries an absolute
// error of about n eps |chi_n|; that moves a_n and b_n by about n eps, which against sums of
// size x^2 Q / 2 stays far below 1e-10 once x is not small.  For smaller |x| (the Rayleigh
// regime, where Q can be tiny) psi_n above |x| is psi_{n-1} / (D_n(x) + n/x) with D_n(x)
// from its downward recurrence.
// With psi_n from the upward recurrence the computed terms do not fall below that error
// past |x|, so the sums cannot end by the size of their terms; they end at order
// |x| + 8 |x|^(1/3) + 8 at the latest.  Past the transition region n ~ |x| the exact terms
// fall like exp(-(4 sqrt(2) / 3) (n - |x|)^(3/2) / sqrt(|x|)) (the Debye asymptotics of
// psi_n and chi_n), which puts every term after that order below 2^-60 of the sums
// (checked against the oracle's coefficients for |x| from 1.5 to 3000, |m| from 0.7 to 4),
// and chi_n, which grows as fast, stays far from overflow there.
constexpr double PSI_UPWARD_MIN_X = 1.5;
__device__ __forceinline__ int psi_upward_last(double ax, int nt) {
    const float a = (float)ax;
    return min(nt, (int)ceilf(a + 8.0f * cbrtf(a) + 8.0f));
}

struct MieArgs {
    int n_wl, n_groups, n_species;
    const double *wl, *nm_re, *nm_im, *np_re, *np_im, *radius, *vol_frac;
    const double *nc_re, *nc_im, *core_radius;   // core-shell species (NULL: none)
    const int* species_group;
    double *q_ext, *q_sca, *g_sp;
    double2* scratch;   // [n_cols * FOS_MIE_MAX_TERMS][T]
    long long T;
    unsigned* status;
    unsigned* large;    // set when some homogeneous sphere needs the chunked pass
    int inject;
};

__device__ __forceinline__ void flag(unsigned* st, unsigned bit, long long idx) {
    atomicOr(&st[ST_CALL], bit);
    atomicMin(&st[ST_INDEX], (unsigned)(idx < 0xffffffffLL ? idx : 0xfffffffeLL));
}

// Downward recurrence D_{n-1} = n/z - 1/(D_n + n/z) from D_{nstart} = 0; D_n stored for
// nlow <= n <= nt at col[(n - nbase) T] (orders below nlow are not needed by the caller;
// nbase = 1 stores order n at row n - 1).
__device__ __forceinline__ void downward_D(cx z, int nstart, int nt, double2* col, long long T,
                                           int nlow = 1, int nbase = 1) {
    const cx zi = crcp(z);
    cx D = mk(0.0, 0.0);
    for (int n = nstart; n >= nlow; --n) {
        if (n <= nt) col[(long long)(n - nbase) * T] = make_double2(D.re, D.im);
        const cx nz = (double)n * zi;
        const cx w = D + nz;   // D_{n-1} = nz - conj(w) / |w|^2
        const int e = max(exponent_field(w.re), exponent_field(w.im));
        if (e > 1023 + 490 || e < 1023 - 490) {
            D = nz - div_smith(mk(1.0, 0.0), w);
        } else {
            const double inv = 1.0 / (w.re * w.re + w.im * w.im);
            D = mk(fma(-w.re, inv, nz.re), fma(w.im, inv, nz.im));
        }
    }
}

// Running sums of Eqs. 11, 12 and 15; Eq. 11 is kept as the complex sum of
// (2n + 1)(a_n + b_n), multiplied by 1/n_m^2 once at the end.
struct Sums {
    double ext_re, ext_im, sca, g;
};

// Order weights of Eq. 15: m (m + 2) / (m + 1) and (2m + 1) / (m (m + 1)), m = 1 .. 511,
// evaluated by the compiler (IEEE double, as the kernel would) into constant memory.
struct Eq15Weights {
    double c1[FOS_MIE_MAX_TERMS], c2[FOS_MIE_MAX_TERMS];
    constexpr Eq15Weights() : c1(), c2() {
        for (int i = 1; i < FOS_MIE_MAX_TERMS; ++i) {
            const double m = (double)i;
            c1[i] = m * (m + 2.0) / (m + 1.0);
            c2[i] = (2.0 * m + 1.0) / (m * (m + 1.0));
        }
    }
};
__constant__ Eq15Weights g_eq15 = Eq15Weights();
// The weights of order m, from the table below FOS_MIE_MAX_TERMS and computed above it
// (large spheres only).
__device__ __forceinline__ double eq15_c1(int m) {
    return m < FOS_MIE_MAX_TERMS ? g_eq15.c1[m] : (double)m * ((double)m + 2.0) / ((double)m + 1.0);
}
__device__ __forceinline__ double eq15_c2(int m) {
    return m < FOS_MIE_MAX_TERMS ? g_eq15.c2[m]
                                 : (2.0 * (double)m + 1.0) / ((double)m * ((double)m + 1.0));
}

// Accumulates Eqs. 11, 12 and the numerator of 15 for order n given a_n, b_n and the
// previous order's coefficients.
__device__ __forceinline__ void accumulate(Sums& S, int n, int nmax, cx an, cx bn, cx a_prev,
                                           cx b_prev) {
    const double dn = (double)n;
    if (n <= nmax) {
        const double wgt = 2.0 * dn + 1.0;
        S.ext_re = fma(wgt, an.re + bn.re, S.ext_re);      // Eq. 11
        S.ext_im = fma(wgt, an.im + bn.im, S.ext_im);
        S.sca = fma(wgt, fma(an.re, an.re, fma(an.im, an.im, fma(bn.re, bn.re, bn.im * bn.im))),
                    S.sca);                                 // Eq. 12
    }
    if (n >= 2) {   // Eq. 15 term of order m = n-1 needs a_n, b_n
        const double t1 = a_prev.re * an.re + a_prev.im * an.im + b_prev.re * bn.re +
                          b_prev.im * bn.im;              // Re(a_m a_n^* + b_m b_n^*)
        const double t2 = a_prev.re * b_prev.re + a_prev.im * b_prev.im;   // Re(a_m b_m^*)
        S.g += eq15_c1(n - 1) * t1 + eq15_c2(n - 1) * t2;
    }
}

// Eqs. 10-12 and 15 from the sums; r is the (outer) radius.
__device__ __forceinline__ void efficiencies(const Sums& S, double lam, double r, cx n_m,
                                             cx inv_nm2, double* qe, double* qs, double* gg) {
    const double alpha = 4.0 * M_PI * r * n_m.im / lam;
    const double gam = gamma_term(alpha);
    const double scale = lam * lam / (2.0 * M_PI * M_PI * r * r);   // lambda^2 / (2 pi area)
    const double ext = S.ext_re * inv_nm2.re - S.ext_im * inv_nm2.im;   // Re(sum / n_m^2)
    *qe = scale * ext;
    *qs = scale * exp(-alpha) * S.sca / (gam * norm2(n_m));
    *gg = (S.sca > 0.0) ? 2.0 * S.g / S.sca : 0.0;
}

// Spheres whose orders exceed the scratch (FOS_MIE_MAX_TERMS orders per column): the same
// sums in chunks of that many orders, each chunk's D_n taken from a downward recurrence
// started at the same N* (so every order has the accuracy of one recurrence from N*), which
// repeats the downward work once per chunk.  It runs in a kernel of its own
// (mie_kernel<false, true>), so that the common single-chunk path keeps its registers.
__device__ bool sphere_eval_large(double lam, double r, cx n_p, cx n_m, double2* colY, double2* colX,
                            long long T, double* qe, double* qs, double* gg) {
    const double k = 2.0 * M_PI * r / lam;
    const cx x = k * n_m;   // Eq. 1
    const cx y = k * n_p;
    const double ay = size_abs(y), ax = size_abs(x);
    const int nmax = nmax_of(ay);
    const int nt = nmax + 1;          // a_{n+1}, b_{n+1} for Eq. 15
    const int nstart = nt + 16;
    const cx xi_ = crcp(x);
    // orders n <= n_up (n <= |x|, or all when |x| >= PSI_UPWARD_MIN_X) take psi_n(x) from
    // the upward recurrence; integer comparisons keep the per-order test off the FP64 pipe
    const bool up_all = ax >= PSI_UPWARD_MIN_X;
    const int n_up = up_all ? nt : (int)fmin(floor(ax), (double)nstart);
    cx psi_m1, psi_0, xi_m1;                                // cos x, sin x, e^{ix}
    start_values(x, psi_m1, psi_0, xi_m1);
    cx xi_0 = psi_0 - mk(-psi_m1.im, psi_m1.re);            // sin x - i cos x
    const cx inv_nm2 = crcp(n_m * n_m);
    const cx q = n_m / n_p, qi = n_p / n_m;
    Sums S{0.0, 0.0, 0.0, 0.0};
    cx a_prev = mk(0.0, 0.0), b_prev = mk(0.0, 0.0);
    // Early end of the sums.  Past n_w = |x| + 4.05 |x|^(1/3) + 2 (Wiscombe's count for the
    // host argument) psi_n(x) falls and xi_n(x) grows super-exponentially, and the terms
    // (2n + 1)(|a_n| + |b_n|) fall faster than geometrically (their ratio tends to
    // (|x| / (2n + 3))^2 < 1/4 there), so once two successive terms are below 2^-60 of the
    // partial sums, everything after them (the rest of Eqs. 11-12, and Eq. 15 with its
    // a_{n+1}) is below 2^-60 of the sums too.  The downward recurrences still start above
    // the n_max of Eq. 12's criterion, so every order used is as accurate as before.
    const int n_w = wiscombe_of(ax);
    const int n_last = up_all ? psi_upward_last(ax, nt) : nt;
    int small = 0;
    bool done = false;
    for (int c0 = 1; c0 <= n_last && !done; c0 += FOS_MIE_MAX_TERMS) {
        const int c1 = min(n_last, c0 + FOS_MIE_MAX_TERMS - 1);
        downward_D(y, nstart, c1, colY, T, c0, c0);
        if (c1 > n_up) downward_D(x, nstart, c1, colX, T, max(c0, n_up + 1), c0);
        for (int n = c0; n <= c1; ++n) {
            const double dn = (double)n;
            const cx c = (double)(2 * n - 1) * xi_, nx = dn * xi_;
            cx psi_n;
            if (n <= n_up) {
                psi_n = mul_sub(c, psi_0, psi_m1);
            } else {
                const double2 d = colX[(long long)(n - c0) * T];
                psi_n = psi_0 / (mk(d.x, d.y) + nx);
            }
            const cx xi_n = mul_sub(c, xi_0, xi_m1);
            // with psi_n' = psi_{n-1} - (n/x) psi_n (and the same for xi_n), q D psi_n - psi_n'
            // = (q D + n/x) psi_n - psi_{n-1}
            const double2 dy = colY[(long long)(n - c0) * T];
            const cx Dy = mk(dy.x, dy.y);
            const cx qa = mul_add(q, Dy, nx), qb = mul_add(qi, Dy, nx);
            cx an, bn;   // Eqs. 2 and 3
            div_pair(mul_sub(qa, psi_n, psi_0), mul_sub(qa, xi_n, xi_0), mul_sub(qb, psi_n, psi_0),
                     mul_sub(qb, xi_n, xi_0), an, bn);
            accumulate(S, n, nmax, an, bn, a_prev, b_prev);
            if (!up_all && n > n_w) {   // (up_all: the sums end at n_last)
                const double t = (2.0 * dn + 1.0) *
                                 (fabs(an.re) + fabs(an.im) + fabs(bn.re) + fabs(bn.im));
                const double ref = fabs(S.ext_re) + fabs(S.ext_im) + S.sca;
                small = (t < 0x1p-60 * ref) ? small + 1 : 0;
                if (small >= 2) {
                    done = true;
                    break;
                }
            }
            a_prev = an;
            b_prev = bn;
            psi_m1 = psi_0;
            psi_0 = psi_n;
            xi_m1 = xi_0;
            xi_0 = xi_n;
        }
    }
    efficiencies(S, lam, r, n_m, inv_nm2, qe, qs, gg);
    return true;
}

// Homogeneous sphere (Eqs. 1-5): D_n(y) downward; psi_n(x) upward (for |x| < 1.5 only
// while n <= |x|, and psi_{n-1}/(D_n(x) + n/x) above, D_n(x) downward); xi_n(x) upward; Eqs. 2-3
// multiplied through by psi_n(x) and xi_n(x), and a_n divided through by n_p, b_n by n_m:
// a_n = (q D_n(y) psi_n - psi_n') / (q D_n(y) xi_n - xi_n'), q = n_m / n_p, and b_n the
// same with 1/q; with the derivatives from the recurrence this is
// a_n = ((q D_n(y) + n/x) psi_n - psi_{n-1}) / ((q D_n(y) + n/x) xi_n - xi_{n-1}).
// Returns false (nothing computed) when n_max + 17 exceeds the scratch: such spheres are
// left to mie_kernel<false, true> and sphere_eval_large.
__device__ bool sphere_eval(double lam, double r, cx n_p, cx n_m, double2* colY, double2* colX,
                            long long T, double* qe, double* qs, double* gg) {
    const double k = 2.0 * M_PI * r / lam;
    const cx x = k * n_m;   // Eq. 1
    const cx y = k * n_p;
    const double ay = size_abs(y), ax = size_abs(x);
    const int nmax = nmax_of(ay);
    const int nt = nmax + 1;          // a_{n+1}, b_{n+1} for Eq. 15
    const int nstart = nt + 16;
    if (nstart > FOS_MIE_MAX_TERMS) return false;
    const cx xi_ = crcp(x);
    downward_D(y, nstart, nt, colY, T);
    // orders n <= n_up (n <= |x|, or all when |x| >= PSI_UPWARD_MIN_X) take psi_n(x) from
    // the upward recurrence; integer comparisons keep the per-order test off the FP64 pipe
    const bool up_all = ax >= PSI_UPWARD_MIN_X;
    const int n_up = up_all ? nt : (int)fmin(floor(ax), (double)nstart);
    if (!up_all) downward_D(x, nstart, nt, colX, T, n_up + 1);
    cx psi_m1, psi_0, xi_m1;                                // cos x, sin x, e^{ix}
    start_values(x, psi_m1, psi_0, xi_m1);
    cx xi_0 = psi_0 - mk(-psi_m1.im, psi_m1.re);            // sin x - i cos x
    const cx inv_nm2 = crcp(n_m * n_m);
    const cx q = n_m / n_p, qi = n_p / n_m;
    Sums S{0.0, 0.0, 0.0, 0.0};
    cx a_prev = mk(0.0, 0.0), b_prev = mk(0.0, 0.0);
    // Early end of the sums.  Past n_w = |x| + 4.05 |x|^(1/3) + 2 (Wiscombe's count for the
    // host argument) psi_n(x) falls and xi_n(x) grows super-exponentially, and the terms
    // (2n + 1)(|a_n| + |b_n|) fall faster than geometrically (their ratio tends to
    // (|x| / (2n + 3))^2 < 1/4 there), so once two successive terms are below 2^-60 of the
    // partial sums, everything after them (the rest of Eqs. 11-12, and Eq. 15 with its
    // a_{n+1}) is below 2^-60 of the sums too.  The downward recurrences still start above
    // the n_max of Eq. 12's criterion, so every order used is as accurate as before.
    const int n_w = wiscombe_of(ax);
    const int n_last = up_all ? psi_upward_last(ax, nt) : nt;
    int small = 0;
    for (int n = 1; n <= n_last; ++n) {
        const double dn = (double)n;
        const cx c = (double)(2 * n - 1) * xi_, nx = dn * xi_;
        cx psi_n;
        if (n <= n_up) {
            psi_n = mul_sub(c, psi_0, psi_m1);
        } else {
            const double2 d = colX[(long long)(n - 1) * T];
            psi_n = psi_0 / (mk(d.x, d.y) + nx);
        }
        const cx xi_n = mul_sub(c, xi_0, xi_m1);
        // with psi_n' = psi_{n-1} - (n/x) psi_n (and the same for xi_n), q D psi_n - psi_n'
        // = (q D + n/x) psi_n - psi_{n-1}
        const double2 dy = colY[(long long)(n - 1) * T];
        const cx Dy = mk(dy.x, dy.y);
        const cx qa = mul_add(q, Dy, nx), qb = mul_add(qi, Dy, nx);
        cx an, bn;   // Eqs. 2 and 3
        div_pair(mul_sub(qa, psi_n, psi_0), mul_sub(qa, xi_n, xi_0), mul_sub(qb, psi_n, psi_0),
                 mul_sub(qb, xi_n, xi_0), an, bn);
        accumulate(S, n, nmax, an, bn, a_prev, b_prev);
        if (!up_all && n > n_w) {   // (up_all: the sums end at n_last)
            const double t = (2.0 * dn + 1.0) *
                             (fabs(an.re) + fabs(an.im) + fabs(bn.re) + fabs(bn.im));
            const double ref = fabs(S.ext_re) + fabs(S.ext_im) + S.sca;
            small = (t < 0x1p-60 * ref) ? small + 1 : 0;
            if (small >= 2) break;
        }
        a_prev = an;
        b_prev = bn;
        psi_m1 = psi_0;
        psi_0 = psi_n;
        xi_m1 = xi_0;
        xi_0 = xi_n;
    }
    efficiencies(S, lam, r, n_m, inv_nm2, qe, qs, gg);
    return true;
}

// Riccati-Bessel psi_n(z), chi_n(z) = z y_n(z) one order up: psi by upward recurrence
// while n <= |z| and psi_{n-1}/(D_n + n/z) above; chi by upward recurrence.
struct RB {
    cx zi;
    int n_up;                        // orders n <= |z|: psi by the upward recurrence
    cx psi_m1, psi0, chi_m1, chi0;   // orders n-2, n-1
};
__device__ __forceinline__ void rb_init(RB& R, cx z) {
    R.zi = crcp(z);
    R.n_up = (int)fmin(floor(cabs_(z)), (double)FOS_MIE_MAX_TERMS);
    R.psi_m1 = ccos(z);
    R.psi0 = csin(z);
    R.chi_m1 = csin(z);
    R.chi0 = mk(0.0, 0.0) - ccos(z);
}
// advances to order n; returns psi_n, chi_n and their derivatives
__device__ __forceinline__ void rb_step(RB& R, int n, const double2* colD, long long T, cx& psi,
                                        cx& dpsi, cx& chi, cx& dchi) {
    const double dn = (double)n;
    const cx c = (double)(2 * n - 1) * R.zi;
    const cx nz = dn * R.zi;
    if (n <= R.n_up) {
        psi = mul_sub(c, R.psi0, R.psi_m1);
    } else {
        const double2 d = colD[(long long)(n - 1) * T];
        psi = R.psi0 / (mk(d.x, d.y) + nz);
    }
    chi = mul_sub(c, R.chi0, R.chi_m1);
    dpsi = sub_mul(R.psi0, nz, psi);
    dchi = sub_mul(R.chi0, nz, chi);
    R.psi_m1 = R.psi0;
    R.psi0 = psi;
    R.chi_m1 = R.chi0;
    R.chi0 = chi;
}

// Core-shell sphere (supplement Eqs. S1-S9): core radius a (index n_c), outer radius b
// (shell index n_s), host n_m; m1 = n_c/n_m, m2 = n_s/n_m, x = k a, y = k b.
// A_n, B_n (S3, S4) divided through by psi_n(m1 x), i.e. with D_n(m1 x); chi_n = z y_n(z)
// (S8); xi_n = psi_n + i chi_n (S9).  Four downward D columns: m1 x, m2 x, m2 y, y.
__device__ bool coated_eval(double lam, double a, double b, cx n_c, cx n_s, cx n_m,
                            double2* col0, double2* col1, double2* col2, double2* col3,
                            long long T, double* qe, double* qs, double* gg) {
    const double kv = 2.0 * M_PI / lam;
    const cx x = (kv * a) * n_m, y = (kv * b) * n_m;
    const cx inv_nm = crcp(n_m);
    const cx m1 = n_c * inv_nm, m2 = n_s * inv_nm;
    const double ymax = kv * b * fmax(cabs_(n_c), cabs_(n_s));
    const int nmax = (int)ceil(2.0 + ymax + 4.3 * cbrt(ymax));
    const int nt = nmax + 1;
    const int nstart = nt + 16;
    if (nstart > FOS_MIE_MAX_TERMS) return false;
    const cx z1 = m1 * x, z2x = m2 * x, z2y = m2 * y;
    downward_D(z1, nstart, nt, col0, T);
    downward_D(z2x, nstart, nt, col1, T);
    downward_D(z2y, nstart, nt, col2, T);
    downward_D(y, nstart, nt, col3, T);
    RB r2x, r2y, ry;
    rb_init(r2x, z2x);
    rb_init(r2y, z2y);
    rb_init(ry, y);
    const cx inv_nm2 = inv_nm * inv_nm;
    const cx I = mk(0.0, 1.0);
    Sums S{0.0, 0.0, 0.0, 0.0};
    cx a_prev = mk(0.0, 0.0), b_prev = mk(0.0, 0.0);
    for (int n = 1; n <= nt; ++n) {
        cx ps2x, dps2x, ch2x, dch2x, ps2y, dps2y, ch2y, dch2y, psy, dpsy, chy, dchy;
        rb_step(r2x, n, col1, T, ps2x, dps2x, ch2x, dch2x);
        rb_step(r2y, n, col2, T, ps2y, dps2y, ch2y, dch2y);
        rb_step(ry, n, col3, T, psy, dpsy, chy, dchy);
        const double2 d1 = col0[(long long)(n - 1) * T];
        const cx D1 = mk(d1.x, d1.y);                        // psi'/psi at m1 x
        const cx D2x = dps2x / ps2x;
        const cx m2D1 = m2 * D1, m1D2 = m1 * D2x;
        const cx An = ps2x * (m2D1 - m1D2) / (m2D1 * ch2x - m1 * dch2x);            // S3
        const cx Bn = ps2x * (m2 * D2x - m1 * D1) / (m2 * dch2x - m1 * D1 * ch2x);  // S4
        const cx xi = psy + I * chy, dxi = dpsy + I * dchy;                          // S9
        const cx Ua = dps2y - An * dch2y, Va = ps2y - An * ch2y;
        const cx Ub = dps2y - Bn * dch2y, Vb = ps2y - Bn * ch2y;
        const cx an = (psy * Ua - m2 * dpsy * Va) / (xi * Ua - m2 * dxi * Va);       // S1
        const cx bn = (m2 * psy * Ub - dpsy * Vb) / (m2 * xi * Ub - dxi * Vb);       // S2
        accumulate(S, n, nmax, an, bn, a_prev, b_prev);
        a_prev = an;
        b_prev = bn;
    }
    efficiencies(S, lam, b, n_m, inv_nm2, qe, qs, gg);
    return true;
}

// CS = false: homogeneous spheres only (the core-shell code is compiled out, which keeps
// the register count of the common case low); CS = true: either kind per species.
// LARGE = false: every species whose orders fit the scratch; homogeneous spheres that do
// not are left for the LARGE = true pass (flagged in A.large), which does only those, in
// chunks of orders, and returns at once when there are none.
template <bool CS, bool LARGE = false>
__global__ void __launch_bounds__(128) mie_kernel(MieArgs A) {
    if (LARGE && *A.large == 0u) return;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (!LARGE && A.inject && tid == 0) atomicOr(&A.status[ST_CALL], DEV_INJECTED);
    const long long n_eval = (long long)A.n_species * A.n_wl;
    const long long col = (long long)FOS_MIE_MAX_TERMS * A.T;
    double2* c0 = A.scratch + tid;
    for (long long ev = tid; ev < n_eval; ev += A.T) {
        const int s = (int)(ev / A.n_wl), w = (int)(ev % A.n_wl);
        const int gi = A.species_group[s];
        const double lam = A.wl[w], r = A.radius[s];
        bool ok = gi >= 0 && gi < A.n_groups && (s == 0 || A.species_group[s - 1] <= gi);
        const long long gw = ok ? (long long)gi * A.n_wl + w : 0;
        const cx n_p = mk(A.np_re[ev], A.np_im[ev]);
        const cx n_m = mk(A.nm_re[gw], A.nm_im[gw]);
        const double f = A.vol_frac[s];
        const double a = CS ? A.core_radius[s] : 0.0;
        cx n_c = mk(1.0, 0.0);
        if (a > 0.0) n_c = mk(A.nc_re[ev], A.nc_im[ev]);
        ok = ok && isfinite(lam) && lam > 0.0 && isfinite(r) && r > 0.0 &&
             isfinite(n_p.re) && n_p.re > 0.0 && isfinite(n_p.im) && n_p.im >= 0.0 &&
             isfinite(n_m.re) && n_m.re > 0.0 && isfinite(n_m.im) && n_m.im >= 0.0 &&
             f >= 0.0 && f < 1.0 && a >= 0.0 && a < r && isfinite(n_c.re) && n_c.re > 0.0 &&
             isfinite(n_c.im) && n_c.im >= 0.0;
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        double qe = nanv, qs = nanv, gg = nanv;
        if (LARGE) {
            // homogeneous spheres beyond the scratch only (the first pass validated them)
            if (!ok || a > 0.0) continue;
            // the same test as sphere_eval's (the same arithmetic)
            if (nmax_of(size_abs((2.0 * M_PI * r / lam) * n_p)) + 17 <= FOS_MIE_MAX_TERMS) continue;
            sphere_eval_large(lam, r, n_p, n_m, c0, c0 + col, A.T, &qe, &qs, &gg);
        } else if (!ok) {
            flag(A.status, DEV_INVALID, ev);
        } else {
            bool fit;
            if (CS && a > 0.0) {
                fit = coated_eval(lam, a, r, n_c, n_p, n_m, c0, c0 + col, c0 + 2 * col,
                                  c0 + 3 * col, A.T, &qe, &qs, &gg);
                if (!fit) flag(A.status, DEV_RANGE, ev);
            } else {
                fit = sphere_eval(lam, r, n_p, n_m, c0, c0 + col, A.T, &qe, &qs, &gg);
                if (!fit) {   // left to the LARGE pass
                    atomicOr(A.large, 1u);
                    continue;
                }
            }
        }
        A.q_ext[ev] = qe;
        A.q_sca[ev] = qs;
        A.g_sp[ev] = gg;
    }
}

struct EmtArgs {
    int n_wl, n_groups, n_species;
    const double *wl, *nm_im, *nm_re, *radius, *vol_frac;
    const int* species_group;
    const double *q_ext, *q_sca, *g_sp;
    double *mu_s, *mu_a, *g;
    unsigned* status;
};

__device__ __forceinline__ int lower_bound(const int* a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void emt_kernel(EmtArgs A) {
    const long long total = (long long)A.n_groups * A.n_wl;
    for (long long gw = blockIdx.x * (long long)blockDim.x + threadIdx.x; gw < total;
         gw += (long long)gridDim.x * blockDim.x) {
        int gi, w;
        if (total <= 0xffffffffLL) {   // 32-bit division where the count allows it
            gi = (int)((unsigned)gw / (unsigned)A.n_wl);
            w = (int)((unsigned)gw - (unsigned)gi * (unsigned)A.n_wl);
        } else {
            gi = (int)(gw / A.n_wl);
            w = (int)(gw % A.n_wl);
        }
        const int s0 = lower_bound(A.species_group, A.n_species, gi);
        const int s1 = lower_bound(A.species_group, A.n_species, gi + 1);
        const double lam = A.wl[w];
        double sum_f = 0.0, ms = 0.0, ma = 0.0, mg = 0.0;
        for (int s = s0; s < s1; ++s) {
            const long long sw = (long long)s * A.n_wl + w;
            const double f = A.vol_frac[s], rr = A.radius[s];
            const double qe = A.q_ext[sw], qs = A.q_sca[sw], gg = A.g_sp[sw];
            const double k = 0.75 * f / rr;            // 3 f / (4 r): one division
            sum_f += f;
            ms += qs * k;                              // Eq. 13
            ma += (qe - qs) * k;                       // Eq. 14
            mg += qs * gg * k;                         // numerator of Eq. 16
        }
        const double km = A.nm_im[gw], nr = A.nm_re[gw];
        if (!(sum_f < 1.0) || !(isfinite(km) && km >= 0.0) || !(isfinite(nr) && nr > 0.0) ||
            !(isfinite(lam) && lam > 0.0)) {
            atomicOr(&A.status[ST_CALL], DEV_INVALID);
        }
        double gv = (ms > 0.0) ? mg / ms : 0.0;        // Eq. 16
        if (ms < 0.0) ms = 0.0;                        // negative coefficients -> 0
        if (ma < 0.0) ma = 0.0;
        if (sum_f > 0.08) {                            // Eqs. 17-19
            const double C = 1.0 + 1.5 * sum_f - 0.75 * sum_f * sum_f;
            ms *= C;
            ma *= C;
        }
        ma += 4.0 * M_PI * km * (1.0 - sum_f) / lam;   // Eq. 20
        A.mu_s[gw] = ms;
        A.mu_a[gw] = ma;
        A.g[gw] = gv;
    }
}

}  // namespace mie
}  // namespace fos

using namespace fos;

static fos_status mie_impl(int n_wl, const double* wl, int n_groups, const double* nm_re,
                           const double* nm_im, int n_species, const int* species_group,
                           const double* np_re, const double* np_im, const double* nc_re,
                           const double* nc_im, const double* radius, const double* core_radius,
                           const double* vol_frac, double* mu_s, double* mu_a, double* g,
                           double* q_ext, double* q_sca, double* g_species, unsigned flags,
                           void* stream) {
    NvtxRange nvtx("fos_mie_properties");
    if (n_wl < 1 || n_groups < 1 || n_species < 0) return FOS_ERR_INVALID_ARG;
    if ((long long)n_groups * n_wl > 0x7fffffffLL || (long long)n_species * n_wl > 0x7fffffffLL)
        return FOS_ERR_INVALID_ARG;
    if (!wl || !nm_re || !nm_im || !mu_s || !mu_a || !g) return FOS_ERR_INVALID_ARG;
    if (n_species > 0 && (!species_group || !np_re || !np_im || !radius || !vol_frac))
        return FOS_ERR_INVALID_ARG;
    if (core_radius && n_species > 0 && (!nc_re || !nc_im)) return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    if (ws->cc_major != 10) return FOS_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n_eval = (long long)n_species * n_wl;
    const int block = 128;
    const int n_cols = core_radius ? 4 : 2;   // downward log-derivative columns per thread
    // 4 blocks of 128 threads per SM, so that several warps hide the FP64 latency; the
    // scratch holds the log-derivative columns of every thread (n_cols x 512 orders x
    // 16 B each)
    long long T = (long long)ws->num_sms * 128 * 4;
    const long long need_T = ((n_eval + block - 1) / block) * block;
    if (need_T < T) T = need_T > 0 ? need_T : block;
    const size_t scratch_bytes = (size_t)n_cols * FOS_MIE_MAX_TERMS * T * sizeof(double2);
    const bool own_q = !(q_ext && q_sca && g_species);
    const size_t qbytes = own_q ? (size_t)3 * n_eval * sizeof(double) + 1024 : 0;
    st = ensure_buffer(ws, &ws->mie_scratch, &ws->mie_bytes, scratch_bytes + qbytes);
    if (st != FOS_OK) return st;
    double* qbase = (double*)((char*)ws->mie_scratch + scratch_bytes);
    double* qe = q_ext ? q_ext : qbase;
    double* qs = q_sca ? q_sca : qbase + n_eval;
    double* gs = g_species ? g_species : qbase + 2 * n_eval;
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_CALL, 0, sizeof(unsigned), s));
    FOS_CUDA_TRY(cudaMemsetAsync(ws->status + ST_INDEX, 0xff, sizeof(unsigned), s));
    if (n_eval > 0 || (flags & FOS_TEST_INJECT)) {
        mie::MieArgs ma;
        ma.n_wl = n_wl;
        ma.n_groups = n_groups;
        ma.n_species = n_species;
        ma.wl = wl;
        ma.nm_re = nm_re;
        ma.nm_im = nm_im;
        ma.np_re = np_re;
        ma.np_im = np_im;
        ma.nc_re = nc_re;
        ma.nc_im = nc_im;
        ma.core_radius = core_radius;
        ma.radius = radius;
        ma.vol_frac = vol_frac;
        ma.species_group = species_group;
        ma.q_ext = qe;
        ma.q_sca = qs;
        ma.g_sp = gs;
        ma.scratch = (double2*)ws->mie_scratch;
        ma.T = T;
        ma.status = ws->status;
        ma.large = ws->status + 3;   // spare word of the status region
        ma.inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
        FOS_CUDA_TRY(cudaMemsetAsync(ma.large, 0, sizeof(unsigned), s));
        if (core_radius)
            mie::mie_kernel<true><<<(unsigned)(T / block), block, 0, s>>>(ma);
        else
            mie::mie_kernel<false><<<(unsigned)(T / block), block, 0, s>>>(ma);
        FOS_CUDA_TRY(cudaGetLastError());
        mie::mie_kernel<false, true><<<(unsigned)(T / block), block, 0, s>>>(ma);
        FOS_CUDA_TRY(cudaGetLastError());
    }
    mie::EmtArgs ea;
    ea.n_wl = n_wl;
    ea.n_groups = n_groups;
    ea.n_species = n_species;
    ea.wl = wl;
    ea.nm_im = nm_im;
    ea.nm_re = nm_re;
    ea.radius = radius;
    ea.vol_frac = vol_frac;
    ea.species_group = species_group;
    ea.q_ext = qe;
    ea.q_sca = qs;
    ea.g_sp = gs;
    ea.mu_s = mu_s;
    ea.mu_a = mu_a;
    ea.g = g;
    ea.status = ws->status;
    const long long total = (long long)n_groups * n_wl;
    long long eb = (total + 255) / 256;
    if (eb > (long long)ws->num_sms * 32) eb = (long long)ws->num_sms * 32;
    mie::emt_kernel<<<(unsigned)eb, 256, 0, s>>>(ea);
    FOS_CUDA_TRY(cudaGetLastError());
    return finish_call(ws, s, flags);
}

extern "C" fos_status fos_mie_properties(int n_wl, const double* wl, int n_groups,
                                         const double* nm_re, const double* nm_im,
                                         int n_species, const int* species_group,
                                         const double* np_re, const double* np_im,
                                         const double* radius, const double* vol_frac,
                                         double* mu_s, double* mu_a, double* g, double* q_ext,
                                         double* q_sca, double* g_species, unsigned flags,
                                         void* stream) {
    return mie_impl(n_wl, wl, n_groups, nm_re, nm_im, n_species, species_group, np_re, np_im,
                    nullptr, nullptr, radius, nullptr, vol_frac, mu_s, mu_a, g, q_ext, q_sca,
                    g_species, flags, stream);
}

extern "C" fos_status fos_mie_properties_cs(int n_wl, const double* wl, int n_groups,
                                            const double* nm_re, const double* nm_im,
                                            int n_species, const int* species_group,
                                            const double* ns_re, const double* ns_im,
                                            const double* nc_re, const double* nc_im,
                                            const double* radius, const double* core_radius,
                                            const double* vol_frac, double* mu_s, double* mu_a,
                                            double* g, double* q_ext, double* q_sca,
                                            double* g_species, unsigned flags, void* stream) {
    if (n_species > 0 && !core_radius) return FOS_ERR_INVALID_ARG;
    return mie_impl(n_wl, wl, n_groups, nm_re, nm_im, n_species, species_group, ns_re, ns_im,
                    nc_re, nc_im, radius, core_radius, vol_frac, mu_s, mu_a, g, q_ext, q_sca,
                    g_species, flags, stream);
}

// Particle-size distribution (section "Scattering properties", last paragraph): one
// diameter D with standard deviation sigma becomes n diameters evenly spaced over
// D +- 3 sigma; each carries the share of the volume fraction given by its Gaussian
// weight exp(-(D_i - D)^2 / (2 sigma^2)), the weights normalised to sum to 1.
// Diameters <= 0 are dropped and the remaining weights renormalised.  Host arrays.
extern "C" fos_status fos_size_distribution(double diameter, double sigma, double vol_frac,
                                            int n, double* radius, double* vol_fracs,
                                            int* n_out) {
    if (!radius || !vol_fracs || !n_out) return FOS_ERR_INVALID_ARG;
    if (!(diameter > 0.0) || !(sigma >= 0.0) || !(vol_frac >= 0.0 && vol_frac < 1.0) || n < 1)
        return FOS_ERR_INVALID_ARG;
    if (sigma == 0.0 || n == 1) {
        radius[0] = 0.5 * diameter;
        vol_fracs[0] = vol_frac;
        *n_out = 1;
        return FOS_OK;
    }
    if (n % 2 == 0) return FOS_ERR_INVALID_ARG;   // odd: the centre size is one of them
    const double step = 6.0 * sigma / (double)(n - 1);
    double wsum = 0.0;
    int k = 0;
    for (int i = 0; i < n; ++i) {
        const double d = diameter - 3.0 * sigma + step * (double)i;
        if (!(d > 0.0)) continue;
        const double u = (d - diameter) / sigma;
        const double w = exp(-0.5 * u * u);
        radius[k] = 0.5 * d;
        vol_fracs[k] = w;
        wsum += w;
        ++k;
    }
    for (int i = 0; i < k; ++i) vol_fracs[i] = vol_frac * (vol_fracs[i] / wsum);
    *n_out = k;
    return FOS_OK;
}
