// Mie theory + effective medium on GB300, FP64 (arxiv 2409.00165, section
// "Scattering properties", Eqs. 1-20).
//
// mie_kernel: one thread per (species, wavelength), grid-stride.  The logarithmic
//   derivative D_n(z) = psi_n'(z)/psi_n(z) of psi_n(z) = z j_n(z) (A_n of Eq. 4) comes
//   from the downward recurrence D_{n-1} = n/z - 1/(D_n + n/z) started at
//   N* = n_max + 17 with D = 0, for the particle argument y and the host argument x.
//   The values are kept in a scratch laid out [order][thread] so that a warp's
//   accesses coalesce.  An upward sweep then builds psi_n(x) (upward recurrence
//   while n <= |x|, psi_{n-1}/(D_n(x) + n/x) above) and xi_n(x) = x h^(1)_n(x)
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
// (no intermediate overflow) when |b| is outside [1e-150, 1e150].
__device__ __forceinline__ cx div_smith(cx a, cx b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return cx{(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    } else {
        const double r = b.re / b.im, d = b.re * r + b.im;
        return cx{(a.re * r + a.im) / d, (a.im * r - a.re) / d};
    }
}
__device__ __forceinline__ cx operator/(cx a, cx b) {
    const double m = fmax(fabs(b.re), fabs(b.im));
    if (m > 1e150 || m < 1e-150) return div_smith(a, b);
    const double inv = 1.0 / (b.re * b.re + b.im * b.im);
    return cx{(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}
__device__ __forceinline__ double norm2(cx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double cabs_(cx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ cx csin(cx z) {
    return cx{sin(z.re) * cosh(z.im), cos(z.re) * sinh(z.im)};
}
__device__ __forceinline__ cx ccos(cx z) {
    return cx{cos(z.re) * cosh(z.im), -sin(z.re) * sinh(z.im)};
}

// Geometric term of Eq. 10 with alpha = 4 pi r k_m / lambda.  Below alpha = 0.5 the
// bracket cancels, so its Taylor series 2 sum_{k>=2} (k-1)/k! alpha^(k-2) is used
// (19 terms: the next one is < 1e-18 at alpha = 0.5).
__device__ __forceinline__ double gamma_term(double a) {
    if (a < 0.5) {
        double sum = 0.0, pw = 1.0, fact = 2.0;   // i = 0: 2 * 1 / 2!
        for (int i = 0; i < 19; ++i) {
            if (i > 0) {
                pw *= a;
                fact *= (double)(i + 2);
            }
            sum += 2.0 * (double)(i + 1) / fact * pw;
        }
        return sum;
    }
    return 2.0 * (1.0 + (a - 1.0) * exp(a)) / (a * a);
}

struct MieArgs {
    int n_wl, n_groups, n_species;
    const double *wl, *nm_re, *nm_im, *np_re, *np_im, *radius, *vol_frac;
    const int* species_group;
    double *q_ext, *q_sca, *g_sp;
    double2* scratch;   // [2*FOS_MIE_MAX_TERMS][T]
    long long T;
    unsigned* status;
    int inject;
};

__device__ __forceinline__ void flag(unsigned* st, unsigned bit, long long idx) {
    atomicOr(&st[ST_CALL], bit);
    atomicMin(&st[ST_INDEX], (unsigned)(idx < 0xffffffffLL ? idx : 0xfffffffeLL));
}

__global__ void __launch_bounds__(128) mie_kernel(MieArgs A) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (A.inject && tid == 0) atomicOr(&A.status[ST_CALL], DEV_INJECTED);
    const long long n_eval = (long long)A.n_species * A.n_wl;
    double2* colY = A.scratch + tid;                                    // D_n(y) at [n-1][T]
    double2* colX = A.scratch + (long long)FOS_MIE_MAX_TERMS * A.T + tid;  // D_n(x)
    for (long long ev = tid; ev < n_eval; ev += A.T) {
        const int s = (int)(ev / A.n_wl), w = (int)(ev % A.n_wl);
        const int gi = A.species_group[s];
        const double lam = A.wl[w], r = A.radius[s];
        bool ok = gi >= 0 && gi < A.n_groups && (s == 0 || A.species_group[s - 1] <= gi);
        const long long gw = ok ? (long long)gi * A.n_wl + w : 0;
        const cx n_p = mk(A.np_re[ev], A.np_im[ev]);
        const cx n_m = mk(A.nm_re[gw], A.nm_im[gw]);
        const double f = A.vol_frac[s];
        ok = ok && isfinite(lam) && lam > 0.0 && isfinite(r) && r > 0.0 &&
             isfinite(n_p.re) && n_p.re > 0.0 && isfinite(n_p.im) && n_p.im >= 0.0 &&
             isfinite(n_m.re) && n_m.re > 0.0 && isfinite(n_m.im) && n_m.im >= 0.0 &&
             f >= 0.0 && f < 1.0;
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        if (!ok) {
            flag(A.status, DEV_INVALID, ev);
            A.q_ext[ev] = nanv;
            A.q_sca[ev] = nanv;
            A.g_sp[ev] = nanv;
            continue;
        }
        const double k = 2.0 * M_PI * r / lam;
        const cx x = k * n_m;   // Eq. 1
        const cx y = k * n_p;
        const double ay = cabs_(y), ax = cabs_(x);
        const int nmax = (int)ceil(2.0 + ay + 4.3 * cbrt(ay));
        const int nt = nmax + 1;          // a_{n+1}, b_{n+1} for Eq. 15
        const int nstart = nt + 16;
        if (nstart > FOS_MIE_MAX_TERMS) {
            flag(A.status, DEV_RANGE, ev);
            A.q_ext[ev] = nanv;
            A.q_sca[ev] = nanv;
            A.g_sp[ev] = nanv;
            continue;
        }
        const cx yi = mk(1.0, 0.0) / y;
        const cx xi_ = mk(1.0, 0.0) / x;
        // downward recurrences, D_{nstart} = 0
        {
            cx Dy = mk(0.0, 0.0), Dx = mk(0.0, 0.0);
            for (int n = nstart; n >= 1; --n) {
                if (n <= nt) {
                    colY[(long long)(n - 1) * A.T] = make_double2(Dy.re, Dy.im);
                    colX[(long long)(n - 1) * A.T] = make_double2(Dx.re, Dx.im);
                }
                const cx ny = (double)n * yi, nx = (double)n * xi_;
                Dy = ny - mk(1.0, 0.0) / (Dy + ny);
                Dx = nx - mk(1.0, 0.0) / (Dx + nx);
            }
        }
        // upward sweep
        cx psi_m1 = ccos(x), psi_0 = csin(x);
        const double eb = exp(-x.im);
        cx xi_m1 = mk(eb * cos(x.re), eb * sin(x.re));        // e^{ix}
        cx xi_0 = psi_0 - mk(-psi_m1.im, psi_m1.re);            // sin x - i cos x
        const cx inv_nm2 = mk(1.0, 0.0) / (n_m * n_m);
        double s_ext = 0.0, s_sca = 0.0, s_g = 0.0;
        cx a_prev = mk(0.0, 0.0), b_prev = mk(0.0, 0.0);
        for (int n = 1; n <= nt; ++n) {
            const double dn = (double)n;
            cx psi_n;
            if (dn <= ax) {
                psi_n = (double)(2 * n - 1) * xi_ * psi_0 - psi_m1;
            } else {
                const double2 d = colX[(long long)(n - 1) * A.T];
                psi_n = psi_0 / (mk(d.x, d.y) + dn * xi_);
            }
            const cx xi_n = (double)(2 * n - 1) * xi_ * xi_0 - xi_m1;
            const cx dpsi = psi_0 - dn * xi_ * psi_n;
            const cx dxi = xi_0 - dn * xi_ * xi_n;
            const double2 dy = colY[(long long)(n - 1) * A.T];
            const cx Dy = mk(dy.x, dy.y);
            const cx mDy = n_m * Dy, pDy = n_p * Dy;
            const cx an = (mDy * psi_n - n_p * dpsi) / (mDy * xi_n - n_p * dxi);   // Eq. 2
            const cx bn = (pDy * psi_n - n_m * dpsi) / (pDy * xi_n - n_m * dxi);   // Eq. 3
            if (n <= nmax) {
                const double wgt = 2.0 * dn + 1.0;
                s_ext += wgt * ((an + bn) * inv_nm2).re;           // Eq. 11
                s_sca += wgt * (norm2(an) + norm2(bn));             // Eq. 12
            }
            if (n >= 2) {   // Eq. 15 term of order m = n-1 needs a_n, b_n
                const double m = dn - 1.0;
                const double t1 = a_prev.re * an.re + a_prev.im * an.im +
                                  b_prev.re * bn.re + b_prev.im * bn.im;   // Re(a_m a_n^* + b_m b_n^*)
                const double t2 = a_prev.re * b_prev.re + a_prev.im * b_prev.im;  // Re(a_m b_m^*)
                s_g += m * (m + 2.0) / (m + 1.0) * t1 + (2.0 * m + 1.0) / (m * (m + 1.0)) * t2;
            }
            a_prev = an;
            b_prev = bn;
            psi_m1 = psi_0;
            psi_0 = psi_n;
            xi_m1 = xi_0;
            xi_0 = xi_n;
        }
        const double alpha = 4.0 * M_PI * r * n_m.im / lam;
        const double gam = gamma_term(alpha);
        const double c_ext = lam * lam / (2.0 * M_PI) * s_ext;
        const double c_sca = lam * lam * exp(-alpha) / (2.0 * M_PI * gam * norm2(n_m)) * s_sca;
        const double area = M_PI * r * r;
        A.q_ext[ev] = c_ext / area;
        A.q_sca[ev] = c_sca / area;
        A.g_sp[ev] = (s_sca > 0.0) ? 2.0 * s_g / s_sca : 0.0;
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
        const int gi = (int)(gw / A.n_wl), w = (int)(gw % A.n_wl);
        const int s0 = lower_bound(A.species_group, A.n_species, gi);
        const int s1 = lower_bound(A.species_group, A.n_species, gi + 1);
        const double lam = A.wl[w];
        double sum_f = 0.0, ms = 0.0, ma = 0.0, mg = 0.0;
        for (int s = s0; s < s1; ++s) {
            const long long sw = (long long)s * A.n_wl + w;
            const double f = A.vol_frac[s], rr = A.radius[s];
            const double qe = A.q_ext[sw], qs = A.q_sca[sw], gg = A.g_sp[sw];
            sum_f += f;
            ms += 1.5 * qs * f / (2.0 * rr);           // Eq. 13
            ma += 1.5 * (qe - qs) * f / (2.0 * rr);    // Eq. 14
            mg += 1.5 * qs * f * gg / (2.0 * rr);      // numerator of Eq. 16
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

extern "C" fos_status fos_mie_properties(int n_wl, const double* wl, int n_groups,
                                         const double* nm_re, const double* nm_im,
                                         int n_species, const int* species_group,
                                         const double* np_re, const double* np_im,
                                         const double* radius, const double* vol_frac,
                                         double* mu_s, double* mu_a, double* g, double* q_ext,
                                         double* q_sca, double* g_species, unsigned flags,
                                         void* stream) {
    if (n_wl < 1 || n_groups < 1 || n_species < 0) return FOS_ERR_INVALID_ARG;
    if ((long long)n_groups * n_wl > 0x7fffffffLL || (long long)n_species * n_wl > 0x7fffffffLL)
        return FOS_ERR_INVALID_ARG;
    if (!wl || !nm_re || !nm_im || !mu_s || !mu_a || !g) return FOS_ERR_INVALID_ARG;
    if (n_species > 0 && (!species_group || !np_re || !np_im || !radius || !vol_frac))
        return FOS_ERR_INVALID_ARG;
    Workspace* ws = nullptr;
    fos_status st = get_workspace(&ws);
    if (st != FOS_OK) return st;
    if (ws->cc_major != 10) return FOS_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n_eval = (long long)n_species * n_wl;
    const int block = 128;
    long long T = (long long)ws->num_sms * 128;
    const long long need_T = ((n_eval + block - 1) / block) * block;
    if (need_T < T) T = need_T > 0 ? need_T : block;
    const size_t scratch_bytes = (size_t)2 * FOS_MIE_MAX_TERMS * T * sizeof(double2);
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
        ma.radius = radius;
        ma.vol_frac = vol_frac;
        ma.species_group = species_group;
        ma.q_ext = qe;
        ma.q_sca = qs;
        ma.g_sp = gs;
        ma.scratch = (double2*)ws->mie_scratch;
        ma.T = T;
        ma.status = ws->status;
        ma.inject = (flags & FOS_TEST_INJECT) ? 1 : 0;
        mie::mie_kernel<<<(unsigned)(T / block), block, 0, s>>>(ma);
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
