/*
 * fos.h - C ABI of libfos: the GB300 hot path of FOS (arxiv 2409.00165, "FOS: Fast
 * Optical Spectrum calculations of nanoparticle media").
 *
 * The library computes the spectral reflectance, absorptance and transmittance of
 * particle-filled layers:
 *   fos_mie_properties  Mie theory + effective medium -> mu_s, mu_a, g per layer and
 *                       wavelength (section "Scattering properties", Eqs. 1-20);
 *                       fos_mie_properties_cs adds core-shell spheres (supplement Eqs.
 *                       S1-S9) and fos_size_distribution expands a size distribution.
 *   fos_mc_spectrum     Monte Carlo photon transport through layer stacks -> integer
 *                       photon counts R, A, T per (stack, wavelength), at normal or
 *                       oblique incidence, over a dielectric, a conductor or a reflector
 *                       (section "Photon transport").
 *   fos_solar_weighted  solar-weighted R, A, T of a spectrum (section "Output", Eq. 21).
 *   fos_surrogate_*     a learned MLP that predicts R, A, T from (wavelength, n, k,
 *                       radius, volume fraction, thickness, g, mu_s, mu_a), or from the
 *                       slab inputs of Table 1, trained on spectra from fos_mc_spectrum
 *                       (the paper's "machine learning method" of section "Photon
 *                       transport").
 *   diagnostics         fos_philox4x32_10, fos_walk_math_f32, fos_walk_math_fast_f32
 *                       and fos_gemm_bf16 expose building blocks to the parity tests;
 *                       fos_mc_walk_times the per-block timing of a walk launch.
 *
 * Conventions for every entry point:
 *   - Plain C types only.  Pointers documented "device" point to CUDA device memory
 *     of the current device; pointers documented "host" to host memory.
 *   - The caller owns every buffer it passes.  The library owns only a per-device
 *     workspace (work queue, status word, packed item tables, Mie scratch) that it
 *     allocates on first use, grows when needed and frees at unload.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All device work
 *     is ordered on it.
 *   - Every argument is validated before results are produced.  Host-visible problems
 *     (NULL pointers, bad sizes) return FOS_ERR_INVALID_ARG before any launch.
 *     Values that live in device memory (NaN, negative coefficients, ...) are checked
 *     by the first kernel of the call, which sets a device status word; the later
 *     kernels then do no work and the call returns FOS_ERR_INVALID_ARG.
 *   - Calls are synchronous (they wait for their stream and return the device
 *     status) unless FOS_ASYNC is given; then the status of the work is returned by
 *     the next fos_sync_status(stream) call.
 *   - No call traps, asserts on the device or waits without a bound.
 */
#ifndef FOS_H
#define FOS_H

#ifdef __cplusplus
extern "C" {
#endif

#define FOS_API_VERSION 1

typedef int fos_status;
enum {
    FOS_OK = 0,
    FOS_ERR_INVALID_ARG = 1,   /* bad argument (host check or device validation)     */
    FOS_ERR_CUDA = 2,          /* a CUDA runtime call failed                          */
    FOS_ERR_NOMEM = 3,         /* workspace allocation failed                          */
    FOS_ERR_STEP_LIMIT = 4,    /* some photon hit max_events; counted as "runaway"    */
    FOS_ERR_TIMEOUT = 5,       /* a bounded wait ran out (host wait for the stream, or
                                  an in-kernel wait that gave up and returned)         */
    FOS_ERR_OUT_OF_RANGE = 6,  /* input outside what a kernel supports (e.g. Mie order) */
    FOS_ERR_INJECTED = 7,      /* test-only failure injected by FOS_TEST_INJECT       */
    FOS_ERR_UNSUPPORTED = 8    /* device is not sm_103 / feature not built            */
};

/* Flags (bitwise OR). */
#define FOS_ASYNC        0x1u  /* return after enqueueing; status via fos_sync_status  */
#define FOS_NO_GRAPH     0x2u  /* launch kernels directly instead of a cached CUDA graph */
#define FOS_AUTOTUNE     0x4u  /* re-run the launch autotuner for this batch shape     */
#define FOS_FAST_WALK    0x8u  /* fos_mc_spectrum: the fast walk (SFU log/cos, approximate
                                  reciprocal and square root); statistically equal to the
                                  exact walk, not bit for bit                         */
#define FOS_RECORD_TIMES 0x10u /* fos_mc_spectrum: record each walk block's start and end
                                  time (read back with fos_mc_walk_times)             */
#define FOS_TEST_INJECT  0x10000u /* test only: the first kernel reports a failure      */
#define FOS_TEST_STALL   0x20000u /* test only (fos_gemm_bf16, fos_surrogate_predict): a
                                     pipeline stage is never loaded, so its bounded wait
                                     runs out -> FOS_ERR_TIMEOUT                        */

#define FOS_MAX_LAYERS   8     /* layers per stack                                     */
#define FOS_NCOUNT       6     /* counts per item: R, A, T, runaway, collisions, interface events */
#define FOS_MIE_MAX_TERMS 512  /* Mie: orders the scratch holds per chunk; homogeneous
                                  spheres of any size are summed in chunks of this many
                                  orders; core-shell spheres need n_max + 16 <= this    */

const char* fos_status_string(fos_status s);
int fos_api_version(void);
/* Name and message of the last CUDA runtime error a library call on this host thread
 * met (the cause behind FOS_ERR_CUDA / FOS_ERR_NOMEM); "" if none. */
const char* fos_last_cuda_error(void);

/* Waits (bounded by timeout_ms; <= 0 -> 600000) for `stream` and returns the status of
 * the library work enqueued on the current device since the last check (FOS_ASYNC
 * calls), then clears it. */
fos_status fos_sync_status(void* stream, int timeout_ms);

/* --------------------------------------------------------------------------------
 * fos_mie_properties: scattering properties of particle-filled media.
 *
 * Follows section "Scattering properties" of arxiv 2409.00165:
 *   size parameters x = 2 pi r n_m / lambda, y = 2 pi r n_p / lambda (Eq. 1); Mie
 *   coefficients a_n, b_n (Eqs. 2-5) with the logarithmic derivative of psi_n(z) =
 *   z j_n(z) from a downward recurrence in FP64; the absorbing-host geometric term
 *   (Eq. 10, read with alpha = 4 pi r k_m / lambda); Q_ext, Q_sca (Eqs. 11-12 with
 *   n_max = ceil(2 + |y| + 4.3 |y|^(1/3))); g_i (Eq. 15); then per group (a layer
 *   matrix with its particles) the effective medium mu_s, mu_a (Eqs. 13-14), g (Eq.
 *   16), negative coefficients set to 0, the dependent-scattering factor C = 1 + 1.5F
 *   - 0.75F^2 when F = sum f > 0.08 (Eqs. 17-19) and the matrix absorption 4 pi k_m
 *   (1 - F)/lambda (Eq. 20).
 *
 * Units: wavelength and radius in one length unit (um in the paper); outputs in the
 * inverse of that unit.  All arrays are device, FP64, row-major:
 *   wl            [n_wl]                 vacuum wavelengths, > 0
 *   nm_re, nm_im  [n_groups*n_wl]        matrix n + ik per group (k >= 0)
 *   species_group [n_species]            group of each particle species, non-decreasing
 *   np_re, np_im  [n_species*n_wl]       particle n + ik (k >= 0)
 *   radius        [n_species]            sphere radius, > 0
 *   vol_frac      [n_species]            volume fraction in [0,1); per-group sum < 1
 *   mu_s, mu_a, g [n_groups*n_wl]        outputs (overwritten)
 *   q_ext, q_sca, g_species [n_species*n_wl]  optional outputs (NULL to skip)
 * The sums end early once two successive terms past |x| + 4.05 |x|^(1/3) + 2 fall below
 * 2^-60 of the partial sums (the rest is smaller still); spheres of any size are
 * computed (their orders in chunks of FOS_MIE_MAX_TERMS).
 * Errors: FOS_ERR_INVALID_ARG (sizes, NULL, bad values), FOS_ERR_CUDA.
 * ------------------------------------------------------------------------------ */
fos_status fos_mie_properties(int n_wl, const double* wl,
                              int n_groups, const double* nm_re, const double* nm_im,
                              int n_species, const int* species_group,
                              const double* np_re, const double* np_im,
                              const double* radius, const double* vol_frac,
                              double* mu_s, double* mu_a, double* g,
                              double* q_ext, double* q_sca, double* g_species,
                              unsigned flags, void* stream);

/* fos_mie_properties_cs: as fos_mie_properties, with core-shell particles (supplement
 * of arxiv 2409.00165, Eqs. S1-S9): a core of radius a and index n_c inside a shell of
 * outer radius b and index n_s.  With m1 = n_c/n_m, m2 = n_s/n_m, x = 2 pi a n_m /
 * lambda and y = 2 pi b n_m / lambda, a_n and b_n come from S1-S2, the shell
 * coefficients A_n, B_n from S3-S4 (evaluated divided by psi_n(m1 x), i.e. with the
 * log-derivative D_n(m1 x), which keeps them finite for absorbing cores), chi_n = z y_n(z)
 * (S8) and xi_n = psi_n + i chi_n (S9); n_max uses 2 pi b max(|n_c|,|n_s|)/lambda in
 * place of |y| of Eq. 4.  The efficiencies (Eqs. 10-12, 15) and the effective medium
 * (Eqs. 13-20) use the outer radius b, as the paper's hollow-sphere example does.
 *   ns_re, ns_im  [n_species*n_wl]   shell index (the np_* of fos_mie_properties)
 *   nc_re, nc_im  [n_species*n_wl]   core index (read only where core_radius > 0)
 *   radius        [n_species]        outer radius b
 *   core_radius   [n_species]        a, 0 <= a < b; a = 0 is a homogeneous sphere of n_s
 * All device FP64.  Errors as fos_mie_properties; core_radius NULL with n_species > 0
 * is FOS_ERR_INVALID_ARG, a < 0 or a >= b is FOS_ERR_INVALID_ARG (reported by the
 * kernel). */
fos_status fos_mie_properties_cs(int n_wl, const double* wl,
                                 int n_groups, const double* nm_re, const double* nm_im,
                                 int n_species, const int* species_group,
                                 const double* ns_re, const double* ns_im,
                                 const double* nc_re, const double* nc_im,
                                 const double* radius, const double* core_radius,
                                 const double* vol_frac,
                                 double* mu_s, double* mu_a, double* g,
                                 double* q_ext, double* q_sca, double* g_species,
                                 unsigned flags, void* stream);

/* Particle-size distribution (section "Scattering properties", last paragraph): one
 * particle of diameter D with standard deviation sigma becomes n (101 in the paper; odd)
 * diameters evenly spaced over D +- 3 sigma.  Each size gets the share
 * w_i / sum(w) of vol_frac, w_i = exp(-(D_i - D)^2 / (2 sigma^2)); diameters <= 0 are
 * dropped (n_out < n).  sigma = 0 gives one size.  radius, vol_fracs: host double[n]
 * outputs, to be passed as species of one group to fos_mie_properties, whose effective
 * medium (Eqs. 13-16) sums over them. */
fos_status fos_size_distribution(double diameter, double sigma, double vol_frac, int n,
                                 double* radius, double* vol_fracs, int* n_out);

/* --------------------------------------------------------------------------------
 * fos_mc_spectrum: Monte Carlo photon transport (section "Photon transport").
 *
 * An item is one (stack, wavelength) pair, item = stack * n_wl + w.  A stack is
 * 1..max_layers homogeneous layers (layer 0 on top) between a medium above and a
 * medium below (refractive index; default air n = 1), a conductor below (complex
 * index n + ik, k > 0) or an opaque specular reflector below.  Photons arrive at the
 * top surface at incidence cosine cos_incidence (default 1, normal).  Only the depth z
 * and the direction cosine mu_z are tracked.  Each photon:
 *   1. meets the top surface: reflected with the unpolarised Fresnel reflectance
 *      (drawn; always under total internal reflection) -> R; otherwise enters layer 0
 *      with mu_z = the refraction cosine (1 at normal incidence);
 *   2. flies an optical depth tau = -ln u; inside layer j it collides after tau /
 *      mu_t; a boundary reached first is crossed with the rest of tau carried on;
 *   3. at a collision is absorbed with probability mu_a/mu_t -> A, else is deflected
 *      by a Henyey-Greenstein angle (g) and a uniform azimuth;
 *   4. at a boundary between different indices is reflected (total internal
 *      reflection, or Fresnel draw) or refracted (Snell); leaving the top -> R,
 *      leaving the bottom -> T; at a reflector or a conductor below it is reflected
 *      with R_sub or with the conductor's unpolarised Fresnel reflectance at mu_z
 *      (drawn), and otherwise enters the substrate -> T;
 *   5. after max_events collisions + boundary arrivals is stopped -> runaway.
 * The walk is FP32 with a fixed operation order; random numbers come from
 * Philox4x32-10 with key = seed and counter = (photon id, item id, event, stream):
 * collision e uses the 4 words of counter (p, item, e, 0) (free path, absorption,
 * deflection, azimuth; at normal incidence word 3 of block 0 is the entry Fresnel test,
 * since the first collision has mu_z = +-1 and needs no azimuth; at oblique incidence the
 * entry test is word 0 of counter (p, item, 0, 2)), boundary draw k uses word k mod 4 of
 * counter (p, item, k/4, 1).  Results depend only on (seed, item id, photon id), not
 * on launch shape, and agree bit for bit with any implementation of the same
 * operation order.  With FOS_FAST_WALK the same walk evaluates -ln u and cos 2 pi u on
 * the special-function unit and the deflection's division and the direction's square
 * root approximately: same random numbers and decisions up to those roundings, so its
 * counts agree with the exact walk's within binomial noise, not bit for bit.
 *
 * Property layout (device, FP64): layer j of stack s at wavelength w is element
 * (s*max_layers + j)*n_wl + w of mu_s, mu_a, g, n_layer (the layout of the
 * fos_mie_properties outputs with group = s*max_layers + j).
 * ------------------------------------------------------------------------------ */
typedef struct fos_mc_batch {
    int n_stacks;                 /* >= 1                                              */
    int n_wl;                     /* >= 1                                              */
    int max_layers;               /* 1..FOS_MAX_LAYERS, row stride of the layer tables */
    const int* n_layers;          /* device [n_stacks] in 1..max_layers, or NULL (= max_layers) */
    const double* mu_s;           /* device, scattering coefficient >= 0, 1/length     */
    const double* mu_a;           /* device, absorption coefficient >= 0, 1/length     */
    const double* g;              /* device, HG asymmetry in (-1, 1)                   */
    const double* n_layer;        /* device, real refractive index of the layer, > 0   */
    const double* thickness;      /* device [n_stacks*max_layers], > 0, length         */
    const double* n_above;        /* device [n_items] index above the stack, or NULL (= 1) */
    const double* n_below;        /* device [n_items] index below the stack, or NULL (= 1) */
    const double* substrate_R;    /* device [n_items] in [0,1]: opaque reflector below
                                     (replaces n_below), or NULL (none)               */
    const long long* n_photons;   /* device [n_items] in 0..2^32-1, or NULL (= photons_per_item) */
    long long photons_per_item;   /* used when n_photons is NULL; 0..2^32-1            */
    const long long* photon_first;/* device [n_items] first photon id, or NULL (= 0);
                                     first + count <= 2^32                            */
    const int* item_list;         /* device [n_list] items to run, or NULL (all, in order) */
    int n_list;
    unsigned long long seed;      /* Philox key                                       */
    unsigned int item_id_base;    /* added to the item index in the Philox counter    */
    long long max_events;         /* per-photon cap, 1..2^32-1; 0 -> 100000000        */
    const double* cos_incidence;  /* device [n_items] in (0, 1]: cosine of the incidence
                                     angle in the medium above, or NULL (= 1)         */
    const double* k_below;        /* device [n_items] >= 0: imaginary index below
                                     (k > 0: conductor n_below + i k), or NULL (= 0);
                                     k > 0 with substrate_R is FOS_ERR_INVALID_ARG     */
} fos_mc_batch;

/* counts: device int64 [n_run * FOS_NCOUNT], n_run = n_list (item_list given) or
 *   n_stacks*n_wl; row r holds R, A, T, runaway, collisions, interface events of the
 *   r-th item run.  R + A + T + runaway = photons of that item exactly.  Overwritten.
 * photon_log: optional device int32 [n_run * log_stride]: photon i of row r writes
 *   min(collisions << 2 | outcome, 2^31-1) at r*log_stride + i (outcome 0 R, 1 A,
 *   2 T, 3 runaway).  NULL to skip.  Requires every count <= log_stride.
 * Returns FOS_OK, FOS_ERR_STEP_LIMIT (counts valid; some photons hit max_events),
 * FOS_ERR_INVALID_ARG, FOS_ERR_CUDA, FOS_ERR_NOMEM, FOS_ERR_TIMEOUT, FOS_ERR_INJECTED. */
fos_status fos_mc_spectrum(const fos_mc_batch* batch, long long* counts, int* photon_log,
                           long long log_stride, unsigned flags, void* stream);

/* fos_solar_weighted: solar-weighted totals (section "Output", Eq. 21).  For each stack
 * s and each of R, A, T: the integral over the wavelength grid of the spectral fraction
 * times G, divided by the integral of G, both by the trapezoidal rule on the grid
 * points.  The spectral fraction is count / (R + A + T) of item s*n_wl + w (0 where that
 * sum is 0); with n_wl = 1 the totals are the fractions there.
 *   wl      device double [n_wl], strictly increasing
 *   G       device double [n_wl], >= 0, with a positive integral (spectral irradiance)
 *   counts  device int64 [n_stacks*n_wl*FOS_NCOUNT], the fos_mc_spectrum output
 *   out     device double [n_stacks*3] (R_s, A_s, T_s per stack)
 * Errors: FOS_ERR_INVALID_ARG (sizes, NULL, unordered wl, bad G), FOS_ERR_CUDA.
 * Synchronous unless FOS_ASYNC. */
fos_status fos_solar_weighted(int n_stacks, int n_wl, const double* wl, const double* G,
                              const long long* counts, double* out, unsigned flags,
                              void* stream);

/* Launch shape of the walk kernel: threads per block (multiple of 32, 32..256; the
 * kernel is compiled for 64, 96, 128 and 256 and a smaller block runs the next larger
 * variant) and photons per thread per work unit (a warp claims 32*ppt photons at a
 * time).  fos_mc_set_tuning(0, 0) returns to autotuned/default shapes (128, 8).  A shape
 * set here runs with the default refill cadence (8 events per live photon between a
 * warp's refill votes); autotuned shapes carry the cadence the autotuner chose.
 * fos_mc_get_tuning reports the shape a call with `flags` (FOS_FAST_WALK or 0) would use
 * for this batch shape. */
fos_status fos_mc_set_tuning(int block, int photons_per_thread);
fos_status fos_mc_get_tuning(const fos_mc_batch* batch, unsigned flags, int* block,
                             int* photons_per_thread);

/* The launch-shape autotuner: times every (block in 64, 96, 128, 256) x (photons per
 * thread in 4, 8, 16) at 8 events per live photon between a warp's refill votes, then 4
 * and 16 events at the fastest of those, on a copy of `batch` whose photon budgets are all
 * scaled by one factor (to about 2^26 photons in total, each non-empty item keeping at
 * least one), so the probe keeps the batch's budget distribution, and caches the fastest
 * for batches of this shape and walk (flags: FOS_FAST_WALK or 0).  The cadence changes no
 * result (every photon's walk is a function of its seed, item and id).  Writes it to *block, *ppt if
 * non-NULL.  fos_mc_spectrum with FOS_AUTOTUNE runs it first. */
fos_status fos_mc_autotune(const fos_mc_batch* batch, unsigned flags, void* stream, int* block,
                           int* photons_per_thread);

/* Per-block timing of the last walk launched with FOS_RECORD_TIMES on the current device
 * (diagnostic of the persistent grid's load balance): *n_blocks = its grid size (0 if
 * none); start_end_ns (host int64 [2 * capacity]) receives each block's start and end
 * in ns of the GPU's global timer; start_end_ns = NULL only queries *n_blocks.  A
 * capacity below the grid size is FOS_ERR_INVALID_ARG.  Call after the walk has
 * finished. */
fos_status fos_mc_walk_times(long long* start_end_ns, int capacity, int* n_blocks);

/* --------------------------------------------------------------------------------
 * Diagnostics of the walk's building blocks (used by the parity tests).
 * fos_philox4x32_10: out[4i..4i+3] = Philox4x32-10(counter = ctr[4i..4i+3],
 *   key = (k0, k1)); device uint32 arrays of 4n words (Salmon et al., SC'11).
 * fos_walk_math_f32: for u[i] in (0,1): neg_log[i] = -ln u, cos2pi[i] = cos(2 pi u),
 *   as the walk evaluates them (device float arrays [n]; either output may be NULL).
 * fos_walk_math_fast_f32: the same as the fast walk (FOS_FAST_WALK) evaluates them.
 * fos_philox4x32_10_curand: the same outputs as fos_philox4x32_10, computed by cuRAND's
 *   device Philox4x32-10 (a library routine), an independent check of the walk's generator.
 * ------------------------------------------------------------------------------ */
fos_status fos_philox4x32_10(const unsigned* ctr, unsigned k0, unsigned k1, unsigned* out,
                             long long n, void* stream);
fos_status fos_philox4x32_10_curand(const unsigned* ctr, unsigned k0, unsigned k1,
                                    unsigned* out, long long n, void* stream);
fos_status fos_walk_math_f32(const float* u, float* neg_log, float* cos2pi, long long n,
                             void* stream);
fos_status fos_walk_math_fast_f32(const float* u, float* neg_log, float* cos2pi, long long n,
                                  void* stream);

/* --------------------------------------------------------------------------------
 * Surrogate of the photon walk (section "Photon transport": a network trained on Monte
 * Carlo simulations predicts R, A, T; Table 1 lists the ranges it was trained on).
 *
 * Network: 9 raw features -> standardised -> [Linear 256, GELU] x 4 -> Linear 3 ->
 * softmax = (R, A, T), summing to 1 (GELU in its tanh form z/2 (1 + tanh(sqrt(2/pi)
 * (z + 0.044715 z^3)))).  Products run on the tensor cores (tcgen05.mma,
 * BF16 operands, FP32 accumulation in tensor memory); master weights and Adam state are
 * FP32.  Features of a row (stack of one layer, wavelength): lambda, n_p, log10 k_p,
 * radius, volume fraction, log10 thickness, g, log10(mu_s d + 1e-6), log10(mu_a d + 1e-6).
 *
 * Model storage: a caller-owned device buffer of n_members * fos_surrogate_model_bytes()
 * bytes.  Member k starts at k * fos_surrogate_model_bytes(); its first
 * fos_surrogate_param_count() floats are the FP32 parameters theta, with weight l
 * (row-major [out][in], padded to [256][64], [256][256] x 3, [64][256]; padding is zero)
 * at w_off[l] and bias l at b_off[l] (fos_surrogate_param_offsets).  The rest holds Adam
 * state, BF16 copies and the feature statistics.
 * ------------------------------------------------------------------------------ */
size_t fos_surrogate_model_bytes(void);
long long fos_surrogate_param_count(void);
fos_status fos_surrogate_param_offsets(long long* w_off, long long* b_off);   /* host [5] each */

/* Initialises n_members members: He-uniform weights from a hash of (seed, member,
 * index), zero biases and Adam state.  feat_stats: host float[64] = mean[16] | std[16] |
 * lo[16] | hi[16] of the 9 raw features (first 9 of each used; std > 0, lo <= hi);
 * rows outside [lo, hi] are flagged for Monte Carlo by fos_surrogate_predict.
 * Synchronous. */
fos_status fos_surrogate_init(void* model, int n_members, unsigned long long seed,
                              const float* feat_stats, void* stream);

/* Loads member `member` of a model buffer from caller parameters: theta is a device
 * float[fos_surrogate_param_count()] in the padded layout above (entries outside the real
 * rows and columns are ignored and stored as 0), e.g. weights trained elsewhere or saved
 * from the theta region of another model.  Adam state and the step count are reset, the
 * BF16 copies rebuilt; feat_stats as for fos_surrogate_init.  Synchronous. */
fos_status fos_surrogate_load(void* model, int member, const float* theta,
                              const float* feat_stats, void* stream);

/* Raw features of the n_designs x n_wl rows (row = design * n_wl + w) of single-layer
 * designs: wl [n_wl]; np_re, np_im, g, mu_s, mu_a [n_designs*n_wl] (the layout of
 * fos_mie_properties outputs with one group per design); radius, vol_frac, thickness
 * [n_designs].  features: device float [rows * 9].  All inputs device FP64. */
fos_status fos_surrogate_features(int n_designs, int n_wl, const double* wl,
                                  const double* np_re, const double* np_im,
                                  const double* radius, const double* vol_frac,
                                  const double* thickness, const double* g,
                                  const double* mu_s, const double* mu_a, float* features,
                                  unsigned flags, void* stream);

/* Raw features of homogeneous slabs given by their optical properties, the inputs of
 * the paper's network (section "Photon transport", Table 1: matrix index, mu_s, mu_a, g,
 * thickness), one row per slab: [n, log10(mu_s + 1e-4), log10(mu_a + 1e-4), g, log10 d,
 * log10(mu_s d + 1e-6), log10(mu_a d + 1e-6), log10(1 - g + 1e-3),
 * log10(mu_s (1 - g) d + 1e-6)] with mu in 1/um and d in um (1e-4 per um = 1 per cm).
 * Each input maps monotonically to one of the first five features, so the range gate of
 * fos_surrogate_predict (feature lo/hi) can hold exactly the ranges of Table 1.
 * n_layer, mu_s, mu_a, g, thickness: device double [n_rows]; features: device float
 * [n_rows*9].  Non-positive d or n, negative mu, non-finite values: FOS_ERR_INVALID_ARG. */
fos_status fos_surrogate_features_slab(long long n_rows, const double* n_layer,
                                       const double* mu_s, const double* mu_a, const double* g,
                                       const double* thickness, float* features,
                                       unsigned flags, void* stream);

/* Statistics of raw feature rows [n_rows*9] (device float) into stats (device float[64]
 * = mean[16] | std[16] | lo[16] | hi[16], first 9 of each used; std floored at 1e-3;
 * [lo, hi] is the observed range widened by 1 % of its span on each side), the layout
 * fos_surrogate_init takes.  Synchronous. */
fos_status fos_surrogate_feature_stats(const float* features, long long n_rows, float* stats,
                                       void* stream);

/* (R, A, T) / (R + A + T) of counts row r (device int64 [n_rows*FOS_NCOUNT]) into row
 * rows[r] of fractions (device float [*3]; row r when rows is NULL): turns photon counts
 * into the spectra and scatters Monte Carlo fallback results into a prediction.
 * Asynchronous on stream. */
fos_status fos_counts_to_fractions(const long long* counts, long long n_rows, const int* rows,
                                   float* fractions, void* stream);

/* The indices of the nonzero bytes of mask [n] (device) into rows (device int32,
 * capacity n) and their number into *count (device int64): the work list of the rows
 * fos_surrogate_predict flagged for Monte Carlo.  Order: ascending within blocks of 1024
 * rows, blocks in any order.  Asynchronous on stream. */
fos_status fos_mask_to_rows(const unsigned char* mask, long long n, int* rows, long long* count,
                            void* stream);

/* One Adam step (lr, beta 0.9/0.999, eps 1e-8, bias-corrected with t = step + 1) of
 * member `member` on a batch of `batch` rows (multiple of 256, <= 65536) of features
 * [n_rows*9] / targets [n_rows*3] (device float; target rows sum to 1).  Rows are
 * batch_rows [batch] (device int32) if given, else drawn uniformly with replacement
 * from a hash of (seed, member, step, slot).  Loss: mean soft-label cross-entropy,
 * written to loss_out (device float) if non-NULL; it is summed with atomics, so its last
 * bits may differ between runs (the parameter update does not).  If grad_out (device float
 * [fos_surrogate_param_count()]) is non-NULL the gradient is written there and the
 * parameters are NOT updated (diagnostic); otherwise the member's step count kept in
 * the model (see fos_surrogate_fit) is set to step + 1.  Synchronous unless FOS_ASYNC.
 * The library keeps one activation workspace per member slot (member mod 4): steps of
 * members in different slots may run concurrently on different streams (with
 * FOS_ASYNC); steps of members in the same slot must be ordered (one stream). */
fos_status fos_surrogate_train_step(void* model, int member, const float* features,
                                    const float* targets, long long n_rows, int batch,
                                    const int* batch_rows, unsigned long long seed, int step,
                                    float lr, float* loss_out, float* grad_out,
                                    unsigned flags, void* stream);

/* n_steps Adam steps of every member 0..n_members-1 with no host work per step (the
 * training loop of the surrogate; the same arithmetic as fos_surrogate_train_step).  Each
 * member continues from its own step count g, kept in the model buffer (0 after
 * fos_surrogate_init / fos_surrogate_load, saved with the buffer): step g draws its batch
 * from a hash of (seed, member, g), uses Adam's t = g + 1 and the cosine learning rate
 * lr_min + (lr_max - lr_min)(1 + cos(pi min(g - schedule_origin, schedule_total) /
 * schedule_total))/2 (g - schedule_origin clamped at 0).  Ensemble steps are captured
 * once into CUDA graphs of 8 steps and of 1 step (each step: the two halves of the
 * ensemble on parallel branches; the step counts live on the device, and the learning
 * rate and bias corrections of the call's steps are a table the call writes first, after
 * waiting for the device's earlier work), launched on `stream` as often as n_steps needs.
 *   loss_out: device float [n_members] or NULL: each member's loss of its last step.
 * Errors of the device work are reported like FOS_ASYNC calls (fos_sync_status); without
 * FOS_ASYNC the call waits for the stream and returns that status itself.  Batch as for
 * fos_surrogate_train_step; flags: 0 or FOS_ASYNC. */
fos_status fos_surrogate_fit(void* model, int n_members, const float* features,
                             const float* targets, long long n_rows, int batch,
                             unsigned long long seed, int n_steps, float lr_max, float lr_min,
                             int schedule_origin, int schedule_total, float* loss_out,
                             unsigned flags, void* stream);

/* Ensemble prediction with members 0..n_members-1 (1..16): rat [n_rows*3] = mean of the
 * members' (R, A, T); spread [n_rows] (or NULL) = max over R, A, T of (max - min across
 * members); needs_mc [n_rows] (or NULL) = 1 where spread > threshold or a raw feature is
 * outside the training range [lo, hi], else 0.  Device buffers.  Synchronous unless
 * FOS_ASYNC. */
fos_status fos_surrogate_predict(void* model, int n_members, const float* features,
                                 long long n_rows, float* rat, float* spread,
                                 unsigned char* needs_mc, float threshold, unsigned flags,
                                 void* stream);

/* Diagnostic: the surrogate's tensor-core product on its own.  C[s][M][N] (device fp32,
 * s = 0..splits-1 partial sums over K ranges of K/splits) = A[M][K] * B[N][K]^T with A, B
 * device BF16 row-major; K a multiple of 64*splits, N a multiple of 64.  flags: 0,
 * FOS_ASYNC or FOS_TEST_STALL (every in-kernel wait is bounded: a stage that never fills
 * makes the kernel give up, drain its copies, free its tensor memory and report
 * FOS_ERR_TIMEOUT).  Synchronous unless FOS_ASYNC. */
fos_status fos_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K,
                         int splits, unsigned flags, void* stream);


/* --------------------------------------------------------------------------------
 * fos_mc_spectrum_noalloc: fos_mc_spectrum for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a property of the library only.
 *
 * Some callers cannot call cudaMalloc: a process whose device memory is all reserved
 * by another allocator (for example a framework's caching pool), or a host under a
 * fixed memory budget where an allocation may fail or stall.  This entry point
 * allocates nothing: no cudaMalloc, cudaFree, allocating library routine, stream or
 * graph.  Its scratch (work-queue counter, status words, packed item tables) is a
 * file-scope device array of about 1.2 MB, which a GPU holds from the first call on it
 * until the process exits.  The caller still passes the inputs (batch, as for
 * fos_mc_spectrum) and the output counts (device int64 [n_run * FOS_NCOUNT]).
 *   - n_run (items run) must be <= FOS_NOALLOC_MAX_ITEMS, else FOS_ERR_OUT_OF_RANGE
 *     is returned before any device work; any max_layers up to FOS_MAX_LAYERS.
 *   - flags: 0 or FOS_TEST_INJECT.  The call is synchronous (bounded wait on stream).
 *   - Set-up: CUDA loads code and device arrays lazily, and loading takes device
 *     memory.  So the first call on each device, with that device current, loads the
 *     array and every kernel the call uses and looks up the array's device address
 *     (cudaGetSymbolAddress).  Make that first call before the caller's allocator takes
 *     the device's memory, and before any stream capture.  A call with an empty batch
 *     (item_list with n_list = 0) does the set-up and nothing else.
 *   - Every call on a device shares the one array and each call clears what must start
 *     at zero; calls that overlap on the GPU (other streams, other host threads) race
 *     on it and must be serialised by the caller.
 *   - A call whose bounded wait runs out returns FOS_ERR_TIMEOUT while its kernels may
 *     still use the array; until that stream has drained, later calls on the device
 *     return FOS_ERR_TIMEOUT without touching the array.
 *   - Results are identical to fos_mc_spectrum's for the same batch.
 * ------------------------------------------------------------------------------ */
#define FOS_NOALLOC_MAX_ITEMS 4096
fos_status fos_mc_spectrum_noalloc(const fos_mc_batch* batch, long long* counts,
                                   unsigned flags, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FOS_H */
