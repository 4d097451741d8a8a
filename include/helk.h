/*
 * helk.h -- C ABI of the GB300 (sm_103a) HELIOS-K hot path.
 *
 * Method: Grimm & Heng 2015, "HELIOS-K: an ultrafast, open-source opacity
 * calculator for radiative transfer" (arXiv:1503.03806).
 *   Opacity  kappa(nu) = sum_lines S Phi(nu)              Sec. 2.3 (kappa = S Phi)
 *   Voigt    Phi = sqrt(ln2/pi) H_V(a,u) / Gamma_D        Sec. 2.3
 *   H_V by Algorithm 916 for a^2+u^2 < 100, 3-node Gauss-Hermite for
 *   100 <= a^2+u^2 < 1e6 and 1-node Gauss-Hermite beyond  Sec. 2.4
 *   line-wing cutoff                                       Sec. 2.4
 *   k-distribution: per-bin sort, k(g), Chebyshev fit      Sec. 2.2, 2.6
 *   transmission T(m) = int_0^1 exp(-k(g) m) dg            Sec. 2.1
 *
 * Conventions common to every entry point:
 *  - All entry points return helk_status; none aborts.  On failure the
 *    context keeps a message readable with helk_last_error().
 *  - Work is enqueued on the context's CUDA stream and the call returns
 *    before it finishes, unless stated otherwise.  Errors raised by kernels
 *    (for example a bounded wait that gave up: HELK_ERR_TIMEOUT) are reported
 *    by the next helk_sync() or by any call that reads results to the host.
 *  - "device pointer" means memory of the context's device (e.g. a torch
 *    tensor's data_ptr()); the caller owns it and keeps it alive until the
 *    work that uses it has completed.  Host pointers are only read during
 *    the call (data are copied before it returns).
 *  - Units: wavenumber cm^-1, T in K, P in atm (P0 = 1 atm), mass in amu,
 *    S in cm/molecule; opacities are cross-sections in cm^2/molecule.
 *  - Grid sizes are limited to 2^31 - 1 points, line lists to 2^31 - 1
 *    lines.
 */
#ifndef HELK_H
#define HELK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helk_ctx helk_ctx;

typedef enum {
    HELK_OK = 0,
    HELK_ERR_INVALID_ARG = -1, /* bad value, size or pointer               */
    HELK_ERR_OOM = -2,         /* device or host allocation failed         */
    HELK_ERR_CUDA = -3,        /* CUDA runtime error (text in last_error)  */
    HELK_ERR_STATE = -4,       /* call order (e.g. opacity before upload)  */
    HELK_ERR_TIMEOUT = -5,     /* a kernel's bounded wait gave up          */
    HELK_ERR_UNSUPPORTED = -6  /* option not available in this build       */
} helk_status;

/* Uniform wavenumber grid nu_i = nu_min + i * dnu, i = 0 .. n-1
 * (Sec. 2.2: equal intervals delta x).  dnu > 0, 0 < n < 2^31. */
typedef struct {
    double nu_min;
    double dnu;
    int64_t n;
} helk_grid;

/* Line-wing cutoff (Sec. 2.4).  A grid point i belongs to a line's window
 * when |nu_i - nu0'| <= C, realised as the integer bounds
 *   i_lo = max(0, ceil((nu0' - C - nu_min)/dnu)),
 *   i_hi = min(n-1, floor((nu0' + C - nu_min)/dnu)).
 *   HELK_CUT_ABS:     C = value                     [cm^-1]
 *   HELK_CUT_LORENTZ: C = min(value * Gamma_L, cap)  (e.g. 500 Gamma_L, 100)
 *   HELK_CUT_NONE:    every grid point (the full Voigt profile)
 * The truncated profile is not renormalised. */
enum { HELK_CUT_ABS = 0, HELK_CUT_LORENTZ = 1, HELK_CUT_NONE = 2 };
typedef struct {
    int32_t kind;
    double value;
    double cap;
} helk_cutoff;

/* Line list as structure-of-arrays of n doubles each (Sec. 2.3).
 *   nu0        line-centre wavenumber [cm^-1]                 (required)
 *   S0         integrated strength [cm/molecule] at T0 = 296 K if E_lower
 *              is given, else at the requested T               (required)
 *   E_lower    lower-state energy [cm^-1]; NULL: no T scaling of S
 *   gamma_air  air-broadening coefficient [cm^-1/atm]          (required)
 *   gamma_self self-broadening coefficient; NULL: = gamma_air
 *   n_coll     temperature exponent; NULL: 0.5
 *   delta      pressure shift [cm^-1/atm]; NULL: 0
 *   mass       molecular mass of the line's species [amu]; NULL: the mass
 *              passed to helk_opacity
 *   weight     abundance (mixing ratio) of the line's species; multiplies S;
 *              NULL: 1.  With mass and weight one list holds several species,
 *              whose opacities are then added before the k-distribution
 *              (Sec. 2.1)
 * All values must be finite, nu0 > 0, S0 >= 0, gamma_* >= 0, mass > 0,
 * weight >= 0. */
typedef struct {
    const double *nu0, *S0, *E_lower, *gamma_air, *gamma_self, *n_coll, *delta;
    const double *mass, *weight;
} helk_lines;

/* Arithmetic of the Voigt stage.
 *   HELK_PREC_F64:       FP64 throughout (reference form).
 *   HELK_PREC_F32_KAHAN: FP32 profile evaluation and Kahan-compensated FP32
 *                        accumulation, output converted to FP64.  Error vs the
 *                        FP64 form <= 1e-5 relative where kappa exceeds 1e-8
 *                        of its k-bin maximum.  Needs every line's core
 *                        (a^2 + u^2 < 100) within 2^23 grid points of its
 *                        centre, i.e. a Doppler width below ~7e5 grid steps
 *                        (point offsets are exact in FP32 only up to 2^24);
 *                        otherwise the next helk_sync (or a call that reads
 *                        results) returns HELK_ERR_UNSUPPORTED. */
enum { HELK_PREC_F64 = 0, HELK_PREC_F32_KAHAN = 1 };

typedef struct {
    int32_t precision;  /* HELK_PREC_*                                      */
    int32_t accumulate; /* 0: kappa = weight*sigma, 1: kappa += weight*sigma */
    double weight;      /* abundance weight X of Sec. 2.1 (mix before k-dist) */
    double q_ratio;     /* Q(T0)/Q(T), used only when E_lower was uploaded   */
    int32_t count_regions; /* 1: also count evaluations per method (slower;
                              read with helk_opacity_stats)                   */
    int32_t surrogate;  /* FP32 form only: 1 routes Algorithm-916 evaluations
                           that fall in the surrogate network's validated
                           cells to the network (helk_surrogate_*); error
                           <= 1e-4 relative per routed term.  The routed
                           terms are added with atomics, so results are no
                           longer bitwise reproducible.  0 (the default)
                           keeps Algorithm 916: on GB300 the network is
                           slower than the FP32 Algorithm 916 it replaces
                           (its 192 SiLU activations take more MUFU time
                           than a whole FP32 evaluation).                  */
} helk_opts;

/* Create a context on CUDA device `device`, enqueueing on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  No counterpart in
 * the paper (context plumbing, as are helk_destroy, helk_last_error,
 * helk_set_stream and helk_sync).  *out receives the
 * context; release it with helk_destroy. */
helk_status helk_create(helk_ctx **out, int device, void *stream);

/* Free the context and every device buffer it owns (synchronises first).
 * No counterpart in the paper. */
void helk_destroy(helk_ctx *ctx);

/* Last error message of this context ("" if none).  Valid until the next
 * call on the context.  No counterpart in the paper. */
const char *helk_last_error(const helk_ctx *ctx);

/* Change the stream later work is enqueued on.  No counterpart in the
 * paper. */
helk_status helk_set_stream(helk_ctx *ctx, void *stream);

/* Wait for all work of the context and report kernel-side errors, each
 * once (the context stays usable): a bounded wait that gave up
 * (HELK_ERR_TIMEOUT); an FP32-form call outside that form's range
 * (HELK_ERR_UNSUPPORTED, see HELK_PREC_F32_KAHAN).  No counterpart in the
 * paper. */
helk_status helk_sync(helk_ctx *ctx);

/* Failure-detection self-test (no counterpart in the paper): launches a
 * kernel whose bounded wait, the
 * one every staged copy of the Voigt kernels uses, waits on a barrier that
 * nothing completes.  The wait is bounded in time, by the GPU's global timer:
 * it gives up after limit_us microseconds (1 .. 1e7; the Voigt kernels use
 * 100 ms) and sets the timeout flag, so the next helk_sync returns
 * HELK_ERR_TIMEOUT.  No fault, no hang. */
helk_status helk_selftest_timeout(helk_ctx *ctx, int32_t limit_us);

/* Upload (copy) a line list -- the per-line parameters of Sec. 2.3 -- into
 * context-owned device memory and order it by nu0 (stable), replacing any
 * previous list.  `on_device` = 0: the
 * pointers in *lines are host memory; 1: device memory.  n >= 0.
 * Validation of values runs on the device and is reported here (the call
 * synchronises the stream). */
helk_status helk_lines_upload(helk_ctx *ctx, const helk_lines *lines,
                              int64_t n, int32_t on_device);

/* Opacity of the uploaded lines at one condition (Sec. 2.3-2.4):
 *   kappa_out[i] (=|+=) weight * sum_lines S' H_V(a, u_i),
 *   S' = S sqrt(ln2/pi)/Gamma_D, u_i = sqrt(ln2)(nu_i - nu0')/Gamma_D.
 * kappa_out: device pointer to grid->n doubles, or NULL to use a buffer
 * owned by the context (read by helk_kdist with kappa == NULL).
 * T > 0, P >= 0, mass > 0.  opts may be NULL (FP64, weight 1, q_ratio 1). */
helk_status helk_opacity(helk_ctx *ctx, double T, double P_atm,
                         double mass_amu, const helk_cutoff *cut,
                         const helk_grid *grid, const helk_opts *opts,
                         double *kappa_out);

/* Opacities of the uploaded lines at n_cond conditions (T[k], P_atm[k]) on
 * one grid, in one persistent launch (Sec. 2.3-2.4; the paper's many (T, P)
 * points).  kappa_out: device pointer to n_cond * grid->n doubles, row k =
 * condition k (NULL: the context's buffer, read by helk_kdist with
 * kappa == NULL and n = n_cond * grid->n -- the k-tables of all conditions
 * then come from one helk_kdist call with n_cond * nbins bins).  q_ratio:
 * per-condition Q(T0)/Q(T) or NULL (opts->q_ratio for all).  T, P, q_ratio
 * are host arrays, read during the call.  The whole sequence is captured
 * once per call shape (n_cond, line list, grid, cutoff, options, output
 * pointer, tile shape) into a CUDA graph and replayed on later calls with the
 * same shape; only the condition values change between replays.  The
 * per-condition line records take 64 B (FP64 form) or 120 B (FP32 form) per
 * line; when those of all n_cond conditions exceed the record budget
 * (64 GiB unless set by helk_set_batch_budget), the conditions run in the
 * fewest equal chunks that fit, each chunk its own captured graph and
 * persistent launch, one after the other on the stream (the context keeps
 * the 16 most recent graphs).  The results equal those of n_cond
 * helk_opacity calls bit for bit.  A call waits until the previous batch call
 * has read its conditions. */
helk_status helk_opacity_batch(helk_ctx *ctx, int32_t n_cond, const double *T,
                               const double *P_atm, const double *q_ratio,
                               double mass_amu, const helk_cutoff *cut,
                               const helk_grid *grid, const helk_opts *opts,
                               double *kappa_out);

/* Line-record budget of one chunk of helk_opacity_batch, in bytes (0: the
 * default, 64 GiB); no counterpart in the paper.  A chunk always holds at least one condition, so a
 * budget below one condition's records runs the conditions one by one.
 * Host-only. */
helk_status helk_set_batch_budget(helk_ctx *ctx, int64_t bytes);

/* Evaluation counts (of the Sec. 2.4 methods; a measurement with no
 * counterpart in the paper) of the first n_cond conditions of the last
 * opacity call
 * (n_evals[k]; region_counts[4k..4k+3] as in helk_opacity_stats when that call
 * counted regions, else pass NULL).  Synchronises. */
helk_status helk_opacity_batch_stats(helk_ctx *ctx, int32_t n_cond,
                                     int64_t *n_evals, int64_t *region_counts);

/* Statistics of the last helk_opacity (a measurement with no counterpart
 * in the paper): number of (line, grid point) Voigt evaluations within the
 * Sec. 2.4 windows and, if region_counts != NULL (4 entries; the last opacity
 * must have run with count_regions), how many fell in each method
 * [Algorithm 916, GH3, GH1] plus the number of Algorithm 916 series terms
 * summed.  Synchronises. */
helk_status helk_opacity_stats(helk_ctx *ctx, int64_t *n_evals,
                               int64_t *region_counts);

/* k-distribution tables (Sec. 2.2, 2.6) of an opacity array of n points cut
 * into nbins equal contiguous bins (n % nbins == 0, N_b = n/nbins):
 *   - each bin sorted ascending: k_j, j = 0..N_b-1, on g_j = (j + 1/2)/N_b;
 *   - ncheb coefficients c_k of the least-squares fit
 *       ln max(k(g), kappa_floor) ~ sum_k c_k T_k(2g - 1);
 *   - the bin mean of kappa (= int_0^1 k(g) dg, Sec. 2.1).
 * kappa: device pointer (NULL = the context's buffer from helk_opacity).
 * coeffs: nbins*ncheb doubles, row-major [bin][k]; mean: nbins doubles or
 * NULL; both host memory if out_on_host != 0 (the call then synchronises)
 * else device memory.  kg_out: optional device pointer to n doubles that
 * receives the sorted values.  1 <= ncheb <= 32, ncheb <= N_b.
 * The sorted values equal those of any correct ascending sort, bit for
 * bit.  kappa holds non-negative values, as helk_opacity writes them (the
 * sort orders the IEEE bit patterns); for negative or NaN values the tables
 * are unspecified (an infinite or NaN largest value gives that mean).
 * Arithmetic: the pseudo-inverse of the Chebyshev design matrix is built
 * once per (N_b, ncheb) in FP64 (Householder QR) and kept as FP32 (high, low)
 * pairs; per point, ln max(k_j, kappa_floor) is a float-float logarithm
 * (absolute error < 2e-12 for |ln k| < 70) and c = P L a double-float dot
 * product (relative error ~2^-46 of sum |P_kj L_j|); the mean is an exact
 * 128-bit integer sum, rounded once to FP64.  Coefficients agree with an
 * FP64 least-squares fit to ~1e-12 of max |c|. */
helk_status helk_kdist(helk_ctx *ctx, const double *kappa, int64_t n,
                       int32_t nbins, int32_t ncheb, double kappa_floor,
                       double *coeffs, double *mean, int32_t out_on_host,
                       double *kg_out);

/* Autotuner of the Voigt kernel's shape (no counterpart in the paper; the
 * helk_tile_* calls and helk_set_tile below belong to it).  A shape is one
 * built
 * configuration of a precision's persistent Voigt kernel: the tile (grid
 * points per CTA tile), the warps per CTA and the candidate lines per
 * pipeline stage; it is named by a shape code (helk_tile_shape decodes it).
 * Runs the line preparation of this condition once, then times every
 * candidate shape of opts->precision on it (three launches each, CUDA events
 * on the context stream) and keeps the fastest for later helk_opacity calls
 * with the same precision and grid size; other sizes fall back to the
 * built-in choice (tiles filling whole waves of resident CTAs).  *tile_out
 * (optional) receives the chosen shape code.  Overwrites the context's own
 * opacity buffer; synchronises. */
helk_status helk_autotune(helk_ctx *ctx, double T, double P_atm,
                          double mass_amu, const helk_cutoff *cut,
                          const helk_grid *grid, const helk_opts *opts,
                          int32_t *tile_out);

/* The shape codes of a precision that the autotuner times (no counterpart
 * in the paper; FP32: the
 * 1-based positions of its built shapes; FP64: slots per warp, 4, 6, 8):
 * writes up to `max` of them to out (host memory) and returns how many there
 * are.  No device work; returns 0 for an unknown precision or out == NULL. */
int32_t helk_tile_candidates(int32_t precision, int32_t *out, int32_t max);

/* Decodes a shape code of `precision` (no counterpart in the paper):
 * points per CTA tile, warps per CTA
 * and candidate lines per pipeline stage (each output optional, host
 * memory).  HELK_ERR_INVALID_ARG for an unknown precision or code.  No
 * device work. */
helk_status helk_tile_shape(int32_t precision, int32_t code, int32_t *points,
                            int32_t *warps, int32_t *lines_per_stage);

/* Fixes the Voigt kernel shape of `precision` (no counterpart in the paper)
 * for grids of n points (what
 * helk_autotune would store), or, with tile == 0, returns to the built-in
 * choice.  tile must be one of helk_tile_candidates(precision); anything
 * else returns HELK_ERR_INVALID_ARG.  The shape changes no FP64 result and
 * FP32 results only at rounding level (Kahan-compensated sums in another
 * grouping). */
helk_status helk_set_tile(helk_ctx *ctx, int32_t precision, int64_t n, int32_t tile);

/* Number of CUDA kernels the context has launched since it was created
 * (tracing, no counterpart in the paper: a caller can bracket a region
 * with two calls).  Launches that a replayed CUDA graph makes
 * (helk_opacity_batch after its first call with given sizes) are counted
 * when the graph is captured, not at each replay.
 * Host-only; returns -1 for ctx == NULL. */
int64_t helk_launch_count(const helk_ctx *ctx);

/* Stage timing (tracing: the paper's per-stage breakdown of Sec. 3.5).
 * With profiling on, the library records a CUDA
 * event pair on the context stream around each stage it launches:
 *   HELK_STAGE_LINEPREP  line preparation and the tile map (Sec. 2.3-2.4)
 *   HELK_STAGE_VOIGT     the Voigt/opacity kernel (Sec. 2.3-2.4)
 *   HELK_STAGE_KDIST     per-bin sort and Chebyshev fit (Sec. 2.6)
 *   HELK_STAGE_SETUP     one-time pseudo-inverse of the Chebyshev basis
 * helk_stage_times synchronises and writes, for each stage, the summed
 * device time in ms (ms[HELK_NSTAGES]) and launch count (count, optional)
 * since profiling was last switched on; at most 65536 pairs per stage are
 * kept (later ones are dropped and flagged by count < 0). */
enum { HELK_STAGE_LINEPREP = 0, HELK_STAGE_VOIGT = 1, HELK_STAGE_KDIST = 2,
       HELK_STAGE_SETUP = 3, HELK_NSTAGES = 4 };
helk_status helk_set_profiling(helk_ctx *ctx, int32_t on);
helk_status helk_stage_times(helk_ctx *ctx, double *ms, int64_t *count);

/* ----------------------------------------------------------------------
 * Surrogate network for the Voigt function (an addition to the paper's
 * method: a 2 -> 64 -> 64 -> 64 -> 1 SiLU network, BF16 tensor-core MMAs with
 * FP32 accumulation, that stands in for Algorithm 916 (Sec. 2.4, the region
 * a^2 + u^2 < 100) as K(x, y) = K_ref(x, y) exp(net(f1, f2)),
 *   K_ref = e^{-x^2} erfcx(y) + (1 - e^{-x^2}) y / (sqrt(pi)(x^2 + y^2)),
 *   f1 = 2 asinh|x| / asinh(10) - 1,  f2 = 2 (log10 y + 4) / 5 - 1,
 * for 1e-4 <= y < 10.  Parameters: 8577 floats, W1[2][64], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4 (W[in][out]).
 * Training targets are this library's FP64 Algorithm 916; the same checks
 * the network cell by cell (helk_surrogate_validate), and only validated
 * cells are routed to it (helk_opts.surrogate).
 * ------------------------------------------------------------------- */
/* (Re)initialise the network with seeded normal weights, zero biases.
 * Surrogate calls have no counterpart in the paper (see above). */
helk_status helk_surrogate_init(helk_ctx *ctx, uint64_t seed);
/* (Surrogate, no counterpart in the paper.)  Copy the parameters to
 * get_host (8577 floats) and/or replace them from
 * set_host (resets the optimiser state); either may be NULL.  Synchronises. */
helk_status helk_surrogate_params(helk_ctx *ctx, float *get_host,
                                  const float *set_host);
/* (Surrogate, no counterpart in the paper.)  n seeded samples of the
 * Sec. 2.4 core region (|x| asinh-uniform in [0, 10], y
 * log-uniform in [1e-4, 10), x^2 + y^2 < 100): features feat[2i], feat[2i+1],
 * target ln(K/K_ref) with K by FP64 Algorithm 916, and optionally x, y.
 * Device pointers. */
helk_status helk_surrogate_samples(helk_ctx *ctx, int64_t n, uint64_t seed,
                                   float *feat, float *target, double *x,
                                   double *y);
/* (Surrogate, no counterpart in the paper.)  Gradient of the mean squared
 * residual error over n samples (device
 * feat/target) at the current parameters, to grad_host (8577 floats) and
 * the loss to loss_host; no update.  Synchronises. */
helk_status helk_surrogate_grad(helk_ctx *ctx, int64_t n, const float *feat,
                                const float *target, float *grad_host,
                                double *loss_host);
/* (Surrogate, no counterpart in the paper.)  Train with Adam on n_samples
 * fresh samples (seed) for `epochs` passes in
 * minibatches of `batch` (>= 128), learning rate lr with cosine decay to 1 %.
 * final_loss (host, optional): mean squared residual error of the last
 * epoch.  Synchronises after every epoch. */
helk_status helk_surrogate_train(helk_ctx *ctx, int64_t n_samples,
                                 uint64_t seed, int32_t epochs, int32_t batch,
                                 double lr, double *final_loss);
/* (Surrogate, no counterpart in the paper.)  K(x_i, y_i) by the network for
 * n points (device arrays). */
helk_status helk_surrogate_eval(helk_ctx *ctx, int64_t n, const double *x,
                                const double *y, double *k);
/* (Surrogate, no counterpart in the paper.)  Held-out check on an nx x ny
 * partition of the feature square with
 * per_cell^2 points at sub-cell centres (points with x^2 + y^2 >= 100 are
 * skipped): a cell is validated when every checked point has
 * |K_net - K_916| <= tol K_916.  Writes mask_host[cy*nx + cx] (0/1) and
 * err_host (max relative error, -1 for cells with no point), both optional,
 * and keeps the mask for routing.  Synchronises. */
helk_status helk_surrogate_validate(helk_ctx *ctx, int32_t nx, int32_t ny,
                                    int32_t per_cell, double tol,
                                    uint8_t *mask_host, double *err_host);

/* Throughput probe of one arithmetic unit (no counterpart in the paper: the
 * measured peaks the roofline fractions of the Voigt kernels are taken
 * against).  kind:
 *   HELK_PROBE_FFMA      FP32 fused multiply-add (the FP32 form's pipe)
 *   HELK_PROBE_DFMA      FP64 fused multiply-add (the FP64 form's pipe)
 *   HELK_PROBE_MUFU_RCP  MUFU reciprocal (rcp.approx; GH1/GH3 of the FP32 form)
 *   HELK_PROBE_MUFU_EX2  MUFU base-2 exponential (ex2.approx)
 * Fills every SM with independent dependency chains of that instruction,
 * calibrates the loop to ~20 ms a launch, then times three launches with
 * CUDA events on the context stream.  *ops_per_s: flops per second for the
 * FMA kinds (an FMA counts 2), results per second for the MUFU kinds;
 * *ms_per_launch (optional): the mean launch time.  Synchronises; uses the
 * context's scratch buffer. */
enum { HELK_PROBE_FFMA = 0, HELK_PROBE_DFMA = 1, HELK_PROBE_MUFU_RCP = 2, HELK_PROBE_MUFU_EX2 = 3 };
helk_status helk_peak_probe(helk_ctx *ctx, int32_t kind, double *ops_per_s,
                            double *ms_per_launch);

/* Transmission of every bin for nm column masses m (Sec. 2.1, Eq. for T:
 * T(m) = int_0^1 exp(-k(g) m) dg; the paper's "Transmission" stage).
 *   sorted (device, nbins*nb doubles, e.g. kg_out of helk_kdist) or NULL:
 *     direct[b*nm + i] = (1/nb) sum_j exp(-k_j m_i), the midpoint rule on
 *     g_j = (j + 1/2)/nb; by Sec. 2.1 this equals the band-mean transmission
 *     of the unsorted bin.
 *   coeffs (device, nbins*ncheb) or NULL: fit[b*nm + i] by the midpoint rule
 *     on ng points of the resampled k(g) = exp(sum_k c_k T_k(2g - 1)).
 * m: host array of nm column masses (cm^2/molecule units inverse to kappa),
 * finite and >= 0.  direct, fit: device arrays of nbins*nm doubles.
 * Arithmetic: the bin's smallest term e^{-k_0 m} in FP64 is factored out;
 * the others, e^{-(k_j - k_0) m}, are left out below e^-87 of it and
 * otherwise evaluated as float-float pairs (relative error ~5e-15 a term),
 * the differences k_j - k_0 formed in FP64.  `sorted` must hold each bin's
 * values in ascending order (as kg_out does) for the terms past e^-87 to be
 * found by a search; a bin that is not sorted, or holds a negative or
 * non-finite value, is summed plainly in FP64.  Each result agrees with the
 * FP64 sum to ~1e-13 relative (the sum of the fit's points also carries the
 * FP64 rounding of k(g), ~1e-14 relative, times k m).  Uses context scratch
 * of 8 B per sorted value. */
helk_status helk_transmission(helk_ctx *ctx, int32_t nbins, int64_t nb,
                              const double *sorted, const double *coeffs,
                              int32_t ncheb, int32_t ng, int32_t nm,
                              const double *m, double *direct, double *fit);

/* Allocation-free k-distribution tables.  The paper has no counterpart: this
 * is an interface addition.  Same computation and outputs as helk_kdist with
 * device-pointer outputs, for callers that cannot call cudaMalloc: code that
 * runs inside a framework whose caching allocator owns the device memory
 * (a cudaMalloc beside it may fail once the pool has taken the memory, and
 * cudaFree synchronises the whole device, stalling the framework's other
 * streams), and host programs that allow no allocation once their set-up is
 * done (fixed-budget or real-time loops).  The caller still allocates the
 * inputs and outputs.
 *
 * It needs no context and calls no cudaMalloc, cudaFree or allocating
 * library routine.  Its scratch (the pseudo-inverse of the Chebyshev basis,
 * its QR work array, the logarithm's table and the sizes they were built for)
 * lives in a fixed 6 MiB device array that every GPU loading the library
 * holds until the process exits.  Limits: N_b = n/nbins <= 12288 points per
 * bin and 1 <= ncheb <= 32 (the bin sort then runs in shared memory); larger
 * requests return HELK_ERR_INVALID_ARG before any GPU work, as do null
 * kappa/coeffs, n % nbins != 0 and kappa_floor <= 0.  Runs on the current
 * CUDA device and on `stream` (a cudaStream_t, NULL = legacy default).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  All calls share the array,
 * which keeps the last call's contents: each call launches a set-up kernel
 * that rebuilds the pseudo-inverse when the sizes recorded in the array
 * differ from its own and returns at once otherwise, so nothing in the array
 * needs to start at zero.  Calls whose work overlaps on the GPU (other
 * streams, other host threads) race on the array: order them on one stream
 * or synchronise between them.
 *
 * kappa: device, n doubles.  coeffs: device, nbins*ncheb doubles.  mean,
 * kg_out: device or NULL, as in helk_kdist. */
helk_status helk_kdist_static(const double *kappa, int64_t n, int32_t nbins,
                              int32_t ncheb, double kappa_floor,
                              double *coeffs, double *mean, double *kg_out,
                              void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HELK_H */
