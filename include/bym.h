/*
 * bym.h -- C ABI of the GB300 (sm_103a) pairwise line-of-sight multipole library.
 *
 * Power-spectrum multipoles P_ell(k) and correlation-function multipoles
 * xi_ell(r) of a galaxy catalog with random catalog, for the line-of-sight
 * choices of Philcox & Slepian, "Beyond Yamamoto" (arXiv:2102.08384):
 *
 *   BYM_LOS_YAMAMOTO  n = hat r_2                 Sec. 2, eq. Yamamoto-estimator / eq. 2pcf-yama
 *   BYM_LOS_MIDPOINT  n = hat(r_1 + r_2)          Secs. 3-4, eq. FFT-midpoint / eq. xi-parity-all-estimator
 *   BYM_LOS_BISECTOR  n = hat(hat r_1 + hat r_2)  Secs. 5-6, eq. bisector-pk-fft / Sec. 6 boxed estimator
 *
 * expanded to order K in the pair opening angle theta ("order"): the midpoint
 * series keeps alpha <= K (eq. Ylm-shift-theorem, eq. Legendre-shift-theorem-
 * all-parity), the bisector series keeps beta <= floor(K/2) (eq.
 * bisector-ylm-expan, beta <-> theta^(2 beta)).  The auto-spectrum calls return the even
 * ell = 0, 2, .., ell_max, as the paper assumes (Sec. 3.2); the cross spectra of two
 * tracers have even (bym_pk_xi_cross) and odd (bym_pk_xi_cross_odd) multipoles.
 *
 * Conventions shared by every entry point:
 *   - The observer sits at the origin.  Mesh node i (per axis) is at
 *     box_lo + i * box_len / n_mesh; the mesh is periodic.
 *   - delta = paint(galaxies, w) - alpha_r paint(randoms, w), alpha_r =
 *     sum w_g / sum w_r (Sec. 2.1); CIC (assign = 2) or TSC (assign = 3).
 *   - Forward transforms use e^{-i k.x} (Sec. 2, first equation).
 *   - |k| = (2 pi / box_len) sqrt(n.n), |Delta| = (box_len / n_mesh) sqrt(j.j)
 *     with integer labels n, j in [-n_mesh/2, n_mesh/2); a bin b collects
 *     magnitudes in [edges[b], edges[b+1]); k = 0 and Delta = 0 never enter.
 *   - Normalisation (norm = 1): P_ell = 4 pi / A * (bin mean), xi_ell =
 *     4 pi / (A V_cell) * (bin mean), A = alpha_r sum_r nbar_r w_r^2 (FKP);
 *     norm = 0 sets A = V_cell = 1.  norm = 2: P as norm = 1; xi_ell divided
 *     instead by the random-random count, xi_ell(r_b) = S_ell[delta](b) /
 *     (alpha_r^2 S_0[n_r](b)) with S the raw bin sums of the same mesh
 *     estimator (the Landy-Szalay form of the pair counts Sec. 2.2 refers to;
 *     S_0 is line-of-sight independent and taken with the Yamamoto form, one
 *     more painting and two more transforms); bins with no random pairs give 0.
 *   - Outputs are host arrays owned by the caller, laid out [ell/2][bin].
 *   - Calls are synchronous on the given CUDA stream (NULL: the context's
 *     stream) unless submitted through bym_submit.  The context's stream is an
 *     ordinary blocking stream, so it orders after work the caller queued on
 *     the legacy default stream (device catalogs produced there are safe to
 *     pass); device inputs produced on other streams must be complete first.
 *
 * Every function returns BYM_OK (0) or a negative BYM_E_* code; the message
 * of the last failure on a context is available from bym_last_error.  A
 * context is not thread-safe except for bym_submit / bym_poll / bym_wait.
 */
#ifndef BYM_H
#define BYM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BYM_OK = 0,
  BYM_E_INVAL = -1,        /* bad argument (null pointer, bad size, unsorted edges, ...) */
  BYM_E_OUT_OF_BOX = -2,   /* a particle lies outside [box_lo, box_lo + box_len) or is not finite */
  BYM_E_NOMEM = -3,        /* device allocation failed or the request exceeds the HBM budget */
  BYM_E_CUDA = -4,         /* CUDA runtime / cuFFT / NVRTC failure */
  BYM_E_TIMEOUT = -5,      /* bym_wait deadline passed (the request keeps running) */
  BYM_E_UNSUPPORTED = -6,  /* odd ell_max (outside bym_pk_xi_cross_odd), order > 12 (> 4 parity-even),
                              ell_max > 8, n_mesh out of range, a combination a call does not offer */
  BYM_E_BUSY = -7          /* no free serving slot */
};

/* BYM_LOS_MIDPOINT_EVEN is the parity-even form of the midpoint series (Sec. 3.3 and Sec. 4.3
 * boxed estimators; coefficients Phi and F of Appendices D and F.2): even alpha <= order only,
 * available to order 4. */
typedef enum { BYM_LOS_YAMAMOTO = 0, BYM_LOS_MIDPOINT = 1, BYM_LOS_BISECTOR = 2, BYM_LOS_MIDPOINT_EVEN = 3 } bym_los;

typedef struct bym_ctx bym_ctx;

/* A catalog: n objects as (x, y, z, w) float quadruples, row major, and an
 * optional per-object nbar (needed for the randoms when norm = 1 or 2).
 * on_device = 1: the pointers are device pointers of the context's GPU.
 * The caller owns the memory; it is only read during the call. */
typedef struct {
  const float *xyzw;
  const float *nbar;
  int64_t n;
  int on_device;
} bym_catalog;

typedef struct {
  double box_lo[3];   /* position of mesh node (0,0,0) */
  double box_len;     /* cubic box side */
  int n_mesh;         /* N, even, 8 <= N <= 1024 */
  int assign;         /* 2 = CIC, 3 = TSC */
  int ell_max;        /* even, 0..8 */
  int los;            /* bym_los */
  int order;          /* K = highest power of theta kept, 0..12 */
  int compensate;     /* 1: divide each painted-field transform by the assignment window W(k) */
  int precision;      /* 32: FP32 fields and FFTs; 64: FP64 throughout. Shell sums are FP64 either way */
  int norm;           /* 1: FKP normalisation A; 0: raw (A = V_cell = 1); 2: FKP for P, RR for xi */
  int interlace;      /* 1: every painted-field transform averaged with the one on the mesh shifted by
                         half a cell, (F_1 + P F_2) / 2, P(k) = prod_d exp(-i pi n_d / N) (0 at the
                         Nyquist index): cancels the aliased images of odd index sum.  Doubles the
                         paintings, field generations and forward transforms and the field memory;
                         not combined with field ranges (bym_set_field_chunk) */
} bym_params;

typedef struct {
  const double *edges;   /* nbins + 1 increasing edges, host memory */
  int nbins;             /* 1..1024 */
} bym_bins;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the context may hold for requests (0: all free memory).
 * *out receives the context (NULL on failure). */
int bym_create(bym_ctx **out, int device, size_t hbm_budget_bytes);

/* Destroy a context: waits for its work, frees its memory, plans and kernels. */
void bym_destroy(bym_ctx *ctx);

/* Message of the last failure on ctx (owned by ctx, valid until the next call). */
const char *bym_last_error(const bym_ctx *ctx);

/* Library version string (static storage). */
const char *bym_version(void);

/* Projected device bytes one request with these parameters and catalog
 * sizes holds at its peak (the admission test of the serving loop). */
int bym_footprint(const bym_params *p, int64_t n_gal, int64_t n_ran, int want_pk, int want_xi,
                  size_t *bytes);

/* Power-spectrum multipoles, Sec. 2 eq. Pk-def with the LOS of p->los:
 *   pk[(ell/2) * nbins + b]  P_ell in bin b
 *   k_mean[b]                mean |k| of the modes in bin b (may be NULL)
 *   n_modes[b]               number of modes in bin b, full grid (may be NULL)
 * ran may be NULL (no randoms, alpha_r = 0; requires norm = 0). */
int bym_pk_multipoles(bym_ctx *ctx, const bym_catalog *gal, const bym_catalog *ran,
                      const bym_params *p, const bym_bins *kbins, double *pk,
                      double *k_mean, int64_t *n_modes, void *cuda_stream);

/* Correlation-function multipoles, Sec. 2.2 eq. general-2pcf-form with the bin
 * replacement Theta^a / v^a, v^a = n_cells * V_cell:
 *   xi[(ell/2) * nbins + b], r_mean[b], n_cells[b] (last two may be NULL). */
int bym_xi_multipoles(bym_ctx *ctx, const bym_catalog *gal, const bym_catalog *ran,
                      const bym_params *p, const bym_bins *rbins, double *xi,
                      double *r_mean, int64_t *n_cells, void *cuda_stream);

/* Both at once from one painting and one set of fields (the midpoint g
 * functions of eq. g-JM-form and the bisector transforms F[Y_J^M delta] serve
 * P and xi alike).  Same output conventions as the two calls above. */
int bym_pk_xi_multipoles(bym_ctx *ctx, const bym_catalog *gal, const bym_catalog *ran,
                         const bym_params *p, const bym_bins *kbins, const bym_bins *rbins,
                         double *pk, double *k_mean, int64_t *n_modes,
                         double *xi, double *r_mean, int64_t *n_cells, void *cuda_stream);

/* Cross spectra of two tracers on one mesh (even ell): delta_A painted from
 * (gal_a, ran_a) and delta_B from (gal_b, ran_b), each with its own alpha_r.
 * The estimators are those above with delta(r_1) delta(r_2) replaced by
 * delta_A(r_1) delta_B(r_2).  With two densities the two anchored terms of the
 * midpoint series (Sec. 3.2, the bracket before eq. P-ell-k-symm) differ and both
 * are kept: for even ell the g functions become (g^AB + g^BA) / 2 with
 * g^XY = (-1)^J IFFT[delta_X*(k) F[(2r)^-alpha Y_J^M delta_Y](k)] (eq. g-JM-form);
 * the Yamamoto forms take the mean of the lines of sight through either galaxy;
 * the bisector forms pair F[Y delta_A](-k) with F[Y delta_B](k) (eq.
 * bisector-pk-fft, Sec. 6).  Normalisation (norm = 1): A = sqrt(A_A A_B).
 * kbins or rbins may be NULL (that statistic is skipped; its outputs are then
 * not written); outputs as for bym_pk_xi_multipoles.  Both field sets stay
 * resident: the request holds 1 + (number of fields) more mesh slots than the
 * auto spectrum.  BYM_E_UNSUPPORTED with norm = 2, interlacing, or field ranges
 * forced by bym_set_field_chunk (midpoint forms and bisector). */
int bym_pk_xi_cross(bym_ctx *ctx, const bym_catalog *gal_a, const bym_catalog *ran_a,
                    const bym_catalog *gal_b, const bym_catalog *ran_b, const bym_params *p,
                    const bym_bins *kbins, const bym_bins *rbins,
                    double *pk, double *k_mean, int64_t *n_modes,
                    double *xi, double *r_mean, int64_t *n_cells, void *cuda_stream);

/* Odd multipoles ell = 1, 3, .., p->ell_max (p->ell_max odd, 1..7) of the cross spectra
 * of two tracers, for the Yamamoto, midpoint (all-parity series) and bisector lines of
 * sight.  The relabelling (Delta -> -Delta, k -> -k) that brings the first-galaxy terms to
 * the form of the second-galaxy ones leaves a factor (-1)^ell (Sec. 3.2, before eq.
 * P-ell-k-symm), so the Yamamoto form is [Q^AB - Q^BA] / 2, Q^XY = F[Y delta_Y](k)
 * conj(delta_X(k)), the midpoint g fields (J - alpha odd) are [-g^AB + g^BA] / 2, and the
 * bisector sum of eq. bisector-pk-fft contributes its part odd in k.  P_ell is the
 * imaginary part of the shell mean (real densities make it imaginary); xi_ell is real.
 * Odd multipoles change sign under A <-> B and vanish for one tracer.  Arguments and
 * outputs as for bym_pk_xi_cross, laid out [(ell - 1) / 2][bin]; the even multipoles are
 * not computed (call bym_pk_xi_cross).  BYM_E_UNSUPPORTED for the parity-even midpoint
 * form, norm = 2, interlacing, or field ranges / blocks forced by bym_set_field_chunk. */
int bym_pk_xi_cross_odd(bym_ctx *ctx, const bym_catalog *gal_a, const bym_catalog *ran_a,
                        const bym_catalog *gal_b, const bym_catalog *ran_b, const bym_params *p,
                        const bym_bins *kbins, const bym_bins *rbins,
                        double *pk, double *k_mean, int64_t *n_modes,
                        double *xi, double *r_mean, int64_t *n_cells, void *cuda_stream);

/* Compile (without running) the runtime-specialised kernels for these
 * parameters (for the midpoint forms and the bisector also the kernels of
 * field ranges, see bym_set_field_chunk, for the bisector the two-tracer
 * contraction of bym_pk_xi_cross, and except for the parity-even form the odd-multipole
 * kernels of bym_pk_xi_cross_odd with ell_max + 1); works without a GPU.  Used by build
 * checks. */
int bym_jit_check(const bym_params *p, char *log, size_t log_len);

/* Shot-noise level of P_0 (Sec. 2.1: eq. Pk-def includes a shot-noise term that
 * does not depend on the line of sight; the estimators above do not subtract
 * it): *shot = (sum_g w^2 + alpha_r^2 sum_r w^2) / A, with A the FKP
 * normalisation for norm = 1 or 2 and A = 1 for norm = 0 (same conventions as
 * the estimators; ran may be NULL, alpha_r = 0).  The sums run on the GPU.
 * Returns BYM_E_OUT_OF_BOX like the estimators. */
int bym_shot_noise(bym_ctx *ctx, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                   double *shot);

/* Memory bound (Sec. 2.2 and Sec. 6: the g^alpha_{J M} functions of eq.
 * g-JM-form, 145 meshes at ell_max = 4, order 4, and the bisector's F[Y_J^M
 * delta] transforms are the largest memory items).  The paper keeps every
 * field resident; the library can instead hold them in ranges of at most
 * max_fields fields.
 *   Midpoint forms: H_{ell m} of eq. FFT-midpoint and the xi shell sums of
 *   eq. xi-parity-all-estimator are sums over the fields, so the ranges are
 *   generated, convolved and consumed one after another and add up to the same
 *   result; a request holds two delta meshes, one range and the 15 H meshes.
 *   Bisector: the bilinear sum of eq. bisector-pk-fft runs over field pairs,
 *   so two blocks are resident and every block pair adds its share; a block is
 *   transformed again for every earlier block (nb + nb (nb - 1) / 2 block
 *   transforms for nb blocks); a request holds delta, two blocks and, for xi,
 *   the 15 X meshes.
 * max_fields = 0 (the default): ranges only when the whole set does not fit
 * the context's budget (or, with no budget, the device memory free at the
 * start of the request, less room for the FFT work area), sized to fit;
 * > 0: always, with ranges of that many fields.  No effect on the Yamamoto
 * line of sight.  Returns BYM_E_INVAL for max_fields < 0. */
int bym_set_field_chunk(bym_ctx *ctx, int max_fields);

/* FFT backend of ctx.  The library has its own FP32 3D FFT kernels for
 * n_mesh = 512: an x pass (C2C along x of tiles of 16 columns moved by the
 * tensor memory accelerator), a y pass (the same along y) and a z pass (R2C /
 * C2R along z of blocks of 32 rows moved by bulk copies), and a plane pass
 * (R2C along z and C2C along y of one x-plane per thread-block cluster of 8
 * or 16 CTAs); in the midpoint convolution steps the product with conj(delta)
 * sits inside the x pass, between its forward and inverse transforms.
 * mode 0: cuFFT 3D transforms always; 1: the library's plane pass and x pass
 * wherever they apply, 8-CTA clusters; 3: the same with 16-CTA clusters (a
 * non-portable cluster size: a launch the device refuses returns
 * BYM_E_CUDA); 4: cuFFT 2D transforms of the (y, z) planes with the library's
 * x pass; 5: cuFFT 2D plane transforms with cuFFT 1D transforms along x (any
 * n_mesh and precision); 6: the library's z, y and x passes; 2 (the default):
 * whichever bym_autotune measured fastest for the request's shape; if it has
 * not been tuned, mode 6 where the library's kernels apply (n_mesh = 512,
 * FP32), else cuFFT 3D.  With modes 4, 5 and 6 the forward transforms of
 * painted fields skip the x planes that hold no painted value (zero planes,
 * zero transforms), and with mode 6 also the rows y that hold none in any
 * plane (not in requests enqueued into CUDA graphs).  Returns BYM_E_INVAL for
 * other modes. */
int bym_set_fft_backend(bym_ctx *ctx, int mode);

/* Autotuner.  Runs the given request (which must be valid) several times on
 * ctx under candidate launch shapes -- blocks per SM of the grid-stride
 * kernels, cuFFT batch size, library FFT kernels or cuFFT -- timing every
 * kernel with the tracer, and keeps the fastest choice per kernel for requests
 * with the same (n_mesh, precision, los) on ctx.  cache_path (may be NULL): a
 * text file of earlier choices; a matching entry is used without measuring,
 * a new choice is appended.  report (may be NULL) receives a one-line JSON
 * summary of the choice. */
int bym_autotune(bym_ctx *ctx, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                 const bym_bins *kbins, const bym_bins *rbins, const char *cache_path, char *report,
                 size_t report_len);

/* In-place batched FP32 3D FFTs of `count` meshes at `data` (device), each
 * n_mesh * n_mesh * (n_mesh + 4) floats (rows of n_mesh values and 4 of
 * padding): forward R2C (inverse = 0) gives the half-spectrum in the same
 * memory, rows of n_mesh/2 + 2 complex values of which kz = 0..n_mesh/2 are
 * the transform (the last is padding); inverse C2R (inverse = 1) is
 * unnormalised.  Sign e^{-i k.x} forward (Sec. 2 Fourier convention). */
int bym_fft3d(bym_ctx *ctx, void *data, int n_mesh, int count, int inverse, void *cuda_stream);

/* Kernel tracing.  While enabled, every launch of the library's own kernels
 * and every cuFFT execution on ctx is bracketed by CUDA events on its stream;
 * bym_profile_read writes a JSON object
 *   {"<kernel>": {"launches": n, "ms": total, "bytes": algorithmic bytes}, ...}
 * into json (truncated to len) and, if reset != 0, clears the totals.
 * Algorithmic bytes are the bytes each launch must move at minimum (inputs
 * read once, outputs written once). */
int bym_profile_enable(bym_ctx *ctx, int enable);
int bym_profile_read(bym_ctx *ctx, char *json, size_t len, int reset);

/* ---------------------------------------------------------------------------
 * Serving and batching.  A context can run a serving loop: n_slots worker
 * slots, each with its own CUDA stream, cuFFT plans and work area, take
 * requests from a queue as slots and HBM budget free up (continuous
 * batching; first request that fits is admitted, so a large request does not
 * block small ones behind it).  Work of different slots overlaps on the GPU.
 * Each request's projected footprint (bym_footprint) is charged against the
 * budget while it runs.  The caller owns every array a request points to and
 * must keep it alive and unchanged until the request is done.
 * ------------------------------------------------------------------------- */
typedef struct {
  bym_catalog gal, ran;   /* ran.n = 0: no randoms */
  bym_params params;
  bym_bins kbins, rbins;  /* nbins = 0: that statistic is not requested */
} bym_request;

typedef struct {          /* caller-allocated host outputs, as for bym_pk_xi_multipoles */
  double *pk, *k_mean;
  int64_t *n_modes;
  double *xi, *r_mean;
  int64_t *n_cells;
} bym_result;

/* Start the serving loop (n_slots 1..16; hbm_budget_bytes 0: 90 % of the
 * free device memory).  BYM_E_BUSY if a loop is already running. */
int bym_serve_start(bym_ctx *ctx, int n_slots, size_t hbm_budget_bytes);
/* Stop after the queued and running requests have finished. */
int bym_serve_stop(bym_ctx *ctx);
/* Queue a request; *ticket identifies it.  BYM_E_NOMEM if its footprint can
 * never fit the budget; BYM_E_INVAL for bad arguments (checked at submit). */
int bym_submit(bym_ctx *ctx, const bym_request *req, const bym_result *out, uint64_t *ticket);
/* *done = 1 once the request has finished (successfully or not). */
int bym_poll(bym_ctx *ctx, uint64_t ticket, int *done);
/* Wait up to timeout_s seconds (< 0: forever).  Returns BYM_E_TIMEOUT if the
 * request is still queued or running (it keeps going); otherwise BYM_OK with
 * the request's own return code in *status, and forgets the ticket. */
int bym_wait(bym_ctx *ctx, uint64_t ticket, double timeout_s, int *status);
/* Latency statistics of the requests finished since the loop started:
 * stats[0] count, [1] p50 and [2] p99 of submit-to-done seconds, [3] p50 and
 * [4] p99 of run (start-to-done) seconds, [5] mean queueing seconds,
 * [6] peak HBM bytes charged at once. */
int bym_serve_stats(bym_ctx *ctx, double stats[7]);
/* Forget the latency records and restart the peak at the bytes charged now
 * (e.g. after warm-up requests).  BYM_E_INVAL if no loop is running. */
int bym_serve_reset_stats(bym_ctx *ctx);
/* Run n requests through the serving loop (started with 4 slots and the
 * default budget for the call if none is running) and wait for all;
 * status[i] receives each request's return code. */
int bym_batch_run(bym_ctx *ctx, int n, const bym_request *reqs, const bym_result *outs, int *status);
/* Run n requests as one CUDA graph: host catalogs are first copied to the
 * device, one request of every distinct shape (mesh, precision, LOS, ell_max,
 * order, compensation, box, bins) runs uncaptured so that its kernels, bin
 * tables, FFT plans and work area exist, then every request (and, for
 * norm = 2, its random-random pass) is enqueued under stream capture on four
 * parallel branches (as bym_batch_plan_create below), the graph is launched
 * once, and the results are normalised on the host.  Suits many mocks of few shapes (the warm-up is paid once per shape
 * and process).  The context's serving loop, if running, is not used.
 * status[i] receives each request's return code; a failure of the capture or
 * of the graph is reported for every request.  Returns the first error. */
int bym_batch_graph(bym_ctx *ctx, int n, const bym_request *reqs, const bym_result *outs, int *status);

/* The same batch kept as an instantiated graph for repeated launches (a
 * persistent batch of mocks: new catalog contents written into the same
 * device buffers, same sizes, between launches).  The graph has n_streams
 * parallel branches (0: 4), each with its own engine (FFT plans, work area,
 * bin tables, settings copied from ctx) like a serving slot; requests go to
 * the least loaded branch, largest first, so their work overlaps on the GPU.
 * create captures and instantiates (status[i]: each request's validation /
 * warm-up outcome; the others are captured); launch runs the graph once and
 * fills the result arrays given at creation (status may be NULL); destroy
 * frees the plan (branch engines, device copies of host catalogs, pinned
 * areas, graph).  Host catalogs are copied to the device once, at creation.
 * The context must outlive the plan. */
typedef struct bym_batch bym_batch;
int bym_batch_plan_create(bym_ctx *ctx, int n, const bym_request *reqs, const bym_result *outs, int n_streams,
                          bym_batch **plan, int *status);
int bym_batch_plan_launch(bym_batch *plan, int *status);
void bym_batch_plan_destroy(bym_batch *plan);

/* Yamamoto P_ell(k) from field spectra the caller already holds, for callers
 * that cannot allocate device memory (an allocator owned by another framework,
 * a fixed memory budget carved out up front, code that runs while allocation
 * is not allowed).  The paper has no counterpart of this entry point; it is
 * the k-space contraction and FP64 shell binning of bym_pk_multipoles with
 * LOS = Yamamoto, run on the caller's data without any cudaMalloc.
 *   F: device memory, (ell_max/2+1)^2 consecutive half-spectra of
 *      n_mesh * n_mesh * (n_mesh/2 + 1) complex floats (re, im interleaved,
 *      kz fastest), the forward transforms of Y_{l mu}(hat x) delta(x) for
 *      even l <= ell_max, mu = -l..l, in that order.  Y_{l mu} are the real
 *      spherical harmonics Y_{l,0} = Y_l^0, Y_{l,m} = sqrt2 (-1)^m Re Y_l^m,
 *      Y_{l,-m} = sqrt2 (-1)^m Im Y_l^m (m > 0), Y_l^m as in DLMF 14.30.
 *   D: device memory, the half-spectrum of delta in the same layout.
 *   pk, n_modes: host outputs as for bym_pk_multipoles; P_ell = 4 pi / norm_A
 *      times the bin mean (no compensation).
 * Limits: FP32 spectra, n_mesh <= 512, ell_max <= 4, nbins <= 1024; larger
 * requests return BYM_E_UNSUPPORTED.  Scratch lives in one static device array
 * of 1 MiB that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other streams, other host
 * threads) race and corrupt each other's sums.  The current device is used;
 * the call is synchronous on cuda_stream (NULL: the legacy default stream). */
int bym_pk_yamamoto_from_spectra_noalloc(const void *F, const void *D, int n_mesh, double box_len,
                                         int ell_max, const bym_bins *kbins, double norm_A, double *pk,
                                         int64_t *n_modes, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BYM_H */
