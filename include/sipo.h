/*
 * sipo.h -- C ABI of the GB300 (sm_103a) SiPO projection-LP solver.
 *
 * SiPO (scale-invariant projection optimisation for tomographic volumetric
 * additive manufacturing) designs a projection sinogram y >= 0 by solving a
 * linear program over the linear dose model f = A^T y, A^T = K P^T (Sec. 2.3,
 * Eqs. 2-3).  This library implements the matrix-free primal-dual hybrid
 * gradient (PDHG) solve of that LP (Sec. 2.8, KKT conditions of Sec. 6.1) for
 * the general form (Eqs. 19-24), Case 1 (Eqs. 32-37) and Case 2 (Eqs. 40-45),
 * plus the forward and adjoint operators themselves.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layouts: a volume is [ny][nx][nz] and a sinogram [n_angles][n_det][nz],
 *   C-contiguous with z (the rotation axis) fastest.  Voxel centres sit at
 *   (i - (n-1)/2); angle k has detector coordinate
 *   u = x cos(theta_k) + y sin(theta_k) + (n_det-1)/2, and P^T interpolates
 *   linearly between bins floor(u) and floor(u)+1; P is its exact transpose.
 * Attenuation (vial radius R > 0, coefficient mu): the tap from voxel (x,y) to
 *   bin j is weighted by exp(-mu (t + sqrt(R^2 - s_j^2))), t = -x sin + y cos,
 *   s_j = j - (n_det-1)/2; 0 when |s_j| > R; voxels with x^2+y^2 > R^2 are
 *   outside the operator.
 * PSF K: separable Gaussian per axis, sigma = (sigma_x, sigma_y, sigma_z),
 *   radius R_a = ceil(trunc * sigma_a) fixed at creation, taps normalised to
 *   sum 1, zero padding (so K is symmetric); sigma_a = 0 is the identity.
 * Return codes: every function returns SIPO_OK (0) or a negative SIPO_ERR_*;
 *   the thread-local message of the last failure is sipo_last_error().
 *   Failures leave the context usable unless the code is SIPO_ERR_CUDA from
 *   a sticky device error.
 * Streams: a NULL stream means the context's own stream.  Calls that take a
 *   stream enqueue their work on it and return without synchronising unless
 *   stated.
 * Ownership: the library never frees caller memory; device buffers passed in
 *   are caller-owned and must stay valid until the enqueued work completes.
 */
#ifndef SIPO_H
#define SIPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SIPO_OK 0
#define SIPO_ERR_INVALID_ARG (-1)
#define SIPO_ERR_CUDA (-2)
#define SIPO_ERR_OOM (-3)
#define SIPO_ERR_TIMEOUT (-4)
#define SIPO_ERR_NUMERIC (-5)
#define SIPO_ERR_UNSUPPORTED (-6)

/* solve status (sipo_result.status); infeasibility is a result, not an error
 * (Secs. 2.7.1 and 2.7.2 read an infeasible LP as a process diagnostic) */
#define SIPO_OPTIMAL 0
#define SIPO_PRIMAL_INFEASIBLE 1
#define SIPO_DUAL_INFEASIBLE 2
#define SIPO_ITER_LIMIT 3

/* LP forms */
#define SIPO_GENERAL 0 /* Eqs. 19-24: min w1 u~ + w2 v~ */
#define SIPO_CASE1 1   /* Eqs. 32-37: min u~ under dose tolerances (Eqs. 29-31) */
#define SIPO_CASE2 2   /* Eqs. 40-45: min v~ under the inhibition bound (Eq. 39) */

/* element types */
#define SIPO_F32 0
#define SIPO_F64 1
#define SIPO_BF16 2

/* where a pointer lives */
#define SIPO_HOST 0
#define SIPO_DEVICE 1

/* region labels (Sec. 2.2, Fig. 2) */
#define SIPO_EXT 0
#define SIPO_BAND 1
#define SIPO_GEL 2

typedef struct sipo_ctx sipo_ctx;

/* Geometry (Secs. 2.2-2.3).  `angles` is a host array of n_angles radians,
 * copied at creation.  vial_radius <= 0 means no vial (then mu must be 0).
 * psf_sigma[a] = 0 disables the PSF along axis a (x, y, z order); psf_trunc
 * is the truncation in sigmas (4 if <= 0). */
typedef struct sipo_geometry {
  int nx, ny, nz;
  int n_angles;
  const double *angles;
  int n_det;
  double vial_radius;
  double mu;
  double psf_sigma[3];
  double psf_trunc;
} sipo_geometry;

/* LP form and its data.  General: weights w1, w2 (Eq. 19).  Case 1: dose
 * tolerances f_L = (1 - tol_lo) f_T, f_U = (1 + tol_hi) f_T (Eq. 29),
 * f_crit = min_gel f_L (Eq. 30).  Case 2: f_crit = inhibit_ratio *
 * min_gel f_T (the inhibition threshold of Sec. 2.7.2).  band_width: the band
 * is the non-gel voxels within Euclidean distance <= band_width of the gel,
 * plus the support of K f_T (Sec. 2.2); band_width < 0 means band-free
 * (every non-gel voxel inside the vial is band). */
typedef struct sipo_case_params {
  int kase;
  double w1, w2;
  double tol_lo, tol_hi;
  double inhibit_ratio;
  int band_width;
} sipo_case_params;

/* Solver controls.  kkt_tol: relative KKT tolerance (primal, dual and gap
 * each <= kkt_tol; 0 runs to max_iter).  check_every: iterations between KKT
 * and restart checks (64 if <= 0).  storage: element type of the iterates
 * (SIPO_F32, SIPO_BF16 with FP32 arithmetic, or SIPO_F64); residuals, gap,
 * step sizes, restart logic and the u~/v~ scalars are FP64 in every mode.
 * tile_cfg: -1 lets the library choose the backprojector's tile shape,
 * otherwise an index into its tile table (see sipo_tile_count).
 * primal_weight: initial primal weight omega of the preconditioned PDHG (<= 0:
 * the library's default rule). */
typedef struct sipo_tolerances {
  double kkt_tol;
  long long max_iter;
  int check_every;
  int storage;
  int tile_cfg;
  double primal_weight;
} sipo_tolerances;

/* Result of sipo_solve.  kkt = max(rel_primal, rel_dual, rel_gap) of the
 * returned point; pobj/dobj are the primal/dual objectives of the normalised
 * LP; u, v are u~*, v~*.  Metrics of the dose d = A^T y (Eqs. 6-8, 46):
 * dtvr_f, dsr, psr_f; alpha: the dose-domain post-scaling factor of Eq. 27
 * with unit weights; s: min_gel(d / f~_L), the recovered Charnes-Cooper scale
 * (t = 1/s, Eq. 18; 1 at an optimum). */
typedef struct sipo_result {
  int status;
  int restarts;
  long long iters;
  double kkt, rel_primal, rel_dual, rel_gap;
  double r_primal, r_dual, gap, pobj, dobj;
  double u, v, omega;
  double f_crit, alpha, dtvr_f, dsr, psr_f, s;
  double solve_ms;
  long long kernel_launches;
  int tile_cfg; /* backprojector tile table entry in use */
  int cert_slice; /* PRIMAL_INFEASIBLE proved by the bound-based test on one
                     z-slice (operators without z coupling): that slice's
                     index; -1 otherwise */
} sipo_result;

/* Creates a solver context: copies the geometry and the target dose f_T
 * ([ny][nx][nz] float32, host or device per f_T_location), builds the region
 * labels, the active-ray mask (Pi_act = {[P f_T]_j != 0}, Sec. 2.2), the
 * normalised target (Sec. 2.5 / Eqs. 30-31 / Eq. 39) and the diagonal
 * preconditioners, all on the device.  `stream` (cudaStream_t or NULL) is the
 * context's stream for solves; creation itself synchronises it.  The context
 * lives on the device current at creation; every later call on it must be
 * made with that device current.  On success *out owns all internal device
 * memory until sipo_destroy.  Errors:
 * INVALID_ARG (sizes, NaN/negative target, empty gel, mu > 0 without vial, an
 * empty band in Case 1 or the general form: the band maximum u~ is then in no
 * row and the LP is unbounded),
 * OOM, CUDA. */
int sipo_create(const sipo_geometry *geo, const float *f_T, int f_T_location,
                const sipo_case_params *cp, const sipo_tolerances *tol,
                void *stream, sipo_ctx **out);

/* Case 1 with explicit per-voxel dose bounds (Sec. 2.7.1 with response-domain
 * tolerances: f_L = M^-1(m_L), f_U = M^-1(m_U), Eq. 5, which are in general
 * not proportional to f_T).  As sipo_create, plus f_L and f_U ([ny][nx][nz]
 * float32, host or device per `location`, like f_T): the gel rows become
 * f_L,i / f_crit <= [A^T y]_i <= f_U,i / f_crit with f_crit = min_gel f_L
 * (the weakest admissible part).  f_T still defines the labels (gel =
 * f_T > 0), the active rays and the dose metrics; case->kase must be
 * SIPO_CASE1 and its tol_lo / tol_hi are not used.  Errors: as sipo_create,
 * and INVALID_ARG where a gel voxel has f_L <= 0, f_U < f_L or a bound that
 * is not finite. */
int sipo_create_bounded(const sipo_geometry *geo, const float *f_T, const float *f_L, const float *f_U,
                        int location, const sipo_case_params *cp, const sipo_tolerances *tol, void *stream,
                        sipo_ctx **out);

/* Material response model (Sec. 2.1): Richards' generalised logistic curve,
 * Eq. 4, m = M(f) = alpha + (k - alpha) / [1 + exp(-beta (f - f0))]^(1/gamma),
 * with lower and upper asymptotes alpha < k, growth rate beta > 0, shape
 * gamma > 0 and location f0 (resin constants supplied by the caller). */
typedef struct sipo_response {
  double alpha, k, beta, gamma, f0;
} sipo_response;

/* Response-domain post-scaling and metrics of a solved dose (Sec. 2.7, Eq. 28
 * with unit weights, Eq. 46).  alpha: the post-scaling factor used (physical
 * dose = alpha * d with d the normalised dose A^T y*); phi: Phi_m(alpha);
 * psr_m: min_gel M(alpha d) / max_band M(alpha d); dtvr_m and its two parts
 * ratio_max / ratio_min: max and min over gel of M(alpha d_i) / m_T,i;
 * m_band_max, m_gel_min: max over band and min over gel of M(alpha d). */
typedef struct sipo_response_result {
  double alpha, phi, psr_m, dtvr_m, ratio_min, ratio_max, m_band_max, m_gel_min;
} sipo_response_result;

/* Elementwise response map on the device, for the front end (target
 * response to target dose, Eq. 5; tolerance bounds (1 -+ eps) m_T through
 * `scale`) and for reading doses as responses (Eq. 4).  With v = scale * in:
 * inverse = 0: out = M(v); inverse = 1: out = M^-1(v)
 * = f0 - ln[((k - alpha) / (v - alpha))^gamma - 1] / beta for
 * alpha < v < k, 0 for v <= alpha (no prescription: outside the part).
 * in, out: n float32 device values (may alias); computed in FP64; enqueued on
 * `stream` and synchronised.  Errors: INVALID_ARG (bad model, null, scale not
 * finite, or, with inverse = 1, a value >= k or NaN: outside the invertible
 * range; out is then written with 0 there), CUDA. */
int sipo_response_map(const sipo_response *M, const float *in, float *out, long long n, double scale,
                      int inverse, void *stream);

/* The inhibition ratio of Case 2 for a threshold given as a response
 * (Sec. 2.7.2 mapped through Eq. 5): r = M^-1(m_crit) / M^-1(min m_T), the
 * minimum over the device float32 array m_T (n values) of the responses above
 * the lower asymptote alpha (the part; M is increasing, so this is the
 * part's smallest prescribed dose).  *ratio receives r, *gel_min (nullable)
 * that minimum response.  Synchronises `stream`.  Errors: INVALID_ARG (bad
 * model, null, n <= 0, m_crit outside (alpha, k), no response inside
 * (alpha, k)), CUDA. */
int sipo_response_inhibit_ratio(const sipo_response *M, const float *m_T, long long n, double m_crit,
                                double *ratio, double *gel_min, void *stream);

/* Response-domain back end of ctx's last solve: m_T ([ny][nx][nz] float32,
 * host or device per `location`, positive on gel) is the target response.
 * alpha > 0 is used as the post-scaling factor; otherwise (0, negative or
 * not finite) alpha minimises Phi_m(alpha) = sum_gel (M(alpha d_i) -
 * m_T,i)^2 (Eq. 28, unit weights) by a grid search: 32 factors spaced
 * geometrically from 1/16 to 16 times the dose-domain factor of Eq. 27, then
 * six rounds of 32 linearly spaced factors between the best one's
 * neighbours.  Synchronises ctx's stream.  Errors: INVALID_ARG (bad model,
 * null, ctx not solved), CUDA. */
int sipo_response_metrics(sipo_ctx *ctx, const sipo_response *M, const float *m_T, int location, double alpha,
                          sipo_response_result *out);

/* Runs the restarted Halpern PDHG (Sec. 2.8) from a zero start until the
 * KKT tolerance, a primal-infeasibility certificate or max_iter, then the
 * post-solve metrics of f~* = A^T y* (recomputed by one operator application
 * at the returned point).  Without a PSF extent along z the bound-based
 * certificate is tested slice by slice (the forward model is slice-separable,
 * Sec. 2.3: one infeasible slice makes the LP infeasible), and
 * res->cert_slice names the slice.  y_out (nullable) receives y*, the normalised
 * projection of Eq. 18, as [n_angles][n_det][nz] in FP32 (FP64 when storage
 * is SIPO_F64), host or device per y_location.  Blocks until done.  Errors:
 * INVALID_ARG, CUDA, TIMEOUT (a bounded device-side wait of the staged
 * backprojector gave up), NUMERIC (a check found NaN or infinite residuals,
 * e.g. from an infinite imported start; or the staged backprojector's rows did
 * not fit its box, which the geometry cannot produce); the context stays
 * usable. */
int sipo_solve(sipo_ctx *ctx, void *y_out, int y_location, sipo_result *res);

/* Warm start, for precision escalation (a reading of the mixed-precision
 * requirement: iterates stored in BF16 stall above tight tolerances, so a
 * BF16 solve is continued in FP32 from where it stopped).  Copies the point
 * T(z) of the last KKT check of `src`'s most recent solve, with its scalars
 * u~, v~ and its primal weight, into `dst`, converting the storage type; the
 * next sipo_solve or sipo_solve_batched of `dst` starts from it, as a restart
 * point (iterate and anchor), instead of from zero.  Both contexts must hold
 * the same problem (sizes, angles, case parameters, labels; checked through
 * a fingerprint), must have been created with the same device current, and
 * may differ in storage and tile settings.  Synchronises
 * both contexts' work.  Errors: INVALID_ARG (null, same context, different
 * problems, src never solved), CUDA. */
int sipo_warm_start(sipo_ctx *dst, const sipo_ctx *src);

/* Checkpoint (no passage of the paper: solver state for resume).  Copies the
 * point T(z) of the last KKT check of ctx's most recent solve — the point a
 * warm start or a resume continues from — out in the compute type (FP32, or
 * FP64 when storage is SIPO_F64), host or device per `location`: y
 * [n_angles][n_det][nz], lam_up and lam_lo [ny][nx][nz] (each nullable), and
 * scalars[4] = {u~, v~, omega, iterations} (nullable).  Synchronises ctx's
 * stream.  Errors: INVALID_ARG (null ctx, bad location, ctx never solved),
 * CUDA. */
int sipo_get_state(sipo_ctx *ctx, void *y, void *lam_up, void *lam_lo, int location, double *scalars);

/* Resume: the next sipo_solve or sipo_solve_batched of ctx starts from the
 * point (y, lam_up, lam_lo) with scalars[0..2] = {u~, v~, omega} (layouts and
 * type as sipo_get_state; scalars[3] is not read: the resumed solve counts
 * its iterations from 0), instead of from zero.  The point is projected onto
 * the domains of Eqs. 20-24 (y >= 0 on active rays; lam_up >= 0 on band and
 * gel rows, lam_lo >= 0 on gel rows; other entries 0); A^T y and
 * A (lam_up - lam_lo) are recomputed; u~, v~ out of their bounds (u~ < 0,
 * v~ < 1, not finite) become the smallest the point allows, as for
 * sipo_set_primal, and omega <= 0 the default.  The point becomes iterate and
 * restart anchor.  Synchronises ctx's stream.  Errors: INVALID_ARG (null, bad
 * location), CUDA. */
int sipo_set_state(sipo_ctx *ctx, const void *y, const void *lam_up, const void *lam_lo, int location,
                   const double *scalars);

/* Primal start, for the two-stage design of Sec. 3.2 (a Case-1 solve fixes
 * the process bound, a Case-2 solve at that bound then recovers conformity,
 * starting from the Case-1 point rescaled).  The next sipo_solve or
 * sipo_solve_batched of `ctx` starts from the primal point y, a normalised
 * projection as sipo_solve returns it ([n_angles][n_det][nz], FP32, or FP64
 * when storage is SIPO_F64, host or device per y_location, read before the
 * call returns), instead of from zero.  y is projected onto the primal domain
 * (negative, NaN and inactive-ray values become 0).  u and v are u~ (general,
 * Case 1) and v~ (general, Case 2); a negative or non-finite value asks for
 * the smallest the point allows (u~ = max of A^T y on band rows, v~ = max of
 * A^T y / f~ on gel rows and at least 1); the one a case lacks is ignored.
 * Duals start at zero, the primal weight at its default, and the point is
 * both iterate and restart anchor.  Synchronises ctx's stream.  Errors:
 * INVALID_ARG (null, bad location), CUDA. */
int sipo_set_primal(sipo_ctx *ctx, const void *y, int y_location, double u, double v);

/* Primal start taken from another context on the device, for the two-stage
 * design of Sec. 3.2 without a host round trip: the point y that src's most
 * recent sipo_solve returned (its last check's T(z), in src's storage type),
 * multiplied by `scale` (finite, > 0), becomes dst's primal start exactly as
 * sipo_set_primal would make it (projected onto the primal domain; u, v as
 * there; duals zero).  The Case-1 -> Case-2 transfer passes scale = 1 / r,
 * the stage-1 dose over (1 - d_lo) in stage-2 normalised units.  Both
 * contexts must have the same geometry (sizes, angles, vial, attenuation,
 * PSF) and device; their LP cases may differ.  Synchronises both streams.
 * Errors: INVALID_ARG (null, same context, scale, geometry mismatch, src not
 * solved), CUDA. */
int sipo_set_primal_from(sipo_ctx *dst, const sipo_ctx *src, double scale, double u, double v);

/* Farkas test with a dual point from another context, for the infeasibility
 * diagnostic of Secs. 2.7.1-2.7.2.  The dual point (lam_up, lam_lo) of src's
 * most recent solve (its last check's T(z)) is tested once as a ray proving
 * ctx's LP (Case 1 or Case 2) primal infeasible, with the bound-based test
 * that sipo_solve runs at every check (slice by slice when the PSF has no z
 * extent).  The test is homogeneous in the ray, so src may normalise the same
 * part differently: the general form with w1 = 1, w2 = 0 on the same target
 * and band minimises the band-to-gel dose ratio, and when its optimum u~*
 * exceeds a Case-2 ratio r its optimal dual is a Farkas ray of Case 2 at r
 * (Eqs. 40-45: band d <= 1 and gel d >= f_T / (r min f_T) cannot both hold).
 * *certified = 1 if the test proves infeasibility (then *slice, if non-null,
 * receives the slice that carries it, or -1 for a whole-volume proof), else
 * 0.  Both contexts must have the same geometry, device and region labels.
 * Resets ctx's solver state (a later sipo_solve starts from zero).
 * Synchronises both streams.  Errors: INVALID_ARG (null, same context,
 * mismatch, general-form ctx, src not solved), CUDA, TIMEOUT. */
int sipo_farkas_from(sipo_ctx *ctx, const sipo_ctx *src, int *certified, int *slice);

/* sipo_solve of ctx that probes target's infeasibility along the way: every
 * probe_every iterations (rounded up to check periods) and when the solve
 * stops, the dual point of ctx's last check is tested as a Farkas ray of
 * target's LP (as sipo_farkas_from does); the solve stops at the first
 * certificate, with *certified = 1 and *slice as in sipo_farkas_from, else
 * *certified = 0.  res receives ctx's result as from sipo_solve (status
 * ITER_LIMIT when a certificate ended it early; the returned point, and the
 * state sipo_get_state exports, are then the check whose dual passed).  For the separation solve of
 * Case 2: ctx holds the same part as Case 1 with tol_lo = 0 (gel dose at least
 * its target, band dose at most u~), target the Case-2 LP.  Errors: as
 * sipo_solve and sipo_farkas_from (a target whose LP cannot test ctx's duals
 * is refused before any iteration runs). */
int sipo_solve_probe(sipo_ctx *ctx, sipo_ctx *target, long long probe_every, sipo_result *res, int *certified,
                     int *slice);

/* sipo_solve_probe of ctx (Farkas probes of target) while a third context,
 * rival, is solved at the same time on its own stream: each round launches
 * one check period of every context still running (ctx and rival overlap on
 * the device), then reads both states.  A context stops running at its own
 * decision or its iteration cap while the other goes on.  The call ends at
 * the first probe certificate (*certified = 1, *slice as in sipo_farkas_from;
 * rival stopped at its last check), at the rival's own decision (optimal,
 * infeasible by its own certificate, or non-finite; ctx stopped at its last
 * check), or when both have stopped.  res and rival_res receive the two
 * results as from sipo_solve (ITER_LIMIT for a solve the other one ended).
 * For Case 2 with its feasibility settled (Secs. 2.7.1-2.7.2): ctx holds the
 * separation LP, target and rival the Case-2 LP at ratio r (two contexts: a
 * probe resets target's solver state); a feasible r ends with the rival's
 * optimum, an infeasible one with the separation dual's certificate.  The
 * three contexts must be distinct, ctx and rival on one device.  Errors: as
 * sipo_solve and sipo_farkas_from (a target whose LP cannot test ctx's duals
 * is refused before any iteration runs). */
int sipo_solve_race(sipo_ctx *ctx, sipo_ctx *target, sipo_ctx *rival, long long probe_every, sipo_result *res,
                    sipo_result *rival_res, int *certified, int *slice);

/* Solves n independent contexts as one batch (a parameter sweep): one CUDA
 * graph holds one check period of every context as parallel branches (each on
 * its context's stream), so small LPs share the device and the host waits
 * once per period.  When contexts finish, the graph is captured again without
 * them.
 * In a batch the iteration limit of each context is rounded up to a whole
 * number of its check periods.  Each context must appear once, all must have
 * been created on one device; contexts created on the same stream run one
 * after another.  y_outs may be NULL or an
 * array of n nullable pointers (same rules as sipo_solve).  results: n
 * entries. */
int sipo_solve_batched(sipo_ctx **ctxs, int n, void **y_outs, int y_location,
                       sipo_result *results);

/* A vol = P_mu K vol (the adjoint of Eq. 3): vol is a device volume, sino a
 * device sinogram, both of `dtype` (SIPO_F32 or SIPO_F64).  Enqueued on
 * `stream`.  With a PSF, uses a context-owned temporary volume, so calls on
 * one context must not overlap in time on different streams. */
int sipo_project(sipo_ctx *ctx, const void *vol, void *sino, int dtype, void *stream);

/* A^T sino = K P_mu^T sino (Eq. 3); arguments as sipo_project. */
int sipo_backproject(sipo_ctx *ctx, const void *sino, void *vol, int dtype, void *stream);

/* K vol (deriv_axis < 0) or (dK/dsigma_a) vol for a = deriv_axis in {0:x,
 * 1:y, 2:z} with the radii frozen at creation; device volumes of `dtype`. */
int sipo_psf_apply(sipo_ctx *ctx, const void *in, void *out, int dtype, int deriv_axis,
                   void *stream);

/* PSF-sigma gradient of the bilinear form <sino, A vol> = <sino, P_mu K vol>:
 * grad[a] = < P_mu^T sino, (dK/dsigma_a) vol > for a = 0 (x), 1 (y), 2 (z),
 * written to host memory (synchronises `stream`).  P_mu^T sino is recomputed
 * into a context-owned temporary rather than stored.  With sino = dL/d(A p)
 * and vol = p this is dL/dsigma of a projection; with sino = y and vol =
 * dL/d(A^T y) it is dL/dsigma of a backprojection (K is symmetric).  sino and
 * vol are device arrays of `dtype`; axes without a PSF get 0. */
int sipo_psf_grad(sipo_ctx *ctx, const void *sino, const void *vol, int dtype, double *grad,
                  void *stream);

/* Replaces the PSF sigmas (radii stay frozen); affects later operator calls. */
int sipo_set_psf_sigma(sipo_ctx *ctx, const double sigma[3]);

/* Copies internal arrays out (synchronous).  which: 0 region labels (uint8,
 * volume), 1 active-ray mask (uint8, sinogram), 2 y (compute type, sinogram),
 * 3 lambda_up, 4 lambda_lo (compute type, volume; the duals of the up rows
 * -- band and gel upper bounds -- and of the gel lower bound), 5 dose
 * d = A^T y (compute type, volume).  After sipo_solve, 2-5 hold the returned
 * point.  location: SIPO_HOST or SIPO_DEVICE. */
int sipo_get_array(sipo_ctx *ctx, int which, void *out, int location);

/* Runs `iters` PDHG iterations without graph capture, timing every kernel
 * phase with CUDA events on the context stream; phase_ms[i] receives the
 * average milliseconds per iteration of phase i for i < n_phases (at most
 * sipo_phase_count()).  Leaves the solver state advanced by `iters`. */
int sipo_profile(sipo_ctx *ctx, int iters, double *phase_ms, int n_phases);
int sipo_phase_count(void);
const char *sipo_phase_name(int i);

/* Number of entries in the backprojector tile table (for sipo_tolerances.tile_cfg):
 * 0 = 8 voxel columns per warp at 2 blocks/SM, 1 = 4 columns at 2 blocks/SM,
 * 2 = 4 columns at 3 blocks/SM, 3 and 4 = the single-precision row-pattern
 * kernel (4 columns, the rows of each angle in registers, packed FP32
 * multiply-adds) at 2 and 3 blocks/SM, 5 and 6 = the row-pattern kernel fed
 * by tensor-memory (TMA) copies of each angle's detector rows into shared
 * memory, at 3 and 2 blocks/SM, when nz is a multiple of 256 (else entry 4).
 * FP64 contexts run entry 2 for 3-6.  Every entry gives the same sums bit for
 * bit within one precision. */
int sipo_tile_count(void);

/* Checked builds (compiled with -DSIPO_CHECKED, the library
 * libsipo_checked.so): synchronises the device and returns the bits of the
 * index and finiteness checks the kernels recorded since the last call (bit 0
 * projector tap column or z offset, bit 1 backprojector detector or staged
 * row, bit 2 epilogue z offset, bit 3 non-finite FP64 block sum), with bit 30
 * set to mark a checked build, and clears them.  A plain build returns 0.
 * The checks never trap: a violation is recorded and the kernel goes on. */
unsigned int sipo_check_flags(void);

/* Self-test of the bounded waits of the staged backprojector (table entries 5
 * and 6): one block of `threads` threads (1..1024) on the current device waits
 * on an mbarrier's first phase with a budget of `budget_cycles` SM clock cycles
 * (> 0).  With `arrive` != 0 thread 0 makes the one arrival the barrier expects
 * and every wait ends at once; with `arrive` == 0 nothing completes the phase
 * and every wait gives up after its budget, as a wait on a tensor-memory copy
 * that never lands does in the kernel (where it sets the fault that makes the
 * solve return SIPO_ERR_TIMEOUT).  *timed_out receives the number of threads
 * whose wait gave up.  Returns SIPO_ERR_TIMEOUT when every wait gave up,
 * SIPO_OK when none did, SIPO_ERR_CUDA on a CUDA error, SIPO_ERR_INVALID_ARG
 * for bad arguments.  Synchronises the device; no solver state is touched. */
int sipo_wait_selftest(long long budget_cycles, int arrive, int threads, unsigned int *timed_out);

/* Total kernels this library has launched in this process (graph nodes count
 * once per graph launch). */
long long sipo_kernel_launch_count(void);

/* Convergence trace of the last solve: one entry per KKT check (at most
 * 4096), 10 doubles each: iteration, relative KKT, relative primal
 * residual, relative dual residual, relative gap, primal objective, primal
 * weight, restarts so far, and the relative violations of the two Farkas
 * candidates tested for primal infeasibility (dual difference since the last
 * restart, dual part of T(z) - z; -1 when a candidate's dual objective is not
 * positive).  Copies min(entries, max_entries) entries to host `out`
 * and returns that count (>= 0), or a negative error code. */
int sipo_get_trace(sipo_ctx *ctx, double *out, int max_entries);

/* Replaces kkt_tol and max_iter for later solves (check_every, storage and
 * tile_cfg are fixed at creation; changing them is INVALID_ARG). */
int sipo_set_tolerances(sipo_ctx *ctx, const sipo_tolerances *tol);

/* Dose-field metrics for callers that cannot allocate device memory.
 * The paper has no counterpart to this entry point.  It repeats the metrics
 * pass that ends sipo_solve for callers that may not call cudaMalloc -- a
 * print controller that must not allocate once its real-time loop runs, or
 * code living inside a framework whose caching allocator owns the device
 * memory budget.  The five outputs, over gel voxels (label 2) and band voxels
 * (label 1) of the dose d: dtvr_f = max(d / f~_T) / min(d / f~_T) with
 * f~_T = f_T / f_crit; dsr = max_band d / min_gel(d / f~_T); psr_f =
 * min_gel d / max_band d; alpha = sum_gel d f_T / sum_gel d^2; s =
 * min_gel d / (lower_scale f_T).  It calls no cudaMalloc, cudaFree or other
 * allocating routine: its per-block partial sums live in a static device
 * array of the library (8 x 8192 + 8 doubles, 512 KiB, held by every GPU that
 * loads the library until the process exits).
 * dose: device volume of n_voxels elements of `dtype` (SIPO_F32 or SIPO_F64),
 *   e.g. sipo_get_array(ctx, 5, ...); labels: device uint8 region labels of
 *   n_voxels bytes (sipo_get_array(ctx, 0, ...)); f_T: device float32 target
 *   of n_voxels elements, same layout.  The caller guarantees those sizes.
 * f_crit: the normalisation dose (sipo_result.f_crit); lower_scale: the ratio
 *   f~_L / f_T of the lower-bound profile, i.e. 1/f_crit for the general form
 *   and Case 2, (1 - tol_lo)/f_crit for Case 1 with tolerances.  s equals
 *   sipo_result.s only when the lower profile is such a multiple of f_T; for a
 *   context made by sipo_create_bounded (explicit per-voxel f_L) it does not.
 * metrics: host array of 5 doubles: dtvr_f, dsr, psr_f, alpha, s.
 * n_voxels above 134217728 (8192 blocks x 256 threads x 64 voxels) is
 * rejected with SIPO_ERR_INVALID_ARG.  The first call with a device current
 * looks up the array's device address for that device (cudaGetSymbolAddress)
 * and keeps it for the life of the process: make that first call before any
 * stream capture, and do not call this entry point again after a
 * cudaDeviceReset of that device.  Calls share the array (each overwrites it
 * completely); calls that overlap on the GPU race on it and must be
 * serialised by the caller.  Synchronises `stream` (NULL: the legacy default
 * stream). */
int sipo_dose_metrics_noalloc(const void *dose, int dtype, const uint8_t *labels, const float *f_T,
                              long long n_voxels, double f_crit, double lower_scale,
                              double *metrics, void *stream);

/* Releases every device buffer and graph of the context (NULL is allowed). */
int sipo_destroy(sipo_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *sipo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SIPO_H */
