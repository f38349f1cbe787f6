/*
 * ffe.h -- C ABI of the GB300 free-energy engine (libffe.so).
 *
 * The engine evaluates the mean-field grand free energy of the two-band
 * iron-pnictide model with intra-band Fulde-Ferrell pairing,
 *
 *   Omega(Delta; Q, h, T) = sum_eps sum_k [ F(E+_{eps k}) + F(E-_{eps k})
 *                                          + E_{eps,-k+Q/2,down} + Delta^2/U ]
 *
 * (Sec. 2, Eq. freeene, with F(E) = -T ln(1 + exp(-E/T)), the Bogoliubov
 * energies E+/- of Eq. enequasiparticle, and the band energies of App. A at
 * k + Q/2 (spin up) and -k + Q/2 (spin down), Zeeman-shifted by -/+ h), as a
 * map-reduce over the N x N lattice k = 2 pi (i, j)/N, and minimises it over
 * Delta (Alg. 1).  Sign of the pairing term: + Delta^2/U per k-point and band
 * (the printed "- 2|Delta|^2/V" would make Omega fall monotonically with
 * Delta; with + it reproduces the BCS gap equation; V = 2U).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an ffe_status; none aborts, exits or traps.
 *  - All array arguments are HOST memory owned by the caller; the library
 *    copies what it needs and never keeps a caller pointer after returning.
 *    `stream` is a cudaStream_t (NULL = the legacy default stream); calls are
 *    synchronous with respect to the host: results are in the caller's
 *    arrays when the call returns.
 *  - Arguments are validated before any device work: N even in [2, 8192],
 *    T > 0, U > 0, lo <= hi, counts >= 1.  Invalid arguments give FFE_EINVAL
 *    and leave outputs untouched.
 *  - A context is not thread-safe; use one context per host thread.  It stays
 *    usable after any error except FFE_ENOMEM during ffe_create.
 *  - Precision: FFE_FP64 evaluates every k-point term in IEEE double.
 *    FFE_FP32C evaluates the k-point terms in FP32 (hardware exp2/log2/rsqrt/
 *    rcp), sums them in a pairwise tree and accumulates across the lattice in
 *    FP64, and re-evaluates in FP64 every value whose FP32 error bound could
 *    change an argmin or a phase label.
 */
#ifndef FFE_H
#define FFE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FFE_API __attribute__((visibility("default")))
#else
#define FFE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFE_OK = 0,
  FFE_EINVAL = 1,        /* invalid argument (checked before device work)    */
  FFE_ENOMEM = 2,        /* host or device allocation failed                 */
  FFE_ECUDA = 3,         /* a CUDA runtime call failed; see ffe_last_error   */
  FFE_ETIMEOUT = 4,      /* a bounded device-side wait ran out               */
  FFE_EUNSUPPORTED = 5,  /* valid but not implemented (e.g. model kind)      */
  FFE_EINTERNAL = 6      /* internal consistency check failed                */
} ffe_status;

typedef enum { FFE_FP64 = 0, FFE_FP32C = 1 } ffe_precision;

typedef enum { FFE_MODEL_RAGHU2 = 0, FFE_MODEL_DAGHOFER3 = 1 } ffe_model_kind;

/* Model plus the pairing channel of Sec. 2.
 * FFE_MODEL_RAGHU2: the two-band model of App. A, hoppings t1..t4 (defaults
 *   t1=-1, t2=1.3, t3=t4=-0.85, mu=1.54: two electrons per site; t5..eps0
 *   unused).
 * FFE_MODEL_DAGHOFER3: the three-band model of App. B, hoppings t1..t12 and
 *   the d_xy level eps0 (printed values in eV: t1=-0.08, t2=0.1825,
 *   t3=0.08375, t4=-0.03, t5=0.15, t6=0.15, t7=-0.12, t8=0.06, t9=0,
 *   t10=-0.024, t11=-0.01, t12=0.0275, eps0=0.75; n = 4 at mu=0.4748).  Its
 *   three bands are the eigenvalues of the 3x3 hopping matrix, ascending;
 *   every band pairs intra-band as in the two-band model.
 * Each band carries the pairing term + Delta^2/U_eps per k-point with its
 * own coupling U_eps = U_band[eps] (U where that is 0); Sec. 2 writes one
 * V_eps per band and minimises every band separately (ffe_minimize_bands). */
typedef struct {
  int32_t kind;      /* ffe_model_kind                                         */
  int32_t prec;      /* ffe_precision used by every call on the context        */
  double t1, t2, t3, t4;
  double mu;         /* chemical potential                                     */
  double U;          /* pairing strength (> 0): + Delta^2/U per k and band     */
  double eta_amp;    /* s+- form factor eta(k) = eta_amp cos kx cos ky (Sec. 1) */
  double t5, t6, t7, t8, t9, t10, t11, t12, eps0;  /* FFE_MODEL_DAGHOFER3 only  */
  double U_band[3];  /* per-band coupling U_eps (the V_eps of Sec. 2, one per
                        band, bands ascending): > 0 replaces U in that band's
                        + Delta^2/U_eps term; 0 = U.  Unused entries (the
                        third of the two-band model) must be 0            */
} ffe_model;

/* One free-energy evaluation point. */
typedef struct {
  int32_t N;         /* lattice is N x N, N even, 2 <= N <= 8192               */
  int32_t reserved;  /* must be 0                                              */
  double qx, qy;     /* Cooper-pair momentum Q (Sec. 2)                        */
  double h;          /* Zeeman field                                           */
  double T;          /* temperature k_B T (> 0)                                */
  double delta;      /* order-parameter amplitude Delta                        */
} ffe_point;

typedef enum {
  FFE_SEARCH_GRID = 0,   /* Omega on linspace(lo, hi, n); lowest, ties -> lowest index   */
  FFE_SEARCH_GOLDEN = 1  /* Delta = lo plus golden-section on [lo, hi], n reductions      */
} ffe_search_kind;

/* One Delta minimisation (the inner loop of Alg. 1). */
typedef struct {
  int32_t N;         /* as in ffe_point                                        */
  int32_t n;         /* GRID: points (1..65536); GOLDEN: reductions (1..200),
                        the same for every param of one call               */
  double qx, qy, h, T;
  double lo, hi;     /* Delta range, lo <= hi                                  */
} ffe_param;

/* Result flags */
#define FFE_FLAG_RESCORED 1   /* omega_star was re-evaluated in FP64           */
#define FFE_FLAG_EDGE 2       /* argmin at the upper end of the Delta range    */
#define FFE_FLAG_LOWER 4      /* argmin at Delta = lo                          */
#define FFE_FLAG_PRUNED 8     /* guided scan: line not evaluated               */
#define FFE_FLAG_INVALID 32   /* stream-ordered calls: the device reported an
                                 internal inconsistency; values are NaN       */

typedef struct {
  double delta_star;   /* minimising Delta                                     */
  double omega_star;   /* Omega at delta_star                                  */
  double omega_lo;     /* Omega at Delta = lo (the normal state when lo = 0)   */
  double err_bound;    /* bound on |omega_star - FP64 value| (0 if FP64)       */
  int32_t idx_star;    /* GRID: index into the Delta grid; GOLDEN: -1          */
  int32_t flags;       /* FFE_FLAG_*                                           */
} ffe_result;

/* Phase labels (Alg. 1, outer loop over q). */
#define FFE_PHASE_NORMAL 0
#define FFE_PHASE_BCS 1
#define FFE_PHASE_FFLO 2

/* A phase-diagram scan: every q of the list against every (h, T) pair of the
 * product h-list x T-list (h-major: point p = ih * n_T + iT), all at one N.
 * Phase labels need Q = (0, 0) in the q list (it defines the normal/BCS
 * reference); a scan without it gives the per-line minima only (labels and
 * best_q must then be NULL; see ffe_label_candidates for split q lists). */
typedef struct {
  int32_t N;
  int32_t n_q;
  const double* qx;    /* [n_q] */
  const double* qy;    /* [n_q] */
  int32_t n_h;
  int32_t n_T;
  const double* h;     /* [n_h] */
  const double* T;     /* [n_T] */
  int32_t search;      /* ffe_search_kind                                      */
  int32_t n;           /* grid points or golden reductions                     */
  double lo, hi;       /* Delta range; lo must be 0 for phase labels           */
} ffe_scan;

typedef struct ffe_context ffe_context;
typedef struct ffe_plan ffe_plan;

/* Create a context on the current CUDA device for model *m.  Reads device
 * properties and allocates nothing large.  *out is NULL on failure. */
FFE_API ffe_status ffe_create(const ffe_model* m, ffe_context** out);

/* Destroy a context and every plan it still owns.  NULL-safe. */
FFE_API void ffe_destroy(ffe_context* ctx);

/* Static description of a status code; never NULL. */
FFE_API const char* ffe_status_string(ffe_status s);

/* Message of the last failing call on ctx (empty string if none). */
FFE_API const char* ffe_last_error(const ffe_context* ctx);

/* Omega (Eq. freeene summed over both bands) at n independent points.
 * omega[n] receives Omega; omega_band (NULL or [n][nb], nb = 2 for the
 * two-band and 3 for the three-band model) receives the per-band Omega_eps,
 * bands in ascending order of energy.
 * Points sharing (N, Q) share the per-k band work. */
FFE_API ffe_status ffe_omega(ffe_context* ctx, const ffe_point* pts, int64_t n,
                     double* omega, double* omega_band, void* stream);

/* Minimise Omega over Delta for n independent parameter points (Alg. 1,
 * inner loop).  All params of one call use the same search kind.  Uneven
 * lattices and grid lengths are packed into one persistent launch.
 * omega_grid (GRID only; NULL or sum_i ps[i].n doubles) receives each
 * parameter point's Omega grid, concatenated in input order; err_grid (NULL
 * or the same size) the FP32 error bound of each grid value (0 where the
 * value was evaluated or re-evaluated in FP64). */
FFE_API ffe_status ffe_minimize(ffe_context* ctx, int32_t search, const ffe_param* ps,
                                int64_t n, ffe_result* out, double* omega_grid,
                                double* err_grid, void* stream);

/* Per-band independent minimisation (Sec. 2: the paper minimises Omega_eps
 * of every band separately).  Omega = Omega_lower(Delta_lower) +
 * Omega_upper(Delta_upper) when each band has its own gap, so the joint
 * minimum is the two one-dimensional minima.  Each band's search runs on its
 * own Omega_eps (its Delta^2/U term included) with the point's search
 * settings; out[n][nb] (nb = 2 or 3 bands of the model) receives each band's
 * result in ascending order of band energy, fields as in ffe_minimize
 * (omega_star and omega_lo are Omega_eps). */
FFE_API ffe_status ffe_minimize_bands(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n,
                                      ffe_result* out, void* stream);

/* Phase-diagram scan (Alg. 1): per (q, h, T) the Delta minimum, then per
 * (h, T) the phase label.  per_point[n_q][n_h*n_T] receives the minima
 * (q-major), labels[n_h*n_T] the FFE_PHASE_* label, best_q[n_h*n_T] the
 * index of the winning q (-1 for normal). */
FFE_API ffe_status ffe_phase_scan(ffe_context* ctx, const ffe_scan* scan,
                          ffe_result* per_point, int8_t* labels,
                          int32_t* best_q, void* stream);

/* ---- stream-ordered forms: device arrays, no host synchronisation ------
 * For callers whose inputs and outputs live in device memory (torch tensors
 * passed by data_ptr(), with torch.cuda.current_stream() as `stream`).  Each
 * call queues its work on `stream` and returns without waiting for the
 * device; results are in the caller's DEVICE arrays once `stream` reaches
 * them (synchronise or record an event as usual).  Descriptions that decide
 * the shape of the work (lattice sizes, grid lengths, pair momenta, the
 * ffe_param / ffe_scan structs and their lists) stay HOST memory.  Errors
 * the device finds cannot be returned: a point with T <= 0 or a non-finite
 * input gets NaN, and a kernel-side inconsistency sets FFE_FLAG_INVALID with
 * NaN values (ffe_minimize_async, ffe_phase_scan_async) or NaN in every
 * output (ffe_omega_async).  The first call of a shape builds and caches a
 * plan on the context (device allocation and an upload that waits); later
 * calls of the same shape stage their values in page-locked memory and only
 * queue copies and kernels.  Calls on one context share its cached plans and
 * scratch: calls on different streams must be ordered by the caller (one
 * context per stream otherwise).  The caller's arrays must stay valid until
 * the stream has passed the call. */

/* Omega (Eq. freeene) at n points (h[i], T[i], delta[i]) of one lattice N and
 * pair momentum Q: h, T, delta are DEVICE arrays of n doubles; omega (n
 * doubles) and omega_band (NULL or [n][nb], nb = 2 or 3 bands ascending) are
 * DEVICE outputs.  Every point is its own (h, T) entry (a distinct h costs one
 * normal-state sum; for grids of parameters prefer ffe_minimize_async).  The
 * job table is written on the device; the context's scratch grows to the
 * largest call (growing waits for the device).  n in [1, 2^24]. */
FFE_API ffe_status ffe_omega_async(ffe_context* ctx, int32_t N, double qx, double qy, const double* h,
                                   const double* T, const double* delta, int64_t n, double* omega,
                                   double* omega_band, void* stream);

/* ffe_minimize with the results left on the device: out[n] (DEVICE) as in
 * ffe_minimize; omega_grid (GRID only; NULL or DEVICE, sum_i ps[i].n doubles)
 * the Omega grids.  ps is host memory. */
FFE_API ffe_status ffe_minimize_async(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n,
                                      ffe_result* out, double* omega_grid, void* stream);

/* ffe_phase_scan with the results left on the device: per_point, labels and
 * best_q (each NULL or DEVICE, sizes as in ffe_phase_scan).  *scan and its
 * lists are host memory. */
FFE_API ffe_status ffe_phase_scan_async(ffe_context* ctx, const ffe_scan* scan, ffe_result* per_point,
                                        int8_t* labels, int32_t* best_q, void* stream);

/* ---- phase labels over q lists split across ranks (Alg. 1, outer argmin) --
 * Host functions (no device work).  A scan's q list may be split across
 * ranks (one process per GPU); each rank scans its own q (a scan without
 * Q = (0, 0) gives no labels) and reduces its lines per (h, T) point to one
 * candidate, then the ranks' candidates are merged.  omega_n[n_pts] is the
 * normal state Omega(q = 0, Delta = 0) of each point (the omega_lo of the
 * q = 0 lines, from the rank that scans q = 0); tau = 1e-12 |omega_n| as in
 * ffe_phase_scan.  A rank's values are those of its own scan: FP32+comp
 * values within their error bound of a competitor's on another rank are not
 * re-evaluated in FP64, as the single-process labels are. */

/* Per point, the lowest omega_star among the rank's lines (per_point
 * [n_q][n_pts], laid out as ffe_phase_scan's) that condense (omega_star <
 * omega_lo - tau), ties to the lowest global q index; q_global[n_q] maps the
 * rank's q to the global list.  best_val[n_pts] (+inf where none) and
 * best_q[n_pts] (the global index, -1 where none). */
FFE_API ffe_status ffe_label_candidates(const ffe_result* per_point, int32_t n_q, int32_t n_pts,
                                        const int32_t* q_global, const double* omega_n, double* best_val,
                                        int32_t* best_q);

/* Labels from the stacked candidates of `world` ranks (best_val, best_q:
 * [world][n_pts]): the lowest candidate (ties to the lowest global q) wins
 * when it lies below omega_n - tau, BCS if its q is zero_q (the global index
 * of Q = (0, 0)), else FFLO; NORMAL otherwise.  labels[n_pts], best_q_out
 * [n_pts] (-1 for normal), as from ffe_phase_scan. */
FFE_API ffe_status ffe_merge_candidates(int32_t world, int32_t n_pts, const double* best_val,
                                        const int32_t* best_q, const double* omega_n, int32_t zero_q,
                                        int8_t* labels, int32_t* best_q_out);

/* ---- device-resident plans (for repeated execution) --------------------
 * A plan holds the packed job table, device buffers and a captured CUDA
 * graph of one scan.  ffe_plan_execute replays the graph on `stream` without
 * any host<->device copy and returns without synchronising; ffe_plan_fetch
 * synchronises the stream and copies the results of the last execution to
 * host arrays laid out as in ffe_phase_scan. */
FFE_API ffe_status ffe_plan_phase_scan(ffe_context* ctx, const ffe_scan* scan,
                               void* stream, ffe_plan** out);
FFE_API ffe_status ffe_plan_execute(ffe_plan* plan, void* stream);
FFE_API ffe_status ffe_plan_fetch(ffe_plan* plan, ffe_result* per_point,
                          int8_t* labels, int32_t* best_q, void* stream);
/* The whole Omega(Delta) grid of every line of a grid phase-scan plan after
 * its last execution: omega_grid[n_q][n_h*n_T][n] (lines as in per_point,
 * grid index fastest); err_grid (NULL or the same size) the FP32 error bound
 * of each value (0 where evaluated or re-evaluated in FP64).  Synchronises
 * `stream`. */
FFE_API ffe_status ffe_plan_fetch_grid(ffe_plan* plan, double* omega_grid, double* err_grid, void* stream);
typedef struct {
  double k_evals;          /* k-point evaluations (one k-point, one Delta, one
                              (q,h,T), both bands) of the main k-sum per execution */
  double device_bytes;     /* device memory held by the plan                  */
  int32_t launches;        /* kernel launches per execution                   */
  int32_t rescored_search; /* FP64 re-evaluations requested by the Delta search
                              in the last fetched execution                   */
  int32_t rescored_labels; /* ... by the phase labels in that execution       */
  int32_t kpt;             /* k-points per thread per k-set of the main k-sum */
  int32_t block, grid;     /* its launch shape (threads, persistent blocks)   */
  int32_t work_items;      /* warp work items in its queue                    */
  int32_t reserved;
  double k_evals_near;     /* FP32: band evaluations (one k, one band, one
                              output) of the last completed execution that took
                              the full term; the others were "far" (log terms 1
                              in FP32, W = c a: one R and a per (k, Delta, band)
                              shared by the outputs).  A k-evaluation covers
                              every band.  0 for FP64, -1 before the first
                              execution                                       */
  double k_evals_single;   /* FP32: those of k_evals_near whose band has
                              c (R + |d|) >= 27 for every output of its work
                              item and that were evaluated with one exponential
                              (the other factor is exactly 1 in FP32); same
                              conventions                                     */
  double k_evals_far_closed; /* FP32: far band evaluations that formed R and a
                              (shared by an output batch's Delta, or per output
                              in the LIST layout); the other far bands, with
                              Delta_max^2 eta^2 / s^2 <= 0.1, enter six moments
                              per k-set (shared Delta) or work item (LIST);
                              same conventions                                */
} ffe_plan_info;

/* Static facts about a plan, the FP64 re-evaluation counts of the last
 * execution whose results were fetched and the full-term count of the last
 * completed execution (this call waits for the device). */
FFE_API ffe_status ffe_plan_stats(const ffe_plan* plan, ffe_plan_info* info);
/* Average duration in milliseconds of the plan's main k-sum kernel over the
 * executions since the last call (CUDA events recorded on the launch stream
 * around that kernel inside the graph); 0 if none. */
FFE_API ffe_status ffe_plan_kernel_ms(ffe_plan* plan, double* ms, int32_t* count);
FFE_API void ffe_plan_destroy(ffe_plan* plan);

/* A device-resident plan of ffe_minimize: the parameter points (uneven
 * lattices and grid lengths allowed) are packed into one job table and one
 * persistent k-sum launch, captured with the Delta search in a CUDA graph.
 * ffe_plan_fetch_minimize returns the results of the last execution as
 * ffe_minimize does. */
FFE_API ffe_status ffe_plan_minimize(ffe_context* ctx, int32_t search, const ffe_param* ps,
                                     int64_t n, void* stream, ffe_plan** out);
FFE_API ffe_status ffe_plan_fetch_minimize(ffe_plan* plan, ffe_result* out, double* omega_grid,
                                           double* err_grid, void* stream);

/* Autotuner (no counterpart in the paper): times the plan's k-sum for a set
 * of launch shapes (k-points per thread 2/4/8, block 128/256 threads, warp
 * work-item sizes), rebuilds the plan with the fastest and remembers it for
 * later plans of the same kind on the context (and in the file named by the
 * environment variable FFE_TUNE_CACHE, read by ffe_create).  Runs the plan
 * about twenty times.  The chosen shape is returned when the pointers are
 * not NULL. */
FFE_API ffe_status ffe_plan_autotune(ffe_plan* plan, void* stream, int32_t* kpt, int32_t* block,
                                     double* item_target);

/* Environment variables read when a plan is built (none is needed):
 *   FFE_KSUM_TUNING_FP32, FFE_KSUM_TUNING_FP64 = "kpt:block:item_target"
 *     force the k-sum launch shape of FP32+comp / FP64 plans;
 *   FFE_KSTATE_TABLE_MAX_BYTES = n
 *     the largest FP32 k-state table (20 bytes per Q, band pair and lattice
 *     point) a plan keeps (default 32 GiB; 0: none, the k-sum then builds
 *     the states itself, with the same results). */

/* ---- learned surrogate of Omega (no counterpart in the paper) ----------
 * A 4 -> 128 -> 128 -> 128 -> 1 MLP with SiLU activations over the raw
 * inputs (q, h, T, Delta), mapped to x = (raw - shift) * scale; it predicts
 * a target divided by y_scale (the library applies both maps).  The two
 * 128 x 128 layers run on the tensor cores in BF16 with FP32 accumulation;
 * master weights and Adam moments are FP32.  Parameters are 33 793 floats:
 * W1[4][128], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 * W4[128], b4[1] (W[i][o] maps input i to output o).  All arrays are host
 * memory; calls are synchronous. */
typedef struct {
  float shift[4], scale[4];
  float y_scale;     /* > 0 */
  int32_t reserved;  /* must be 0 */
} ffe_surrogate_meta;
typedef struct ffe_surrogate ffe_surrogate;

/* params NULL = all zeros. */
FFE_API ffe_status ffe_surrogate_create(ffe_context* ctx, const ffe_surrogate_meta* meta,
                                        const float* params, ffe_surrogate** out);
FFE_API void ffe_surrogate_destroy(ffe_surrogate* s);
/* Replace the weights (resets the Adam moments). */
FFE_API ffe_status ffe_surrogate_set_params(ffe_surrogate* s, const float* params);
FFE_API ffe_status ffe_surrogate_get_params(ffe_surrogate* s, float* params);
/* Checkpoint of the whole training state -- weights, Adam moments and step,
 * input/output maps -- as host bytes: buf NULL returns the size in *bytes;
 * otherwise *bytes is the buffer's size on entry and the bytes written on
 * return.  Training resumed from a loaded checkpoint continues exactly as the
 * saved one would have (the same bits).  load rejects a buffer that is not a
 * checkpoint of this network (FFE_EINVAL). */
FFE_API ffe_status ffe_surrogate_save(ffe_surrogate* s, void* buf, size_t* bytes);
FFE_API ffe_status ffe_surrogate_load(ffe_surrogate* s, const void* buf, size_t bytes);
/* Training targets of the surrogate (data generation, no counterpart in the
 * paper): omega holds n_lines lines of n_per_line free energies of one lattice
 * size N, each line's first value at its reference Delta = 0; y receives the
 * condensation energy per site (omega[l][j] - omega[l][0]) / N^2 of every value,
 * rounded to FP32 from the FP64 difference and quotient.  Host arrays (caller
 * owned, n_lines * n_per_line each); computed by a kernel.  FFE_EINVAL for
 * NULL arrays, n_lines < 1, n_per_line < 1 or N < 1. */
FFE_API ffe_status ffe_surrogate_targets(ffe_context* ctx, const double* omega, int64_t n_lines,
                                         int32_t n_per_line, int32_t N, float* y);
/* y[n] = prediction at x[n][4] = (q, h, T, Delta). */
FFE_API ffe_status ffe_surrogate_predict(ffe_surrogate* s, const float* x, int64_t n, float* y,
                                         void* stream);
/* Gradient (33 793 floats) of the mean squared error over the n samples,
 * in the network's normalised units, and that loss. */
FFE_API ffe_status ffe_surrogate_grad(ffe_surrogate* s, const float* x, const float* t, int64_t n,
                                      float* grad, double* loss, void* stream);
/* Adam training over `epochs` passes of the samples in their given order
 * (epochs in [1, 1000000], batch a multiple of 64; the tail that does not
 * fill a batch is skipped).
 * loss_per_epoch (NULL or [epochs]) receives the mean batch loss. */
FFE_API ffe_status ffe_surrogate_train(ffe_surrogate* s, const float* x, const float* t, int64_t n,
                                       int32_t epochs, int32_t batch, float lr,
                                       float* loss_per_epoch, void* stream);
/* The same with one learning rate per epoch (lr_per_epoch[epochs], host,
 * each > 0): the samples are uploaded once for the whole schedule.  A call
 * with epochs E and rates r gives the same bits as E calls of
 * ffe_surrogate_train with one epoch and rate r[e] each. */
FFE_API ffe_status ffe_surrogate_train_schedule(ffe_surrogate* s, const float* x, const float* t, int64_t n,
                                                int32_t epochs, int32_t batch, const float* lr_per_epoch,
                                                float* loss_per_epoch, void* stream);

/* Phase scan guided by the surrogate, grid or golden-section search.  The
 * surrogate predicts every (q, h, T) line's condensation energy on a Delta
 * grid (the search grid; 256 points on [lo, hi] for golden); with a margin,
 * the exact k-sum evaluates the normal states Omega(q, Delta = lo) of every q
 * at a sample of at most 64 (h, T) points, and at every point when they
 * differ from those of q = 0 by more than a tenth of the margin somewhere
 * in the sample (on a finite lattice the normal states of different q
 * differ, and the labels compare Omega across q).  Per (h, T) the exact k-sum
 * verifies q = 0 and the q_keep lines of lowest predicted minimum (the
 * normal state relative to q = 0's where evaluated, plus the predicted
 * condensation energy), with a margin also every q predicted to condense by more
 * than the margin whose predicted minimum is within the margin of the
 * lowest and every q whose exact normal state lies more than the margin
 * below that of q = 0 (any condensation would make it the winner), each on a
 * window of `window` grid points around its predicted
 * minimum, with Delta = 0 as the reference (with the FP64 re-evaluation and
 * label passes of ffe_phase_scan).  Grid: the window's grid points.  Golden:
 * the window is the initial bracket and takes as many fewer reductions as
 * reach the full search's final bracket width.  An (h, T) point with a line
 * whose verified minimum lies on an inner window edge (or that `margin`
 * flags) is scanned again with all its verified lines over the whole range.
 * Unverified (pruned) lines are reported with idx_star 0 (grid) or -1
 * (golden), flags FFE_FLAG_LOWER | FFE_FLAG_PRUNED and the Delta = lo value
 * of the q = 0 line at the same (h, T); a line
 * whose minimum is its Delta = 0 point never decides a label, so pruning
 * changes a label only where the exact minimum of a pruned q would have
 * beaten the kept ones.  Outputs as in ffe_phase_scan. */
typedef struct {
  int32_t window;       /* grid points per verified line, 2..n               */
  int32_t q_keep;       /* q values kept per (h, T) besides q = 0            */
  double margin;        /* >= 0, |t1| per site: a kept line whose predicted
                           minimum is in the window at Delta = lo but which has
                           a second predicted basin outside it with
                           condensation energy below +margin (the basins may
                           swap within the surrogate's error, as at a
                           first-order transition) is searched over the
                           whole range instead, and beyond q_keep every q
                           predicted to condense by more than margin whose
                           predicted minimum is within margin of the lowest
                           one, and every q whose exact normal state lies
                           more than margin below that of q = 0, is kept
                           too; 0: none of these                          */
} ffe_guide;
typedef struct {
  double k_evals;       /* exact k-point evaluations done (the normal states
                           included)                                         */
  double k_evals_full;  /* those of the unguided grid scan                   */
  int64_t lines_kept, lines_pruned;
  int64_t fallbacks;    /* kept lines searched over the whole range          */
  double rms_error;     /* RMS of predicted - exact condensation energy per
                           site, (Omega(Delta) - Omega(0))/N^2, on the
                           verified window points                            */
  double mlp_flops;     /* multiply-adds x 2 of the predictions              */
} ffe_guide_stats;
FFE_API ffe_status ffe_surrogate_scan(ffe_context* ctx, ffe_surrogate* s, const ffe_scan* scan,
                                      const ffe_guide* guide, ffe_result* per_point, int8_t* labels,
                                      int32_t* best_q, ffe_guide_stats* stats, void* stream);

/* ---- static Cooper pair susceptibility (App. C) ------------------------
 * chi[n_q][nb][nb] (nb = 2 or 3 bands of the model, ascending) at pair
 * momenta q = (qx[i], qy[i]):
 *   chi_{e e'}(q) = (1/N^2) sum_k eta(-k-q)^2 [1 - f(E_{e,k,up}) - f(E_{e',-k-q,down})]
 *                                            / (E_{e,k,up} + E_{e',-k-q,down}),
 * E_{e,k,up} = E_e(k) - mu - h, E_{e',-k-q,down} = E_e'(-k-q) - mu + h, f the
 * Fermi function at T > 0, eta = eta_amp cos kx cos ky of the context (App. C
 * uses eta_amp = 4), k over the N x N lattice; the quotient takes its limit
 * where the denominator vanishes.  FP64.  Host arrays; synchronous on
 * `stream`.  A peak of chi_{ee}(q) at q != 0 indicates the FF phase. */
FFE_API ffe_status ffe_pair_susceptibility(ffe_context* ctx, int32_t N, int32_t n_q, const double* qx,
                                           const double* qy, double h, double T, double* chi, void* stream);

/* ---- Omega without any allocation (no counterpart in the paper) --------
 * For callers that cannot allocate device memory when they need a free
 * energy -- a service that has given all free device memory to its own pool
 * (a cudaMalloc there fails or evicts), or a latency-critical loop in which
 * cudaMalloc/cudaFree would synchronise the device and stall other streams.
 * Computes Omega at n points (h[i], T[i], delta[i]) of one lattice N and one
 * pair momentum Q = (qx, qy) with the precision of m->prec, within the same
 * per-site tolerance as ffe_omega (its own k-chunking, so not always the same
 * bits).  The caller passes DEVICE arrays h, T, delta (n doubles each) and
 * omega (n doubles, written); every intermediate, the job table included,
 * is written by the call's kernels into one fixed 4 MiB __device__ array of
 * the library that each GPU loading the library holds until exit: the call
 * makes no host-to-device copy and allocates nothing.  Limits of that array:
 * N even in [2, 2048] and 1 <= n <= 512; beyond them the call returns
 * FFE_EINVAL before any device work.  The inputs are checked on the device:
 * a point with T <= 0 or a non-finite h, T or delta gets omega = NaN (the
 * other points are computed normally), and if a kernel of the call detects
 * an internal inconsistency every omega of the call is NaN.  The first call
 * on a device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture.  The
 * call returns once the work is queued on `stream`.  All calls share the
 * array, which keeps the last call's contents (counters are cleared at the
 * start of every call): calls that overlap on the GPU race and must be
 * serialised by the caller. */
FFE_API ffe_status ffe_omega_noalloc(const ffe_model* m, int32_t N, double qx, double qy,
                                     const double* h, const double* T, const double* delta,
                                     int32_t n, double* omega, void* stream);

/* ---- device throughput probe (no counterpart in the paper) -------------
 * Measured issue rates, in operations per second over the whole device, of
 * the units the k-sum is bound by: the special-function unit for
 * ex2/lg2/rsqrt/rcp (FP32 approximate), FP32 FMA and FP64 FMA.  Runs short
 * self-contained kernels (~0.1 s) on the current device. */
typedef struct {
  double ex2, lg2, rsqrt, rcp;  /* MUFU results per second            */
  double fma32, fma64;          /* fused multiply-adds per second      */
  int32_t n_sm;                 /* multiprocessors                     */
  int32_t sm_khz_max;           /* maximum SM clock reported (kHz)     */
} ffe_peaks;
FFE_API ffe_status ffe_probe_peaks(ffe_peaks* out);

#ifdef __cplusplus
}
#endif

#endif /* FFE_H */
