/*
 * hse.h -- C ABI of the GB300 (sm_103a) half-space Spectral Ewald library.
 *
 * Computes, on one GPU, the sums of Stokes singularities above a no-slip wall
 * at x3 = 0 in the image representation of Srinivasan & Tornberg (arXiv
 * 1802.07844, Sec. 3, eq. v_sum_halfspace): for every target x
 *
 *   stokeslet  u += S(r) f - S(rt) f^I - x3 grad(phi_S) + e3 phi_S
 *   stresslet  u += T(r)(g q) - T(rt)(g^I q^I) - x3 grad(phi_T) + e3 phi_T
 *   rotlet     u += W(r) tau + W(rt) tau^I - x3 grad(phi_W) + e3 phi_W
 *
 * summed over all sources y (r = x - y, rt = x - y^I, y^I = (y1, y2, -y3)),
 * with the Ewald split of Sec. 4 (real-space erfc-screened neighbour sum within
 * r_c over sources and images, Sec. 5.1) and the Fourier-space Spectral Ewald
 * part of Alg. 1 (Gaussian spreading, zero-padded FFT, scaling by the truncated
 * kernels of Sec. 5.2, inverse FFT, Gaussian quadrature).
 *
 * Units: velocities are returned in "8 pi units", i.e. 8*pi times the physical
 * velocity at unit viscosity, with S(r) f = f/r + r (r.f)/r^3,
 * T(r)(g q) = -6 r (r.g)(r.q)/r^5 and W(r) tau = 2 tau x r / r^3.
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller, in
 * component-major ("SoA") layout: an array "3 x n" holds x[0..n), y[n..2n),
 * z[2n..3n).  The plan owns all of its own device memory (grids, tables,
 * cell lists, cuFFT plans and work areas).  Calls are asynchronous on the
 * given CUDA stream except where stated; no caller memory is touched after
 * the stream work of a call completes.  A plan is not re-entrant: use one
 * plan per concurrent stream.
 *
 * Errors: status codes only; no exceptions cross this ABI and nothing exits.
 * hse_last_error() gives the text of the last failure of a plan.
 */
#ifndef HSE_H
#define HSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hse_plan_s* hse_plan;

typedef enum {
  HSE_OK = 0,
  HSE_ERR_INVALID = 1,     /* argument or input data out of the documented domain */
  HSE_ERR_OOM = 2,         /* a device allocation failed                          */
  HSE_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed         */
  HSE_ERR_CUFFT = 4,       /* a cuFFT call failed                                 */
  HSE_ERR_TIMEOUT = 5,     /* a bounded wait ran out                              */
  HSE_ERR_UNSUPPORTED = 6  /* valid request this build does not support           */
} hse_status;

/* kernel bit mask; several bits may be combined, the sums are added.
 * HSE_FREE_SPACE (with at least one kernel bit) selects the free-space sums of
 * Sec. 2 instead: the same kernels without the wall -- no images, no harmonic
 * corrections (u = sum S8(r) f, T8(r)(g q), W8(r) tau); the box, the Ewald
 * split, the self term and every entry point are otherwise unchanged. */
enum { HSE_STOKESLET = 1, HSE_STRESSLET = 2, HSE_ROTLET = 4, HSE_FREE_SPACE = 8 };
/* arithmetic of the path.
 * HSE_FP64 (any tolerance): real-space pairs closer than rc64 (hse_params) in
 *   FP64 and the outer shell [rc64, r_c) in FP32, its rc64 chosen so that the
 *   FP32 rounding stays below half the real-space truncation estimate; with
 *   HSE_FFT_DF64 (the automatic choice for tol >= 1e-12 or explicit
 *   parameters) the spread and gather grids, the zero-padded transforms and
 *   the scaling run in double-float (~48-bit) arithmetic on the FP32 pipe;
 *   sums, the self term and the combination in FP64.  hse_plan_set_rc64(plan,
 *   rc) with hse_plan_set_fft(plan, HSE_FFT_CUFFT) gives FP64 throughout.
 * HSE_MIXED (tol >= 1e-6): FP32 real-space pairs, spreading, cuFFT single
 *   transforms, scaling and gather; FP64 sums, close image pairs of near-wall
 *   targets, the self term and the tables' construction (rounded to FP32). */
enum { HSE_FP64 = 0, HSE_MIXED = 1 };
/* transforms of the Fourier part (hse_plan_set_fft): HSE_FFT_DF64 runs the
 * grids, zero-padded FFTs and scaling in double-float (~48-bit) arithmetic on
 * the FP32 pipe, HSE_FFT_CUFFT in cuFFT double (HSE_MIXED plans: FP32 grids
 * and cuFFT single); HSE_FFT_AUTO picks HSE_FFT_DF64 for HSE_FP64 plans with
 * tol >= 1e-12 or explicit parameters, HSE_FFT_CUFFT otherwise.  An HSE_MIXED
 * plan with HSE_FFT_DF64 keeps FP32 real space and runs a double-float Fourier
 * part: for the half-space stokeslet with sources spread through the box the
 * FP32 Fourier part loses ~2.5e-8 sqrt(N) of the velocity (FP32 rounding at
 * low wave numbers, where the image system cancels the long-range field and
 * the kernel scales by ~1/k^2), which the double-float part avoids. */
enum { HSE_FFT_AUTO = 0, HSE_FFT_CUFFT = 1, HSE_FFT_DF64 = 2 };

/* Parameters of a plan, as chosen or given (Alg. 1 notation). */
typedef struct {
  int kernel_mask;
  int precision;
  double box[3];     /* L1, L2, L3 of the source box [0,L1) x [0,L2) x (0,L3]    */
  double L;          /* max(L1, L2, L3): side of the cubic Fourier domain         */
  double xi;         /* Ewald parameter                                            */
  double rc;         /* real-space cut-off radius                                  */
  double rc64;       /* HSE_FP64, targets = sources: pairs closer than rc64 are     *
                      * evaluated in FP64, pairs in [rc64, rc) in FP32 (their      *
                      * screened kernels are small enough that FP32 rounding stays  *
                      * below half the real-space truncation estimate); rc64 >= rc  *
                      * means FP64 throughout (also for the spread's small-weight   *
                      * part, which otherwise runs in FP32).  0 under HSE_MIXED.     */
  int P;             /* Gaussian support width in grid points (even)               */
  int M;             /* basic grid size, h = L / M                                 */
  int Mt;            /* extended grid size M + P; grid Mt x Mt x 2 Mt              */
  double h;          /* grid spacing                                               */
  double eta;        /* Gaussian shape parameter P xi^2 h^2 / (c^2 pi), c = 0.95  */
  int ncell[3];      /* real-space cell list dimensions (cell side >= rc / 2)      */
  int n_fft_in;      /* number of forward FFTs per evaluation                      */
  int n_fft_out;     /* number of inverse FFTs per evaluation (6)                  */
  int fft;           /* transforms: HSE_FFT_DF64 or HSE_FFT_CUFFT (see hse_plan_set_fft) */
  size_t grid_bytes; /* device bytes held by grids and tables                      */
  int spread_tile[3];/* grid points along x, y, z that one warp of the spread owns   *
                      * (one per lane; product 32), see hse_plan_set_spread_tile   */
  double rcmid;      /* HSE_FP64, targets = sources: pairs at distance in [rcmid,   *
                      * min(rc64, rc)) are evaluated in double-float arithmetic    *
                      * (hse_plan_set_rcmid); 0: none                              */
} hse_params;

/*
 * hse_plan_create -- choose parameters and build the Fourier-space machinery.
 *   kernel_mask  HSE_STOKESLET | HSE_STRESSLET | HSE_ROTLET (non-zero).
 *   box          host array {L1, L2, L3} > 0; sources must lie in
 *                [0,L1) x [0,L2) x (0,L3], targets in [0,L1) x [0,L2) x [0,L3].
 *   xi, rc, P    Ewald parameter, cut-off radius, support width; a value <= 0
 *                is chosen from tol (tol must then be > 0).  P is rounded up
 *                to an even number.
 *   tol          target relative RMS error (Sec. 6 definition); used to pick
 *                missing parameters and the grid size M (Tables 2-3 estimates).
 *                With tol <= 0 all of xi, rc, P must be given and M is set
 *                with hse_plan_set_grid before the first evaluation.
 *   precision    HSE_FP64 or HSE_MIXED.
 *   out          receives the plan (host pointer).
 * Builds the truncated-kernel tables of Sec. 5.2 on the device (untimed
 * set-up work, synchronous).  Errors: HSE_ERR_INVALID, HSE_ERR_OOM,
 * HSE_ERR_CUDA, HSE_ERR_CUFFT.  On error *out is NULL.
 */
hse_status hse_plan_create(int kernel_mask, const double box[3], double xi, double rc, int P, double tol,
                           int precision, hse_plan* out);

/* Set the basic grid size M explicitly (h = L/M) and rebuild the grids and
 * tables (synchronous).  HSE_ERR_INVALID if M < 4 or the Gaussian shape
 * parameter eta falls outside (0, 1). */
hse_status hse_plan_set_grid(hse_plan plan, int M);

/* Copy the plan's parameters to *out (host). */
hse_status hse_plan_get_params(hse_plan plan, hse_params* out);

/* Override the FP64/FP32 split radius rc64 of an HSE_FP64 plan (see
 * hse_params); rc64 >= rc evaluates everything in FP64.
 * HSE_ERR_INVALID for rc64 < 0 or an HSE_MIXED plan. */
hse_status hse_plan_set_rc64(hse_plan plan, double rc64);
/* Double-float band of the real-space sum (Sec. 5.1) of an HSE_FP64 plan with
 * targets = sources: pairs at distance in [rcmid, min(rc64, rc)) are
 * evaluated in double-float (~48-bit head/tail) arithmetic on the FP32 pipe by
 * a second kernel instead of in FP64: relative error ~1e-11 per pair term
 * (FP64 ~1e-15, the FP32 shell beyond rc64 ~1e-7) at a fraction of the cost,
 * since GB300's FP64 pipe executes 2 multiply-adds per SM and clock against
 * 128 on the FP32 pipe.  Pairs closer than rcmid, and pairs with an end point
 * within 1/64 of their distance of the wall, stay in FP64.  rcmid = 0 (the
 * default) or rcmid >= min(rc64, rc): no band.  HSE_ERR_INVALID for rcmid < 0
 * or an HSE_MIXED plan. */
hse_status hse_plan_set_rcmid(hse_plan plan, double rcmid);

/* Choose the transforms of the Fourier part (HSE_FFT_AUTO, HSE_FFT_CUFFT or
 * HSE_FFT_DF64; hse_params.fft reports the choice).  Builds what the choice
 * needs when the grids exist (synchronous; an HSE_MIXED plan rebuilds its
 * grids and tables, whose element changes between FP32 and double-float).
 * HSE_ERR_INVALID for an unknown mode; HSE_ERR_UNSUPPORTED when the grid has
 * a length with a prime factor other than 2, 3, 5. */
hse_status hse_plan_set_fft(hse_plan plan, int mode);

/*
 * hse_eval -- velocities at the targets.
 *   n_src      number of sources (>= 0).
 *   src_xyz    device, 3 x n_src positions.
 *   strengths  device, rows stacked in the kernel order of the mask:
 *              stokeslet f (3 rows), stresslet g then q (6 rows), rotlet tau
 *              (3 rows); each row has n_src entries.
 *   n_tgt      number of targets; tgt_xyz == NULL means the targets are the
 *              sources (then n_tgt must equal n_src) and the pair of a target
 *              with its own source is excluded from the free-space term
 *              (Sec. 2).  With explicit targets, pairs at exactly zero
 *              separation are excluded in the same way.
 *   vel        device, 3 x n_tgt, overwritten.
 *   cuda_stream  cudaStream_t (NULL = legacy default stream).
 * The input check (finite values inside the box, sources strictly above the
 * wall) synchronises the stream once.  Errors: HSE_ERR_INVALID (bad input;
 * vel is then unspecified), HSE_ERR_OOM, HSE_ERR_CUDA, HSE_ERR_CUFFT.
 */
hse_status hse_eval(hse_plan plan, int64_t n_src, const double* src_xyz, const double* strengths, int64_t n_tgt,
                    const double* tgt_xyz, double* vel, void* cuda_stream);

/*
 * hse_eval_parts -- as hse_eval, but returns the two halves of the split
 * separately (Sec. 4): u_real = real-space sum within r_c plus the stokeslet
 * self term, u_fourier = Fourier-space part (Alg. 1).  Either output pointer
 * may be NULL to skip that half; the real-space half alone needs no grid
 * (a plan created with tol <= 0 and no hse_plan_set_grid).  Same arguments
 * and errors as hse_eval.
 */
hse_status hse_eval_parts(hse_plan plan, int64_t n_src, const double* src_xyz, const double* strengths,
                          int64_t n_tgt, const double* tgt_xyz, double* u_real, double* u_fourier,
                          void* cuda_stream);

/*
 * hse_cell_list -- the real-space cell list of the plan's box (Sec. 5.1).
 *   pos        device, 3 x n positions.
 *   cell_id    device, n int32: cell of each point,
 *              c_d = clamp(floor((x_d - 0) * (1/cell_d)), 0, ncell_d - 1),
 *              id = (c_z ncell_y + c_y) ncell_x + c_x.
 *   perm       device, n int32: point indices sorted by (cell id, index).
 *   cell_start device, ncell_x ncell_y ncell_z + 1 int32: first position in
 *              perm of each cell; the last entry is n.
 * Integer results; identical to a sequential stable counting sort.
 */
hse_status hse_cell_list(hse_plan plan, int64_t n, const double* pos, int32_t* cell_id, int32_t* perm,
                         int32_t* cell_start, void* cuda_stream);

/*
 * hse_neighbor_counts -- per target, the number of free-space pairs and of
 * image pairs inside the cut-off (|d|^2 < r_c^2 with the squared distance
 * formed as ((dx*dx) + (dy*dy)) + (dz*dz) in FP64 without contraction), the
 * same decision the real-space sum takes.  tgt_xyz == NULL: targets are the
 * sources and the self pair is not counted.  n_pairs, n_images: device,
 * n_tgt int32 each.
 */
hse_status hse_neighbor_counts(hse_plan plan, int64_t n_src, const double* src_xyz, int64_t n_tgt,
                               const double* tgt_xyz, int32_t* n_pairs, int32_t* n_images, void* cuda_stream);

/*
 * hse_spread_grids -- the spread grids of Alg. 1 step 5 on the Mt x Mt x 2 Mt
 * grid (z fastest), in the component order: per kernel in the order S, T, W,
 *   S: C1 (3), C2 = f3 (1), C3 = y3 f^I (3)
 *   T: C1 = sym(g q) (6: xx xy xz yy yz zz), C2 = g.q (1), C3 = y3 sym(g^I q^I) (6)
 *   W: C1 = tau (3), C2 = (-tau2, tau1) (2)
 * C1 holds the sources and their images, C2/C3 the images only.  Grid point
 * (i, j, k) sits at (-P h/2 + i h, -P h/2 + j h, -Mt h + k h).
 * grids: device, n_comp x Mt x Mt x 2 Mt doubles; *n_comp receives the count
 * (pass grids = NULL to query it).  Diagnostic entry point (slow path).
 */
hse_status hse_spread_grids(hse_plan plan, int64_t n_src, const double* src_xyz, const double* strengths,
                            double* grids, int* n_comp, void* cuda_stream);

/* Stages of one evaluation, in order (the phases of Sec. 7, Fig. 6). */
enum {
  HSE_STAGE_CHECK = 0,     /* input check (one stream synchronisation)        */
  HSE_STAGE_CELLS = 1,     /* binning, stable sort, cell starts, sorted copy   */
  HSE_STAGE_REAL = 2,      /* real-space neighbour sum and self term           */
  HSE_STAGE_SPREAD = 3,    /* window factors, spreading, image mirror (step 5) */
  HSE_STAGE_FFT = 4,       /* forward zero-padded FFTs (step 6)                */
  HSE_STAGE_SCALE = 5,     /* k-space scaling (steps 7-8)                      */
  HSE_STAGE_IFFT = 6,      /* inverse FFTs (step 9)                            */
  HSE_STAGE_GATHER = 7,    /* quadrature at the targets (step 10)              */
  HSE_N_STAGES = 8
};

typedef struct {
  int n_kernel_launches;            /* kernels of this library launched by the last evaluation */
  int n_fft_execs;                  /* 3-D transforms (one per buffer) of the last evaluation   */
  int timing;                       /* 1 when stage_ms is valid                                 */
  double stage_ms[HSE_N_STAGES];    /* device time of each stage (CUDA events on its stream)   */
  int overlapped;                   /* 1: the real stage ran concurrently with SPREAD..GATHER  */
  double total_ms;                  /* first to last event of the evaluation                   */
} hse_eval_stats;

/* Enable (1) or disable (0) CUDA-event timing of the stages of hse_eval and
 * hse_eval_parts.  Timing adds one event record per stage on the stream; with
 * overlapped halves (hse_plan_set_overlap) stage times are per stream and
 * overlap in time. */
hse_status hse_plan_set_timing(hse_plan plan, int enable);
/* 1: with both halves requested, run the real-space stage on one internal
 * stream and the Fourier stages on another (higher priority), joined on the
 * caller's stream before the call's work ends; 0 (default): one after the
 * other on the caller's stream. */
hse_status hse_plan_set_overlap(hse_plan plan, int enable);
/* Cap the real-space kernel of targets = sources at blocks_per_sm resident
 * blocks per multiprocessor (a persistent grid of blocks_per_sm x SM-count
 * blocks; 0, the default: no cap).  Results are unchanged up to summation
 * order.  With overlapped halves this leaves part of every SM's registers to
 * the Fourier kernels, so the FP64-bound real space and the FP32-bound
 * Fourier part share the SMs instead of running one after the other.
 * HSE_ERR_INVALID for blocks_per_sm outside [0, 64]. */
hse_status hse_plan_set_real_residency(hse_plan plan, int blocks_per_sm);

/* Shape of the grid tile one warp of the spread owns (Alg. 1 step 5: each
 * lane sums the windows of the sources covering its grid point): wx x wy x wz
 * points along x, y, z, each 1, 2, 4, 8 or 16 with wx wy wz = 32; a block of
 * 8 warps owns 2wx x 2wy x 2wz points.  The default 2 x 4 x 4 suits large
 * grids; the batch autotuner (hse_batch_create) picks the shape per group of
 * instances.  Results change only by the rounding of the FP32 small-weight
 * part of the spread (which weights take it depends on the tile), far below
 * the plan's tolerance.  HSE_ERR_INVALID for any other shape. */
hse_status hse_plan_set_spread_tile(hse_plan plan, int wx, int wy, int wz);

/* Statistics of the last evaluation (synchronises on its last event when
 * timing is on).  out: host pointer. */
hse_status hse_get_eval_stats(hse_plan plan, hse_eval_stats* out);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of independent evaluations.                  */
/* ------------------------------------------------------------------------ */
typedef struct hse_server_s* hse_server;

#define HSE_PENDING 7 /* hse_server_poll: the request has not finished yet */

typedef struct {
  int n_slots;              /* concurrent evaluations (one CUDA stream and worker thread each), >= 1 */
  size_t mem_budget_bytes;  /* device memory the server may hold for plans and work areas (0: 60% of free) */
} hse_server_config;

typedef struct {
  int kernel_mask;          /* HSE_STOKESLET / HSE_STRESSLET / HSE_ROTLET bits */
  int precision;            /* HSE_FP64 or HSE_MIXED */
  double tol;               /* target relative RMS error (> 0)                   */
  double box[3];            /* source box, as for hse_plan_create                */
  int64_t n_src;
  const double* src_xyz;    /* device, 3 x n_src (caller-owned until completion) */
  const double* strengths;  /* device, rows x n_src                              */
  int64_t n_tgt;
  const double* tgt_xyz;    /* device or NULL (targets = sources)                */
  double* vel;              /* device, 3 x n_tgt, written on completion          */
} hse_request;

typedef struct {
  int64_t submitted, completed, failed, in_flight;
  double p50_ms, p99_ms, mean_ms;  /* submit -> completion latency of completed requests */
  double busy_s;                   /* wall time from first submission to last completion */
  double targets_per_s;            /* completed targets / busy_s                         */
  int64_t plans_created, plans_evicted;
  size_t resident_bytes;           /* device bytes held by cached plans                  */
  int64_t plan_hits;               /* requests admitted to a resident plan (cache hits)  */
  double plan_build_s;             /* host time spent building plans (incl. prewarm)     */
} hse_server_stats;

/*
 * A server evaluates independent requests (Sec. 3 sums of any kernel mix,
 * size and tolerance) with continuous batching: requests queue on submission;
 * each worker slot takes the oldest request whose estimated device memory
 * (grids, tables and cell-list work areas) fits the budget next to the work
 * already admitted, checks out a resident plan with the request's parameters
 * (or builds one, evicting idle plans least recently used), and evaluates on
 * its own stream, so work of different requests overlaps on the GPU (a
 * request whose plan is busy with another request waits for it rather than
 * building a duplicate).  An HSE_MIXED request with the stokeslet bit (half
 * space) whose modelled FP32 rounding of the Fourier part, 2.5e-8 sqrt(n_src)
 * of the velocity, exceeds tol/3 runs its Fourier part in double-float (see
 * HSE_FFT_DF64; hse_server_request_params reports fft).  xi is
 * chosen from N and the box (xi = 0.7 (N/V)^(1/3) rounded to a factor-sqrt(2)
 * ladder, so plans are shared between requests); r_c, M and P come from tol.
 * The caller keeps the request's arrays alive until the request completes.
 */
hse_status hse_server_create(const hse_server_config* cfg, hse_server* out);
/* Queue a request; *ticket identifies it.  Never blocks on GPU work. */
hse_status hse_server_submit(hse_server srv, const hse_request* req, uint64_t* ticket);
/* Build, synchronously on the calling thread, the plan that a request like
 * *req would use (only kernel_mask, precision, tol, box and n_src are read;
 * no data), so that later requests with the same plan parameters find it
 * resident instead of paying its set-up inside their latency.  HSE_OK when
 * the plan is resident or already being built; HSE_ERR_OOM when it does not
 * fit the memory budget next to the plans already held; the errors of
 * hse_plan_create otherwise.  The calling thread's current device is kept. */
hse_status hse_server_prewarm(hse_server srv, const hse_request* req);
/* Parameters (xi, r_c, P, M, ...) of the plan that evaluated a finished
 * request: HSE_OK, HSE_PENDING while it runs, HSE_ERR_INVALID for an unknown
 * ticket or a request that failed before its plan existed.  out: host. */
hse_status hse_server_request_params(hse_server srv, uint64_t ticket, hse_params* out);
/* HSE_OK when finished, HSE_PENDING while queued or running, else the
 * request's error status. */
hse_status hse_server_poll(hse_server srv, uint64_t ticket);
/* Wait at most timeout_s seconds: HSE_OK, the request's error, or
 * HSE_ERR_TIMEOUT (the request keeps running). */
hse_status hse_server_wait(hse_server srv, uint64_t ticket, double timeout_s);
hse_status hse_server_get_stats(hse_server srv, hse_server_stats* out);
/* Text of a failed request's error ("" when it succeeded or is pending); valid
 * until the server is destroyed. */
const char* hse_server_error_text(hse_server srv, uint64_t ticket);
/* Reset the latency record (not the plan cache). */
hse_status hse_server_reset_stats(hse_server srv);
/* Waits for admitted work, fails queued requests, frees plans. */
hse_status hse_server_destroy(hse_server srv);

/* ------------------------------------------------------------------------ */
/* Batched instances: many small independent systems in few launches.         */
/* ------------------------------------------------------------------------ */
typedef struct hse_batch_s* hse_batch;

typedef struct {
  int kernel_mask;          /* HSE_STOKESLET / HSE_STRESSLET / HSE_ROTLET bits   */
  int64_t n;                /* particles (>= 1); targets are the sources         */
  const double* src_xyz;    /* device, 3 x n                                     */
  const double* strengths;  /* device, rows x n in the order of hse_eval         */
  double* vel;              /* device, 3 x n, overwritten                        */
} hse_instance;

typedef struct {
  int64_t instances, particles;  /* evaluated so far                          */
  int64_t chunks;                /* launch groups (one pass of every stage)   */
  int64_t kernel_launches;       /* this library's kernels                    */
  int64_t fft_execs;             /* batched cuFFT executions                  */
  int64_t plans;                 /* (mask, xi) groups with a resident plan    */
  int64_t autotuned_groups;      /* groups whose xi the autotuner timed       */
  size_t grid_bytes;             /* component-major grids of the largest chunk */
  size_t fft_work_bytes;         /* shared work area of the batched cuFFT plans */
  size_t particle_bytes;         /* per-particle work arrays (grow-only)      */
  size_t plan_bytes;             /* grids and tables held by the group plans  */
  double stage_ms[HSE_N_STAGES]; /* summed stage times of all timed chunks     */
  int64_t graphs_captured;       /* stage sequences captured as CUDA graphs   */
  int64_t graph_launches;        /* chunks run by replaying a captured graph  */
} hse_batch_stats;

/*
 * A batch evaluates many independent instances of the Sec. 3 sums, each a
 * set of particles in the same box (targets = sources, as hse_eval with
 * tgt_xyz == NULL), to one tolerance and precision.  Instances are grouped by
 * kernel mask and xi (xi = 0.7 (N/V)^(1/3) on a factor-sqrt(2) ladder, or the
 * ladder level the autotuner found fastest for the group); each group has one
 * plan (r_c, M, P from tol) and is evaluated in chunks of many instances, every
 * stage of Sec. 4-5 one launch over the whole chunk: one cell list over all
 * instances (key = instance, cell), one real-space launch, one spread, batched
 * pruned FFTs (a few cuFFT executions over all instances' grids), one k-space
 * scaling, one gather.
 * Results equal those of hse_eval on a plan with the same parameters, up to
 * summation order.
 *   tol, precision    as for hse_plan_create (xi, r_c, P chosen from tol).
 *   box               host {L1, L2, L3}, shared by all instances.
 *   mem_budget_bytes  device bytes for the grids of one chunk (0: half the
 *                     free memory at creation).
 *   autotune          1: on the first instances of each group, time xi
 *                     ladder levels walking down from the default while each
 *                     step is faster per particle (else up), and keep the
 *                     fastest; every level meets tol, so results stay valid.
 */
hse_status hse_batch_create(double tol, int precision, const double box[3], size_t mem_budget_bytes, int autotune,
                            hse_batch* out);
/* Evaluate n_inst instances (host array of descriptors, device data) on the
 * stream; returns after the last chunk has been queued (the input check
 * synchronises the stream once per chunk).  Errors: HSE_ERR_INVALID (bad
 * descriptor or data; text from hse_batch_last_error), HSE_ERR_OOM,
 * HSE_ERR_CUDA, HSE_ERR_CUFFT. */
hse_status hse_batch_eval(hse_batch batch, int n_inst, const hse_instance* inst, void* cuda_stream);
hse_status hse_batch_get_stats(hse_batch batch, hse_batch_stats* out);
/* Parameters (xi, r_c, P, M, ...) of the group plan that evaluated instance i
 * (0-based, in the order of the last hse_batch_eval call's array).
 * HSE_ERR_INVALID when i was not evaluated by the last call.  out: host. */
hse_status hse_batch_instance_params(hse_batch batch, int i, hse_params* out);
/* Enable (1) or disable (0) CUDA-event timing of the stages of every chunk
 * (stage_ms of the stats; synchronises the stream once per chunk).  Timed
 * chunks are launched directly, not from graphs. */
hse_status hse_batch_set_timing(hse_batch batch, int enable);
/* Replay (1, the default) or not (0) each chunk's stage sequence from a CUDA
 * graph.  A chunk's stages after the input check (sort, real space, spread,
 * transforms, scaling, gather, scatter) are captured once per chunk shape and
 * replayed when the same instance sizes come again; the graph reads the
 * caller's arrays through a device descriptor table, so they may change. */
hse_status hse_batch_set_graphs(hse_batch batch, int enable);
/* Text of the batch's last failure ("" when none). */
const char* hse_batch_last_error(hse_batch batch);
/* Waits for the device, frees plans, grids and cuFFT plans. */
hse_status hse_batch_destroy(hse_batch batch);

/*
 * hse_cell_list_noalloc -- the cell list of hse_cell_list (same cell ids,
 * permutation and cell starts, bit for bit) without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that may
 * not let a library call cudaMalloc/cudaFree -- applications whose framework
 * or pool allocator owns the device heap, and loops where an allocation,
 * which can synchronise the device, is not allowed.
 *   n           number of points, 0 <= n <= HSE_NOALLOC_MAX_POINTS; larger n
 *               is rejected with HSE_ERR_INVALID (see hse_last_error(NULL)).
 *   pos         device, 3 x n positions.
 *   box, ncell  host arrays: box side L_d > 0 and cells per side
 *               1 <= ncell_d <= 1024; cell side L_d / ncell_d, cell of a point
 *               clamp(floor(x_d * (ncell_d / L_d)), 0, ncell_d - 1) (non-finite
 *               coordinates land in a boundary cell).
 *   cell_id, perm  device, n int32 each; cell_start device, prod(ncell) + 1.
 * Work arrays live in one fixed device array inside the library (3.3 MiB), resident on every GPU that loads the library until the process
 * exits.  The first call on a device looks up that array's device address
 * (no allocation), with the device current; make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents: calls whose work can overlap on the GPU (different streams,
 * threads or devices sharing a context) race -- serialise them.
 */
#define HSE_NOALLOC_MAX_POINTS 262144
hse_status hse_cell_list_noalloc(int64_t n, const double* pos, const double box[3], const int ncell[3],
                                 int32_t* cell_id, int32_t* perm, int32_t* cell_start, void* cuda_stream);

/* Measured arithmetic throughput of the current device (dense multiply-add
 * chains on every SM, best of three launches; synchronous, ~0.1 s).  The
 * paper has no counterpart: these are the roofline denominators of the
 * FP64-bound real-space pairs, the FP32 shell and mixed path, and the
 * double-float (df64) Fourier part (one df64 multiply-add counted as 2 flops,
 * the grid update of the spread and gather).  Allocates and frees a small
 * device buffer.  Errors: HSE_ERR_INVALID (NULL out), HSE_ERR_OOM,
 * HSE_ERR_CUDA. */
typedef struct {
  double fp64_tflops;   /* FP64 FMA, 2 flops each   */
  double fp32_tflops;   /* FP32 FMA, 2 flops each   */
  double df64_tflops;   /* df64 multiply-add, 2 flops each */
  int n_sm;             /* multiprocessors          */
  double sm_clock_mhz;  /* the device's reported maximum SM clock */
} hse_pipe_peaks;
hse_status hse_measure_pipe_peaks(hse_pipe_peaks* out);

/* Release all device memory and cuFFT plans of the plan (synchronises). */
hse_status hse_plan_destroy(hse_plan plan);

/* Static text of a status code. */
const char* hse_status_string(hse_status status);

/* Text of the last failure of a plan (valid until the next call on the plan);
 * "" when none.  A NULL plan gives the calling thread's last failure outside a
 * plan (hse_plan_create, servers, the no-allocation entry point). */
const char* hse_last_error(hse_plan plan);

#ifdef __cplusplus
}
#endif

#endif /* HSE_H */
