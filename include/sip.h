/*
 * sip.h -- C ABI of a GB300 (sm_103a) implementation of PARSDMM, the
 * projection onto an intersection of sets of arXiv:1902.09699.
 *
 * Problem (Eq. proj_intersect, Eq. proj_intersect_indicator):
 *     x = argmin_x 1/2 ||x - m||_2^2   s.t.  A_i x in C_i,  i = 1..p,
 * with A_i an identity or finite-difference operator on a regular 2D/3D grid
 * and C_i a simple set (bounds, l1 ball, l2 ball, cardinality; set table of
 * Sec. "Software and numerical examples").  The user gives m and the pairs
 * (A_i, C_i); the library adds the identity block and the prox of the
 * squared distance (Sec. "Software and numerical examples") and runs
 * Algorithm PARSDMM with Algorithm adapt-rho-gamma and the stopping rule of
 * Eq. stopping_conditions, optionally inside Algorithm ML-PARSDMM.
 *
 * Layout: every grid vector is contiguous with z the fastest index,
 * linear index iz + n_z*(ix + n_x*iy) (Sec. "Notation").  The output of a
 * forward difference along an axis has one sample fewer along that axis
 * (Eq. FD_mat) and the same z-fastest layout on its own grid; the TV
 * operator stacks D_z, D_x (, D_y) outputs in that order.
 *
 * Precision: SIP_F64 stores and computes everything in binary64.
 * SIP_F32 stores vectors and computes element-wise in binary32.  Its sums
 * are formed in two levels: each CTA adds its share (a work item of at most
 * a few thousand entries) in binary32; the CTA totals of the set and final
 * passes (norms, feasibility and adapt-rho-gamma inner products) are added
 * in binary64, those of the CG's inner products in double-binary32 (a
 * hi + lo pair whose rounding error TwoSum keeps), and the CG scalars alpha
 * and beta are binary32.  The l1 threshold's running sums are exact (integer
 * sums of the binary32 significands in the radix selection) and the
 * adapt-rho-gamma ratios are binary64.  Binary64 arithmetic runs at 1/64 of
 * the binary32 rate on this GPU, which is why the CG chain avoids it.
 * Device buffers passed to the library hold elements of the handle's
 * dtype.
 *
 * Errors: every call returns a sip_status; nothing throws across the ABI.
 * sip_last_error() gives a thread-local message for the last failure of
 * the calling thread.  A failed call leaves a handle usable.
 *
 * Threads / streams: calls on one handle must not overlap; distinct
 * handles are independent.  Device work is ordered on the caller's stream
 * (a cudaStream_t passed as void*, NULL for the legacy default stream).
 */
#ifndef SIP_H
#define SIP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIP_MAX_SETS 16
#define SIP_MAX_LEVELS 8  /* ML-PARSDMM levels */

typedef enum {
    SIP_OK = 0,
    SIP_ERR_INVALID_ARG = 1, /* bad pointer, size, set parameter or option */
    SIP_ERR_OOM = 2,         /* device or host allocation failed */
    SIP_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SIP_ERR_TIMEOUT = 4,     /* a bounded wait gave up */
    SIP_ERR_NONFINITE = 5,   /* NaN/Inf met in the model */
    SIP_ERR_BUDGET = 6,      /* request exceeds a memory budget */
    SIP_ERR_INTERNAL = 7     /* a device-side consistency check failed */
} sip_status;

/* Linear operators A_i (Eq. FD_mat; set table). */
typedef enum {
    SIP_OP_I = 0,   /* identity, M = N */
    SIP_OP_DZ = 1,  /* (x[iz+1]-x[iz])/h_z, output (n_z-1) x n_x (x n_y) */
    SIP_OP_DX = 2,  /* (x[ix+1]-x[ix])/h_x, output n_z x (n_x-1) (x n_y) */
    SIP_OP_DY = 3,  /* (x[iy+1]-x[iy])/h_y, 3D only */
    SIP_OP_TV = 4,  /* anisotropic TV stack [D_z; D_x (; D_y)] */
    SIP_OP_BLUR = 5 /* blurring forward operator F of a data-fit set (Sec.
                       "Introduction", the projection / feasibility problem
                       with V_data; the motion blur of Sec. "Joint
                       deblurring-denoising-inpainting"): M = N,
                       (F x)[j] = sum_{|t| <= R} k_|t| x[j + t e_axis], samples
                       outside the grid taken as 0; see sip_set.blur_* */
} sip_op;

/* Simple sets C_i (set table). */
typedef enum {
    SIP_SET_BOUNDS = 0, /* lo <= (Ax)[j] <= hi; lo/hi may be -/+INFINITY */
    SIP_SET_L1 = 1,     /* ||Ax||_1 <= sigma */
    SIP_SET_L2 = 2,     /* ||Ax||_2 <= sigma */
    SIP_SET_CARD = 3,   /* card(Ax) <= k; ties: larger |.| first, then lower index */
    SIP_SET_ANNULUS = 4 /* lo <= ||Ax||_2 <= hi, 0 <= lo <= hi (absolute radii);
                           not convex for lo > 0; Ax = 0 is left at 0 */
} sip_set_type;

/* Where a set applies (the paper's per-column / per-row / per-fiber sets):
 * to A x as a whole, or to every line of A x's output grid along z (the
 * columns of a 2D model), along x (its rows) or along y (3D fibers), each
 * line on its own.  Per-line sets: l1, l2, card or annulus (bounds apply
 * entry-wise anyway); not with SIP_OP_TV (its parts live on different
 * grids); absolute radii only (sigma_rel = 0); k_frac resolves against the
 * line length; card and l1 lines hold at most SIP_MAX_LINE entries. */
typedef enum { SIP_SCOPE_ALL = 0, SIP_SCOPE_Z = 1, SIP_SCOPE_X = 2, SIP_SCOPE_Y = 3 } sip_scope;
#define SIP_MAX_LINE 4096
/* Largest blur radius R (2R + 1 samples: a 25-sample motion blur is R = 12). */
#define SIP_MAX_BLUR_RADIUS 12

typedef enum { SIP_F64 = 0, SIP_F32 = 1 } sip_dtype;

/* SIP_FORM_ALG1: the paper's iteration with the identity block p+1
 * (Eqs. PARSDMM_1, SDMM_adaptive).  SIP_FORM_DIRECT: the distance term kept
 * in the x-step, (I + sum rho_i A_i^T A_i) x = m + sum A_i^T(rho_i y_i + v_i),
 * no block p+1. */
typedef enum { SIP_FORM_ALG1 = 0, SIP_FORM_DIRECT = 1 } sip_form;

typedef struct {
    int ndim;     /* 2 or 3 */
    int64_t n[3]; /* n_z, n_x, n_y (n[2] ignored in 2D); every n >= 1 */
    double h[3];  /* grid spacing per axis, > 0 (Eq. FD_mat) */
} sip_grid;

typedef struct {
    int op;           /* sip_op */
    int type;         /* sip_set_type */
    double lo, hi;    /* SIP_SET_BOUNDS, lo <= hi; SIP_SET_ANNULUS radii */
    double sigma;     /* SIP_SET_L1 / L2 radius (>= 0), used when sigma_rel == 0 */
    double sigma_rel; /* > 0: radius = sigma_rel * ||A m|| (l1 or l2 norm of the
                         set), resolved on the device from each model m */
    int64_t k;        /* SIP_SET_CARD, >= 0, used when k_frac == 0 */
    double k_frac;    /* > 0: k = floor(k_frac * N) with N the grid size (per-line
                         sets: the line length) */
    int scope;        /* sip_scope (SIP_SCOPE_ALL when zero-initialised) */
    /* SIP_SET_BOUNDS only, optional: host arrays of M_i = rows of A_i
     * entries, per-entry bounds lo_vec[j] <= (A x)[j] <= hi_vec[j] in place
     * of lo / hi (either may be NULL: the scalar applies).  This is the
     * paper's point-wise data-fit set {l <= F x - d_obs <= u} for F = A_i
     * (e.g. the identity or a blur, SIP_OP_BLUR; a binary mask is
     * +-INFINITY at unobserved entries), with d_obs folded in:
     * lo_vec = l + d_obs, hi_vec = u + d_obs.
     * Copied when the handle is created; lo_vec <= hi_vec, no NaN.  Not
     * accepted by the server. */
    const double *lo_vec, *hi_vec;
    /* SIP_SET_L2 only, optional: host array of M_i observed values d: the
     * set becomes the paper's l2 data-fit ball {||F x - d||_2 <= sigma} with
     * F = A_i; NaN marks an unobserved entry (a binary mask: left out of
     * the norm, unconstrained).  Absolute sigma, scope SIP_SCOPE_ALL;
     * copied at create; not accepted by the server. */
    const double *center_vec;
    /* SIP_OP_BLUR only: the axis (0 = z, 1 = x, 2 = y; y needs a 3D grid),
     * the radius R (1..SIP_MAX_BLUR_RADIUS) and a host array of the R + 1
     * taps k_0..k_R (finite; copied at create) of the centred symmetric
     * kernel.  F is symmetric, so F^T F adds a band of 4R + 1 samples along
     * the axis to the x-step's system matrix (Eq. sys_mat).  A blur set
     * takes scope SIP_SCOPE_ALL and a single level; at most one blur set
     * per projection.  The single-operator entry points (sip_apply_op,
     * sip_apply_op_t, sip_system_apply, sip_op_norm, sip_prolong) carry no
     * taps and reject SIP_OP_BLUR; the server rejects blur sets. */
    int blur_axis;
    int blur_radius;
    const double *blur_taps;
} sip_set;

typedef struct {
    int max_iter;       /* iterations of Algorithm PARSDMM (>= 1) */
    int cg_iters;       /* > 0: fixed CG steps per x-update; 0: Eq. cg_stop
                           rule ||r_j|| < 0.1 ||r_0||, at most cg_max steps */
    int cg_max;
    double eps_feas;    /* Eq. stopping_conditions (paper: 1e-3) */
    double eps_evol;    /* Eq. stopping_conditions (paper: 1e-2) */
    int check_every;    /* feasibility / evolution tested when k % check_every == 0 */
    int evol_hist;      /* s of Eq. obj_stop, 1..8 */
    int stop;           /* 0: run max_iter; 1: Eq. stopping_conditions; 2: feasibility only */
    int adapt;          /* 0: fixed rho, gamma; 1: adapt rho; 2: adapt rho and gamma */
    int adapt_every;    /* adapt when k % adapt_every == 1 % adapt_every */
    double rho0, gamma0;
    double eps_corr;    /* Algorithm adapt-rho-gamma (0.3) */
    double rho_ratio_max; /* rho_i kept in [rho_{p+1}/R, rho_{p+1} R] */
    double gamma_max;   /* gamma kept below 2 (1.99) */
    int form;           /* sip_form */
    int dtype;          /* sip_dtype */
    int levels;         /* 1, or 2..SIP_MAX_LEVELS for ML-PARSDMM (Sec. "Multilevel
                           PARSDMM"): each coarser grid halves every axis
                           (n -> ceil(n/2), h -> 2h); every level must be a
                           valid grid for the set list */
    int coarse_iter;    /* iterations on the coarse level (0: max_iter) */
    /* Optional host arrays [max_iter][nblocks] of rho_i / gamma_i used in
     * iteration k (row k-1); nblocks = nsets + (form == ALG1).  When set, the
     * values are replayed instead of adapted.  Read during sip_project. */
    const double *rho_schedule;
    const double *gamma_schedule;
    /* Optional host array [max_iter][2*nblocks + 2 + nsets] filled by
     * sip_project (single-level only): per iteration the rho_i and gamma_i
     * used, the CG steps, r_evol and r_feas_i (NaN when not a check
     * iteration). */
    double *trace;
    /* Execution of the iterations: SIP_EXEC_AUTO (currently the graph path),
     * SIP_EXEC_GRAPH (one kernel per phase, replayed from a CUDA graph),
     * SIP_EXEC_PERSISTENT (one cooperative kernel for all iterations, grid
     * barriers between phases) or SIP_EXEC_CLUSTER (one launch for all
     * iterations; each instance runs on one thread-block cluster of
     * cluster_ctas CTAs with the cluster's hardware barrier between phases,
     * and a cluster takes the next instance when its own has stopped; for
     * small grids, where the graph path is bound by launch latency).  Results
     * are the same up to rounding order of the binary64 atomics.  Plans with
     * a blur block take the graph path. */
    int exec;
    /* Top-k selections of cardinality sets (Sec. Notation: projection onto
     * {card(A x) <= k}): 1 (default) starts each iteration's selection from
     * a window around the previous iteration's k-th value; the set pass
     * collects the entries inside it and, when the k-th value falls inside,
     * one CTA selects it there instead of the full radix passes.  0: radix
     * passes only.  The selected key, and so the result, is the same. */
    int select_window;
    /* CTAs per cluster in SIP_EXEC_CLUSTER: 1, 2, 4, 8 or 16; 0 picks one
     * from the instance sizes (about 8192 grid points per CTA). */
    int cluster_ctas;
    /* 1: tune the plan on the handle's first projection (see sip_tuning);
     * 0 (default): the built-in heuristic. */
    int tune;
    /* 1 (SIP_F32 only): BF16 storage trial for m and the duals.  Every
     * store of y_i and v_i (and their adapt-rho-gamma copies) and the model m
     * are rounded to bfloat16 (round to nearest even), so the iteration
     * follows exactly the numbers a BF16 storage of those arrays would hold;
     * the arrays stay binary32 (the trial measures the accuracy, not the
     * bandwidth).  Coarse multilevel models are restricted from the binary32
     * model and then rounded.  Not with per-line sets or blur sets. */
    int store_bf16;
} sip_options;

#define SIP_EXEC_AUTO 0
#define SIP_EXEC_GRAPH 1
#define SIP_EXEC_PERSISTENT 2
#define SIP_EXEC_CLUSTER 3

typedef struct {
    int iters;          /* iterations run (finest level) */
    int cg_steps_total; /* CG steps summed over iterations (finest level) */
    int stop_reason;    /* 0: max_iter reached; 1: stopping rule held */
    int nblocks;
    double r_evol;      /* last computed Eq. obj_stop value */
    double r_feas[SIP_MAX_SETS]; /* last computed Eq. feas_stop values */
    double rho[SIP_MAX_SETS + 1];
    double gamma[SIP_MAX_SETS + 1];
    double sigma[SIP_MAX_SETS];  /* resolved radii (finest level) */
    int64_t k[SIP_MAX_SETS];     /* resolved cardinalities (finest level) */
    float ms;           /* device time of the projection (CUDA events) */
    int window_hits;    /* top-k selections resolved inside their window
                           (summed over the cardinality sets and iterations) */
} sip_info;

typedef struct sip_handle sip_handle;

/* Fill *opts with the defaults (paper values where the paper gives one):
 * max_iter 200, cg_iters 5, cg_max 100, eps_feas 1e-3, eps_evol 1e-2,
 * check_every 5, evol_hist 5, stop 0, adapt 1, adapt_every 2, rho0 1,
 * gamma0 1.5, eps_corr 0.3, rho_ratio_max 1e3, gamma_max 1.99,
 * form ALG1, dtype F32, levels 1, select_window 1, cluster_ctas 0, tune 0,
 * store_bf16 0. */
void sip_options_default(sip_options *opts);

/* Build a projector for one grid and set list.  Validates every argument,
 * resolves the operator / set layout and allocates the device arena that
 * holds x, y_i, v_i, the CG vectors, the adapt state and all scratch
 * (allocation happens here only).  nsets in [1, 16].  Returns
 * SIP_ERR_INVALID_ARG for: NULL pointers, ndim not 2/3, n < 1, h <= 0,
 * unknown op/type, an op that needs an axis of length >= 2 on a shorter
 * axis, lo > hi, sigma < 0, k < 0, k_frac or sigma_rel < 0, bad options. */
sip_status sip_create(const sip_grid *grid, const sip_set *sets, int nsets,
                      const sip_options *opts, sip_handle **out);

/* Project the device vector m_dev (N elements of the handle's dtype) and
 * write the result to x_dev (N elements).  Stream-ordered on `stream`;
 * returns without synchronising unless info != NULL, a trace or schedule
 * is requested, or the stopping rule is on.  m_dev must stay valid until
 * the work completes.  State (x, y_i, v_i) starts from zero on the coarsest
 * level each call. */
sip_status sip_project(sip_handle *h, const void *m_dev, void *x_dev,
                       void *stream, sip_info *info);

sip_status sip_destroy(sip_handle *h);

/* Warm start (the paper starts the iterates from a given state where one is
 * available: ML-PARSDMM hands x, y_i, v_i from one level to the next, Sec.
 * "Multilevel PARSDMM"; an inverse-problem loop projects nearby models
 * one after another).  The state is x (N entries) and y, v (M' entries
 * each: every block's rows in block order, the identity block p + 1 last
 * in SIP_FORM_ALG1), device arrays of the handle's dtype, z fastest.
 * sip_state_rows returns M' (-1 for a batched or multilevel handle).
 * sip_get_state copies the handle's current state out (after a
 * projection: its final iterates); NULL pointers are skipped.
 * sip_set_state loads a state; the next sip_project (that one only) starts
 * from it instead of zeros.  x_dev is required; NULL y_dev / v_dev load
 * zeros.  rho / gamma (host arrays, one value per block in block order,
 * identity block last in SIP_FORM_ALG1; e.g. sip_info.rho / gamma of the
 * projection the state came from) give the starting penalties and
 * relaxations, which adapt-rho-gamma then updates as usual; NULL: rho0 /
 * gamma0, as on a multilevel hand-over.  rho_i > 0, 0 < gamma_i < 2; a
 * rho_schedule, when set, takes precedence.  Both are stream-ordered on `stream`; single-level,
 * single-instance handles only (SIP_ERR_INVALID_ARG otherwise). */
int64_t sip_state_rows(const sip_handle *h);
sip_status sip_get_state(sip_handle *h, void *x_dev, void *y_dev, void *v_dev,
                         void *stream);
sip_status sip_set_state(sip_handle *h, const void *x_dev, const void *y_dev,
                         const void *v_dev, const double *rho,
                         const double *gamma, void *stream);

/* The quantities Algorithm adapt-rho-gamma saved at its last call ("save
 * for next call"): v-hat, y and v at that iteration k0 (M' entries each, the
 * layout of y, v above) and x^{k0} (N entries), from which the set pass
 * forms s^{k0} = A_i x^{k0}.  With them a warm start continues the
 * iteration as if it had not stopped: the next projection's first adapt
 * call forms its differences against them instead of only saving.  (With
 * sip_set_state alone it starts a fresh adapt history.)
 * sip_get_adapt_state copies them out after a projection and sets *have to
 * 1, or to 0 when no adapt call has saved anything yet (the arrays are then
 * not written; NULL pointers are skipped); it synchronises `stream`.
 * sip_set_adapt_state loads them for the next sip_project, together with a
 * state loaded by sip_set_state (call that too: the adapt history belongs
 * to the iterates it came with), copied into a staging buffer that the
 * handle allocates on first use.  For handles whose adapt calls come more
 * often than the x history is long (adapt_every < evol_hist, the default);
 * single-level, single-instance handles with adapt != 0; SIP_ERR_INVALID_ARG
 * otherwise. */
sip_status sip_get_adapt_state(sip_handle *h, void *vhat_dev, void *y_dev, void *v_dev, void *xk0_dev,
                               int *have, void *stream);
sip_status sip_set_adapt_state(sip_handle *h, const void *vhat_dev, const void *y_dev, const void *v_dev,
                               const void *xk0_dev, void *stream);

const char *sip_last_error(const sip_handle *h);

/* ---------------------------------------------------------------------
 * Batched projections: `count` independent problems, each with its own
 * grid and set list, run together.  Every launch of an iteration covers the
 * work items of all instances (a ragged launch: instances of any size share
 * the launch; reductions, selections and the adapt-rho-gamma tail stay per
 * instance), so launch and synchronisation costs are paid once per batch
 * instead of once per problem.  Each instance follows exactly the iteration
 * of a single sip_project with the same options (Algorithm PARSDMM); the
 * results equal the one-at-a-time results up to the rounding order of the
 * binary64 atomics.
 *
 * sets holds the sets of instance 0, then of instance 1, ...; nsets[i] of
 * them for instance i.  opts applies to every instance (single level, no
 * schedules or traces).  Models and results are packed: instance i's N_i
 * elements start at element sip_batch_offset(h, i); sip_batch_offset(h,
 * count) is the total.  infos (host, may be NULL) receives count entries;
 * passing it synchronises the stream.  sip_project on a batched handle
 * returns SIP_ERR_INVALID_ARG. */
sip_status sip_batch_create(int count, const sip_grid *grids, const sip_set *sets,
                            const int *nsets, const sip_options *opts,
                            sip_handle **out);
sip_status sip_batch_project(sip_handle *h, const void *m_dev, void *x_dev,
                             void *stream, sip_info *infos);
int64_t sip_batch_offset(const sip_handle *h, int i);

/* ---------------------------------------------------------------------
 * Parallel Dykstra baseline (Appendix A; the comparison of Sec. "Parallel
 * Dykstra versus PARSDMM").  argmin 1/2 ||x - m||^2 over the intersection
 * of the p sets {x : A_i x in C_i} by parallel Dykstra sweeps: y_i =
 * P_i(v_i), x = (1/p) sum_i y_i, v_i = x + v_i - y_i, from x = v_i = m.
 * Each projection P_i is computed like the paper's sub-problem solver: the
 * same iteration as PARSDMM with the one set i, `inner->max_iter`
 * iterations (or its stopping rule), starting from zero state; the p
 * sub-problems of a sweep run as one batched projection.  The sets must be
 * fixed across sweeps: absolute radii only (sigma_rel = 0).  Errors as
 * sip_create; levels must be 1. */
typedef struct {
    int sweeps;          /* Dykstra sweeps run */
    int64_t cg_steps;    /* per sweep the largest sub-problem's CG steps, summed */
    int64_t l1_projections; /* l1-ball projections: sweeps x sub-problem iterations of l1 sets */
    float ms;            /* device time (CUDA events) */
} sip_dykstra_info;
sip_status sip_dykstra_create(const sip_grid *grid, const sip_set *sets, int nsets, const sip_options *inner,
                              sip_handle **out);
/* m_dev and x_dev: N elements of the handle's dtype; synchronises. */
sip_status sip_dykstra_project(sip_handle *h, const void *m_dev, void *x_dev, int sweeps, void *stream,
                               sip_dykstra_info *info);

/* ---------------------------------------------------------------------
 * Projection server (continuous batching).  Requests may be submitted
 * from any thread at any time; a worker thread admits queued requests as
 * cohorts when the HBM budget has room for a cohort's whole state (sized
 * before allocation, so the budget is never exceeded), runs every cohort as
 * a batched plan on its own stream (cohorts admitted at different times
 * overlap on the device), keeps each request's x, y_i, v_i, rho_i and CG
 * state resident until its own stopping rule holds, then delivers it and
 * records its latency (submission to delivery, queueing included).
 * ------------------------------------------------------------------- */
typedef struct {
    sip_options opts;      /* per-request options (single level; dtype of the
                              models and results; default: stop = 2, i.e.
                              feasibility 1e-3, or max_iter = 500) */
    int64_t budget_bytes;  /* device memory the server may hold (default 120 GiB) */
    int max_batch;         /* requests per cohort (default 64) */
    int max_cohorts;       /* cohorts running at once (default 8) */
    double max_wait_ms;    /* a cohort forms once the oldest request waited
                              this long, even if smaller than max_batch */
    int64_t max_points;    /* grid points per cohort (default 2^24); a cohort
                              takes requests within a factor 4 of the size
                              of the oldest queued request */
} sip_server_config;

typedef struct {
    int64_t completed, failed, queued;
    int running_cohorts;
    int64_t hbm_in_use, hbm_peak;  /* bytes of cohort state */
    double p50_ms, p99_ms;         /* latency of completed requests */
    double projections_per_s;      /* completed / (last completion - first submission) */
} sip_server_stats;

typedef struct sip_server sip_server;

void sip_server_config_default(sip_server_config *cfg);
sip_status sip_server_create(const sip_server_config *cfg, sip_server **out);
/* Queue a projection of the host model m_host (N elements of opts.dtype);
 * the result is written to x_host (N elements) before the request is
 * reported done.  The model is copied; x_host must stay valid until
 * sip_server_wait returns for this request.  A request that does not fit
 * the budget even alone fails with SIP_ERR_BUDGET. */
sip_status sip_server_submit(sip_server *srv, const sip_grid *grid,
                             const sip_set *sets, int nsets,
                             const void *m_host, void *x_host, int64_t *req_id);
/* Block until the request is done (timeout_ms < 0: no limit); returns its
 * status, info and latency, and forgets the request. */
sip_status sip_server_wait(sip_server *srv, int64_t req_id, double timeout_ms,
                           sip_info *info, double *latency_ms);
sip_status sip_server_query_stats(sip_server *srv, sip_server_stats *out);
/* Finishes every queued and running request, then stops the worker. */
sip_status sip_server_destroy(sip_server *srv);

/* Bytes of device memory the handle holds. */
int64_t sip_device_bytes(const sip_handle *h);

/* Algorithmic bytes one PARSDMM iteration must move at the handle's
 * precision (state read and written once per phase; the figure the roofline
 * uses), finest level. */
double sip_bytes_per_iter(const sip_handle *h);

/* Per-kernel device timing.  With timing on, sip_project runs the
 * iterations as a CUDA graph in which every launch records the global timer
 * at its first CTA's start and its last CTA's end, and synchronises after
 * each replay to read them; sip_kernel_times returns, per kernel category
 * (see sip_kernel_name, 0..SIP_KERNEL_CATEGORIES-1), the summed device
 * milliseconds, the launch count since timing was switched on, and the
 * algorithmic bytes one launch moves (the roofline numerator). */
#define SIP_KERNEL_CATEGORIES 9
sip_status sip_set_timing(sip_handle *h, int on);
sip_status sip_kernel_times(const sip_handle *h, double *ms, int64_t *launches,
                            double *bytes_per_launch);
const char *sip_kernel_name(int category);

/* ---------------------------------------------------------------------
 * Single-step entry points.  Each runs the same device code the loop uses
 * on caller buffers, so every step can be checked alone.  All pointers are
 * device pointers of `dtype` elements unless stated; all calls are
 * stream-ordered and synchronise only to return host scalars.
 * ------------------------------------------------------------------- */

/* s = A x (op on grid; Eq. FD_mat).  s has sip_op_rows(grid, op) entries. */
sip_status sip_apply_op(const sip_grid *grid, int op, int dtype,
                        const void *x_dev, void *s_dev, void *stream);
/* x = A^T s. */
sip_status sip_apply_op_t(const sip_grid *grid, int op, int dtype,
                          const void *s_dev, void *x_dev, void *stream);
/* Number of rows of A (M_i), or -1 for an invalid grid/op. */
int64_t sip_op_rows(const sip_grid *grid, int op);

/* out = C x with C = c_identity I + sum_i rho_i A_i^T A_i (Eq. sys_mat),
 * applied as a matrix-free stencil.  ops/rhos are host arrays of nops. */
sip_status sip_system_apply(const sip_grid *grid, const int *ops,
                            const double *rhos, int nops, double c_identity,
                            int dtype, const void *x_dev, void *out_dev,
                            void *stream);

/* y = P_C(w) for one simple set on n entries (set table), computed with the
 * loop's kernels: clip, l2 radial scaling, l1-ball threshold by radix
 * selection with binary64 running sums, top-k by radix selection with the
 * index tie rule.  set->sigma / set->k are used as given (sigma_rel and
 * k_frac ignored).  *scalar_out (host, may be NULL) receives the l1
 * threshold theta, the l2 scale, or for card the |.| of the k-th kept
 * entry. */
sip_status sip_project_set(const sip_set *set, int dtype, const void *w_dev,
                           int64_t n, void *y_dev, void *stream,
                           double *scalar_out);

/* *out (host) = ||A m||_1 (type L1) or ||A m||_2 (type L2), accumulated in
 * binary64: the norm that relative radii (sigma_rel) refer to. */
sip_status sip_op_norm(const sip_grid *grid, int op, int type, int dtype,
                       const void *m_dev, void *stream, double *out);

/* Coarse model for ML-PARSDMM: average over 2x2(x2) blocks; the coarse
 * grid has n_c = ceil(n/2) and twice the spacing (Sec. "Multilevel
 * PARSDMM").  mc_dev has the coarse grid's N entries. */
sip_status sip_restrict(const sip_grid *fine, int dtype, const void *m_dev,
                        void *mc_dev, void *stream);
/* Linear interpolation of a vector on op's output grid from the coarse grid
 * of `fine` to `fine` (same op), extrapolating linearly at the ends. */
sip_status sip_prolong(const sip_grid *fine, int op, int dtype,
                       const void *uc_dev, void *uf_dev, void *stream);

/* ---------------------------------------------------------------------
 * Plan tuning.  The paper has no counterpart (its parallelism is one
 * thread per set, Sec. "Parallelism"); on the GPU the launch shapes decide
 * the speed.  A plan's work items are sized so that one launch fills the
 * GPU once at the kernel's occupancy; the knobs below scale that per launch
 * kind (grid points: right-hand side and CG; set pass; selection passes;
 * final pass), choose the execution form (graph or cluster) and the
 * warm-started top-k window, and switch the staged right-hand side.  Every
 * choice computes the same iteration; results differ only in the rounding
 * order of sums.
 *
 * With sip_options.tune = 1 the handle's first projection (single-level or
 * batched handles) measures candidate plans on its own model, a few
 * iterations each, one knob after another (coordinate search), keeps the
 * fastest, and records it in a process-wide cache keyed by the instances'
 * grids, set lists and options, so later handles of the same shape start
 * from the cached choice without measuring.
 *
 * sip_get_tuning reports the plan's knobs and, after tuning, the measured
 * milliseconds per iteration of the default and of the chosen plan.
 * sip_set_tuning rebuilds the plan with the given knobs (scales in
 * [1/16, 16], exec SIP_EXEC_GRAPH or SIP_EXEC_CLUSTER, cluster_ctas as in
 * sip_options, select_window and stage_rhs 0 or 1); a warm state loaded by
 * sip_set_state is dropped.  Multilevel and parallel-Dykstra handles return
 * SIP_ERR_INVALID_ARG.
 * ------------------------------------------------------------------- */
typedef struct {
    double scale_n, scale_set, scale_sel, scale_fin;
    int exec;
    int cluster_ctas;
    int select_window;
    int stage_rhs;
    /* reported by sip_get_tuning (ignored by sip_set_tuning) */
    int tuned;          /* the knobs come from a measurement (or the cache) */
    int from_cache;     /* ... taken from the process-wide cache */
    int candidates;     /* plans measured */
    double ms_default;  /* ms per iteration of the default plan (measured) */
    double ms_best;     /* ms per iteration of the chosen plan (measured) */
} sip_tuning;

sip_status sip_get_tuning(const sip_handle *h, sip_tuning *out);
sip_status sip_set_tuning(sip_handle *h, const sip_tuning *in);

/* ---------------------------------------------------------------------
 * Test hooks: host-side fault injection for the failure-handling tests.
 * The paper has no counterpart.  Process-wide settings, read when a handle
 * is created (allocation) or a persistent projection is launched
 * (barriers); not synchronised with calls running on other threads.
 *   SIP_HOOK_FAIL_ALLOC, n >= 1: the n-th next device-arena allocation of a
 *     handle (sip_create, sip_batch_create, ...) fails as if the device were
 *     out of memory, and that call returns SIP_ERR_OOM; 0 switches it off.
 *   SIP_HOOK_BARRIER_EXTRA, e >= 1: the grid barriers of the persistent
 *     kernel (SIP_EXEC_PERSISTENT) wait for e arrivals more than its CTAs
 *     make, so the first barrier runs out of polls, every CTA returns, and
 *     sip_project (with info) returns SIP_ERR_TIMEOUT; the handle stays
 *     usable.  0 switches it off.
 *   SIP_HOOK_BARRIER_SPINS, s >= 1: polls (about 0.1 us each) before a
 *     grid barrier gives up; 0 restores the default of 2^26.
 * Returns SIP_ERR_INVALID_ARG for an unknown hook or a value out of range.
 * ------------------------------------------------------------------- */
#define SIP_HOOK_FAIL_ALLOC 1
#define SIP_HOOK_BARRIER_EXTRA 2
#define SIP_HOOK_BARRIER_SPINS 3
sip_status sip_test_hook(int hook, int64_t value);

/* ---------------------------------------------------------------------
 * Allocation-free l1-ball projection.  The paper has no counterpart: this
 * is a deployment variant of sip_project_set with SIP_SET_L1.
 *
 * Same result as sip_project_set(l1 set with sigma = tau) on n device
 * elements w_dev -> y_dev, but the call allocates no memory: no cudaMalloc,
 * cudaFree or allocating library routine (host memory is touched only to
 * format an error message on failure).  It
 * is meant for callers that cannot allocate while they run: code that works
 * inside a fixed memory pool or budget a raw device allocation would bypass,
 * and latency-sensitive loops in which an allocation or free could
 * synchronise the device.  Its scratch (work list, selection state, radix
 * histograms; 89 KB) is one fixed array compiled into the library,
 * held on every GPU that loads the library until the process exits.
 *
 * n must be in [1, SIP_NOALLOC_MAX_N]; larger n returns
 * SIP_ERR_INVALID_ARG.  tau >= 0.  The first call on each device looks up
 * the array's device address (once, with that device current) and may set
 * a kernel attribute; make that first call before any stream capture.
 * Every call on a device shares the array: calls whose device work could
 * overlap (several streams or host threads on one device) race and must be
 * serialised by the caller.  Stream-ordered on `stream`; synchronises only
 * when theta_out (host, may be NULL; receives the threshold, 0 when w is
 * already inside the ball or tau = 0) is requested.  w must be finite: when
 * it holds a NaN or an infinity every y entry is NaN, and a call with
 * theta_out returns SIP_ERR_NONFINITE (theta_out = NaN).  The launches
 * size their grids from the device's SM count.
 * ------------------------------------------------------------------- */
#define SIP_NOALLOC_MAX_N (INT64_C(1) << 24)
sip_status sip_project_l1_noalloc(int dtype, const void *w_dev, int64_t n,
                                  double tau, void *y_dev, void *stream,
                                  double *theta_out);

#ifdef __cplusplus
}
#endif
#endif /* SIP_H */
