/*
 * pdhgc: restarted PDHG for linear programs and the corner-push phase of
 * Rothberg, "Backing PDHG into a Corner" (arXiv 2511.13894), on one GPU.
 *
 * The LP (Section 2) is   min c'x  s.t.  a_i x (=, <=, >=) b_i,  l <= x <= u
 * with A an m x n sparse matrix.  Its canonical form (all '=', l = 0,
 * u = +inf) is the primal of Section 2 with dual  max b'y  s.t.  A'y + z = c,
 * z >= 0.  Inequality rows and bounds are handled implicitly, as Section 2
 * says practical implementations do: no slack columns are added.
 *
 * Conventions of every call:
 *  - Return value: PDHGC_OK (0) or a negative PDHGC_ERR_* code.  Nothing is
 *    modified on an error return unless the call says otherwise.
 *    pdhgc_strerror() gives a message; pdhgc_last_error_detail() gives the
 *    detail of the last error on the calling thread (e.g. the CUDA error).
 *  - All device work is enqueued on the CUDA stream given to
 *    pdhgc_lp_create (NULL = the legacy default stream).  Calls that return
 *    host results synchronise that stream before returning.
 *  - A handle is not thread-safe; different handles are independent.
 *  - Vectors are dense, in the user's row / column order, FP64.  A pointer
 *    argument documented "host or device" is a device pointer when the
 *    call's `on_device` flag is 1 and a host pointer when it is 0.
 *  - Dual signs: y_i >= 0 on '>' rows, y_i <= 0 on '<' rows, free on '='
 *    rows (Lagrangian c'x - y'(Ax - b)).  z = c - A'y projected onto the
 *    cone allowed by the finite bounds (z_j >= 0 at a finite lower bound,
 *    <= 0 at a finite upper bound, 0 for a free column).
 */
#ifndef PDHGC_H
#define PDHGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (return values) ---------------------------------------- */
#define PDHGC_OK                 0
#define PDHGC_ERR_INVALID_ARG   -1  /* NULL handle/pointer, m or n < 1, bad flag, bad parameter value */
#define PDHGC_ERR_INVALID_CSR   -2  /* row_ptr not monotone / not 0-based / nnz mismatch, column out of range */
#define PDHGC_ERR_NONFINITE     -3  /* NaN or Inf in A, b or c; NaN in a bound; l = +inf or u = -inf */
#define PDHGC_ERR_BOUNDS        -4  /* l_j > u_j */
#define PDHGC_ERR_CUDA          -5  /* a CUDA runtime call failed (detail string has the CUDA error) */
#define PDHGC_ERR_OOM           -6  /* device or pinned-host allocation failed */
#define PDHGC_ERR_NO_PHASE1     -7  /* corner phase or PHASE1 report requested before pdhgc_solve */
#define PDHGC_ERR_NO_CORNER     -8  /* CORNER report / solution requested before pdhgc_corner_phase */
#define PDHGC_ERR_TOO_LARGE     -9  /* nnz >= 2^31 or a dimension >= 2^31, or n above the
                                       limit of a fixed-capacity entry point (pdhgc_kkt_eval_noalloc) */
#define PDHGC_ERR_DEVICE        -10 /* a device-side check failed (error word set by a kernel) */
#define PDHGC_ERR_BUFFER        -11 /* a caller buffer is too small (size written back) */
#define PDHGC_ERR_IO            -12 /* a file could not be opened, read or written, or is not in the expected format */

/* ---- solver outcome (pdhgc_report.status) -------------------------------- */
#define PDHGC_STATUS_NONE          0
#define PDHGC_STATUS_OPTIMAL       1  /* the three relative tolerances of Section 2 met */
#define PDHGC_STATUS_ITER_LIMIT    2
#define PDHGC_STATUS_TIME_LIMIT    3
#define PDHGC_STATUS_NUMERICAL     4  /* a non-finite KKT quantity appeared */
#define PDHGC_STATUS_CORNER_DONE   5  /* Section 3.1 stopping rule met */
#define PDHGC_STATUS_CORNER_LIMIT  6  /* corner phase hit a limit; the phase-1 x is returned */

/* ---- precision and which-solution selectors ------------------------------ */
#define PDHGC_FP64       0  /* matrix, iterates and SpMV accumulation in FP64 */
#define PDHGC_FP32_BULK  1  /* FP32 matrix and iterates in the iteration; FP64-class
                               (float-float) row sums and running sums; every KKT,
                               gap, restart, step-size and primal-weight quantity in FP64 */

#define PDHGC_PHASE1  0
#define PDHGC_CORNER  1
#define PDHGC_DUAL_CORNER 2  /* the dual corner push's result (pdhgc_dual_corner_phase) */

/* ---- inner loop (pdhgc_params.algorithm) ---------------------------------
 * PDHGC_ALG_AVERAGED: cuPDLP.jl-style restarted PDHG; restarts compare the
 *   omega-weighted KKT error of the current iterate and of the running
 *   average, and the better of the two is returned.
 * PDHGC_ALG_HALPERN: the form of cuPDLP+, which Section 4.1 says the paper's
 *   PDHG follows.  It runs anchored (Halpern) steps on the reflected PDHG
 *   operator and keeps no averages:
 *     z <- w_t ((1 + rho) T(z) - rho z) + (1 - w_t) z_0,  w_t = (t+1)/(t+2)
 *   z_0 is the last restart point.  Restarts test the fixed-point residual
 *   ||z - T(z)|| in the PDHG metric; the primal weight follows a PID rule on
 *   the anchor's movement; every check evaluates, and returns, the PDHG
 *   output T(z).  FP64 only. */
#define PDHGC_ALG_AVERAGED 0
#define PDHGC_ALG_HALPERN  1

/* Sense codes are ASCII: '=' (61), '<' (60), '>' (62). */

/*
 * Phase-1 parameters.  The paper fixes eps_rel (1e-6, Section 4.1); every
 * other value is the cuPDLP-family reading this library implements (the
 * paper prints no PDHG iteration).  pdhgc_default_params() fills defaults.
 */
typedef struct pdhgc_params {
    double  eps_rel;       /* relative tolerance of the Section 2 test (1e-6); < 0 never stops on it */
    int64_t max_iters;     /* iteration limit (>= 1), default 1,000,000 */
    double  time_limit_s;  /* device-clock time limit, checked at each check period (3600) */
    int32_t check_period;  /* iterations between KKT / restart checks (64, 1..4096) */
    double  beta_suff;     /* restart on sufficient decay of KKT_omega (0.2) */
    double  beta_nec;      /* restart on necessary decay without progress (0.8) */
    double  beta_art;      /* artificial restart when t >= beta_art * k (0.36) */
    double  theta;         /* primal-weight smoothing in log space (0.5) */
    double  eta_factor;    /* step eta = eta_factor / sigma_max(A_hat) (0.998) */
    int32_t ruiz_iters;    /* Ruiz infinity-norm passes (10, 0..100) */
    int32_t power_iters;   /* power iterations for sigma_max (100, 1..10000) */
    int32_t precision;     /* PDHGC_FP64 or PDHGC_FP32_BULK */
    int32_t algorithm;     /* PDHGC_ALG_AVERAGED (default) or PDHGC_ALG_HALPERN (FP64 or FP32 bulk) */
    /* the Halpern loop only: */
    double  reflection;    /* rho in [0, 1]; 1 (default): the reflected operator 2T - I */
    double  pid_kp, pid_ki, pid_kd; /* primal-weight PID gains in log space (0.99, 0.01, 0):
                              e = log(omega) - log(|y+ - y0| / |x+ - x0|) at a restart,
                              I += e, log(omega) -= kp e + ki I + kd (e - e_prev) */
} pdhgc_params;

/*
 * Corner-phase parameters (Algorithm 1 and Section 3.1).
 */
typedef struct pdhgc_corner_params {
    double   eps_abs;      /* reduced-cost threshold of Algorithm 1 (1e-6) */
    double   eps_rel;      /* primal tolerance to regain, Section 3.1 (1e-6) */
    int64_t  min_iters;    /* at least this many corner iterations (100) */
    int64_t  max_iters;    /* corner iteration limit (1,000,000) */
    double   time_limit_s; /* device-clock limit (3600) */
    uint64_t obj_seed;     /* seed of the Uniform([0,1]^n) objective (SplitMix64 stream) */
    double   obj_scale;    /* objective = obj_scale * U[0,1) (1.0; Section 5 studies small scales) */
    int32_t  stop_rule;    /* 0: Section 3.1 primal rule; 1: full relative KKT (a testing aid) */
    int32_t  row_rule;     /* 0 (default): Section 3's rule, an inequality row whose dual is non-trivial
                              (|y_i| > eps_abs) becomes '='; 1 (an option, not the paper's): only when the
                              row also looks active at the phase-1 point, its slack (a_i x - b_i in the '>'
                              form) no larger than |y_i|, so that rows the phase-1 point is clearly off
                              keep their sense */
    int32_t  omega_rule;   /* starting primal weight: 0 (default) ||c_hat'|| / ||b_hat|| of the corner
                              model, as at a phase start; PDHG with omega proportional to ||c|| is
                              scale-equivariant, so obj_scale then changes nothing beyond rounding (and,
                              in the averaged loop, the gap term of its restart test).  1: phase 1's final
                              primal weight, so that obj_scale rescales the dual's share of the
                              iteration, the setting of Section 5's objective-scale study */
    int32_t  reserved;
} pdhgc_corner_params;

/*
 * Result of a phase or a report.  Norms are of the user's (unscaled) model.
 * Metrics follow Section 2.1 and Section 4.2 with tolerance 1e-6, counting
 * one explicit slack per inequality row:
 *   off_bound_p    variables (and inequality slacks) more than 1e-6 from both bounds
 *   zero_rc_d      variables with |z_j| <= 1e-6 plus inequality rows with |y_i| <= 1e-6
 *   candidates     variables (and slacks) off bound with |reduced cost| <= 1e-6
 *   corner_measure max(0, candidates - m)
 *   primal_push_est max(0, p - m);  dual_push_est max(0, m - d)
 *   should_corner  candidates >= max(2m, 100000)
 */
typedef struct pdhgc_report {
    int32_t status;        /* PDHGC_STATUS_* */
    int32_t chosen;        /* 0: current iterate returned, 1: average returned,
                              2: the PDHG output T(z) of the last check (Halpern loop) */
    int64_t iters;         /* PDHG iterations of the phase */
    int64_t restarts;
    double  rP2, rD2;      /* ||r_P||_2, ||r_D||_2 */
    double  rPinf, rDinf;  /* infinity norms */
    double  pobj, dobj;    /* c'x and b'y + sum l_j z_j^+ - sum u_j z_j^- */
    double  gap;           /* pobj - dobj */
    double  rel_p, rel_d, rel_gap, rel_kkt; /* Section 2 ratios; rel_kkt = their max */
    int64_t off_bound_p, zero_rc_d, candidates, corner_measure;
    int64_t primal_push_est, dual_push_est;
    int32_t should_corner;
    int32_t precision;
    double  seconds;       /* device-clock seconds of the phase (0 for a report) */
    double  omega, eta, sigma_max; /* primal weight at exit, step size, norm estimate */
} pdhgc_report;

typedef struct pdhgc_lp pdhgc_lp;   /* opaque; owns all of its device memory */

void pdhgc_default_params(pdhgc_params* p);
void pdhgc_default_corner_params(pdhgc_corner_params* p);

/*
 * pdhgc_lp_create — the problem data of Section 2 (A m x n in CSR, b, c,
 * bounds and row senses).  Validates, copies and lays out the data on the
 * device: rows and columns are renumbered internally by decreasing nnz so
 * that rows of similar length share a warp, an explicit CSR of A' is built,
 * and row tiles for the SpMV kernels are planned.  The caller keeps
 * ownership of every input; the handle owns the device copies.
 *   row_ptr  int64[m+1], 0-based, non-decreasing, row_ptr[m] = nnz
 *   col_idx  int32[nnz] in [0, n); val FP64[nnz], finite
 *   b FP64[m], c FP64[n] finite
 *   lb, ub   FP64[n] or NULL (NULL: l = 0, u = +inf); +-inf allowed
 *   sense    int8[m] of '=', '<', '>' or NULL (all '=')
 *   inputs_on_device  1: the six array arguments are device pointers
 *   cuda_stream       cudaStream_t (as void*) used by every later call
 * Errors: INVALID_ARG, INVALID_CSR, NONFINITE, BOUNDS, TOO_LARGE, CUDA, OOM.
 * The scaling and step size are computed by pdhgc_solve (they are part of
 * the timed solve); create only uploads and lays out the data.
 */
int pdhgc_lp_create(pdhgc_lp** out, int32_t m, int32_t n, int64_t nnz,
                    const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                    const double* b, const double* c, const double* lb, const double* ub,
                    const int8_t* sense, int inputs_on_device, void* cuda_stream);

/*
 * pdhgc_solve — phase 1: scale (Ruiz + Pock-Chambolle), estimate
 * sigma_max(A_hat), then run restarted PDHG on the device until the
 * Section 2 relative test holds with eps_rel (Section 4.1: 1e-6) at a
 * check, or a limit.  The whole loop (iterations, checks, restarts,
 * termination) runs as one CUDA graph with a device-side while condition;
 * no host round trip per iteration.  `out` may be NULL.  Re-solving
 * discards any previous phase-1 and corner result of the handle.
 */
int pdhgc_solve(pdhgc_lp* lp, const pdhgc_params* params, pdhgc_report* out);

/*
 * pdhgc_corner_phase — Algorithm 1 applied to the phase-1 result:
 * ub_j <- x_j where z_j > eps_abs, lb_j <- x_j where z_j < -eps_abs,
 * inequality rows with |y_i| > eps_abs become '=' (Section 3), objective
 * obj_scale * Uniform([0,1]^n) from SplitMix64(obj_seed), PDHG restarted
 * from (x, 0) with the phase-1 step size, stopped by the Section 3.1 rule
 * (k >= min_iters and ||r_P||_2 <= eps_rel (1 + ||b||_2), at a check).
 * Returns (x_hat, y, z) with the phase-1 y and z.  The report's KKT numbers
 * and metrics are those of (x_hat, y, z) on the ORIGINAL model.
 * Errors: NO_PHASE1 before pdhgc_solve.
 */
int pdhgc_corner_phase(pdhgc_lp* lp, const pdhgc_corner_params* params, pdhgc_report* out);

/*
 * pdhgc_kkt_report — residuals, objectives, Section 2 ratios and the
 * Section 2.1 / 4.2 metrics of the PHASE1, CORNER or DUAL_CORNER solution
 * on the original model, computed on the device.  Errors: INVALID_ARG,
 * NO_PHASE1, NO_CORNER (that phase has not run since the last pdhgc_solve).
 */
int pdhgc_kkt_report(pdhgc_lp* lp, int which, pdhgc_report* out);

/*
 * pdhgc_get_solution — x (n), y (m), z (n) of the PHASE1, CORNER or
 * DUAL_CORNER solution in the user's order and scale (CORNER: the corner x
 * with phase 1's y and z; DUAL_CORNER: phase 1's x with the dual corner
 * phase's y and its z).  Any of the three may be NULL.  Errors as
 * pdhgc_kkt_report.
 */
int pdhgc_get_solution(pdhgc_lp* lp, int which, double* x, double* y, double* z, int on_device);

/*
 * pdhgc_get_iterates — the solver's state in scaled space, user order:
 * current x_hat (n), y_hat (m) and the running averages of the iterates
 * since the last restart (zeros when no iteration ran since it).  After a
 * Halpern-loop phase, x_avg / y_avg receive instead the PDHG output T(z) of
 * the last check step, the point the phase returns.  Any pointer may be
 * NULL.  iters_out (may be NULL) receives {k, t, restarts}.  For parity
 * tests against a reference implementation.
 */
int pdhgc_get_iterates(pdhgc_lp* lp, double* x, double* y, double* x_avg, double* y_avg,
                       int64_t* iters_out, int on_device);

/*
 * pdhgc_get_scaling — D_r (m), D_c (n) in user order and the scalars
 * {sigma_max, eta, omega, tau, sigma} (5 doubles).  Any pointer may be NULL.
 */
int pdhgc_get_scaling(pdhgc_lp* lp, double* d_row, double* d_col, double* scalars, int on_device);

/*
 * pdhgc_get_layout — how the matrix passes split the rows of A (out[0..3])
 * and of A' (out[4..7]) over the SpMV's row segments, as planned at
 * lp_create: the number of blocks that each own one row longer than 4096
 * nonzeros (one CTA per row), of blocks of warp-per-row rows (257..4096
 * nonzeros), of SELL-32 blocks (rows of at most 256 nonzeros), and the
 * number of rows in the CTA segment.  `out` is a host array of 8 int64.
 * (The Halpern loop's primal pass can instead run a chunked layout; see
 * pdhgc_set_primal_layout.)
 * A layout query (the paper has no counterpart; the segments implement the
 * CSR passes of the Section 2 iteration).  Errors: INVALID_ARG.
 */
int pdhgc_get_layout(const pdhgc_lp* lp, int64_t* out);

/*
 * pdhgc_set_primal_layout — how the Halpern loop runs its primal pass
 * x+ = proj(x - tau (c - A'y)) (the Section 2 iteration's A' product):
 * chunked = 0 (the default) uses the row segments of pdhgc_get_layout with
 * gathers from global memory; chunked = 1 stages the gathered vector y in
 * shared memory, 200 KB at a time, with one CTA per SM whose warps gather
 * from shared memory (the layout is planned by the first call that selects
 * it, from A' as laid out on the device: work units of one long column or
 * 32 short ones, their entries grouped by chunk).  On the
 * 100k x 400k LP the chunked pass measured 2-2.5 times slower (each warp
 * runs its units' short per-chunk segments one after another), so it is
 * not the default.  The results differ only by the summation order of the
 * row sums.  Takes effect at the next pdhgc_solve or pdhgc_corner_phase.  A
 * layout choice for measurement and tests (the paper has no counterpart).
 * Errors: INVALID_ARG; on the first selection also CUDA, OOM.
 */
int pdhgc_set_primal_layout(pdhgc_lp* lp, int32_t chunked);

/*
 * pdhgc_set_launch_mode — how pdhgc_solve, pdhgc_corner_phase and the dual
 * corner push drive their restarted loop (Section 2's iteration with a check
 * every check_period steps):
 *   PDHGC_LAUNCH_GRAPH (0, the default): one CUDA graph per phase whose
 *     conditional WHILE node repeats the body (check_period iterations, the
 *     check, the decision, the restart) until the device decision sets the
 *     phase's done flag: no host round trip inside the loop;
 *   PDHGC_LAUNCH_STREAM (1): the same kernels, enqueued as plain launches on
 *     the handle's stream, one body at a time; the host reads the done flag
 *     back after each body.  Every kernel is then a separate launch that a
 *     profiler's launch list shows (kernel nodes inside a conditional graph
 *     body are not listed separately).
 * Both modes make the same decisions and give bitwise-equal results.  Takes
 * effect at the next call.  A launch choice (the paper has no counterpart).
 * Errors: INVALID_ARG.
 */
#define PDHGC_LAUNCH_GRAPH  0
#define PDHGC_LAUNCH_STREAM 1
int pdhgc_set_launch_mode(pdhgc_lp* lp, int32_t mode);

/*
 * pdhgc_kkt_eval — the Section 2 residuals, objectives and relative ratios,
 * and the Section 2.1 / 4.2 metrics, of a caller-supplied point (x, y) on an
 * LP given as device arrays, without creating a handle.  The LP arguments
 * mean what they mean for pdhgc_lp_create (row_ptr int64[m+1], col_idx
 * int32[nnz], val, b, c; lb, ub, sense may be NULL for their defaults); x
 * (n) and y (m) are in the user's scale with the dual signs of this header
 * (y <= 0 on '<' rows, y >= 0 on '>' rows); every pointer is a device
 * pointer.  z = proj(c - A'y).  Fills the numeric fields of *out (host);
 * status, iters and the phase fields are zero.  Work is enqueued on
 * `cuda_stream`, which the call synchronises.  The inputs are not
 * validated beyond NULL and size checks (use pdhgc_lp_create for that).
 * Scratch (n + 13 * 1024 + 16 doubles) is taken with cudaMallocAsync on
 * the stream and released before returning.  A'y is accumulated with
 * atomic adds, so results may differ from run to run in the last bits.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int pdhgc_kkt_eval(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* val, const double* b, const double* c, const double* lb, const double* ub,
                   const int8_t* sense, const double* x, const double* y, pdhgc_report* out,
                   void* cuda_stream);

/*
 * pdhgc_kkt_eval_noalloc — pdhgc_kkt_eval for callers that cannot allocate
 * device memory: services that run under a fixed device-memory budget,
 * applications whose device memory is owned by a pool or framework allocator
 * that must account for every byte, and code paths where the implicit
 * synchronisation of cudaMalloc / cudaFree is not acceptable.  (The paper
 * has no counterpart; this is a library convenience.)  Same arguments and
 * results as pdhgc_kkt_eval.  Errors: INVALID_ARG (as pdhgc_kkt_eval),
 * TOO_LARGE (below), CUDA; never OOM.  Further:
 *  - n must be <= 262,144 (1 << 18); a larger n returns PDHGC_ERR_TOO_LARGE
 *    without touching the device.
 *  - The scratch is a file-scope device array of 2,203,776 bytes ((1 << 18)
 *    + 13 * 1024 + 16 doubles) that every GPU which loads the library holds
 *    until the process exits.  The call itself allocates nothing and calls
 *    no cudaMalloc, cudaFree or allocating library routine.
 *  - The first call on a device (the current device of the calling thread)
 *    looks up that array's device address with cudaGetSymbolAddress; make
 *    that first call before any stream capture begins.  Later calls check
 *    with cudaPointerGetAttributes that the address still belongs to the
 *    device's current context (after cudaDeviceReset it does not) and look
 *    it up again when it does not.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents; every call clears the part that must start at zero.  Calls
 *    that overlap on the GPU (different streams, or different host threads
 *    without ordering) race on the array and give wrong results: serialise
 *    them on one stream.
 */
int pdhgc_kkt_eval_noalloc(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                           const double* val, const double* b, const double* c, const double* lb,
                           const double* ub, const int8_t* sense, const double* x, const double* y,
                           pdhgc_report* out, void* cuda_stream);

/*
 * pdhgc_uniform — out[j] = obj_scale * U_j for j < n, where U_j is the top 53
 * bits of the (j+1)-th SplitMix64 output from state `seed`, times 2^-53
 * (the corner objective of Algorithm 1).  `out` is a device pointer; the
 * work is enqueued on `cuda_stream` and the call synchronises it.
 */
int pdhgc_uniform(uint64_t seed, int64_t n, double obj_scale, double* out, void* cuda_stream);

/* ---- batched solve: many independent LPs in one persistent launch ------- */

/*
 * pdhgc_dual_corner_phase — the dual corner push: the dual counterpart of
 * Algorithm 1 that Section 6 (Discussion) proposes for the dual superbasics
 * (the paper gives no construction; this is the reading).  From the phase-1
 * point (x1, y1, z1), complementary slackness decides, in user space: of a
 * pair (the distance of x_j from a bound, the part of z_j that bound
 * allows) or (an inequality row's slack, |y_i|) the first is read as
 * nonzero when it exceeds both eps_abs and the second;
 *   - a bound is removed where x1 is off it in that sense, so a column
 *     strictly inside its bounds becomes free, which fixes its reduced cost
 *     at 0 (the counterpart of fixing x_j where z_j != 0);
 *   - an inequality row whose slack is nonzero in that sense has its dual
 *     fixed at 0 (an inactive row);
 *   - the dual objective becomes b' = obj_scale U[0,1)^m (SplitMix64 of
 *     obj_seed per user row, negated on '<' rows, scaled like b); c stays.
 * PDHG then runs from (proj(0), y1) in the phase-1 inner loop and precision,
 * with omega_0 = ||c_hat|| / ||b_hat'||, and stops at a check once k >=
 * min_iters and the dual residual of the model meets eps_rel (1 + ||c||)
 * (stop_rule 0, the counterpart of Section 3.1's primal rule) or the full
 * Section 2 test holds (stop_rule 1); on a limit y1 is kept
 * (PDHGC_STATUS_CORNER_LIMIT).  The result is (x1, y, z): phase 1's x with
 * the new dual, read with which = PDHGC_DUAL_CORNER.  On the optimal face a
 * converged run ends at a vertex of the dual optimal face (at least m zero
 * reduced costs, dual push estimate 0); the 1e-6 count of zero reduced costs
 * registers it only once the phase has converged beyond 1e-6 (eps_rel, e.g.
 * 1e-9, with stop_rule 1).  Uses corner params eps_abs, eps_rel, min_iters,
 * max_iters, time_limit_s, obj_seed, obj_scale, stop_rule; row_rule and
 * omega_rule must be 0.  Errors: NO_PHASE1, INVALID_ARG, CUDA, OOM.
 */
int pdhgc_dual_corner_phase(pdhgc_lp* lp, const pdhgc_corner_params* params, pdhgc_report* out);

/*
 * pdhgc_batch_create — `count` LPs, each as for pdhgc_lp_create, given by
 * host arrays of per-LP pointers (row_ptr[k], col_idx[k], ... are the k-th
 * LP's arrays; lb, ub and sense may be NULL as a whole or per LP).  Every LP
 * is validated and laid out as in pdhgc_lp_create and packed into one set of
 * device arrays.  nnz summed over the batch must be < 2^31.  The batch owns
 * its device memory; all work goes on `cuda_stream`.
 * Errors: as pdhgc_lp_create (the detail names the offending LP).
 */
typedef struct pdhgc_batch pdhgc_batch;
int pdhgc_batch_create(pdhgc_batch** out, int32_t count, const int32_t* m, const int32_t* n, const int64_t* nnz,
                       const int64_t* const* row_ptr, const int32_t* const* col_idx, const double* const* val,
                       const double* const* b, const double* const* c, const double* const* lb,
                       const double* const* ub, const int8_t* const* sense, void* cuda_stream);

/*
 * pdhgc_batch_solve — phase 1 (as pdhgc_solve, same parameters) for every
 * LP of the batch in one persistent kernel launch, captured with the reset of
 * its work queue in a CUDA graph that is launched on the batch's stream (one
 * graph launch per call): each CTA takes LPs from
 * a work queue, largest first, and runs the whole method on one LP (scaling,
 * power iteration, the restarted PDHG loop with its per-LP step size, primal
 * weight, restarts and termination, then the report); an LP's x_bar and y
 * live in the CTA's shared memory.  `reports` (count entries, may be NULL)
 * receives one report per LP in the caller's order; `seconds` is that LP's
 * device time.  Both precisions and both inner loops are supported.
 * Errors: INVALID_ARG (a parameter out of range), CUDA, OOM, and those of
 * the single-LP path for a handed-off LP.
 */
int pdhgc_batch_solve(pdhgc_batch* batch, const pdhgc_params* params, pdhgc_report* reports);

/* pdhgc_batch_corner_phase — Algorithm 1 for every LP (as pdhgc_corner_phase;
 * omega_rule 0 only, INVALID_ARG otherwise). */
int pdhgc_batch_corner_phase(pdhgc_batch* batch, const pdhgc_corner_params* params, pdhgc_report* reports);

/*
 * pdhgc_batch_solve_corner — phase 1 and Algorithm 1 (Section 3, with the
 * Section 3.1 stopping rule) for every LP in ONE persistent launch: the CTA
 * that finishes an LP's phase 1 goes straight on to that LP's corner phase,
 * so no batch-wide barrier separates the two phases (the results and reports
 * are those of pdhgc_batch_solve followed by pdhgc_batch_corner_phase with
 * the same parameters).  reports1 / reports_c (count entries each, either
 * may be NULL) receive the phase-1 and corner reports in the caller's order.
 * An LP handed off in phase 1 runs both phases on the single-LP path; one
 * handed off in its corner phase runs phase 1 and the corner phase there and
 * keeps the corner result.  Errors: as pdhgc_batch_solve and
 * pdhgc_batch_corner_phase.
 */
int pdhgc_batch_solve_corner(pdhgc_batch* batch, const pdhgc_params* params, const pdhgc_corner_params* cparams,
                             pdhgc_report* reports1, pdhgc_report* reports_c);

/* pdhgc_batch_get_solution — x (n) and y (m) of LP `lp`, user order, host pointers (either may be NULL). */
int pdhgc_batch_get_solution(pdhgc_batch* batch, int32_t lp, int which, double* x, double* y);

/*
 * Schedule knobs of the batched kernel, set by the autotuner: threads per
 * CTA (512 or 1024) and lanes per row of the A and A' passes (1..32, a power
 * of two; 0 = chosen per LP from its mean row length).
 */
int pdhgc_batch_set_block(pdhgc_batch* batch, int32_t threads);
int pdhgc_batch_set_lanes(pdhgc_batch* batch, int32_t lanes_a, int32_t lanes_t);
/* layout of the matrix passes: 1 = SELL-32 slices (lane per row), 0 = CSR rows with the lanes above */
int pdhgc_batch_set_layout(pdhgc_batch* batch, int32_t sell);

/*
 * pdhgc_batch_tune — the schedule autotuner.  For each candidate schedule
 * (threads per CTA x layout x lanes per row; 7 candidates) it times
 * `tune_iters` iterations of the whole batch (setup included, no early
 * termination, so every candidate does the same work) with CUDA events on
 * the batch's stream, and keeps the fastest.  chosen (4 ints, may be NULL)
 * receives {threads, sell, lanes_a, lanes_t}; timings_ms (7 doubles, may be
 * NULL) the candidates' times.  Discards any phase-1 / corner result.
 */
int pdhgc_batch_tune(pdhgc_batch* batch, const pdhgc_params* params, int32_t tune_iters, int32_t* chosen,
                     double* timings_ms);

/*
 * pdhgc_batch_set_handoff — the tail handoff.  Once every LP of the queue has
 * been taken and at most `max_running` LPs are still running, an LP that has
 * done at least `min_iters` iterations of the current phase stops at its next
 * check, and the batch finishes it on the single-LP path (the graph-driven
 * whole-GPU loop of pdhgc_solve / pdhgc_corner_phase), several such LPs
 * concurrently on their own streams, each started as soon as the host sees
 * its handoff status while the batched kernel still runs.  A handed-off LP
 * restarts its phase from the phase's start point on that path; a corner
 * phase handed off there starts from that path's own phase 1 of the LP.  Its
 * report and result are the single-LP path's.  Defaults: 8, 8192 (measured
 * on 512 LPs: 9.3-9.9 s per step at 8; 8.6 s at 16 alone but 14.2 s at 16
 * while another process polled the GPU through NVML; 23 s at 32; 17 s with
 * no handoff); max_running = 0 disables.
 */
int pdhgc_batch_set_handoff(pdhgc_batch* batch, int32_t max_running, int64_t min_iters);

/* pdhgc_batch_handed_off — 1 when LP `lp`'s result of phase `which` came from the single-LP path. */
int32_t pdhgc_batch_handed_off(const pdhgc_batch* batch, int32_t lp, int which);

/* pdhgc_batch_kernel_launches — kernels launched so far: one persistent kernel per graph launch, plus the
 * single-LP kernels of handed-off LPs. */
int64_t pdhgc_batch_kernel_launches(const pdhgc_batch* batch);

void pdhgc_batch_destroy(pdhgc_batch* batch);

/* ---- learned corner guidance (an extension of Algorithm 1; the paper has none) ----
 *
 * A per-column network predicts which columns the corner phase may hold at a
 * bound.  Network: 18 features -> 64 -> 64 -> 1, ReLU hidden layers, sigmoid
 * output read as P(column ends at a bound after the corner phase); BF16
 * weights and activations, FP32 accumulation (tensor cores), trained on the
 * mean binary cross-entropy with Adam (Kingma & Ba 2015: beta1 0.9, beta2
 * 0.999, eps 1e-8).
 *
 * Features of column j (PDHGC_GUIDE_FEATURES = 18), from a phase-1 result and
 * the corner parameters (the objective seed):
 *   [0]      c'_j: Algorithm 1's random objective, scaled like c (the
 *            objective of the LP the corner phase solves);
 *   [1]      ||A_hat_j||_2, the column norm of the scaled matrix;
 *   [2..9]   x_hat_j at the last 8 restart points of phase 1, newest first
 *            (the start point counts as the first; padded with the oldest);
 *   [10..17] z_hat_j = proj(c_hat - A_hat' y_hat)_j at the same points;
 * each of the four groups divided by its root mean square over all columns.
 * Stored as BF16 rows of PDHGC_GUIDE_FEAT_STRIDE (32) values, 64 bytes, the
 * entries 18..31 zero; row-major, 16-byte aligned, in user column order.
 *
 * A column is eligible for holding when Algorithm 1's reduced-cost rule did
 * not fix it and it has a finite bound; a held column gets l_hat = u_hat =
 * the bound of [l_hat, u_hat] nearest to its phase-1 value (ties: lower),
 * and the corner phase starts there.
 *
 * Parameter vector (PDHGC_GUIDE_PARAMS = 5441 FP32): W1 [64][18], b1 [64],
 * W2 [64][64], b2 [64], w3 [64], b3 — row-major, unit-major rows.
 */
#define PDHGC_GUIDE_FEATURES    18
#define PDHGC_GUIDE_FEAT_STRIDE 32
#define PDHGC_GUIDE_PARAMS      5441
#define PDHGC_STATUS_GUIDE_FALLBACK 7  /* pdhgc_guide_report.status: the plain corner result was returned */

typedef struct pdhgc_guide pdhgc_guide;

typedef struct {
    double threshold;          /* hold an eligible column when its probability >= threshold (0.9) */
    int64_t guided_max_iters;  /* iteration limit of the guided run; 0 (default) = the corner limit */
    int32_t fallback;          /* 1 (default): run the plain corner phase when the guided one regresses */
    int32_t reserved;
} pdhgc_guide_params;

typedef struct {
    int32_t status;                 /* guided run's status; PDHGC_STATUS_GUIDE_FALLBACK when replaced */
    int32_t fell_back;              /* 1 when the plain corner phase's result was returned */
    int64_t eligible, held;         /* eligible columns; columns held at a bound */
    int64_t guided_iters;           /* iterations of the guided corner run */
    double guided_seconds;          /* device time of the guided run (features and inference included) */
    double guided_rel_kkt;          /* its relative KKT error on the original model */
    int64_t guided_corner_measure;  /* its corner measure */
    double infer_seconds;           /* features + network inference */
} pdhgc_guide_report;

/* pdhgc_default_guide_params — threshold 0.9, guided_max_iters 0, fallback 1. */
void pdhgc_default_guide_params(pdhgc_guide_params* p);

/*
 * pdhgc_guide_create — a network with He-uniform initial weights drawn from
 * SplitMix64(seed) (biases 0); device memory on the current device, work on
 * `cuda_stream`.  Errors: INVALID_ARG, CUDA, OOM.
 */
int pdhgc_guide_create(pdhgc_guide** out, uint64_t seed, void* cuda_stream);
void pdhgc_guide_destroy(pdhgc_guide* g);

/* set (resets Adam's moments) / read the FP32 parameter vector; host arrays of PDHGC_GUIDE_PARAMS.
 * Errors: INVALID_ARG, NONFINITE (set). */
int pdhgc_guide_set_weights(pdhgc_guide* g, const float* w);
int pdhgc_guide_get_weights(pdhgc_guide* g, float* w);

/*
 * pdhgc_guide_save / pdhgc_guide_load — the network's FP32 parameter vector
 * in a file: the 8 bytes "PDHGCGW1", PDHGC_GUIDE_PARAMS as a little-endian
 * int32, a zero int32, the parameters as little-endian IEEE FP32 in the
 * parameter-vector layout, then the 64-bit FNV-1a hash of those parameter
 * bytes (little-endian).  load checks the header, size and hash, rejects
 * non-finite weights, and resets Adam's moments as set_weights does.
 * Errors: INVALID_ARG (NULL), IO (open / read / write failure, wrong header,
 * size or hash), NONFINITE (load), CUDA.
 */
int pdhgc_guide_save(pdhgc_guide* g, const char* path);
int pdhgc_guide_load(pdhgc_guide* g, const char* path);

/*
 * pdhgc_guide_infer — probabilities p[r] for `rows` feature rows; feat and p
 * are DEVICE pointers (feat: rows x 32 BF16, 16-byte aligned; p: rows FP32).
 * Errors: INVALID_ARG (NULL, rows < 1, misaligned), CUDA.
 */
int pdhgc_guide_infer(pdhgc_guide* g, const uint16_t* feat, int64_t rows, float* p);

/*
 * pdhgc_guide_grad — gradient of the mean binary cross-entropy over the
 * minibatch idx[0..batch-1] (HOST int32 indices into the rows of the DEVICE
 * arrays feat and labels (uint8 0/1)), without updating the weights; grad
 * (host, PDHGC_GUIDE_PARAMS floats) in the parameter-vector layout; loss
 * (host, may be NULL).  Errors: INVALID_ARG (index out of range), CUDA, OOM.
 */
int pdhgc_guide_grad(pdhgc_guide* g, const uint16_t* feat, const uint8_t* labels, int64_t rows,
                     const int32_t* idx, int32_t batch, float* grad, float* loss);

/*
 * pdhgc_guide_train — `steps` Adam steps at learning rate lr on minibatches
 * of `batch` rows drawn with replacement: row SplitMix64(seed, step * batch
 * + s) mod rows for s < batch.  feat and labels are DEVICE arrays as above;
 * losses (host, `steps` floats, may be NULL) receives each step's minibatch
 * loss.  Errors: INVALID_ARG, CUDA, OOM.
 */
int pdhgc_guide_train(pdhgc_guide* g, const uint16_t* feat, const uint8_t* labels, int64_t rows, int32_t batch,
                      int64_t steps, float lr, uint64_t seed, float* losses);

/*
 * pdhgc_guide_features — the feature rows of every column of the handle's
 * phase-1 result for the corner objective of `params` (NULL = defaults):
 * feat (DEVICE, n rows, layout above), eligible (DEVICE uint8 n, may be
 * NULL).  Rebuilds the corner model's bounds and objective (the next corner
 * phase rebuilds them again); the phase-1 and corner results are untouched.
 * Errors: NO_PHASE1, INVALID_ARG, CUDA, OOM.
 */
int pdhgc_guide_features(pdhgc_lp* lp, const pdhgc_corner_params* params, uint16_t* feat, uint8_t* eligible);

/*
 * pdhgc_guide_dataset_append — training rows from the last corner phase:
 * for every eligible column (in user column order) its feature row (for the
 * corner objective that phase used) and its label (1 when the returned
 * corner x_j lies within 1e-6, in user space, of the bound a hold would use:
 * the one nearest to its phase-1 value; on a CORNER_LIMIT status the corner
 * point is the phase-1 x).  Rows are appended to the
 * DEVICE arrays feat / labels at row *count, which is advanced.  Errors:
 * NO_PHASE1, NO_CORNER, BUFFER (capacity - *count too small; *count is left
 * unchanged and nothing is written), INVALID_ARG, CUDA, OOM.
 */
int pdhgc_guide_dataset_append(pdhgc_lp* lp, uint16_t* feat, uint8_t* labels, int64_t capacity, int64_t* count);

/*
 * pdhgc_corner_phase_guided — Algorithm 1 with held columns.  The hold set
 * comes from the network g (eligible columns with probability >=
 * gparams->threshold) or, when g is NULL, from `hold` (uint8 per user
 * column, host or device per hold_on_device; non-eligible entries ignored).
 * Exactly one of g and hold must be given.  With gparams->fallback = 1, a
 * guided result that hit a limit, has a relative KKT error above
 * max(phase-1 rel_kkt, params->eps_rel), or a corner measure above the
 * phase-1 point's is replaced by the plain corner phase's (out then holds
 * the plain run's report and gout->status = PDHGC_STATUS_GUIDE_FALLBACK).
 * out / gout may be NULL.  Errors: as pdhgc_corner_phase, INVALID_ARG.
 */
int pdhgc_corner_phase_guided(pdhgc_lp* lp, const pdhgc_corner_params* params, const pdhgc_guide_params* gparams,
                              pdhgc_guide* g, const uint8_t* hold, int hold_on_device, pdhgc_report* out,
                              pdhgc_guide_report* gout);

/*
 * pdhgc_guide_set_wait_limit — polls each tensor-core completion wait of the
 * inference kernel makes before it gives up (default 2^24; 0: give up at
 * once).  A wait that gives up makes the call return DEVICE; the kernel
 * still lets the pending product land (full limit) and frees its tensor
 * memory, so the context stays usable.  For failure-path tests.
 */
int pdhgc_guide_set_wait_limit(pdhgc_guide* g, int64_t polls);

/* pdhgc_guide_kernel_launches — CUDA kernels launched by this network so far. */
int64_t pdhgc_guide_kernel_launches(const pdhgc_guide* g);

/*
 * pdhgc_get_state / pdhgc_set_state — checkpoint and restore of a handle's
 * results (the paper has no counterpart; a service needs it to resume).  The
 * state is a host byte buffer holding the parameters, the phase-1 and corner
 * reports, the scaling factors, the phase-1 point (x1, y1), the corner x and
 * the phase-1 restart history.  get_state with buf = NULL writes the size to
 * *bytes; with a buffer smaller than that it returns BUFFER (size written
 * back).  set_state restores into a handle created from the same LP: it
 * recomputes the scaling and step size (deterministic) and returns INVALID_ARG
 * when the shape, the format or the recomputed scaling factors differ from the
 * saved ones.  Afterwards get_solution, kkt_report, corner_phase and the
 * guidance calls behave as on the original handle.  The state is not portable
 * across builds that change the scaling arithmetic.
 */
int pdhgc_get_state(pdhgc_lp* lp, void* buf, size_t* bytes);
int pdhgc_set_state(pdhgc_lp* lp, const void* buf, size_t bytes);

/*
 * pdhgc_kernel_launches — number of CUDA kernels this handle has launched
 * so far (kernels inside the solve graph counted once per execution).
 */
int64_t pdhgc_kernel_launches(const pdhgc_lp* lp);

/*
 * pdhgc_probe_gather — the random-gather ceiling the SpMV passes run against
 * (a measurement utility; the paper has no counterpart).  Times `reps`
 * launches of a kernel that makes 16 * `count` loads of elem_bytes (4 or 8)
 * at hashed uniform positions of a device vector of n_vec elements (resident
 * in L2 after a warm launch), 8 independent loads in flight per thread, and
 * writes the mean milliseconds per `count` loads (a launch's time / 16: the
 * steady-state rate, without the launch latency and the grid's tail that a
 * launch of only `count` loads would include).  Allocates and frees the
 * vector.
 * Errors: INVALID_ARG, CUDA, OOM.
 */
int pdhgc_probe_gather(int64_t n_vec, int64_t count, int32_t elem_bytes, int32_t reps, double* ms_out,
                       void* cuda_stream);

/*
 * pdhgc_profile_iteration — replays `iters` PDHG iterations of the last
 * phase's model as plain launches on the handle's stream, each kernel
 * bracketed by CUDA events, and writes the mean duration in milliseconds of
 * one launch of the primal step (the A' pass, ms_out[0]) and of the dual
 * step (the A pass, ms_out[1]).  After a Halpern-loop phase the replayed
 * kernels are that loop's (a step inside a chunk, not a check step).  The
 * replayed iterations are real: they
 * advance the iterate state, which is left inconsistent with the phase's
 * report (x1/y1 and the corner result are not touched).  For profiling.
 * Errors: NO_PHASE1, INVALID_ARG (iters < 1 or ms_out NULL).
 */
int pdhgc_profile_iteration(pdhgc_lp* lp, int32_t iters, double* ms_out);

void pdhgc_lp_destroy(pdhgc_lp* lp);
const char* pdhgc_strerror(int code);
const char* pdhgc_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* PDHGC_H */
