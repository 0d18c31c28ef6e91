/*
 * fgadmm.h -- C-ABI of the GB300 factor-graph ADMM library (libfgadmm.so).
 *
 * The library runs Algorithm 2 of "Testing fine-grained parallelism for the
 * ADMM on a factor-graph" (Hao et al., Sec. II): on a factor graph
 * G = (F, V, E) with per-edge messages x, m, u, n, weights rho, alpha and
 * per-variable z, one iteration is
 *     x_(a,da) = Prox_{f_a,rho}(n_(a,da))    for every factor a
 *     m = x + u                              for every edge
 *     z_b = sum rho m / sum rho              for every variable b
 *     u = u + alpha (x - z_b)                for every edge
 *     n = z_b - u                            for every edge
 * with Prox_{h,rho}(r) = argmin_s h(s) + rho/2 |s - r|^2 (Eq. PO).
 *
 * The call sequence follows the paper's usage description (Sec. III):
 * build the graph factor by factor (the paper's addNode; here factors are
 * registered by type and in batches), copy it to the GPU
 * (CopyGraphFromCPUtoGPU; here fga_finalize), run the update loop
 * (fga_iterate) and read the solution from z (Sec. II, last paragraph).
 *
 * Conventions for every function:
 *   - The return value is a status code (FGA_OK or a negative FGA_E*).
 *     On failure a thread-local message is available from fga_last_error().
 *     Out-parameters are written only on FGA_OK.
 *   - Every host input array is copied before the call returns; the caller
 *     keeps ownership.  Output arrays are caller-allocated.  Where a
 *     function says "host or device", the pointer may be either (the
 *     library asks the CUDA runtime which it is).
 *   - A graph object is not thread-safe; calls on one graph must not run
 *     concurrently.  Different graphs are independent.
 *   - Vector variables are expanded into scalar components.  A "scalar
 *     edge" is one component of one (factor, variable) edge; scalar edges
 *     are numbered in creation order: factor by factor in call order, each
 *     factor's variables in the order given, each variable's components in
 *     order (Sec. III storage order).  z is indexed by scalar variable in
 *     the order variables were added.
 */
#ifndef FGADMM_H
#define FGADMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FGA_OK 0
#define FGA_EINVAL (-1)     /* bad argument, id out of range, arity mismatch  */
#define FGA_ENOMEM (-2)     /* host or device allocation failed               */
#define FGA_ECUDA (-3)      /* a CUDA runtime call failed                     */
#define FGA_ESTATE (-4)     /* call not allowed in the object's current state */
#define FGA_ETIMEOUT (-5)   /* a device-side wait ran out of its time limit   */
#define FGA_ENONFINITE (-6) /* a residual became NaN or infinite              */
#define FGA_EBUDGET (-7)    /* iteration budget spent before the tolerance    */

/* ---- precision of messages and prox evaluations ------------------------ */
#define FGA_F32 0           /* FP32 messages; FP64 residuals and readout      */
#define FGA_F64 1           /* FP64 everywhere                                */

/* ---- factor types (interface numbers) ---------------------------------- */
/* Each entry: variables (dims) ; params per factor ; definition.           */
#define FGA_PACK_PAIR 0       /* (c1:2, r1:1, c2:2, r2:1) ; 0 ; indicator of
                                 |c1-c2| >= r1+r2 (Appendix A, no-collision) */
#define FGA_PACK_WALL 1       /* (c:2, r:1) ; 4 = Qx,Qy,Vx,Vy ; indicator of
                                 Q.(c-V) >= r (Appendix A, wall)             */
#define FGA_PACK_RADIUS_LIN 2 /* (r:1) ; 1 = w ; f = -w r                    */
#define FGA_PACK_RADIUS_QUAD 3 /* (r:1) ; 0 ; f = -r^2/2 (Appendix A); needs
                                 rho > 1 on its edge                          */
#define FGA_SVM_HINGE 4       /* (w:D, b:1) ; D+2 = x[D], y, c ;
                                 f = c max(0, 1 - y (w.x + b))               */
#define FGA_SVM_L2 5          /* (w:any) ; 1 = lambda ; f = lambda/2 |w|^2
                                 (Appendix C, minimal norm two)               */
#define FGA_MPC_DYN 6         /* (x:n, u:m, x':n) ; n*n + n*m = A (row-major),
                                 B (row-major) ; indicator of x' = A x + B u
                                 (Appendix B, linearised dynamics)            */
#define FGA_MPC_QUAD 7        /* (any vars) ; one q per scalar component ;
                                 f = 1/2 sum q_k v_k^2 (Appendix B, cost)     */
#define FGA_MPC_BOX 8         /* (any vars) ; 2 = lo, hi ; indicator of
                                 lo <= v <= hi                                */
#define FGA_FIX 9             /* (any vars) ; one value per scalar component ;
                                 indicator of v = value                       */
#define FGA_SVM_MARGIN 10     /* (w:D, b:1, xi:1) ; D+1 = x[D], y ; indicator
                                 of y (w.x + b) >= 1 - xi (Appendix C, one-
                                 point minimal margin)                        */
#define FGA_SVM_SLACK 11      /* (xi:any) ; 1 = lambda ; f = lambda sum xi_k
                                 on xi >= 0 (Appendix C, minimal error)       */
#define FGA_EQUAL 12          /* (v1:D, v2:D) ; 0 ; indicator of v1 = v2
                                 (Appendix C, equality of two copies)         */
#define FGA_NUM_TYPES 13
#define FGA_USER_TYPE0 64     /* first type number returned by
                                 fga_register_prox (user-supplied operators,
                                 numbered in registration order per graph)   */

/* ---- edge arrays for readout ------------------------------------------- */
#define FGA_EDGE_X 0
#define FGA_EDGE_M 1
#define FGA_EDGE_U 2
#define FGA_EDGE_N 3

/* ---- options (fga_set_option, before fga_finalize) --------------------- */
#define FGA_OPT_ZORDER 0      /* 0 = canonical: each z_b sums its edges one by
                                 one in ascending creation order (bit-exact
                                 with a serial FP64 loop); 1 = fast:
                                 deterministic warp / block / hub trees over
                                 chunks of factors; 2 = disk tiles: circle
                                 packing only (Sec. V-A: disk pairs, walls,
                                 radius rewards), FP32, one rho and one
                                 alpha, m not kept -- a warp holds 32 x 8
                                 disk pairs' state in registers, x is
                                 recomputed from u and the previous z, the
                                 CTAs' per-variable sums exchanged through
                                 count-and-sum words (a grid-wide barrier
                                 on checked iterations only); fused
                                 launches only; 3 = hinge bank: a linear
                                 soft-margin SVM only (Sec. V-C: hinge
                                 factors on one shared (w, b), dim(w) <= 64,
                                 plus L2 factors on w), FP32, one rho,
                                 alpha = 1, m not kept -- each CTA keeps its
                                 slice of the data rows in shared memory and
                                 one value of state per hinge factor in
                                 registers, the sums exchanged as in 2;
                                 fused launches only; 4 =
                                 scatter: each edge's rho*m goes straight to
                                 a per-variable column (the variable's k-th
                                 edge in creation order to column k < W, W
                                 <= 15 chosen at fga_finalize from the
                                 degrees) or past the columns to the
                                 variable's overflow row; z sums the columns
                                 in column order (for a variable of degree
                                 <= W the serial creation-order sum, as in
                                 0), then the overflow row by a warp tree
                                 (hub rows in pieces); items are grid-wide,
                                 factor-major, no chunks -- for graphs of
                                 low-degree variables; fewer than 2^28
                                 scalar variables.  Default: 0 for FGA_F64;
                                 for FGA_F32, 2 or 3 when the graph
                                 qualifies, else 4 when at least three
                                 quarters of the edges fit in the columns
                                 and the columns hold at most twice the
                                 edges, else 1.  Asking for 2 or 3
                                 on a graph that does not qualify makes
                                 fga_finalize return FGA_EINVAL.             */
#define FGA_OPT_STORE_M 1     /* 1 = keep m per edge so FGA_EDGE_M can be read
                                 back (default 1 for FGA_F64, 0 for FGA_F32)  */
#define FGA_OPT_BLOCK 2       /* threads per CTA of the sweep (0 = library
                                 choice; 64..256, multiple of 32); in the
                                 disk-tile order, the most threads per CTA
                                 (a CTA's units beyond its warps take turns) */
#define FGA_OPT_WEIGHTS 3     /* 0 = rho fixed per edge (Algorithm 2 as
                                 printed); 1 = three weights: each x-update
                                 gives every edge a weight class -- infinite
                                 for FGA_FIX, zero on an edge of a disk
                                 pair, wall, box, hinge or margin factor
                                 whose x equals its n (the constraint does
                                 not act on it), standard otherwise; z is
                                 the mean of the infinite-weight messages m
                                 if any, else the rho-weighted mean of the
                                 standard ones, else of all; u is reset to 0
                                 on zero- and infinite-weight edges.  The
                                 paper allows such improved rho schemes
                                 (Sec. II) without stating one; this is the
                                 library's reading.  Canonical z-order only
                                 (FGA_OPT_ZORDER 0, the default with it).   */

typedef struct fga_graph fga_graph; /* opaque, library-owned */

/* Creates an empty graph.  precision: FGA_F32 or FGA_F64.  device: CUDA
 * device ordinal used by every later call.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream) on which all device work of this
 * graph is ordered.  No device memory is touched until fga_finalize. */
int fga_graph_create(fga_graph **out, int32_t precision, int32_t device, void *cuda_stream);

/* Replaces the stream used by later calls. */
int fga_set_stream(fga_graph *g, void *cuda_stream);

/* Sets an FGA_OPT_* option; before fga_finalize only (FGA_ESTATE after). */
int fga_set_option(fga_graph *g, int32_t option, int64_t value);

/* Adds `count` variables of dimension `dim` (>= 1).  *first_var_id gets
 * the id of the first one; ids are consecutive.  Before fga_finalize. */
int fga_add_variables(fga_graph *g, int64_t count, int32_t dim, int64_t *first_var_id);

/* Registers `count` factors of one type (the paper's addNode, by type and
 * in batches).  var_ids: count * n_vars_per_factor variable ids, row-major
 * (factor-major).  params: count * params_per_factor values, row-major, or
 * params_per_factor values shared by all `count` factors when
 * params_shared != 0 (NULL allowed when params_per_factor == 0).  The
 * number of params must match the type's definition above, and variable
 * dimensions must match the type's shape; otherwise FGA_EINVAL.  Scalar
 * edges are numbered in call order.  *first_factor_id may be NULL. */
int fga_add_factors(fga_graph *g, int32_t type, int64_t count, int32_t n_vars_per_factor,
                    const int64_t *var_ids, const double *params, int32_t params_per_factor,
                    int32_t params_shared, int64_t *first_factor_id);

/* Registers a user-supplied proximal operator as a new factor type (the
 * paper's addNode takes the operator of a factor as a function pointer,
 * Sec. III; a GPU cannot call host code, so here it is CUDA source).
 *   cuda_source: NUL-terminated CUDA C++ that defines a function template
 *     template <typename R>
 *     void function_name(int arity, const R *n, const R *rho, const R *params, R *x);
 *   which must write x = argmin_s f(s) + sum_k rho_k/2 (s_k - n_k)^2
 *   (Eq. PO) for one factor: n, rho and x hold the factor's `arity` scalar
 *   edges in creation order (its variables in the order given to
 *   fga_add_factors, each variable's components in order; x holds n on
 *   entry), params its params_per_factor values (R = float for FGA_F32
 *   graphs, double for FGA_F64).  Functions need no __device__ mark; the
 *   CUDA math functions are available; no headers are included.
 *   arity: 1..64 scalar edges per factor; params_per_factor: 0..4096.
 * The source is compiled at once for the graph's device with NVRTC (FP64
 * graphs without multiply-add contraction, so that an operator written
 * the same way as a host implementation gives the same bits; IEEE division
 * and square root in both precisions).  *type_out gets the type number
 * (FGA_USER_TYPE0 + k) to pass to fga_add_factors; every factor of that type
 * must have `arity` scalar edges and params_per_factor parameters.
 * Before fga_finalize.  Errors: FGA_EINVAL with the compiler's log in
 * fga_last_error() when the source does not compile or the name is not a C
 * identifier; FGA_ECUDA when NVRTC (libnvrtc.so.13) cannot be opened.
 * A graph with user types runs in the canonical or scatter z-order
 * (FGA_OPT_ZORDER 0 or 4, the library's choice by default), with fixed
 * weights, one launch per update phase whatever fga_iter_opts.fused says
 * (each user type has its own x-update kernel), and not as a shard. */
int fga_register_prox(fga_graph *g, const char *cuda_source, const char *function_name, int32_t arity,
                      int32_t params_per_factor, int32_t *type_out);

/* Uniform rho > 0 and alpha > 0 on every edge (default 1, 1).  Before
 * fga_finalize. */
int fga_set_rho_alpha(fga_graph *g, double rho, double alpha);

/* Per-scalar-edge rho and alpha (creation order, |E| values each; either
 * may be NULL to keep the uniform value).  Before fga_finalize.  The two
 * coordinates of a disk centre (PACK_PAIR, PACK_WALL) must share one rho. */
int fga_set_edge_rho_alpha(fga_graph *g, const double *rho, const double *alpha);

/* Validates the graph, lays it out for the GPU (type buckets of
 * edge-major arrays, a variable-major edge index for the z-update) and
 * copies it to device memory -- the paper's CopyGraphFromCPUtoGPU.  After
 * this, no variable or factor can be added. */
int fga_finalize(fga_graph *g);

/* Sizes: scalar edges, scalar variables, factors, variables. */
int fga_graph_info(const fga_graph *g, int64_t *num_edges, int64_t *num_scalar_vars,
                   int64_t *num_factors, int64_t *num_vars);

/* Starting point (the paper leaves it open): z = z0 (|Z| values, variable
 * order; NULL = 0), u = u0 (|E| values, creation order; NULL = 0),
 * n = z_b - u, x = 0.  Host or device pointers (FP64).  After finalize. */
int fga_init(fga_graph *g, const double *z0, const double *u0);

typedef struct {
    int64_t max_iters;          /* iterations to run in this call (>= 0)    */
    double tol_pri, tol_dual;   /* stop when RMS primal and dual residuals
                                   are both <= these (0 = never)             */
    int32_t check_every;        /* residuals are evaluated after every
                                   check_every-th iteration and after the
                                   last one (>= 1)                           */
    int32_t fused;              /* 1 = one persistent kernel for the whole
                                   call; 0 = one launch per update phase
                                   (FGA_EINVAL in the disk-tile and hinge
                                   orders)                                  */
    int64_t barrier_timeout_ns; /* limit on one grid-wide wait inside the
                                   persistent kernel (0 = 2e9 ns)            */
    int32_t fault_skip_block;   /* testing: >= 0 makes that CTA skip its
                                   first barrier arrival (the wait then runs
                                   out and FGA_ETIMEOUT is returned); -1 off */
    int32_t reserved;
} fga_iter_opts;

typedef struct {
    int64_t iters;    /* iterations done in this call                      */
    double r_pri;     /* RMS primal residual sqrt(sum_e (x_e-z_b)^2 / |E|)   */
    double r_dual;    /* RMS dual residual sqrt(sum_e rho_e^2 (dz_b)^2 / |E|) */
    int32_t status;   /* FGA_OK, FGA_EBUDGET (tolerances set but not met),
                         FGA_ETIMEOUT or FGA_ENONFINITE                     */
    float ms;         /* device time of the call (CUDA events)             */
} fga_iter_result;

/* Runs Algorithm 2 for up to opts->max_iters iterations on the graph's
 * stream, stopping at the first checked iteration whose residuals meet both
 * tolerances.  The state after the call is exactly the state after
 * result->iters iterations, so calls can be chained (resume) with the same
 * iterates as one long call.  Synchronises the stream before returning.
 * Returns result->status as well (FGA_EBUDGET is reported in the result but
 * the call itself returns FGA_OK). */
int fga_iterate(fga_graph *g, const fga_iter_opts *opts, fga_iter_result *result);

/* Launch configuration chosen at fga_finalize, for reports: info[0] CTAs,
 * info[1] threads per CTA, info[2] dynamic shared memory per CTA (bytes),
 * info[3] co-resident CTAs per SM, info[4] work chunks (fast z-order), disk
 * tiles (tile order), hinge-bank CTAs (hinge order), columns W (scatter
 * order) or 0 (canonical order), info[5] type buckets, and when
 * n >= 7 info[6] the z-order in use (FGA_OPT_ZORDER values).  n >= 6. */
int fga_launch_info(const fga_graph *g, int64_t *info, int32_t n);

/* Latency floor of the disk-tile and hinge-bank orders (FGA_OPT_ZORDER 2
 * and 3) on this graph's grid: device time of `iters` passes that do
 * everything an unchecked pass does except the operators -- mode 1: each CTA
 * adds one count-and-sum contribution (value zero) per variable it holds
 * (every variable, in the hinge bank) and polls its variables' words until
 * every holder's contribution is in (the z exchange); mode 0: the grid-wide
 * barrier alone (which checked passes add).  FGA_EINVAL for other orders, and
 * for a graph not finalized.  A measurement of
 * the hardware's floor under a pass (the paper reports where an
 * iteration's time goes, Sec. V-A); the graph's variables and messages are
 * not changed.  *ms: device time (CUDA events). */
int fga_latency_floor(fga_graph *g, int64_t iters, int32_t mode, float *ms);

/* Residuals of the last checked iteration (NaN before any). */
int fga_residuals(const fga_graph *g, double *r_pri, double *r_dual);

/* z readout in FP64, variable order, n = number of scalar variables. Host or
 * device pointer. */
int fga_read_z(fga_graph *g, double *out, int64_t n);

/* Edge-array readout in FP64, creation order, n = number of scalar edges.
 * which: FGA_EDGE_X/M/U/N.  FGA_EDGE_M needs FGA_OPT_STORE_M.  Host or
 * device pointer. */
int fga_read_edge_state(fga_graph *g, int32_t which, double *out, int64_t n);

/* Frees every host and device resource of the graph. */
int fga_destroy(fga_graph *g);

/* ==========================================================================
 * Shards: one graph split across GPUs (one process per GPU).  The paper
 * names multi-GPU execution as future work (Sec. VI); its z-update is the
 * only step that couples factors, through the sums S_b = sum rho m and
 * R_b = sum rho over each variable's edges (Sec. II), so the factors are cut
 * into contiguous slices in creation order, one per rank, and the ranks
 * exchange only those sums.
 *
 * Each rank builds the same variables (every rank calls fga_add_variables
 * identically) and only its slice of the factors, in creation order, with
 * FGA_OPT_ZORDER 0 or 1.  Its edges are then a contiguous run of the whole
 * graph's creation order: rank r's edges follow rank r-1's.
 *   Set-up: R_b and sum rho^2 are chained through the ranks in rank order
 *     (fga_shard_rho_chain, host arrays: rank 0 from NULL, rank r from rank
 *     r-1's output; the last rank's output is the graph-wide sum) and
 *     handed to every rank by fga_shard_begin.
 *   Iteration: fga_shard_xstep (deferred u- and n-update, x-update, m, and
 *     this rank's running sums of rho m), an exchange of those sums by the
 *     caller, fga_shard_zstep (z from the graph-wide sums).  Two exchanges
 *     are supported:
 *     - chain (canonical order, FGA_OPT_ZORDER 0): rank r passes rank r-1's
 *       output as s_in; each rank adds its terms one by one onto it, so the
 *       last rank's output equals the serial creation-order sum of the
 *       whole graph bit for bit; it is then broadcast to every rank;
 *     - gather (any order): every rank runs s_in = NULL, the outputs are
 *       all-gathered and fga_shard_add_parts sums them in rank order.
 *   Residuals: the x-step that follows a checked z-step (check_prev = 1),
 *     or fga_shard_finish at the end, gives this rank's primal partial sum;
 *     the checked z-step gives the graph-wide dual sum (the same value on
 *     every rank); fga_shard_stop_rule applies the stop rule.  A stop after
 *     an x-step leaves the state of the checked iteration (the x just
 *     computed is discarded), as fga_iterate does.
 * Device work is queued on the graph's stream and these calls return
 * without waiting; s_in, s_out, parts and total are device arrays of the
 * graph's precision (float for FGA_F32, double for FGA_F64) with one value
 * per scalar variable; pri_out and dual_out are device doubles.  A shard
 * graph cannot be run by fga_iterate (FGA_ESTATE).
 * ========================================================================== */

/* Host arrays of n = scalar variables: out = in + this graph's rho (and
 * rho^2) added one by one in creation order (in may be NULL: zeros). */
int fga_shard_rho_chain(const fga_graph *g, const double *srho_in, const double *srho2_in, double *srho_out,
                        double *srho2_out);

/* Switches a finalized graph into shard mode with the graph-wide sums (host
 * arrays).  FGA_EINVAL for the disk-tile or hinge-bank orders. */
int fga_shard_begin(fga_graph *g, const double *srho_total, const double *srho2_total);

/* One x-step: the pending u- and n-update (after a z-step), the x-update of
 * every factor of the shard, m = x + u, and s_out = s_in + this shard's
 * rho m terms.  check_prev = 1 also writes this shard's primal residual sum
 * sum (x - z)^2 of the pending iteration to *pri_out (needs a pending
 * z-step). */
int fga_shard_xstep(fga_graph *g, int32_t check_prev, const void *s_in, void *s_out, double *pri_out);

/* total = parts[0] + parts[1] + ... + parts[n_shards - 1] per variable, in
 * that order (parts: n_shards consecutive arrays). */
int fga_shard_add_parts(fga_graph *g, const void *parts, int32_t n_shards, void *total);

/* z = total / R per variable (a variable with R = 0 keeps z); with check,
 * the graph-wide dual residual sum sum_b (sum_e rho^2) (z_b - z_b^prev)^2 to
 * *dual_out.  Ends the iteration. */
int fga_shard_zstep(fga_graph *g, const void *total, int32_t check, double *dual_out);

/* The pending u-update at the end of a run, and this shard's primal
 * residual sum of the last iteration to *pri_out. */
int fga_shard_finish(fga_graph *g, double *pri_out);

/* Stop rule on host values: RMS primal sqrt(sum_r pri_parts[r] / E) (the
 * parts added in rank order), RMS dual sqrt(dual / E); *stop = 1 when both
 * meet their tolerances or either is not finite. */
int fga_shard_stop_rule(const double *pri_parts, int32_t n_shards, double dual, int64_t num_edges, double tol_pri,
                        double tol_dual, double *r_pri, double *r_dual, int32_t *stop);

/* ==========================================================================
 * One long-horizon MPC (Sec. V-B: the paper's sampled inverted pendulum,
 * A 4 x 4, B 4 x 1, horizons up to 10^5) solved by Algorithm 2 in FP32 with
 * the horizon laid along the grid: the factor graph
 *   FIX(x_0) | DYN(x_t, u_t, x_{t+1}) t<K | QUAD(x_t, u_t) t<K | QUAD(x_K)
 * (creation order; Appendix B operators: fixed value, the rho-weighted
 * projection onto x' = A x + B u, f = 1/2 v' diag(q, r) v), uniform rho and
 * alpha.  E = 14 K + 8 scalar edges, numbered in creation order (FIX 0..3,
 * DYN_t from 4 + 9 t, QUAD_t from 4 + 9 K + 5 t, the terminal cost from
 * 4 + 14 K); z = x_0..x_K (4 each), then u_0..u_{K-1}.  The same graph on
 * the general path (fga_graph_*) gives the same iterates up to FP32
 * rounding.  One thread per step, its messages in registers; one grid-wide
 * barrier per iteration (one more on check iterations).
 * ========================================================================== */
typedef struct fga_horizon fga_horizon; /* opaque, library-owned */

/* nx must be 4 and nu 1 (the pendulum); A (4 x 4) and B (4 x 1) row-major,
 * q (4), r (1) the cost diagonals (>= 0), x0 the fixed state; rho, alpha
 * > 0.  K steps need ceil(K / 224) co-resident CTAs (K up to about 10^5 on
 * 152 SMs; FGA_EINVAL beyond).  Host pointers.  stream NULL: the object
 * creates its own.  The state is undefined until fga_horizon_init. */
int fga_horizon_create(fga_horizon **out, int32_t K, int32_t nx, int32_t nu, const double *A, const double *B,
                       const double *q, const double *r, const double *x0, double rho, double alpha,
                       int32_t device, void *cuda_stream);

/* Cold start: z = 0, u = 0, x = 0 (n = z - u). */
int fga_horizon_init(fga_horizon *h);

/* Runs up to opts->max_iters iterations (opts as for fga_iterate; fused
 * only), stopping at the first checked iteration whose RMS residuals meet
 * both tolerances; the state after the call is the state after
 * result->iters iterations, so calls chain.  FGA_ETIMEOUT when a grid-wide
 * wait runs out (the state then needs fga_horizon_init). */
int fga_horizon_solve(fga_horizon *h, const fga_iter_opts *opts, fga_iter_result *result);

/* Readout in FP64 to host memory (any pointer may be NULL): z ((K+1) 4 + K
 * values, variable order above), x and u (E values each, creation order). */
int fga_horizon_read(fga_horizon *h, double *z, double *x_edges, double *u_edges);

/* info[0] CTAs, info[1] steps (threads) per CTA, info[2] E, info[3] scalar
 * variables.  n >= 4. */
int fga_horizon_info(const fga_horizon *h, int64_t *info, int32_t n);

/* Frees every resource of the object. */
int fga_horizon_destroy(fga_horizon *h);

/* ==========================================================================
 * Batched ragged MPC (Sec. V-B, Appendix B): many independent instances of
 *   minimise 1/2 sum_{t<T} (x_t' Q x_t + u_t' R u_t) + 1/2 x_T' Q x_T
 *   s.t. x_{t+1} = A x_t + B u_t, x_0 fixed, lo <= u_t <= hi (lo = -umax)
 * each written as the factor graph FIX(x_0) | DYN(x_t,u_t,x_{t+1}) t<T |
 * QUAD(x_t,u_t) t<T | QUAD(x_T) | BOX(u_t) t<T (creation order; z per
 * instance = x_0, u_0, x_1, u_1, ..., u_{T-1}, x_T), solved by Algorithm 2
 * with uniform rho, alpha, all instances in one persistent launch (one CTA
 * per instance at a time, state in shared memory), optionally replayed from
 * a CUDA graph.  Per instance: E = 2 nx + 3 (nx + nu) T scalar edges and
 * V = (nx + nu) T + nx scalar variables; instance i's z starts at the sum
 * of the V of instances 0..i-1, its u at the sum of their E.
 * ========================================================================== */
typedef struct fga_mpc_batch fga_mpc_batch; /* opaque, library-owned */

/* n_inst instances of horizons T[i] (1..1e5) on n_sys systems: A (n_sys x
 * nx x nx, row-major), B (n_sys x nx x nu), q (n_sys x nx, diagonal of Q),
 * r (n_sys x nu, diagonal of R).  sys_of_inst[i] picks instance i's system
 * (NULL: all use system 0 when n_sys == 1, instance i uses system i when
 * n_sys == n_inst).  2 nx + nu <= 64.  stream NULL: the batch creates its
 * own stream (needed to capture CUDA graphs).  Host pointers. */
int fga_mpc_batch_create(fga_mpc_batch **out, int32_t precision, int32_t device, void *stream, int32_t n_inst,
                         const int32_t *T, int32_t nx, int32_t nu, int32_t n_sys, const int32_t *sys_of_inst,
                         const double *A, const double *B, const double *q, const double *r, double umax,
                         double rho, double alpha);

/* Initial states x_0 of all instances (n_inst x nx).  Host or device. */
int fga_mpc_batch_set_x0(fga_mpc_batch *b, const double *x0);

/* Start point: z (all instances, concatenated; NULL = 0) and per-edge u
 * (concatenated, creation order; NULL = 0); x = 0.  Host or device. */
int fga_mpc_batch_init(fga_mpc_batch *b, const double *z0, const double *u0);

/* Warm start from a prediction (device pointer, FP32, one row of length
 * >= 2 (nx+nu) Tmax per instance, stride ld): first T(nx+nu) values are
 * (x_{t+1}, u_t) for t = 0..T-1, the next T(nx+nu) are (lambda_t, mu_t),
 * the multipliers of the dynamics and of the input box.  Sets z from the
 * trajectory and every edge's u from the fixed-point relation
 * u = -(1/rho) (sub)gradient of its factor at z (the paper has no warm
 * start; this is the start point a learned model supplies). */
int fga_mpc_batch_warm_start(fga_mpc_batch *b, const float *pred, int64_t ld);

/* Inverse of the warm-start map on the current state: writes, per
 * instance, (x_{t+1}, u_t) and (lambda_t, mu_t) in the layout above (device
 * pointer, FP32, stride ld) -- training targets for the learned model. */
int fga_mpc_batch_targets(fga_mpc_batch *b, float *out, int64_t ld);

typedef struct {
    int64_t max_iters;          /* budget per instance                      */
    double tol_pri, tol_dual;   /* RMS residual tolerances per instance     */
    int32_t check_every;        /* 0 = autotuned value (default 1)          */
    int32_t threads;            /* CTA size 64/128/224/256/448/512 (one CTA
                                   per instance at a time); 32 = one lane
                                   per time step, its state in registers
                                   (FP32, 12 states, 4 inputs, horizons up
                                   to 64: a warp per instance of up to 32
                                   steps, two warps up to 64); 0 =
                                   autotuned (128)                           */
    int32_t use_graph;          /* 1 = launch from a cached CUDA graph      */
    int32_t reserved;
} fga_mpc_opts;

typedef struct {
    int64_t total_iters;        /* sum over instances                       */
    int64_t max_inst_iters;
    int32_t n_converged, n_budget, n_nonfinite;
    float ms;                   /* device time of the solve (CUDA events)   */
    int32_t threads, check_every;
} fga_mpc_result;

/* Solves every instance from the current start point; each instance stops
 * at the first checked iteration whose residuals meet both tolerances
 * (status 0) or at the budget (FGA_EBUDGET).  Synchronises the stream. */
int fga_mpc_batch_solve(fga_mpc_batch *b, const fga_mpc_opts *opts, fga_mpc_result *res);

/* Readout (host pointers, any may be NULL): z (FP64, concatenated), u (FP64,
 * concatenated, creation order), per-instance iterations, status, RMS
 * residuals. */
int fga_mpc_batch_read(fga_mpc_batch *b, double *z, double *u, int64_t *iters, int32_t *status, double *r_pri,
                       double *r_dual);

/* info[0] instances, [1] total edges, [2] total scalar variables, [3] longest
 * horizon, [4] tuned CTA size, [5] tuned check interval.  n >= 6. */
int fga_mpc_batch_info(const fga_mpc_batch *b, int64_t *info, int32_t n);

/* Autotuner: times CTA sizes {32 (where it applies),64,128,224,256,448,512} x check intervals {1,2,5,10} on
 * the batch from its current start point (which it restores) and keeps the
 * fastest for later solves.  cache_path (may be NULL): a text file of
 * previous results keyed by GPU, precision and problem shape; a hit skips
 * the timing, a miss appends the result. */
int fga_mpc_batch_autotune(fga_mpc_batch *b, const char *cache_path, int64_t max_iters, double tol,
                           int32_t *threads_out, int32_t *check_every_out);

int fga_mpc_batch_destroy(fga_mpc_batch *b);

/* Allocation-free batched MPC solve (the paper has no counterpart; this is
 * a deployment variant of fga_mpc_batch_solve).  For callers that cannot
 * call cudaMalloc at solve time -- code running inside a memory arena it
 * does not own, real-time control loops that must not touch the allocator
 * after start-up, plugins whose host forbids device allocations -- this
 * entry point allocates nothing: all scratch (per-edge x and u, instance
 * offsets, the dynamics projector, residuals, the work counter) lives in
 * one 16 MiB device array that every GPU loading the library holds until
 * the process exits.  Limits: n_inst <= 4096, about 2 million scalar edges
 * in total (E = 2 nx + 3 (nx + nu) T per instance); larger batches are
 * rejected with FGA_EINVAL.
 *
 * Cold start (z = u = x = 0) of n_inst instances of ONE system, FP32
 * messages, FP64 residuals; same model, factor graph and stopping rule as
 * fga_mpc_batch_solve with tol_pri = tol_dual = tol.  T: host array of
 * horizons, read once during the call (the launch carries a copy, so the
 * caller may change or free T as soon as the call returns).  A (nx x nx),
 * B (nx x nu), q (nx), r (nu), x0 (n_inst x nx): device FP32, read when the
 * work runs.  Outputs (device): z_out (sum of V = (nx + nu) T + nx values,
 * instances concatenated), iters_out and status_out per instance; a
 * non-finite A or B (a projector that cannot be formed) makes every
 * status_out entry FGA_EINVAL.  The work is queued on `stream` (NULL: legacy
 * default stream) and the call returns without waiting; outputs are valid
 * once the stream has synchronised.  The first call on a device looks up
 * the array's device address (once per device, with that device current)
 * and keeps it for the life of the process: make that first call before any
 * CUDA graph capture, and do not use this entry point across a
 * cudaDeviceReset.  All calls share the one array and every call overwrites
 * it, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. */
int fga_mpc_solve_noalloc(int32_t n_inst, const int32_t *T, int32_t nx, int32_t nu, const float *A, const float *B,
                          const float *q, const float *r, const float *x0, float umax, float rho, float alpha,
                          int64_t max_iters, double tol, int32_t check_every, float *z_out, int64_t *iters_out,
                          int32_t *status_out, void *stream);

/* ==========================================================================
 * Learned warm start: a ReLU MLP in -> h1 -> h2 -> out, BF16 weights and
 * activations on the tcgen05 tensor cores with FP32 accumulation in tensor
 * memory, FP32 master weights and Adam (beta 0.9, 0.999, eps 1e-8), MSE loss
 * on standardised targets.  Not in the paper; it supplies
 * fga_mpc_batch_warm_start's prediction.  Parameters are packed as W1 (h1 x
 * in, row-major), b1, W2 (h2 x h1), b2, W3 (out x h2), b3.  h1, h2, out and
 * every batch: multiples of 8.  Every wait inside a GEMM is bounded (about
 * one second); a call that synchronises (fga_mlp_forward,
 * fga_mlp_gradients, fga_mlp_train_step with a loss) returns FGA_ETIMEOUT
 * if a GEMM since the previous such call gave up, and its outputs are then
 * not valid.
 * ========================================================================== */
typedef struct fga_mlp fga_mlp; /* opaque, library-owned */

/* He-initialised (seeded splitmix64 + Box-Muller) network; buffers for up
 * to max_batch rows. */
int fga_mlp_create(fga_mlp **out, int32_t in, int32_t h1, int32_t h2, int32_t out_dim, int32_t max_batch,
                   uint64_t seed, int32_t device, void *stream);
int fga_mlp_num_params(const fga_mlp *m, int64_t *n);
/* FP32 master weights from / to host memory (packed order above). */
int fga_mlp_set_params(fga_mlp *m, const float *params, int64_t n);
int fga_mlp_get_params(fga_mlp *m, float *params, int64_t n);
/* Per-output mean and standard deviation of Y (device, rows x out FP32);
 * Y is standardised in place, and fga_mlp_forward de-standardises. */
int fga_mlp_fit_normalization(fga_mlp *m, float *Y, int64_t rows);
int fga_mlp_get_normalization(fga_mlp *m, float *mean, float *stdv);
/* Loss (mean squared error against standardised targets Y) and the
 * gradient of every parameter, into host `grads` (packed order).  X, Y:
 * device, FP32, batch x in / batch x out. */
int fga_mlp_gradients(fga_mlp *m, const float *X, const float *Y, int32_t batch, float *grads, double *loss);
/* One Adam step on a minibatch (device X, Y); loss may be NULL (no sync). */
int fga_mlp_train_step(fga_mlp *m, const float *X, const float *Y, int32_t batch, float lr, double *loss);
/* Prediction in target units (de-standardised), device X and Y. */
int fga_mlp_forward(fga_mlp *m, const float *X, float *Y, int32_t batch);
int fga_mlp_destroy(fga_mlp *m);

/* Message describing the last failure on this thread ("" if none). */
const char *fga_last_error(void);

/* Library version string. */
const char *fga_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FGADMM_H */
