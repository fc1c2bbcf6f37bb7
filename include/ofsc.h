/*
 * ofsc.h - C ABI of the GB300 (sm_103a) library for spectral clustering via
 * orthogonalization-free methods (Pang and Yang, arXiv 2305.10356).
 *
 * The calls follow the four steps of Algorithm 1:
 *   1. ofsc_graph_build     S and D from an edge list; A = L - 2I with L = I - D^-1/2 S D^-1/2 (Eq. (1))
 *   2. ofsc_iterate         OFM-f1 / TriOFM-f1 / OFM-f2 / TriOFM-f2 by Algorithm 2
 *      ofsc_objective_grad  f1 (Eq. (2)) or f2 (Eq. (3)) and its gradient (Eq. (5) / Eq. (10))
 *   3. ofsc_row_normalize   row normalisation of the feature block
 *   4. ofsc_kmeans          Euclidean K-means on the rows
 * and beyond them:
 *      ofsc_iterate_batched many independent graphs in one call (streams, CUDA-graph replay)
 *      ofsc_autotune        the sparse product's row partition and gathers in flight, by timing
 *      ofsc_weight_grad     df/dw for the edge weights of a weighted S
 *      ofsc_unrolled_grad   d f1(X_T)/dX_0 (and /dw) through T updates of Algorithm 2
 *      ofsc_rayleigh_ritz   Ritz values and relerr of Sec. 5 for a feature block
 *      ofsc_gram            the k x k dot-product blocks on the tensor cores
 *      ofsc_set_allocator   the caller's device allocator for every block the library allocates
 *
 * Conventions (all calls):
 *   - Every call returns an ofsc_status. No C++ exception crosses this boundary. On an error
 *     ofsc_last_error() returns a message for the calling host thread.
 *   - Array arguments are DEVICE pointers owned by the caller, unless a comment says "host".
 *     Dense blocks are row-major n x k FP32 with leading dimension k (row l = node l).
 *     Pointers to FP32 data must be 4-byte aligned; they need not be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *     queued on it. A call that returns a host value (f_out, ofsc_result, inertia, counts)
 *     synchronises that stream before it returns. Calls that allocate or free device memory
 *     (the first call on a handle for a given k, ofsc_graph_build/free, ofsc_unrolled_grad,
 *     ofsc_autotune, ofsc_weight_grad, ofsc_rayleigh_ritz, ofsc_gram) carry the device-wide
 *     synchronisation of cudaMalloc/cudaFree (or of ofsc_set_allocator's frees); no other call
 *     synchronises the whole device.
 *   - Host phases of the longer calls are marked with NVTX ranges ("ofsc_iterate", "update",
 *     "exact refresh", "report", "ofsc_graph_build", ...) for Nsight tools.
 *   - ofsc_graph handles are owned by the library: create with ofsc_graph_build, release with
 *     ofsc_graph_free. A handle also caches the device workspace of ofsc_iterate and
 *     ofsc_objective_grad, so calls that share one handle must be ordered by the caller
 *     (one stream, or explicit events); calls on different handles are independent.
 *   - The current CUDA device at the time of the call is used; all pointers must live on it.
 */
#ifndef OFSC_H
#define OFSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ofsc_status;
enum {
  OFSC_OK = 0,
  OFSC_ERR_INVALID_ARG = 1,   /* bad size, id out of range, bad weight, NULL where required */
  OFSC_ERR_OOM = 2,           /* device allocation failed */
  OFSC_ERR_NONFINITE = 3,     /* NaN/Inf met in the input block or in the iteration */
  OFSC_ERR_TIMEOUT = 4,       /* a bounded device wait ran out */
  OFSC_ERR_NOT_CONVERGED = 5, /* warning only: maxit reached before tol; the result is valid */
  OFSC_ERR_CUDA = 6           /* a CUDA runtime call failed (message in ofsc_last_error) */
};

/* Methods of Sec. 2: gradient of f1 (Eq. (5)), g1 (Eq. (7)), gradient of f2 (Eq. (10)), g2 (Eq. (12)). */
enum { OFSC_OFM_F1 = 0, OFSC_TRI_F1 = 1, OFSC_OFM_F2 = 2, OFSC_TRI_F2 = 3 };
/* Objectives: f1 = ||A + XX^T||_F^2 (Eq. (2)), f2 = tr((2I - X^T X) X^T A X) (Eq. (3)). */
enum { OFSC_F1 = 1, OFSC_F2 = 2 };
/* Storage of the block gathered by the sparse product: FP32, or BF16 with FP32 accumulation. */
enum { OFSC_GATHER_FP32 = 0, OFSC_GATHER_BF16 = 1 };
/* Engine of the k x k Gram reductions: FP32 CUDA cores, or tcgen05 tensor cores (3-term TF32). */
enum { OFSC_GRAM_AUTO = 0, OFSC_GRAM_SIMT = 1, OFSC_GRAM_TC = 2 };
/* Row gathers of the sparse product: CUDA-core loads, or TMA tile::gather4 into shared memory. */
enum { OFSC_SPMM_AUTO = 0, OFSC_SPMM_SIMT = 1, OFSC_SPMM_TMA = 2 };

typedef struct ofsc_graph ofsc_graph;
/* The state of Algorithm 2's conjugate-gradient recurrence between calls (ofsc_state_create). */
typedef struct ofsc_state ofsc_state;

typedef struct {
  int64_t n;            /* nodes */
  int64_t m_in;         /* edges in the input list */
  int64_t nnz;          /* stored entries of S (2 x distinct undirected non-loop pairs) */
  int64_t n_selfloops;  /* input edges with src == dst (dropped) */
  int64_t n_duplicates; /* directed entries merged into another (repeated pairs) */
  int64_t n_isolated;   /* nodes of degree 0 (they get D^-1/2 = 0, so L_ii = 1) */
  int32_t weighted;     /* 1 if S carries FP32 weights */
  double normA_fro2;    /* ||A||_F^2 = n + sum_ij (D^-1/2 S D^-1/2)_ij^2, FP64 */
} ofsc_graph_info;

/*
 * ofsc_graph_build - S, D and D^-1/2 from an undirected edge list (Eq. (1); Algorithm 1, step 2).
 *   n        number of nodes (>= 0, < 2^31)
 *   m        number of input edges (>= 0)
 *   src,dst  device int32 [m]; edge e joins src[e] and dst[e]; ids must lie in [0, n)
 *   w        device float32 [m] edge weights (finite, > 0), or NULL for a binary S
 *   flags    reserved, must be 0
 *   out      host pointer that receives the new handle
 * Each input edge {u, v} sets S_uv = S_vu. Self-loops are dropped and counted. A pair listed
 * more than once (in either direction) is one entry: weight 1 for a binary S; for a weighted S
 * the listed FP32 weights are summed in FP64 in input order and rounded once to FP32.
 * D_ii = sum_j S_ij (integer count, or FP64 sum in column order); D^-1/2 = (float)(1/sqrt(D_ii))
 * in IEEE FP64, and 0 for an isolated node. CSR columns are ascending within each row.
 * Errors: OFSC_ERR_INVALID_ARG (bad n/m/flags, id out of range, bad weight), OFSC_ERR_OOM.
 * Synchronises `stream` (the validation result and sizes are read back).
 */
ofsc_status ofsc_graph_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                             const float* w, uint32_t flags, void* stream, ofsc_graph** out);

/* Releases a handle and its device memory (NULL is allowed). Synchronises the device memory
 * owned by the handle only after queued work on every stream has finished (cudaFree rules). */
ofsc_status ofsc_graph_free(ofsc_graph* g);

/* Sizes and counts of a built graph (host struct). */
ofsc_status ofsc_graph_get_info(const ofsc_graph* g, ofsc_graph_info* info);

/*
 * ofsc_graph_csr - device pointers into the handle's CSR (owned by the handle, valid until
 * ofsc_graph_free): row_ptr int64 [n+1], col int32 [nnz], val float32 [nnz] (NULL if binary),
 * dinv float32 [n] = D^-1/2, deg float64 [n] = D_ii. Any output pointer may be NULL.
 */
ofsc_status ofsc_graph_csr(const ofsc_graph* g, const int64_t** row_ptr, const int32_t** col,
                           const float** val, const float** dinv, const double** deg);

/*
 * ofsc_objective_grad - f and its gradient at X (Eqs. (2)/(3), (5)/(10)).
 *   objective  OFSC_F1 or OFSC_F2
 *   k          columns of X (1 <= k <= 128)
 *   X          device float32 [n x k]
 *   f_out      HOST double*: receives f (nullable)
 *   G_out      device float32 [n x k]: receives the gradient with its factor 4 (nullable)
 * f1 uses ||A + XX^T||^2 = ||A||^2 + 2 tr(X^T A X) + ||X^T X||^2. Synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_OOM, OFSC_ERR_NONFINITE (NaN/Inf in X or f).
 */
ofsc_status ofsc_objective_grad(ofsc_graph* g, int32_t objective, int32_t k, const float* X,
                                double* f_out, float* G_out, void* stream);

/*
 * ofsc_objective_grad_noalloc - the same f and gradient as ofsc_objective_grad, computed
 * without allocating any device memory. The paper has no counterpart: this is a library entry
 * point for callers that must not call cudaMalloc while they run, such as a process whose device
 * memory is already reserved by another allocator (cudaMalloc would fail there) or a
 * latency-bound loop that cannot afford an allocation's driver call and implicit
 * synchronisation.
 *   Arguments, layout and results are those of ofsc_objective_grad; the graph is only read.
 *   Temporary storage comes from one static device array of about 30 MiB inside the library,
 *   which every GPU that loads the library holds until the process exits.
 *   Limit: n * kp <= 2^20 with kp = k rounded up to a multiple of 8 (k <= 128); larger sizes
 *   return OFSC_ERR_INVALID_ARG with a message (use ofsc_objective_grad for them).
 *   The first call on a device looks up the array's device address with that device current;
 *   make that first call before any stream capture. The address is kept for the life of the
 *   process, so after a cudaDeviceReset of a device this entry point must not be called on it
 *   again. The graph must belong to the current device (OFSC_ERR_INVALID_ARG otherwise). All
 *   calls share the array and it keeps the previous call's contents, so calls that overlap on
 *   the GPU (several streams or host threads) race with one another: order them.
 *   Synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_NONFINITE, OFSC_ERR_CUDA.
 */
ofsc_status ofsc_objective_grad_noalloc(const ofsc_graph* g, int32_t objective, int32_t k,
                                        const float* X, double* f_out, float* G_out, void* stream);

/* Phases of one update, for the optional per-phase device timing of ofsc_iterate. */
enum {
  OFSC_PHASE_DIRECTION = 0,    /* update X, AX; G = g(X); column sums (the direction pass) */
  OFSC_PHASE_BETA = 1,         /* beta and the stop test */
  OFSC_PHASE_SPMM = 2,         /* A G gather with the fused V, AV epilogue */
  OFSC_PHASE_GRAM = 3,         /* k x k Gram partials over all rows */
  OFSC_PHASE_GRAM_REDUCE = 4,  /* fixed-order FP64 sum of the Gram partials */
  OFSC_PHASE_LINESEARCH = 5,   /* FP64 cubic coefficients, roots, alpha */
  OFSC_PHASE_REFRESH = 6,      /* exact A X recomputation with its Grams */
  OFSC_PHASE_OTHER = 7,        /* padding copies, control, update-only passes */
  OFSC_NUM_PHASES = 8
};

/* Accumulated device time per phase, measured with CUDA events on the call's stream. */
typedef struct {
  double ms[OFSC_NUM_PHASES];
  int64_t launches[OFSC_NUM_PHASES];
} ofsc_profile;

typedef struct {
  int32_t gather;      /* OFSC_GATHER_FP32 (default) or OFSC_GATHER_BF16 */
  int32_t y_refresh;   /* AX is carried by the recurrence AX += AV diag(alpha); it is recomputed
                          exactly every y_refresh iterations (<= 0: default 32) */
  int32_t check_every; /* host reads the stop flag every check_every iterations (<= 0: 16) */
  double alpha0;       /* > 0: fixed step for step 0 of Algorithm 2; else exact line search */
  double* trace;       /* device float64 [trace_cap x (3 + 2k)] or NULL: per update t the record
                          {t, ||G_t||/||G_0||, f(X_t), alpha_t[0..k-1], beta_t[0..k-1]} */
  int32_t trace_cap;   /* records available in `trace` */
  ofsc_profile* profile; /* HOST struct or NULL: the call ADDS its per-phase device times
                            (events around every launch; adds a little host overhead) */
  int32_t gram_engine;   /* OFSC_GRAM_AUTO (tensor cores when k > 64), OFSC_GRAM_SIMT, OFSC_GRAM_TC */
  int32_t spmm_engine;   /* OFSC_SPMM_AUTO (= OFSC_SPMM_SIMT: one warp per row, CUDA-core gathers),
                            OFSC_SPMM_TMA (tile::gather4 into shared memory; padded k 64 or 128) */
  int32_t direct_launch; /* 0 (default): the updates whose launches repeat are captured once into a
                            CUDA graph and replayed (ofsc_iterate does so unless `profile` is set);
                            1: every kernel is launched directly (same results, bit for bit) */
  int32_t cg_restart;    /* 0 (default): beta exactly as Algorithm 2 prints it. 1: an optional
                            restart that is NOT in the paper: a column whose new direction would
                            not descend (V_t,i . G_t,i >= 0) takes beta_i = 0. Runs far past the
                            FP32 rounding floor can see noise-level beta compound in V until it
                            overflows (OFSC_ERR_NONFINITE); the restart prevents that */
  double refine_tol;     /* gather = OFSC_GATHER_BF16 only; 0 (default): BF16 gathers to the end.
                            > 0: the FP32 refinement sweep: once a host check (every check_every
                            updates) reads ||G_t||_F <= refine_tol ||G_0||_F, every later update
                            gathers D^-1/2 V in FP32, so the run ends on FP32 products. The switch
                            point depends only on check_every and the iterates */
  double exact_tail;     /* 0 (default): 1e3 tol when tol > 0, else never. > 0: once a host check
                            reads ||G_t||_F <= exact_tail ||G_0||_F, every later update recomputes
                            AX = A X, X^T X and X^T AX exactly, as Algorithm 2 states it, instead of
                            carrying them by the recurrences (whose FP32 drift is near the size of
                            G at tolerances of 1e-6). < 0: never */
  int32_t vscale_exp;    /* 0 (default 20), else in [-60, 60]: V is stored in FP32 as V diag(1/s)
                            with s_j a power of two, 1 until |V_j| would exceed
                            2^vscale_exp ||G_0||_F (Algorithm 2's beta can compound past the FP32
                            range where FP64 still holds it). Scaling by powers of two is exact,
                            so the results do not depend on this value unless FP32 would
                            overflow or underflow */
  int64_t spin_limit;    /* polls allowed per bounded mbarrier wait of the tensor-core kernels
                            (0: the compiled default, 2^22); a wait that runs out ends its kernel
                            with OFSC_ERR_TIMEOUT after its own copies and MMAs have completed */
  int32_t withhold_arrivals; /* test hook, 0 (default) or 1: the converter warps of the tensor-core
                            direction pass (OFM-f1, TriOFM-f1 at padded k = 128) never signal a full
                            stage, so its MMA warp's first bounded wait runs out before any MMA is
                            issued and the call returns OFSC_ERR_TIMEOUT (exercises the timeout
                            path without a fault; use with a small spin_limit) */
  int32_t merge_path;    /* 0 (default): the direction product (Sec. 3.3) splits its work by merge
                            path (equal shares of rows + nonzeros, so a long row spans several
                            warps, whose partial sums are added in warp order) when ofsc_autotune
                            chose it for this k and gather storage, or, untuned, when the graph
                            holds at least 2^23 stored entries or its longest row holds at least
                            1024 nonzeros and more than four warps' shares of the row partition;
                            else by whole rows; 1: always by merge path; -1: never */
  int32_t group_launches; /* replayed updates: 0 (default) one launch per graph and kernel, on
                            the graphs' own streams; n in [1, 64]: grouped launches, where one
                            launch runs a kernel of the update for up to 32 graphs, its blocks a
                            work list of (graph, block) pairs, with the same results bit for bit;
                            the graphs are dealt into n lanes of similar work, grouped within a
                            lane, and the lanes overlap */
  ofsc_state* state;     /* ofsc_iterate only (NULL: none): the CG state to resume and to leave
                            for the next call. If it holds a run (t > 0) the call continues that
                            run: X must be the X that run returned, and the first update takes
                            beta from the saved G_{t-1} and extends the saved V_{t-1} (no step of
                            steepest descent); relative norms stay relative to that run's
                            ||G_0||. A call that performs all maxit > 0 updates without stopping
                            leaves its own state in it (t grows by maxit); a call that stops or
                            fails leaves it empty. */
  int32_t overlap_gram;  /* where each update's Grams V^T X, V^T V (Sec. 3.3) run. 1: on a second
                            stream of the graph, at the same time as the direction product (both
                            read the V that the V pass wrote; neither writes what the other reads),
                            and the line search waits for both; -1: after the product on the
                            call's stream; 0 (default): 1 for a call on one graph with n kp <= 2^23
                            (padded k), else -1. Same kernels, same results bit for bit. Ignored
                            with group_launches > 0 or `profile`; for the f2 methods only with the
                            tensor-core Grams, whose V^T AX, V^T AV launch follows the product */
} ofsc_opts;

typedef struct {
  int32_t iterations;   /* updates X <- X + V diag(alpha) performed */
  int32_t status;       /* OFSC_OK (converged), OFSC_ERR_NOT_CONVERGED, or an error */
  double rel_dir_norm;  /* ||g(X)||_F / ||g(X_0)||_F at the returned X (AX recomputed exactly) */
  double g0_norm;       /* ||g(X_0)||_F */
  double f;             /* objective of the method (f1 or f2) at the returned X */
  int64_t kernel_launches; /* device kernels this call launched (in a batch, a grouped launch
                              serving several graphs is counted once, for the first of them) */
  int32_t refined_at;   /* first update of the FP32 refinement sweep (opts->refine_tol), or -1 */
  int32_t exact_at;     /* first update of the exact tail (opts->exact_tail), or -1 */
} ofsc_result;

/*
 * ofsc_iterate - Algorithm 2 (column-wise nonlinear CG with the exact line search of Sec. 3.2).
 *   method   OFSC_OFM_F1, OFSC_TRI_F1, OFSC_OFM_F2 or OFSC_TRI_F2
 *   k        columns (1 <= k <= 128; internally padded to a multiple of 8 with zero columns,
 *            which stay zero)
 *   X        device float32 [n x k]: in = X0 (warm start allowed), out = final X
 *   tol      stop when ||G_t||_F <= tol * ||G_0||_F (tol <= 0: run maxit updates)
 *   maxit    maximum number of updates t_max (>= 0)
 *   opts     host struct or NULL for defaults
 *   out      HOST ofsc_result (nullable)
 * G_0 = g(X_0), V_0 = -G_0, X_1 = X_0 + V_0 diag(alpha_0); for t >= 1: G_t = g(X_t);
 * beta_i = sum_l (G_t - G_{t-1})_li G_t,li / sum_l G_{t-1,li}^2 (0 if the denominator is 0; with
 * opts->cg_restart also 0 where the column of V_t would not descend);
 * V_t = -G_t + V_{t-1} diag(beta); alpha_t from the exact line search (one alpha for OFM, one
 * per column for TriOFM, with X_i, V_i the first i columns); X_{t+1} = X_t + V_t diag(alpha_t).
 * Only an update with an exact AX (every y_refresh updates, the exact tail, or one scheduled at the
 * next host check after ||G_t|| <= tol ||G_0|| was seen on a recurrence update) may stop the run,
 * so rel_dir_norm <= tol whenever the status is OFSC_OK.
 * Returns OFSC_OK when tol was met, OFSC_ERR_NOT_CONVERGED when maxit was reached first (X is
 * still the valid final iterate). Synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_OOM, OFSC_ERR_NONFINITE.
 */
ofsc_status ofsc_iterate(ofsc_graph* g, int32_t method, int32_t k, float* X, double tol,
                         int32_t maxit, const ofsc_opts* opts, ofsc_result* out, void* stream);

/*
 * ofsc_iterate_batched - ofsc_iterate (Algorithm 2) on `count` independent graphs in one call, for
 * many small independent problems of uneven sizes.
 *   count    number of problems (>= 0)
 *   graphs   HOST array [count] of distinct handles
 *   method   one method for every problem
 *   ks       HOST int32 [count]: columns of each problem (1 <= k <= 128)
 *   Xs       HOST array [count] of device float32 [n_i x k_i]: in = X0, out = final X
 *   tol, maxit, opts   as for ofsc_iterate, shared by every problem; opts->trace and
 *            opts->profile must be NULL
 *   outs     HOST ofsc_result [count] (nullable), one per problem, in input order
 * Each problem runs on a stream owned by its handle, ordered after `stream` on entry and before it
 * on return; the problems advance in lockstep and share the SMs. Every problem gets exactly the
 * launches, in the same order, that ofsc_iterate would give it, so each result and each X equals
 * that of ofsc_iterate on the same problem bit for bit. The call returns when every problem has
 * met tol or maxit is reached. Synchronises `stream`.
 * Returns OFSC_OK when every problem converged, else the first error among them, else
 * OFSC_ERR_NOT_CONVERGED. Errors: OFSC_ERR_INVALID_ARG (any problem's arguments, a repeated
 * handle, trace or profile set), OFSC_ERR_OOM, OFSC_ERR_NONFINITE, OFSC_ERR_CUDA.
 */
ofsc_status ofsc_iterate_batched(int32_t count, ofsc_graph* const* graphs, int32_t method,
                                 const int32_t* ks, float* const* Xs, double tol, int32_t maxit,
                                 const ofsc_opts* opts, ofsc_result* outs, void* stream);

/*
 * ofsc_unrolled_grad - the gradient, with respect to the starting block X_0, of f1 (Eq. (2)) at
 * the block X_T reached by T updates of OFM-f1 (Algorithm 2 with the exact line search of
 * Eq. (15), beta as Algorithm 2 prints it (no restart), A X recomputed every update, no stopping
 * test).
 *   k        columns (1 <= k <= 128)
 *   X0       device float32 [n x k]
 *   T        updates to differentiate through (0 <= T <= 4096; T = 0 gives grad f1(X_0))
 *   ckpt     checkpoint interval (0: 5): the forward sweep keeps X_t, V_{t-1}, G_{t-1} every ckpt
 *            updates and the reverse sweep recomputes one segment at a time, so the working set is
 *            about 4 ckpt + 13 + 3 T / ckpt row blocks of n x k FP32 (k padded to a multiple of 8).
 *            The result does not depend on ckpt (the recomputation repeats the same arithmetic).
 *   m, src, dst  the edge list the (weighted) graph was built from, device int32 [m]; used only
 *            with grad_w
 *   f_out    HOST double* (nullable): f1(X_T)
 *   grad     device float32 [n x k] (nullable): d f1(X_T) / d X_0
 *   grad_w   device float32 [m] (nullable; weighted graphs only): d f1(X_T) / d w_e for every
 *            listed edge, with A depending on the weights through S and D (listings of one pair
 *            share a value, self-loops get 0), as for ofsc_weight_grad
 * The step alpha_t is differentiated through the implicit-function theorem on the cubic, beta_t
 * through its quotient (a column whose denominator is 0 carries no derivative), G_t through
 * its Hessian-vector product; for grad_w, A's adjoint collects 4 Gbar_t X_t^T from every G_t,
 * c_t V_t X_{t+1}^T from every step's cubic and f1(X_T)'s own term, and is mapped to the
 * weights per stored entry (an SDDMM per update). Allocates its working set for the call.
 * Synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG (also grad_w on an unweighted graph, an endpoint outside [0, n)),
 * OFSC_ERR_OOM, OFSC_ERR_NONFINITE (non-finite value, or a step whose cubic has zero slope at
 * its root, where the step is not differentiable), OFSC_ERR_CUDA.
 */
ofsc_status ofsc_unrolled_grad(ofsc_graph* g, int32_t k, const float* X0, int32_t T, int32_t ckpt,
                               int64_t m, const int32_t* src, const int32_t* dst, double* f_out,
                               float* grad, float* grad_w, void* stream);

/*
 * ofsc_state_create - an empty CG state for ofsc_iterate on graph g with k columns (opts.state):
 * the last direction V_{t-1}, gradient G_{t-1}, V's column scales and V_{t-1}^T V_{t-1} of a run
 * of Algorithm 2, with its update count t and ||G_0||. Owns 8 n kp + 8 kp (kp + 1) bytes of device
 * memory (kp = k rounded up to a multiple of 8) on g's device; usable with g (or a graph of the
 * same n) and the same k and method. Resuming continues the CG recurrence exactly (Algorithm 2
 * as one run); the first update of a resumed call evaluates G_t from an exact A X, as every call
 * does at its start. Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_OOM, OFSC_ERR_CUDA.
 */
ofsc_status ofsc_state_create(const ofsc_graph* g, int32_t k, ofsc_state** out);
ofsc_status ofsc_state_free(ofsc_state* st);
/* t_out: updates of the run the state holds (0: empty); bytes_out: size of its host image. */
ofsc_status ofsc_state_info(const ofsc_state* st, int64_t* t_out, int64_t* bytes_out);
/* The state to a HOST buffer of exactly ofsc_state_info's bytes (a checkpoint), and back into a
 * state created for the same n and k (load checks the image's header: OFSC_ERR_INVALID_ARG on a
 * mismatch). Both synchronise `stream`. */
ofsc_status ofsc_state_save(const ofsc_state* st, void* host, int64_t bytes, void* stream);
ofsc_status ofsc_state_load(ofsc_state* st, const void* host, int64_t bytes, void* stream);

/*
 * ofsc_autotune/*
 * ofsc_autotune - picks, by timing, the shape of the direction product (the sparse product of
 * Sec. 3.3, the largest part of an update of Algorithm 2) for this graph, k columns and the given
 * gather storage: how finely its rows are split among warps (4, 8, 16 or 32 warps per SM, coarser
 * ones only while each warp keeps at least 16 nonzeros) and how many row gathers each lane keeps
 * in flight (2, 4, 6 or 8, as many as one step of at most 32 nonzeros allows), and, for each number
 * of warps, the merge-path split (equal shares of rows + nonzeros, default gathers in flight). Every
 * combination is timed (3 launches after one warm-up); the fastest is kept in the handle and used
 * by every later call on it with the same padded k and gather storage whose merge_path option is 0.
 * Each warp sums its rows' share of diag(V^T AV) before a fixed-order fold, so a new choice can
 * change the last bits of later results (and the split of a long row those of its row of A V).
 *   k         columns (1 <= k <= 128)
 *   gather    OFSC_GATHER_FP32 or OFSC_GATHER_BF16
 *   warps_out HOST int32* (nullable): the chosen number of warps
 *   slots_out HOST int32* (nullable): the chosen gathers in flight per lane
 *   merge_out HOST int32* (nullable): 1 if the merge-path split was chosen, else 0
 *   ms_out    HOST double* (nullable): its time per product in milliseconds
 * Uses the handle's workspace (allocated for k if needed; its blocks are overwritten).
 * Synchronises `stream`. Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_OOM, OFSC_ERR_CUDA.
 */
ofsc_status ofsc_autotune(ofsc_graph* g, int32_t k, int32_t gather, int32_t* warps_out, int32_t* slots_out,
                          int32_t* merge_out, double* ms_out, void* stream);

/*
 * ofsc_weight_grad - gradient of f1 (Eq. (2)) or f2 (Eq. (3)) at X with respect to the weight of
 * every listed edge of a weighted graph: with A_hat = D^-1/2 S D^-1/2 and Gamma = df/dA_hat
 * (2(I + A_hat - X X^T) for f1, -X(2I - X^T X)X^T for f2), a listing e of the pair {a, b}, a != b,
 * gets 2 Gamma_ab / sqrt(d_a d_b) - r_a / d_a - r_b / d_b with r_a = sum_j Gamma_aj A_hat_aj.
 * Listings of the same pair share one value (S sums them); self-loops get 0.
 * g: built with weights from the same edge list. X: device float32 [n x k], 1 <= k <= 128.
 * src, dst: device int32 [m], the edge list given to ofsc_graph_build. grad: device float32 [m],
 * written. Synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG (unweighted graph, NULL pointers, an endpoint outside [0, n)),
 * OFSC_ERR_OOM.
 */
ofsc_status ofsc_weight_grad(ofsc_graph* g, int32_t objective, int32_t k, const float* X, int64_t m,
                             const int32_t* src, const int32_t* dst, float* grad, void* stream);

/*
 * ofsc_rayleigh_ritz - the eigensolver view of a feature block (Sec. 5): Ritz values of
 * B = 2I - L = -A on span(X) and relerr = ||B U - U Lam||_F / ||U Lam||_F with U = X Z the
 * B-Ritz vectors (Z^T X^T X Z = I). Computed from the Grams X^T X, X^T A X (exact A X) by k x k
 * FP64 algebra on the device (Cholesky, cyclic Jacobi) and one row pass for the residual
 * A X - X (X^T X)^-1 X^T A X; U itself is not formed.
 * X: device float32 [n x k] (n = the graph's node count, 1 <= k <= 128), read only, full column
 * rank. ritz: device float64 [k], written with the Ritz values in ascending order. relerr: host,
 * written. Uses the graph's cached workspace; synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG (NULL pointers, k out of range, X rank deficient), OFSC_ERR_OOM,
 * OFSC_ERR_NONFINITE.
 */
ofsc_status ofsc_rayleigh_ritz(ofsc_graph* g, int32_t k, const float* X, double* ritz, double* relerr,
                               void* stream);

/*
 * ofsc_row_normalize - X_l <- X_l / ||X_l||_2 for every row; zero rows stay zero
 * (Algorithm 1, step 3). X is device float32 [n x k], in place. Asynchronous.
 */
ofsc_status ofsc_row_normalize(int64_t n, int32_t k, float* X, void* stream);

/*
 * ofsc_kmeans - Euclidean K-means on the rows of X (Algorithm 1, step 4).
 *   X        device float32 [n x d]
 *   n_clusters  1 <= n_clusters <= n
 *   seed     key of the Philox-4x32-10 stream that drives K-means++ seeding
 *   n_init   independent seeded runs (>= 1); the lowest inertia wins (ties: earlier run)
 *   maxit    maximum Lloyd assignments per run (>= 1)
 *   labels   device int32 [n], receives the cluster of each row
 *   inertia  HOST double* (nullable): sum of squared distances to the assigned centroids
 * Seeding: run r, draw c uses u = word0(Philox4x32-10(ctr = {c, r, 0, 0}, key = {seed_lo,
 * seed_hi})) / 2^32; centre 0 = row floor(u N); centre c = first row whose running sum of D^2
 * exceeds u * sum D^2. Lloyd: nearest centroid (ties: lowest index), stop when no label
 * changes; an empty cluster takes the row farthest from its own centroid. Synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_OOM.
 */
ofsc_status ofsc_kmeans(int64_t n, int32_t d, const float* X, int32_t n_clusters, uint64_t seed,
                        int32_t n_init, int32_t maxit, int32_t* labels, double* inertia,
                        void* stream);

/*
 * ofsc_gram - the k x k dot-product blocks of Sec. 3.3, out_b = L^T R_b (b < nr), summed over all
 * n rows on the tcgen05 tensor cores: each FP32 value is split into two TF32 parts and the three
 * leading products are accumulated in FP32 tensor memory per block of rows; the per-block
 * partials are added in FP64 in a fixed order (deterministic for a given rows_per_block).
 *   n, k     rows and features (1 <= k <= 128)
 *   ld       row stride of L and every R_b in floats (ld >= k, ld % 4 == 0, 16-byte aligned rows)
 *   L        device float32 [n x ld]
 *   nr, R    1 <= nr <= 4; HOST array of nr device pointers, each float32 [n x ld]
 *   rows_per_block  rows per tensor-memory accumulation (multiple of 32), 0 = default
 *   out      device float64 [nr][k][k], row-major
 * Allocates its scratch with cudaMallocAsync on `stream`; synchronises `stream`.
 * Errors: OFSC_ERR_INVALID_ARG, OFSC_ERR_TIMEOUT (a bounded tensor-core wait ran out), OFSC_ERR_CUDA.
 */
ofsc_status ofsc_gram(int64_t n, int32_t k, int32_t ld, const float* L, int32_t nr, const float* const* R,
                      int64_t rows_per_block, double* out, void* stream);

/*
 * ofsc_line_search_step - the step of the exact line search (Sec. 3.2) for n cubics
 * c3 a^3 + c2 a^2 + c1 a + c0 (the derivative of the objective along the direction, up to a
 * positive factor): among the real roots (Cardano's formula, each root polished by two Newton
 * steps), the one where q(a) = c3 a^4/4 + c2 a^3/3 + c1 a^2/2 + c0 a is smallest, ties to the
 * smaller |a| and then the smaller a; 0 when the cubic has no real root or is identically zero.
 * These are the solvers ofsc_iterate runs: solver 0 takes one thread per cubic (the per-column
 * cubics of TriOFM, Eqs. (16)/(18)), solver 1 one warp per cubic, the three roots of a cubic with
 * three real roots in three lanes (the single cubic of OFM, Eqs. (15)/(17)); both give the same
 * bits.
 *   coef   device float64 [n][4], {c3, c2, c1, c0} per cubic
 *   steps  device float64 [n] (written)
 *   bad    device int32 [n] or NULL: 1 where a coefficient is not finite (its step is then 0)
 * Asynchronous on `stream`; allocates nothing.
 * Errors: OFSC_ERR_INVALID_ARG (n < 0, NULL coef or steps with n > 0, solver not 0 or 1),
 * OFSC_ERR_CUDA.
 */
ofsc_status ofsc_line_search_step(int64_t n, const double* coef, int32_t solver, double* steps, int32_t* bad,
                                  void* stream);

/*
 * ofsc_set_allocator - makes the library take every device block it allocates (graph arrays,
 * workspaces, scratch) from the caller's allocator instead of cudaMalloc, for a process whose device
 * memory belongs to another allocator (a framework's caching pool). Not in the paper.
 *   alloc(bytes, user)  returns a device pointer on the current device, 256-byte aligned, or NULL
 *                       when it cannot (the calling entry point then returns OFSC_ERR_OOM and
 *                       frees what it had taken)
 *   free(ptr, user)     returns a block that alloc gave
 *   Both NULL: back to cudaMalloc/cudaFree for later allocations. One of them NULL: INVALID_ARG.
 * A block is always returned to the allocator that made it, also after a later change of
 * allocator. Before calling `free` the library synchronises the device, so no queued kernel still
 * uses the block. Applies process-wide; not thread-safe against concurrent library calls.
 * Errors: OFSC_ERR_INVALID_ARG.
 */
typedef void* (*ofsc_alloc_fn)(size_t bytes, void* user);
typedef void (*ofsc_free_fn)(void* ptr, void* user);
ofsc_status ofsc_set_allocator(ofsc_alloc_fn alloc, ofsc_free_fn free, void* user);

/* Message of the last failing call on this host thread ("" if none). */
const char* ofsc_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t ofsc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OFSC_H */
