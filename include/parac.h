/*
 * parac.h -- C ABI of libparac: randomized approximate Cholesky (rchol's
 * elimination, scheduled by ParAC's dynamic dependency tracking) and PCG,
 * on one GB300 GPU (sm_103a).
 *
 * Problem statement (ParAC paper, Sec. I, Eq. 1-2): solve L x = b for a graph
 * Laplacian or SDDM matrix L, using a randomized factor L ~ G G^T as the PCG
 * preconditioner.  The factor is kept in the scaled form of Sec. IV:
 * L ~ F D F^T with F unit lower triangular and D diagonal (G = F D^{1/2}).
 *
 * Conventions shared by every entry point
 *   Matrices    Full symmetric CSC: colptr int64[n+1] (colptr[0] = 0,
 *               non-decreasing), rowind int32[nnz] in [0, n), val double[nnz].
 *               Sign convention of Sec. V: positive diagonal, off-diagonal
 *               entries <= 0 (explicit zeros are ignored).  Both triangles
 *               must be stored; the library reads the strict lower triangle
 *               in elimination-label order and the column sums.
 *   Pointers    Every array argument may be host or device memory; the
 *               library checks which with cudaPointerGetAttributes and copies
 *               host data itself.  Inputs are read during the call only; the
 *               caller keeps ownership.  Output arrays are written only on
 *               PARAC_OK.
 *   Handles     parac_factor_t is owned by the library; release it with
 *               parac_factor_free.  A handle is bound to the device that was
 *               current when it was created.
 *   Streams     All device work of a call is ordered on opts->stream (the
 *               legacy default stream if NULL); calls return after that work
 *               has completed.
 *   Errors      Every call returns a parac_status; no exception crosses the
 *               ABI.  parac_last_error() gives a thread-local message.
 *   Determinism The factor (F, D) is a deterministic function of (L,
 *               ordering, seed, kind) whatever the GPU schedule: it is
 *               bit-identical to a sequential elimination in label order.
 */
#ifndef PARAC_H
#define PARAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct parac_factor_s *parac_factor_t;

typedef enum {
    PARAC_OK = 0,
    PARAC_EINVAL = 1,    /* malformed arguments, ordering not a permutation, kind mismatch */
    PARAC_ENOT_SDD = 2,  /* positive off-diagonal entry or negative row excess */
    PARAC_ENOMEM = 3,    /* device or host allocation failed */
    PARAC_EPOOL = 4,     /* fill workspace still overflowed after the allowed regrowths */
    PARAC_ETIMEOUT = 5,  /* a device wait exceeded opts->spin_limit polls (watchdog) */
    PARAC_ECUDA = 6,     /* a CUDA runtime call failed */
    PARAC_ENOCONV = 7    /* PCG reached maxit before the tolerance (outputs still written) */
} parac_status;

enum { PARAC_KIND_AUTO = 0, PARAC_KIND_LAPLACIAN = 1, PARAC_KIND_SDDM = 2 };
/* Triangular-solve strategies (all sync-free, rows in dependency-level
 * order): WARP gives each row a warp of 32 lanes (and a whole block to a row
 * of more than 512 entries); SUB8 / SUB4 give each row 8 / 4 lanes, so a warp
 * works on 4 / 8 short rows at once; THREAD is the hybrid: a dependency level
 * with more rows than the solve grid has warps is cut into runs of up to 32
 * rows, one lane per row (rows of more than 64 entries go to the whole warp),
 * and every row of a narrower level gets a warp (for factors without rows or
 * columns of more than 2048 entries; others fall back to WARP).  AUTO is
 * THREAD where it applies, else WARP. */
enum { PARAC_SPTRSV_AUTO = 0, PARAC_SPTRSV_WARP = 1, PARAC_SPTRSV_SUB8 = 2, PARAC_SPTRSV_SUB4 = 3,
       PARAC_SPTRSV_THREAD = 4 };
/* Tri-state switches of parac_opts: 0 = the library default. */
enum { PARAC_DEFAULT = 0, PARAC_ON = 1, PARAC_OFF = 2 };
/* Elimination order: the caller's ordering array (NULL = identity), or Sec.
 * V's NNZ-sorted ordering computed on the device (the ordering array must
 * then be NULL). */
enum { PARAC_ORDER_GIVEN = 0, PARAC_ORDER_NNZ = 1 };

/*
 * Options.  parac_opts_default() fills the defaults; a NULL opts pointer
 * means the defaults.
 *   kind            AUTO: SDDM when some row excess exceeds 1e-12 of its
 *                   diagonal, else Laplacian.  SDDM rows with positive excess
 *                   get an edge to a ground node labelled last (Sec. V); the
 *                   ground row and column are removed from the factor.
 *   g_precision     64: PCG applies F in FP64.  32: F values are stored as
 *                   FP32 and the triangular solves run in FP32, while PCG's
 *                   SpMV, residual update and dot products stay FP64.
 *   pool_mult       Initial fill-workspace capacity, in units of the strict
 *                   lower input entries; 0 (default) picks 5, or 10 when the
 *                   longest lower column exceeds 16x the average (grids use
 *                   ~3.5, R-MAT graphs ~8 with the overflow slabs' rounding;
 *                   an overflow reruns the whole elimination, larger).
 *   max_pool_regrow Reruns with a 2x larger workspace after an overflow (the
 *                   rerun gives the same factor).
 *   spin_limit      Polls any device wait may take before PARAC_ETIMEOUT
 *                   (0: library default, 2^24).  Waits on the ready queue
                   count only polls during which no vertex was published.
 *   warps_per_block, blocks, queue_chunk, big_threshold
 *                   Elimination schedule (0 = autotuned/default): worker warps
 *                   per CTA, CTAs (0 = all co-resident), ready-queue slots a
 *                   worker claims at once, gathered-entry count above which a
 *                   vertex leaves the per-warp shared-memory path.
 *   sptrsv          Triangular-solve strategy (PARAC_SPTRSV_*).
 *   check_every     PCG iterations between host convergence checks (0 = 8).
 *   stream          cudaStream_t to order all work on.
 *   timing          Nonzero: record per-phase device times in the stats.
 *   samples         Samples drawn per clique-tree slot (0 or 1: Alg. 2).  k > 1
 *                   is per-slot multi-sampling MS(k): every slot p of every
 *                   pivot draws k neighbours, sample q with Philox counter
 *                   (k_label, p, sys, q), each edge weighted c_p / k -- a denser
 *                   factor for fewer iterations.  MS(k) is this library's
 *                   variant, not Sec. VI's AC(2), which doubles the samples
 *                   of the input's own entries only: MS(k) also multiplies
 *                   the samples of fill entries.
 *   fill_store      Where fill waits for its column's pivot: 0 = per-column
 *                   slabs (inline 16 entries, then geometrically growing
 *                   overflow slabs); 1 = the hashmap W of Sec. IV-C (open
 *                   addressing: an entry of column c is inserted from step
 *                   fill_count(c) of c's probe sequence hash(c), hash(c) + s_c,
 *                   ... with a per-column odd stride s_c, and gathered by
 *                   parallel scans of that sequence).  The factor is the same
 *                   either way.
 * Finer elimination schedule (0 = default; none changes the factor):
 *   block_cap       entries of a CTA's shared working-set buffer, rounded up
 *                   to a power of two in [256, 8192] (default: 2048, or less
 *                   when it would cost resident blocks)
 *   coop            PARAC_ON / PARAC_OFF: a working set above the warp buffer
 *                   is eliminated by all warps of the CTA (default on) or by
 *                   its warp alone through global scratch
 *   sample_sort     PARAC_ON / PARAC_OFF: sample sort for working sets held
 *                   in global scratch (default on) instead of bitonic sorts
 *   idle_ns         sleep of a worker that found no ready vertex (default 512)
 *   trace_path      NULL (default), or a file that receives one line per
 *                   vertex: ready / start / end times, gathered and merged
 *                   sizes, the pivot that made it ready and its level
 * Solve schedule (kept in the handle; none changes the preconditioner beyond
 * the order of the row sums):
 *   trsv_blocks     persistent grid of the triangular solves (0: sized to
 *                   the dependency frontier; capped at the co-resident blocks)
 *   poll_ns         cap of the solves' polling back-off in ns (0: 64)
 *   pcg_graph       PARAC_ON / PARAC_OFF: parac_pcg replays its iterations
 *                   from a captured CUDA graph (default on) or launches them
 *   pcg_many        parac_pcg_many (read from the first handle): PARAC_ON /
 *                   default = one block-diagonal solve when the handles allow
 *                   it; PARAC_OFF = one parac_pcg per system on worker threads
 *   pcg_workers     worker threads of that per-system path (0: 4)
 *   order           PARAC_ORDER_GIVEN (default) or PARAC_ORDER_NNZ: vertices
 *                   by ascending count of stored entries in their column
 *                   (Sec. V, the paper's choice for the GPU), ties by the top
 *                   31 bits of the (v+1)-th output of a splitmix64 generator
 *                   started from `seed` (v = the vertex's index in its
 *                   system), then by v; each system of a batch separately.
 *   grid_help       a vertex whose working set lives in global scratch (more
 *                   gathered entries than the CTA buffer) is offered to the
 *                   grid's idle warps, which take chunks of its gather,
 *                   sorts, scan, sampling and counter releases while its CTA
 *                   runs the serial steps; one such vertex at a time.
 *                   Default: on for hub-dominated inputs (longest lower
 *                   column above 16x the average); PARAC_ON / PARAC_OFF
 *                   force it.  The factor is the same either way.
 *   grid_help_min   gathered entries from which a vertex is offered (0: every
 *                   working set in global scratch)
 *   host_tables     PARAC_ON: the group tables of the warp-per-row solves
 *                   (factors with rows of more than 2,048 entries) are built
 *                   by a host pass over the factor's pointers, as a reference
 *                   for the default device builder; the tables are the same.
 */
typedef struct {
    int32_t kind;
    int32_t g_precision;
    double pool_mult;
    int32_t max_pool_regrow;
    int32_t warps_per_block;
    int64_t spin_limit;
    int32_t blocks;
    int32_t queue_chunk;
    int32_t big_threshold;
    int32_t sptrsv;
    int32_t check_every;
    int32_t timing;
    void *stream;
    int32_t samples;
    int32_t fill_store;
    int32_t block_cap;
    int32_t coop;
    int32_t sample_sort;
    int32_t idle_ns;
    const char *trace_path;
    int32_t trsv_blocks;
    int32_t poll_ns;
    int32_t pcg_graph;
    int32_t pcg_many;
    int32_t pcg_workers;
    int32_t order;
    int32_t grid_help;
    int32_t grid_help_min;
    int32_t host_tables;
} parac_opts;

void parac_opts_default(parac_opts *opts);

/*
 * parac_factor -- randomized approximate Cholesky of one matrix
 * (Alg. 1 with Alg. 2 per pivot, run by the dependency-counter schedule of
 * Sec. III on the GPU, Alg. 4's structure re-derived for sm_103a).
 *   n         order of L (0 <= n < 2^31 - 1)
 *   colptr, rowind, val   L in the convention above
 *   ordering  ordering[k] = original vertex eliminated k-th (a permutation of
 *             0..n-1); NULL means the identity.  Labels are positions in
 *             this ordering.
 *   seed      keys the Philox4x64-10 stream: slot p of pivot k draws counter
 *             (k, p, 0, 0) under key (seed, 0).
 *   opts      NULL for defaults.
 *   out       receives a new handle on PARAC_OK (NULL otherwise).
 * Errors: EINVAL, ENOT_SDD, ENOMEM, EPOOL, ETIMEOUT, ECUDA.
 */
parac_status parac_factor(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                          const int32_t *ordering, uint64_t seed, const parac_opts *opts,
                          parac_factor_t *out);

/*
 * parac_pcg -- preconditioned conjugate gradients for L X = B (Sec. V),
 * preconditioner M^{-1} = P^T F^{-T} D^+ F^{-1} P (D^+ skips zero pivots).
 *   G         handle from parac_factor / parac_factor_many
 *   n, colptr, rowind, val   the matrix to solve with (normally the one that
 *             was factored); colptr == NULL uses the device copy kept in G.
 *   B         n x nrhs right-hand sides, column-major, leading dimension ldb
 *   nrhs      1..32
 *   tol       stop when ||r_j|| <= tol ||b_j|| for the recurrence residual
 *             and then for the recomputed true residual b_j - L x_j
 *   maxit     iteration cap (per right-hand side)
 *   X         n x nrhs output, column-major, leading dimension ldx (x0 = 0)
 *   iters     [nrhs] iterations taken (may be NULL)
 *   true_relres [nrhs] ||b_j - L x_j|| / ||b_j|| at exit (may be NULL)
 * For singular Laplacians each b_j must be orthogonal to the constant vector.
 * Returns PARAC_ENOCONV (with X, iters, true_relres written) when some
 * right-hand side has not converged within maxit.
 */
parac_status parac_pcg(parac_factor_t G, int64_t n, const int64_t *colptr, const int32_t *rowind,
                       const double *val, const double *B, int32_t nrhs, int64_t ldb, double tol,
                       int32_t maxit, double *X, int64_t ldx, int32_t *iters, double *true_relres);

/* One system of a batch. */
typedef struct {
    int64_t n;
    const int64_t *colptr;
    const int32_t *rowind;
    const double *val;
    const int32_t *ordering;   /* NULL = identity */
} parac_system;

/*
 * parac_factor_many -- factor `count` independent systems in ONE persistent
 * elimination launch sharing one ready queue (batched form of Alg. 4).
 * System s draws its randomness from counter (k, p, s, 0) under key
 * (seed, 0), so its factor equals the one a sequential elimination of that
 * system alone with system index s gives.  out[s] receives the handles
 * (all NULL on error).  Errors as parac_factor.
 */
parac_status parac_factor_many(int32_t count, const parac_system *systems, uint64_t seed,
                               const parac_opts *opts, parac_factor_t *out);

/*
 * parac_precond_apply -- z = M^{-1} r = P^T F^{-T} D^+ F^{-1} P r with the
 * factor in G (the preconditioner PCG applies; Sec. IV scaled form, D^+ = 0
 * on zero pivots).  r and z are n-vectors in the original numbering, host or
 * device memory.  Errors: EINVAL, ETIMEOUT, ECUDA.
 */
parac_status parac_precond_apply(parac_factor_t G, const double *r, double *z);

/*
 * parac_precond_apply_noalloc -- the same z = M^{-1} r as parac_precond_apply
 * (same kernels, same result), for callers that cannot allocate device memory
 * when they need the preconditioner: code that must not enter a memory
 * allocator once its solve loop is running (fixed memory budgets, latency-
 * critical inner loops, host code driving its own Krylov method around an
 * allocator it does not control).  The ParAC paper has no counterpart; this
 * entry point is an interface convenience of this library.
 *   Allocation  none: the two work vectors of the triangular solves live in a
 *               fixed device array of 4 MiB inside the library (every GPU
 *               that loads the library holds it until the process exits).
 *   Limit       the factor's order n must be at most 262,144 (2^18);
 *               larger factors return PARAC_EINVAL.
 *   Pointers    r and z are n-vectors of DEVICE memory in the original
 *               numbering; host pointers return PARAC_EINVAL.
 *   Set-up      the first call on a device looks up the array's device
 *               address (cudaGetSymbolAddress) with that device current;
 *               make that first call before any stream capture.
 *   Sharing     every call uses the same array and leaves the last call's
 *               values in it (each call resets what it reads); calls whose
 *               work overlaps on the GPU (other streams, other threads) race
 *               on it and must be serialised by the caller.
 * Errors: EINVAL, ETIMEOUT, ECUDA.
 */
parac_status parac_precond_apply_noalloc(parac_factor_t G, const double *r, double *z);

/*
 * parac_autotune -- choose the schedule for a class of inputs by timing
 * candidates on representative systems (the batched form's autotuned
 * schedule).  The factor never depends on the schedule, so tuning changes
 * only time.
 *   count, systems, seed   as for parac_factor_many (count >= 1)
 *   base      options to start from (NULL: defaults); kind, precision,
 *             workspace sizes and stream are kept
 *   best      receives base with warps_per_block, queue_chunk, big_threshold
 *             (timed on parac_factor_many) and sptrsv (timed on
 *             parac_precond_apply with the fastest factor) set
 *   report    optional JSON of every candidate's time, cap bytes (NULL / 0:
 *             none)
 * Factors and work space made while tuning are freed before returning.
 * Errors: EINVAL (also when report is too small), and any error of
 * parac_factor_many or parac_precond_apply.
 */
parac_status parac_autotune(int32_t count, const parac_system *systems, uint64_t seed, const parac_opts *base,
                            parac_opts *best, char *report, size_t cap);

/*
 * parac_pcg_many -- parac_pcg (one right-hand side each, with the matrix kept
 * in each handle) on several factored systems, e.g. the handles of one
 * parac_factor_many call.  Handles on one device with one g_precision are
 * solved as one block-diagonal system: their matrices, factors and vectors
 * are concatenated for the call, every SpMV and triangular-solve launch
 * advances all systems (the solves' schedule interleaves the systems'
 * dependency levels, and skips the systems that already stopped), and each
 * system keeps its own CG scalars, stopping test and true-residual check.  A
 * system's preconditioner applies are the same arithmetic as in its own
 * parac_pcg call; its dot products are reduced over row chunks of its own, so
 * iterates agree with separate calls up to rounding (iteration counts within
 * one).  The batched solves use the hybrid layout of PARAC_SPTRSV_THREAD
 * whenever no handle's factor has a row or column of more than 2048 entries
 * (whatever the handles' sptrsv), else one row per warp.  Otherwise (mixed
 * devices or precisions, or pcg_many = PARAC_OFF in
 * the options the first handle was made with) host worker threads run the
 * systems' parac_pcg calls concurrently, with results equal to separate
 * calls.
 *   count     number of systems; G[count] distinct handles
 *   b[s], x[s]   right-hand side / solution of system s (n_s entries; host or
 *             device memory)
 *   tol, maxit   as for parac_pcg
 *   iters, true_relres   [count] outputs (may be NULL)
 * Returns PARAC_OK when every system converged; otherwise the first error of
 * the lowest-numbered failing system (PARAC_ENOCONV only if no other error),
 * with every system's outputs written.  Device memory for the concatenated
 * system is allocated for the call (about the factors' and matrices' size
 * again) and released before it returns; when it cannot be allocated, the
 * systems are solved by the worker threads instead.
 */
parac_status parac_pcg_many(int32_t count, const parac_factor_t *G, const double *const *b, double *const *x,
                            double tol, int32_t maxit, int32_t *iters, double *true_relres);

/*
 * parac_factor_export -- copy the factor out (label space, ground removed).
 *   nnz       receives the strict-lower entry count of F
 *   colptr    int64[n+1], rowind int32[nnz], Fval double[nnz] (rows ascending
 *             within each column), D double[n]
 * Pass colptr == NULL to query nnz (and n via parac_factor_stats) first.
 * Arrays may be host or device memory.
 */
parac_status parac_factor_export(parac_factor_t G, int64_t *nnz, int64_t *colptr, int32_t *rowind,
                                 double *Fval, double *D);

/*
 * parac_factor_stats -- JSON object with sizes and timings of the factor
 * (n, nnz_F, nnz_G = nnz_F + n, fill entries, pool use, per-phase times in
 * ms when opts->timing was set).  Writes at most cap bytes including the
 * terminating NUL; returns PARAC_EINVAL if cap is too small.
 */
parac_status parac_factor_stats(parac_factor_t G, char *json, size_t cap);

/* Release a handle (NULL is ignored). */
void parac_factor_free(parac_factor_t G);

/* Static description of a status code. */
const char *parac_status_string(parac_status s);

/* Message describing the last failing call on this thread ("" if none). */
const char *parac_last_error(void);

/* Diagnostics: number of GPU kernels this library has launched in the
 * process so far (all threads and devices). */
uint64_t parac_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* PARAC_H */
