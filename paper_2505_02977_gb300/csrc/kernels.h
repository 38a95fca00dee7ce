// kernels.h -- host-side launchers of libparac's device kernels (internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "schedule.h"

namespace parac {

struct ElimArgs;

// Process-wide count of kernels launched by the library (diagnostics).
void count_launches(unsigned n);
void count_graph_launches(unsigned long long n);
void capture_launch_counts(unsigned long long *acc);   // nullptr: count globally again
unsigned long long launch_count();

// ---------------------------------------------------------------- scan.cu
// out[0] = 0, out[i+1] = out[i] + in[i] for i < n (n+1 outputs).  tmp must
// hold scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(int64_t n);
cudaError_t scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t st);

// ---------------------------------------------------------------- ingest.cu
// Ingest flags (OR-ed into the ingest status word; priority in this order).
enum : int32_t { INGEST_BAD_INDEX = 1, INGEST_NOT_SDD = 2, INGEST_KIND = 4 };
// Single input system or a block-diagonal concatenation of systems
// (sys_of_orig / sys_ground_label describe the batch; nullptr = one system).
struct IngestArgs {
    int64_t n;                  // original vertices (all systems)
    const int64_t *colptr;      // [n+1]
    const int32_t *rowind;      // global row indices
    const double *val;
    const int32_t *sys_of_orig; // [n] system of each vertex (nullptr: system 0)
    const int32_t *sys_obase;   // [S] first original vertex of each system
    const int32_t *sys_n;       // [S] vertices per system
    const int32_t *sys_ground;  // [S] ground label of each system (-1: none)
    int32_t single_ground;      // ground label when sys_of_orig == nullptr (-1: none)
    int32_t kind;               // 0 auto, 1 laplacian, 2 sddm
    int32_t *iperm;             // [n] original vertex -> label
    int32_t *lcnt;              // [nl] strict-lower entries per label column
    int32_t *dp;                // [nl] dependency counters (zeroed by caller)
    double *gw;                 // [n] ground-edge weight per original vertex (0 = none)
    int32_t *status;
};

// ordering (global: label k <- original vertex ord[k]); iperm must be filled
// with -1 first.  label_of_k maps position k of the concatenated ordering to
// its label (nullptr: identity).
cudaError_t launch_iperm(int64_t n, const int32_t *ord, const int32_t *label_of_k, int32_t *iperm,
                         int32_t *status, cudaStream_t st);
cudaError_t launch_identity_iperm(int64_t n, int32_t *iperm, cudaStream_t st);
cudaError_t launch_ingest_count(const IngestArgs &a, cudaStream_t st);
cudaError_t launch_ingest_scatter(const IngestArgs &a, const int64_t *lcp, int32_t *lrow, double *lw,
                                  cudaStream_t st);
cudaError_t launch_queue_init(int32_t nl, const int32_t *dp, int32_t *queue, uint32_t *q_tail, cudaStream_t st);
cudaError_t launch_add_offset_i32(const int32_t *in, int32_t *out, int64_t n, int32_t off, cudaStream_t st);
cudaError_t launch_add_offset_i64(const int64_t *in, int64_t *out, int64_t n, int64_t off, cudaStream_t st);
cudaError_t launch_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t st);
cudaError_t launch_iota_i32(int32_t *p, int64_t n, int32_t base, cudaStream_t st);
// NNZ-sorted ordering (ascending stored entries per column, ties by a seeded
// splitmix64 key, then index) of n vertices, or of each system of a batch
// (sys_of_v / sys_obase non-null: keys use local indices, systems stay in
// order); ord receives global vertex indices; tmp holds nnz_order_tmp_bytes(n).
size_t nnz_order_tmp_bytes(int64_t n);
cudaError_t nnz_sorted_order(int64_t n, const int64_t *colptr, const int32_t *sys_of_v, const int32_t *sys_obase,
                             int32_t nsys, uint64_t seed, int32_t *ord, void *tmp, cudaStream_t st);

// ---------------------------------------------------------------- elim.cu
size_t elim_smem_bytes(int warps_per_block, int warp_cap, int block_cap);
cudaError_t elim_configure(int warps_per_block, int warp_cap, int block_cap, int *blocks_per_sm);
cudaError_t elim_launch(const ElimArgs &a, int blocks, int warps_per_block, int fchunk, cudaStream_t st);

// ---------------------------------------------------------------- compact.cu
// out_of_label: label -> output column (-1 for ground labels).
cudaError_t launch_out_len(int32_t nl, const int32_t *out_of_label, const int64_t *f_start, const int32_t *f_len,
                           const int32_t *f_row, int32_t *olen, cudaStream_t st);
cudaError_t launch_gather_factor(int32_t nl, const int32_t *out_of_label, const int64_t *f_start,
                                 const int32_t *f_row, const double *f_val, const double *D, const int64_t *fcp,
                                 int32_t *Frow, double *Fval, double *Dout, cudaStream_t st);
cudaError_t launch_out_of_label_single(int32_t nl, int32_t n, int32_t *out_of_label, cudaStream_t st);
cudaError_t launch_out_of_label_batch(int32_t nl, const int32_t *sys_of_label, const int32_t *sys_lbase,
                                      const int32_t *sys_obase, const int32_t *sys_n, int32_t *out_of_label,
                                      cudaStream_t st);
cudaError_t launch_row_count(int64_t nnz, const int32_t *rows, int32_t *cnt, cudaStream_t st);
cudaError_t launch_transpose_scatter(int32_t n, const int64_t *cp, const int32_t *rows, const double *vals,
                                     const int64_t *rp, int32_t *cursor, int32_t *cols_out, double *vals_out,
                                     cudaStream_t st);
cudaError_t launch_sort_rows(int32_t n, const int64_t *rp, int32_t *cols, double *vals, cudaStream_t st);
// rows of 257..2048 entries (launch_sort_rows sorts those up to 256)
cudaError_t launch_sort_long_rows(int32_t n, const int64_t *rp, int32_t *cols, double *vals, cudaStream_t st);
// Stable sort of n (key, value) pairs by the low key_bits bits of the
// non-negative keys (LSD radix, 8 bits per pass), in place; tmp holds
// radix_tmp_bytes(n) bytes.
size_t radix_tmp_bytes(int64_t n);
cudaError_t stable_sort_pairs(int32_t n, int32_t *keys, int32_t *vals, int key_bits, void *tmp, cudaStream_t st);
// CSR rows of more than 2,048 entries sorted by column (a segmented sort:
// by column, then stably by row).  huge_rows_count finds them with scans in
// tmp (huge_rows_tmp_bytes(n)) and returns their number and total entries;
// huge_rows_sort then sorts them with `work` of huge_rows_sort_bytes bytes.
size_t huge_rows_tmp_bytes(int64_t n);
cudaError_t huge_rows_count(int32_t n, const int64_t *rp, void *tmp, int64_t *nrows, int64_t *entries,
                            cudaStream_t st);
size_t huge_rows_sort_bytes(int64_t nrows, int64_t entries);
cudaError_t huge_rows_sort(int32_t n, const int64_t *rp, int32_t *cols, double *vals, const void *tmp, int64_t nrows,
                           int64_t entries, void *work, cudaStream_t st);
cudaError_t launch_scatter_levels(int32_t nl, const int32_t *out_of_label, const int32_t *lvl, int32_t *lev_out,
                                  cudaStream_t st);
cudaError_t launch_max_i32(const int32_t *a, int64_t n, int32_t *mx, cudaStream_t st);
cudaError_t launch_inverse_perm(int32_t n, const int32_t *order, int32_t *posof, cudaStream_t st);
cudaError_t launch_relabel_lengths(int32_t n, const int32_t *order, const int64_t *cp, int32_t *len, cudaStream_t st);
cudaError_t launch_relabel_gather(int32_t n, const int32_t *order, const int32_t *posof, const int64_t *cp,
                                  const int32_t *rows, const double *vals, const int64_t *ncp, int32_t *nrows,
                                  double *nvals, cudaStream_t st);
cudaError_t launch_gather_i32(int32_t n, const int32_t *idx, const int32_t *src, int32_t *dst, cudaStream_t st);
cudaError_t launch_gather_f64(int32_t n, const int32_t *idx, const double *src, double *dst, cudaStream_t st);
cudaError_t launch_to_f32(const double *in, float *out, int64_t n, cudaStream_t st);
cudaError_t launch_dinv(int32_t n, const double *D, double *Dinv, cudaStream_t st);
cudaError_t launch_sys_of_label(int32_t S, const int32_t *sys_lbase, int32_t nl, int32_t *sys_of_label,
                                cudaStream_t st);

// ---------------------------------------------------------------- solve.cu
// device-resident scalars of one PCG run (solve.cu)
struct PcgState {
    double rz, alpha, beta, bb, rr, tol2bb, true_rr, pad0;
    int32_t done, iters, maxit, converged;
};

struct SolveArgs {
    int32_t n;                    // rows (original numbering)
    // the matrix (symmetric CSC = CSR)
    const int64_t *Lp; const int32_t *Li; const double *Lv;
    // factor relabelled into dependency-level order (position space)
    const int64_t *Fcp; const int32_t *Frow; const double *Fval64; const float *Fval32;   // CSC (backward)
    const int64_t *Frp; const int32_t *Fcol; const double *Fvalr64; const float *Fvalr32; // CSR (forward)
    const double *Dinv;           // [n] 1/D or 0, by position
    const int32_t *operm;         // [n] original index of each position
    int32_t prec;                 // 64 or 32
    int32_t lanes_spmv;           // lanes per row for SpMV (4, 8, 16, 32)
    int32_t lanes_trsv;           // lanes per row for the triangular solves
    int32_t trsv_blocks;          // persistent grid of the triangular solves
    int32_t trsv_warps;           // warps per block of the triangular solves
    int32_t tpr_blocks;           // > 0: one lane per row (thread-per-row solves) on this many blocks of 256
    const int2 *tpr_chunks;       // their chunks: (first position, rows <= 32), never across a level
    int32_t ntpr;
    long long spin_limit;
    int32_t *status;
    // optional group tables of the one-row-per-warp solves (row_groups with the
    // _SINGLE sizes and trsv_warps warps); nullptr: fixed groups of rows
    const int4 *gt_f, *gt_b;
    int32_t ng_f, ng_b;
    void *part_f, *part_b;        // partial sums of split rows (XT), nslot_f / nslot_b
    int32_t nslot_f, nslot_b;
    // batched solves: stop flag of each system (groups of a stopped system are
    // skipped); the tables then carry the system in the kind's upper bits and
    // the solves run one row per warp.  nullptr: none.
    const int32_t *skip;
};

// one right-hand side: rows above LONG_ROW_SINGLE entries get a block, above
// SPLIT_ROW_SINGLE they are split into chunks of CHUNK_SINGLE; block solves
// (nrhs columns, 32 x the bytes per entry) use the _BLOCK sizes
constexpr int LONG_ROW_SINGLE = 512, SPLIT_ROW_SINGLE = 32768, CHUNK_SINGLE = 8192;
constexpr int LONG_ROW_BLOCK = 64, SPLIT_ROW_BLOCK = 1024, CHUNK_BLOCK = 512;
constexpr int SOLVE_WARPS = 8;        // warps per block of the solves (default)
// Group table of the one-row-per-warp solves (row_groups of schedule.cpp)
// built on the device: row_groups_count runs the scans in tmp
// (row_groups_tmp_bytes(n)) and returns the group and slot counts;
// row_groups_write then fills table[4 * ngroups] from the same tmp.
size_t row_groups_tmp_bytes(int64_t n);
cudaError_t row_groups_count(const int64_t *ptr, int64_t n, bool descending, int warps, int long_row, int split_row,
                             int chunk, void *tmp, int64_t *ngroups, int64_t *nslots, cudaStream_t st);
cudaError_t row_groups_write(const int64_t *ptr, int64_t n, bool descending, int warps, int split_row, int chunk,
                             const void *tmp, int32_t *table, cudaStream_t st);
// thread-per-row solves: used for factors whose rows and columns all have at
// most TPR_MAX_ROW entries; blocks of 256 threads
constexpr int TPR_MAX_ROW = 2048, TPR_THREADS = 256;
int tpr_blocks_per_sm(int prec);

struct PcgBuffers {
    double *x, *r, *z, *p, *q, *b;  // [n]
    double *yl64, *zl64;            // label-space work (FP64 apply)
    float *yl32, *zl32;             // label-space work (FP32 apply)
    double *partials;               // [3 * pstride]
    PcgState *state;
    int32_t vec_blocks;             // grid of the vector kernels
    int32_t pstride;                // >= max(vec_blocks, trsv_blocks)
};

size_t pcg_state_bytes();
cudaError_t set_poll_backoff(unsigned max_ns);
cudaError_t pcg_init(const SolveArgs &A, const PcgBuffers &B, double tol, int32_t maxit, cudaStream_t st);
cudaError_t pcg_iteration(const SolveArgs &A, const PcgBuffers &B, cudaStream_t st);
cudaError_t pcg_true_residual(const SolveArgs &A, const PcgBuffers &B, cudaStream_t st);
// host view of the scalars after a sync
struct PcgHostState { int32_t done; int32_t iters; double rr; double bb; double true_rr; int32_t maxit; };
cudaError_t pcg_read_state(const PcgBuffers &B, PcgHostState *h, cudaStream_t st);
cudaError_t pcg_clear_done(const PcgBuffers &B, cudaStream_t st);
cudaError_t pcg_resume(const SolveArgs &A, const PcgBuffers &B, cudaStream_t st);
cudaError_t precond_apply(const SolveArgs &A, const PcgBuffers &B, const double *r, double *z, cudaStream_t st);
// ---------------------------------------------------------------- block.cu
// PCG on nrhs <= 32 right-hand sides at once: row-major n x nrhs blocks, one
// lane per column, per-column scalars and stopping.
struct BlockState;
struct BlockBuffers {
    double *x, *r, *z, *p, *q, *b;  // [n * nrhs] row-major
    double *yl64, *zl64;            // [n * nrhs] position-space unknowns (FP64 apply)
    float *yl32, *zl32;             // [n * nrhs] (FP32 apply)
    double *partials;               // [3 * 32 * pstride]
    BlockState *state;
    const int4 *gt_f, *gt_b;        // group tables of the forward / backward SpTRSM
    int32_t ng_f, ng_b;
    void *part_f, *part_b;          // partial sums of split rows: nslot_* x 32 values (XT)
    int32_t nslot_f, nslot_b;
    int32_t nrhs;
    int32_t vec_blocks;             // grid of the vector kernels
    int32_t pstride;                // >= max(vec_blocks, trsv grid)
};
struct BlockHostState {
    int32_t all_done;
    int32_t iters[32], converged[32], done[32];
    double bb[32], true_rr[32];
};
size_t block_state_bytes();

int btrsm_blocks_per_sm(int warps, int prec);
cudaError_t bpack(int32_t n, int nrhs, const double *B, int64_t ldb, double *Bt, cudaStream_t st);
cudaError_t bunpack(int32_t n, int nrhs, const double *Xt, double *X, int64_t ldx, cudaStream_t st);
cudaError_t bpcg_init(const SolveArgs &A, const BlockBuffers &B, double tol, int32_t maxit, cudaStream_t st);
cudaError_t bpcg_iteration(const SolveArgs &A, const BlockBuffers &B, cudaStream_t st);
cudaError_t bpcg_true_residual(const SolveArgs &A, const BlockBuffers &B, cudaStream_t st);
cudaError_t bpcg_reopen(const SolveArgs &A, const BlockBuffers &B, cudaStream_t st);
cudaError_t bpcg_read_state(const BlockBuffers &B, BlockHostState *h, cudaStream_t st);

cudaError_t solve_spmv(const SolveArgs &A, const double *x, double *y, const PcgState *st, int blocks, cudaStream_t s);
cudaError_t solve_apply(const SolveArgs &A, const PcgBuffers &B, const double *r, double *z, const PcgState *st,
                        cudaStream_t s);
cudaError_t solve_fill_sentinels(const SolveArgs &A, const PcgBuffers &B, cudaStream_t s);

// ---------------------------------------------------------------- batch.cu
// PCG on many systems at once (one right-hand side each): the systems' factors
// concatenated (global positions, rows interleaved by dependency level in the
// schedule table), per-system scalars and stopping, dot products over fixed
// row chunks that never straddle two systems.
struct SysState {
    double rz, alpha, beta, bb, rr, tol2bb, true_rr, pad0;
    int32_t done, iters, converged, pad1;
};
struct BatchState {
    PcgState gate;                // gate.done = every system stopped (gates the shared kernels)
    int32_t count, maxit, pad0, pad1;
};
struct BatchBuffers {
    int32_t count;                // systems
    int32_t nchunks;              // row chunks
    const int64_t *clo;           // [nchunks + 1] chunk row bounds (original order)
    const int32_t *csys;          // [nchunks] system of each chunk
    const int32_t *sys_c0;        // [count + 1] first chunk of each system
    double *x, *r, *z, *p, *q, *b;   // [n] concatenated vectors
    int32_t *stop;                // [count] 1 once a system stopped (read by the solves)
    PcgBuffers solve;             // yl/zl work of the solves
    double *partials;             // [3 * nchunks]
    SysState *sys;                // [count]
    BatchState *st;
    int32_t spmv_blocks;
};
size_t batch_state_bytes();
cudaError_t spcg_init(const SolveArgs &A, const BatchBuffers &B, double tol, int32_t maxit, cudaStream_t st);
cudaError_t spcg_iteration(const SolveArgs &A, const BatchBuffers &B, cudaStream_t st);
cudaError_t spcg_true_residual(const SolveArgs &A, const BatchBuffers &B, cudaStream_t st);
cudaError_t spcg_reopen(const SolveArgs &A, const BatchBuffers &B, cudaStream_t st);
// dst[seg.dst + i] = src[i] + seg.add for every segment (elem 4 or 8 bytes;
// integer add, or a plain copy of floats); seg[] in device memory
struct CatSeg { const void *src; int64_t count, dst, add; };
cudaError_t launch_cat(const CatSeg *seg, int32_t nseg, int64_t max_count, int elem, bool is_float, void *dst,
                       cudaStream_t st);
// the inverse: dst_k[i] = src[seg_k.src + i] + seg_k.add, i < seg_k.count (seg[] in device memory)
struct SplitSeg { void *dst; int64_t count, src, add; };
cudaError_t launch_split(const SplitSeg *seg, int32_t nseg, int64_t max_count, int elem, bool is_float,
                         const void *src, cudaStream_t st);
// out[i] = ptr[i][idx[i]] for i < m (ptr, idx, out in device memory)
cudaError_t launch_gather_ends(const int64_t *const *ptr, const int64_t *idx, int32_t m, int64_t *out,
                               cudaStream_t st);
// out[seg_of[i]] = max(out[..], val[i]); hist[seg_off[seg_of[i]] + val[i]] += 1
cudaError_t launch_seg_max(int64_t n, const int32_t *val, const int32_t *seg_of, int32_t *out, cudaStream_t st);
cudaError_t launch_seg_hist(int64_t n, const int32_t *val, const int32_t *seg_of, const int64_t *seg_off,
                            int32_t *hist, cudaStream_t st);
// Allocation-free variant: work vectors in a fixed device array (n <= NOALLOC_MAX_N).
constexpr int NOALLOC_MAX_N = 1 << 18;
constexpr int NOALLOC_MAX_DEVICES = 64;
cudaError_t precond_apply_noalloc(const SolveArgs &A, const double *r, double *z, cudaStream_t st);
int trsv_configure(int lanes, int warps, int *blocks_per_sm, int prec, bool skip = false);

}  // namespace parac
