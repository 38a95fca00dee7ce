// solve.cu -- PCG with the randomized factor as preconditioner (Sec. V):
// SpMV on L, sync-free triangular solves with F (forward, pull over CSR rows)
// and F^T (backward, pull over CSC columns) around the D^+ scaling, and the
// PCG vector/scalar steps, all on device-resident scalars so that one
// iteration can be captured in a CUDA graph.
//
// Sync-free solves: every unknown starts as a signalling-NaN sentinel (never
// produced by arithmetic); a row's lanes poll the unknowns they need until the
// sentinel is gone, so the value itself is the ready flag.  Rows are visited
// in the order of their dependency level (computed during the elimination:
// the forward solve's DAG is the elimination DAG) -- the factor is relabelled
// into that order once, at setup -- ascending for the forward solve and
// descending for the backward one, handed to a persistent, fully co-resident
// grid in a static round-robin of row groups.  Every dependency sits at an
// earlier position, so the smallest unfinished group never waits on an
// unfinished group and the solve always progresses; every wait is bounded by
// the spin limit.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace parac {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int VEC_THREADS = 256;
__constant__ unsigned g_poll_max_ns = 64;    // cap of the polling back-off

__device__ __forceinline__ double sentinel64() { return __longlong_as_double((long long)0xfff7ffffffffffffull); }
__device__ __forceinline__ float sentinel32() { return __int_as_float((int)0xffbfffffu); }
__device__ __forceinline__ bool is_sentinel(double x) { return __double_as_longlong(x) == (long long)0xfff7ffffffffffffull; }
__device__ __forceinline__ bool is_sentinel(float x) { return __float_as_int(x) == (int)0xffbfffffu; }

template <typename T> __device__ __forceinline__ T sentinel();
template <> __device__ __forceinline__ double sentinel<double>() { return sentinel64(); }
template <> __device__ __forceinline__ float sentinel<float>() { return sentinel32(); }

__device__ __forceinline__ double ld_poll(const double *p) { return ld_relaxed_f64(p); }
__device__ __forceinline__ float ld_poll(const float *p) { return ld_relaxed_f32(p); }
__device__ __forceinline__ void st_pub(double *p, double v) { st_relaxed_f64(p, v); }
__device__ __forceinline__ void st_pub(float *p, float v) { st_relaxed_f32(p, v); }

// block-wide sum; result valid in thread 0
__device__ double block_sum(double v)
{
    __shared__ double ws[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------- SpMV: y = L x (+ partial x.y)
// S lanes per row; a lane group owns rows i, i + R, i + 2R, ... (R = lane
// groups in the grid) and works SPMV_ROWS of them at a time, so that their
// pointer, index/value and x loads are in flight together.  Each row's sum
// is the same in any case: lane sl adds entries sl, sl + S, ... in order,
// then the lanes' sums meet in a fixed shuffle tree.
constexpr int SPMV_ROWS = 4;

template <int S>
__global__ void k_spmv(int32_t n, const int64_t *Lp, const int32_t *Li, const double *Lv, const double *x, double *y,
                       double *partial, const PcgState *st)
{
    if (st && st->done) return;
    const unsigned lane = threadIdx.x & 31;
    const int sub = lane / S, sl = lane % S;
    const unsigned smask = (S == 32) ? FULL : (((1u << S) - 1u) << (sub * S));
    const int64_t R = ((int64_t)gridDim.x * blockDim.x) / S;
    double dotacc = 0.0;
    for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / S; i0 < n; i0 += SPMV_ROWS * R) {
        int64_t b[SPMV_ROWS], e[SPMV_ROWS];
        double acc[SPMV_ROWS];
        int64_t len = 0;
#pragma unroll
        for (int u = 0; u < SPMV_ROWS; ++u) {
            const int64_t i = i0 + u * R;
            b[u] = i < n ? Lp[i] : 0;
            e[u] = i < n ? Lp[i + 1] : 0;
            acc[u] = 0.0;
            len = max(len, e[u] - b[u]);
        }
        for (int64_t k = sl; k < len; k += S) {
            double vv[SPMV_ROWS], xv[SPMV_ROWS];
            int32_t cc[SPMV_ROWS];
#pragma unroll
            for (int u = 0; u < SPMV_ROWS; ++u) {
                const bool in = k < e[u] - b[u];
                cc[u] = in ? Li[b[u] + k] : -1;
                vv[u] = in ? Lv[b[u] + k] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < SPMV_ROWS; ++u) xv[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < SPMV_ROWS; ++u)
                if (cc[u] >= 0) acc[u] += vv[u] * xv[u];
        }
#pragma unroll
        for (int u = 0; u < SPMV_ROWS; ++u) {
            double a = acc[u];
#pragma unroll
            for (int off = S / 2; off > 0; off >>= 1) a += __shfl_xor_sync(smask, a, off);
            const int64_t i = i0 + u * R;
            if (sl == 0 && i < n) {
                y[i] = a;
                dotacc += a * x[i];
            }
        }
    }
    if (partial) {
        const double s = block_sum(dotacc);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------- scalar kernels (one block)
__device__ double reduce_partials(const double *partial, int nb)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    return block_sum(s);
}

__global__ void k_alpha(PcgState *st, const double *partial_pq, int nb)
{
    if (st->done) return;
    const double pq = reduce_partials(partial_pq, nb);
    if (threadIdx.x == 0) st->alpha = st->rz / pq;
}

__global__ void k_check(PcgState *st, const double *partial_rr, int nb)
{
    if (st->done) return;
    const double rr = reduce_partials(partial_rr, nb);
    if (threadIdx.x == 0) {
        st->rr = rr;
        st->iters += 1;
        if (rr <= st->tol2bb) { st->done = 1; st->converged = 1; }
        else if (st->iters >= st->maxit) st->done = 1;
    }
}

__global__ void k_beta(PcgState *st, const double *partial_rz, int nb)
{
    if (st->done) return;
    const double rz = reduce_partials(partial_rz, nb);
    if (threadIdx.x == 0) {
        st->beta = rz / st->rz;
        st->rz = rz;
    }
}

__global__ void k_init_scalars(PcgState *st, const double *partial_bb, int nb, const double *partial_rz, int nbz,
                               double tol, int32_t maxit)
{
    const double bb = reduce_partials(partial_bb, nb);
    const double rz = reduce_partials(partial_rz, nbz);
    if (threadIdx.x == 0) {
        st->bb = bb; st->rz = rz; st->rr = bb;
        st->tol2bb = tol * tol * bb;
        st->iters = 0; st->maxit = maxit; st->converged = 0;
        st->done = (bb == 0.0 || maxit <= 0) ? 1 : 0;
        if (bb == 0.0) st->converged = 1;
        st->alpha = st->beta = 0.0;
        st->true_rr = 0.0;
    }
}

__global__ void k_true_rr(PcgState *st, const double *partial, int nb)
{
    const double s = reduce_partials(partial, nb);
    if (threadIdx.x == 0) st->true_rr = s;
}

// ---------------------------------------------------------------- vector kernels
__global__ void k_update_xr(int32_t n, double *x, double *r, const double *p, const double *q, double *partial_rr,
                            const PcgState *st)
{
    if (st->done) return;
    const double a = st->alpha;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial_rr[blockIdx.x] = s;
}

__global__ void k_update_p(int32_t n, double *p, const double *z, const PcgState *st)
{
    if (st->done) return;
    const double b = st->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + b * p[i];
}

__global__ void k_init_vectors(int32_t n, const double *b, double *x, double *r, double *partial_bb)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        x[i] = 0.0; r[i] = bi;
        acc += bi * bi;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial_bb[blockIdx.x] = s;
}

__global__ void k_copy(int32_t n, const double *a, double *b)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

template <typename T>
__global__ void k_fill_part(T *a, int32_t na, T *b, int32_t nb)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (na > nb ? na : nb); i += gridDim.x * blockDim.x) {
        if (i < na) a[i] = sentinel<T>();
        if (i < nb) b[i] = sentinel<T>();
    }
}

template <typename T>
__global__ void k_fill_sentinel(int32_t n, T *a, T *b)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a[i] = sentinel<T>();
        b[i] = sentinel<T>();
    }
}

// block partials of r . z over a grid that depends only on n (vec_blocks), so
// the dot product's rounding does not depend on the solves' launch shape
__global__ void k_dot(int32_t n, const double *a, const double *b, double *partial, const PcgState *st)
{
    if (st && st->done) return;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i] * b[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_resid_sq(int32_t n, const double *b, const double *Lx, double *partial)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = b[i] - Lx[i];
        acc += d * d;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// ---------------------------------------------------------------- triangular solves
template <typename XT> __device__ __forceinline__ XT to_x(double v);
template <> __device__ __forceinline__ double to_x<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_x<float>(double v) { return __double2float_rn(v); }

// Wait for an unknown published by another row: polls separated by an
// exponentially growing sleep; false when the wait is abandoned.
template <typename XT>
__device__ __forceinline__ bool poll_ready(const XT *p, XT &v, long long spin_limit, const int32_t *status)
{
    v = ld_poll(p);
    long long spins = 0;
    unsigned ns = 16;
    while (is_sentinel(v)) {
        ++spins;
        // the shared status word is read only now and then: every poller
        // reading it on every spin would turn its cache line into a hot spot
        if ((spins & 127) == 0 && (spins > spin_limit || read_status(status) != ST_OK)) return false;
        __nanosleep(ns);                   // back off: pollers must not crowd out the producers
        if (ns < g_poll_max_ns) ns <<= 1;
        v = ld_poll(p);
    }
    return true;
}

// This lane's share of sum_u v[t(u)] x[idx[t(u)]] over u = sl, sl+stride, ...
// < e-b, where t(u) = b+u, or e-1-u when REV (the backward solve walks a
// column from its last entry, whose unknown was published first), waiting
// for each x to be published.  Entries are taken in chunks of PF per lane: a
// chunk's indices and values are fetched together, then the chunk's x loads
// are issued in rounds -- every entry still unpublished is re-loaded in the
// same round -- so a chunk costs one round trip for its indices and one per
// round of waiting, whatever the row length; the terms are added in a fixed
// order once all are known.
template <bool REV, typename VT, typename XT>
__device__ __forceinline__ bool dot_ready(int64_t b, int64_t e, int sl, int stride, const int32_t *idx,
                                          const VT *v, const XT *x, XT &acc, long long spin_limit,
                                          const int32_t *status, long long *t_seen = nullptr,
                                          int32_t *seen_idx = nullptr)
{
    constexpr int PF = 8;
    const int64_t len = e - b;
    for (int64_t base = sl; base < len; base += (int64_t)PF * stride) {
        int32_t cc[PF];
        VT vv[PF];
        XT xx[PF];
#pragma unroll
        for (int r = 0; r < PF; ++r) {
            const int64_t u = base + (int64_t)r * stride;
            const int64_t t = REV ? e - 1 - u : b + u;
            cc[r] = u < len ? idx[t] : -1;
            vv[r] = u < len ? v[t] : (VT)0;
        }
#pragma unroll
        for (int r = 0; r < PF; ++r) xx[r] = cc[r] >= 0 ? ld_poll(x + cc[r]) : (XT)0;
        long long spins = 0;
        unsigned ns = 16;
        for (;;) {
            int last = -1;
#pragma unroll
            for (int r = 0; r < PF; ++r)
                if (cc[r] >= 0 && is_sentinel(xx[r])) last = r;
            if (last < 0) break;
            ++spins;
            if ((spins & 127) == 0 && (spins > spin_limit || read_status(status) != ST_OK)) return false;
            __nanosleep(ns);               // back off: pollers must not crowd out the producers
            if (ns < g_poll_max_ns) ns <<= 1;
            bool seen = false;
            int32_t seen_c = -1;
#pragma unroll
            for (int r = 0; r < PF; ++r) {
                if (cc[r] >= 0 && is_sentinel(xx[r])) {
                    xx[r] = ld_poll(x + cc[r]);
                    if (!is_sentinel(xx[r])) { seen = true; seen_c = cc[r]; }
                }
            }
            if (t_seen && seen) { *t_seen = global_ns(); *seen_idx = seen_c; }
        }
#pragma unroll
        for (int r = 0; r < PF; ++r) acc += (XT)vv[r] * xx[r];
    }
    return true;
}

// Sum over the block of one value per warp (lane 0's), in warp order, for a
// row shared by the whole block; the result is valid in thread 0.
template <typename XT>
__device__ __forceinline__ XT block_row_sum(XT acc, XT *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    XT s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// The factor is stored relabelled by dependency level (position j holds the
// column of the j-th vertex in level order), so F stays unit lower triangular
// with every row's dependencies at earlier positions and the rows of one
// level contiguous.  operm[j] is the original index of position j.
//
// Each row is handled by S lanes (S = 32: a warp).  A warp works ahead: it
// issues the loads of its current row's unknowns, then the loads its next
// rows need (which depend on no other row; see k_trsv_fwd), and only then
// waits for the current unknowns -- so when a row's dependencies are
// published, its own data is already in registers and it costs one round of
// polls.  Each lane prefetches RPF entries of a row; rows beyond S*RPF
// entries continue with dot_ready.
//
// With a group table (schedule.h), rows are handed out in its groups: up to
// one row per lane group, or one row longer than LONG_ROW_SINGLE entries
// shared by every warp of the block (the rows that collect the most fill,
// e.g. of hub vertices, would otherwise leave one warp to walk them alone on
// the critical path), or chunks of a longer row and their combine.
constexpr int RPF = 1;     // measured: 1 beats 2 and 4 (fewer instructions per row; long rows go on in dot_ready)

template <int S, bool REV, typename VT>
__device__ __forceinline__ void fetch_chunk(int64_t b, int64_t e, int sl, const int32_t *idx, const VT *v,
                                            int32_t (&cc)[RPF], VT (&vv)[RPF])
{
    const int64_t len = e - b;
#pragma unroll
    for (int r = 0; r < RPF; ++r) {
        const int64_t u = sl + (int64_t)r * S;
        const int64_t t = REV ? e - 1 - u : b + u;
        cc[r] = u < len ? idx[t] : -1;
        vv[r] = u < len ? v[t] : (VT)0;
    }
}

template <typename XT>
__device__ __forceinline__ void issue_x(const XT *x, const int32_t (&cc)[RPF], XT (&xx)[RPF])
{
#pragma unroll
    for (int r = 0; r < RPF; ++r) xx[r] = cc[r] >= 0 ? ld_poll(x + cc[r]) : (XT)0;
}

// Wait until the chunk's unknowns are published (polls in rounds with
// back-off), then add its terms in entry order.
template <typename VT, typename XT>
__device__ __forceinline__ bool finish_chunk(const XT *x, const int32_t (&cc)[RPF], const VT (&vv)[RPF],
                                             XT (&xx)[RPF], XT &acc, long long spin_limit, const int32_t *status)
{
    long long spins = 0;
    unsigned ns = 16;
    for (;;) {
        bool pending = false;
#pragma unroll
        for (int r = 0; r < RPF; ++r)
            if (cc[r] >= 0 && is_sentinel(xx[r])) pending = true;
        if (!pending) break;
        ++spins;
        if ((spins & 127) == 0 && (spins > spin_limit || read_status(status) != ST_OK)) return false;
        __nanosleep(ns);
        if (ns < g_poll_max_ns) ns <<= 1;
#pragma unroll
        for (int r = 0; r < RPF; ++r)
            if (cc[r] >= 0 && is_sentinel(xx[r])) xx[r] = ld_poll(x + cc[r]);
    }
#pragma unroll
    for (int r = 0; r < RPF; ++r) acc += (XT)vv[r] * xx[r];
    return true;
}

// A row's last TAIL entries in walk order (forward: the highest positions;
// backward, walked from its last entry: the lowest) hold its dependencies
// published last.  The lanes sum the other entries (their dependencies are
// usually published long before) and reduce them while the row still waits;
// lane 0 then adds the tail entries one by one in walk order, each as soon as
// its unknown is published.  So after the last dependency arrives only an FMA
// and the publication remain, not a batch of FMAs and the shuffle tree (an
// FP64 add costs ~100 cycles on this chip).  The order of the sum is fixed:
// the tree over the head, then the tail in order.
// The batched solves (many systems' levels interleaved: thousands of rows in
// flight, throughput-bound) keep the plain lane-strided sum (TN = 0).
constexpr int TAIL = 4;

template <int TN = TAIL>
__device__ __forceinline__ int64_t head_len(int64_t len) { return len > TN ? len - TN : 0; }

template <bool REV, typename VT, typename XT>
__device__ __forceinline__ bool tail_sum(int64_t b, int64_t e, const int32_t *idx, const VT *v, const XT *x, XT &acc,
                                         long long spin_limit, int32_t *status)
{
    const int64_t len = e - b, h = head_len(len);
    int32_t c[TAIL];
    VT w[TAIL];
    XT xv[TAIL];
#pragma unroll
    for (int k = 0; k < TAIL; ++k) {
        const int64_t u = h + k;
        const int64_t t = REV ? e - 1 - u : b + u;
        c[k] = u < len ? idx[t] : -1;
        w[k] = u < len ? v[t] : (VT)0;
    }
#pragma unroll
    for (int k = 0; k < TAIL; ++k) xv[k] = c[k] >= 0 ? ld_poll(x + c[k]) : (XT)0;
#pragma unroll
    for (int k = 0; k < TAIL; ++k) {
        if (c[k] >= 0) {
            if (is_sentinel(xv[k]) && !poll_ready(x + c[k], xv[k], spin_limit, status)) return false;
            acc += (XT)w[k] * xv[k];
        }
    }
    return true;
}

// Group g of the schedule as seen by one lane group: its row (position) for
// GK_ROWS (-1: none), the group's row for the block-wide kinds.
struct Grp {
    int64_t j;
    int32_t kind, arg, slot;
    int32_t aux;              // SKIP solves: the group's system, then its stop flag
};

// Table entry of group g: from the table, or the fixed group of
// rows_per_group consecutive positions; past the end, an empty group.
__device__ __forceinline__ int4 group_entry(int64_t g, int64_t ngroups, const int4 *gt, int32_t n, int rows_per_group)
{
    if (g >= ngroups) return make_int4(0, GK_ROWS, 0, 0);
    if (gt) return __ldg(gt + g);
    const int64_t k0 = g * rows_per_group;
    const int64_t cnt = (int64_t)n - k0 < rows_per_group ? (int64_t)n - k0 : rows_per_group;
    return make_int4((int32_t)k0, GK_ROWS, (int32_t)cnt, 0);
}

__device__ __forceinline__ Grp group_decode(int4 t, int32_t n, int my, bool rev)
{
    Grp r{-1, t.y & GK_KIND_MASK, t.z, t.w, t.y >> GK_SYS_SHIFT};
    if (r.kind == GK_ROWS) {
        const int64_t kk = (int64_t)t.x + my;
        r.j = my < t.z ? (rev ? (int64_t)n - 1 - kk : kk) : -1;
    } else {
        r.j = rev ? (int64_t)n - 1 - t.x : (int64_t)t.x;
    }
    return r;
}

// A block-wide group of a row of [b, e): the whole row (GK_SHARED) or chunk
// `arg` of it (GK_CHUNK, entries arg*CHUNK_SINGLE .. in walk order), summed by
// every thread of the block in a fixed order; valid in thread 0.
template <bool REV, typename VT, typename XT>
__device__ __forceinline__ XT block_part(const Grp &q, int64_t b, int64_t e, const int32_t *idx, const VT *v,
                                         const XT *x, XT *red, long long spin_limit, int32_t *status)
{
    int64_t lo = b, hi = e;
    if (q.kind == GK_CHUNK) {
        const int64_t c0 = (int64_t)q.arg * CHUNK_SINGLE, c1 = c0 + CHUNK_SINGLE < e - b ? c0 + CHUNK_SINGLE : e - b;
        if (REV) { lo = e - c1; hi = e - c0; } else { lo = b + c0; hi = b + c1; }
    }
    XT acc = 0;
    if (!dot_ready<REV, VT, XT>(lo, hi, threadIdx.x, blockDim.x, idx, v, x, acc, spin_limit, status))
        set_status(status, ST_TIMEOUT);
    return block_row_sum(acc, red);
}

// GK_COMBINE, thread 0: the row's chunk partials summed in chunk order (each
// awaited, then reset to the sentinel for the next solve).
template <typename XT>
__device__ __forceinline__ XT combine_parts(const Grp &q, XT *part, long long spin_limit, int32_t *status)
{
    XT acc = 0;
    for (int c = 0; c < q.arg; ++c) {
        XT v;
        if (!poll_ready(part + q.slot + c, v, spin_limit, status)) { set_status(status, ST_TIMEOUT); v = 0; }
        acc += v;
        part[q.slot + c] = sentinel<XT>();
    }
    return acc;
}

// Forward: y[j] = rhs[operm[j]] - sum_{c<j} F(j,c) y[c] over CSR row j; also
// resets the backward unknown z[j] to the sentinel.
//
// Loads are pipelined over a lane group's successive groups g, g+G, g+2G,
// g+3G (G = gridDim.x): while row g waits for its unknowns, the lanes fetch
// the indices and values of row g+G, the bounds (and operm) of row g+2G and
// the table entry of group g+3G, so each load is issued a step before its
// consumer needs it.  (Unrolling the loop by two over two register sets that
// swap roles was measured slower: more registers, no fewer stalls.)
template <int S, typename VT, typename XT, bool SKIP>
__global__ void k_trsv_fwd(int32_t n, const int64_t *rp, const int32_t *ci, const VT *v, const int32_t *operm,
                           const double *rhs, XT *y, XT *zreset, const int4 *gt, int32_t ngs, XT *part,
                           const PcgState *st, long long spin_limit, int32_t *status, const int32_t *skip)
{
    __shared__ XT red[32];
    if (st && st->done) return;
    const unsigned lane = threadIdx.x & 31;
    const int sub = lane / S, sl = lane % S;
    const unsigned smask = (S == 32) ? FULL : (((1u << S) - 1u) << (sub * S));
    const int rows_per_group = (blockDim.x / 32) * (32 / S);
    const int my = (threadIdx.x >> 5) * (32 / S) + sub;
    const int64_t ngroups = gt ? (int64_t)ngs : ((int64_t)n + rows_per_group - 1) / rows_per_group;
    const int64_t G = gridDim.x;
    auto bounds = [&](Grp &r, int64_t &bb, int64_t &ee, int32_t &o) {
        if constexpr (SKIP) r.aux = skip[r.aux];
        if (r.kind == GK_ROWS && r.j >= 0) {
            bb = rp[r.j]; ee = rp[r.j + 1];
            if (sl == 0) o = operm[r.j];
        }
    };
    auto data = [&](Grp &r, int64_t bb, int64_t ee, int32_t o, double &rr, int32_t (&c)[RPF], VT (&w)[RPF]) {
        if constexpr (SKIP)
            if (r.aux) { r.kind = GK_ROWS; r.j = -1; }      // a stopped system's group: nothing to do
        if (r.kind == GK_ROWS && r.j >= 0) {
            if (sl == 0) rr = rhs[o];
            fetch_chunk<S, false, VT>(bb, bb + head_len<SKIP ? 0 : TAIL>(ee - bb), sl, ci, v, c, w);
        }
    };
    int64_t g = blockIdx.x;
    Grp q = group_decode(group_entry(g, ngroups, gt, n, rows_per_group), n, my, false);
    Grp q1 = group_decode(group_entry(g + G, ngroups, gt, n, rows_per_group), n, my, false);
    int4 t2 = group_entry(g + 2 * G, ngroups, gt, n, rows_per_group);
    int64_t b = 0, e = 0, b1 = 0, e1 = 0;
    int32_t o = 0, o1 = 0;
    double rj = 0.0;
    int32_t cc[RPF];
    VT vv[RPF];
    XT xx[RPF];
    bounds(q, b, e, o);
    bounds(q1, b1, e1, o1);
    data(q, b, e, o, rj, cc, vv);
    while (g < ngroups) {
        const int64_t j = q.j;
        const bool rows = q.kind == GK_ROWS;
        if (rows && j >= 0) issue_x(y, cc, xx);
        // advance the pipeline: data of g+G, bounds of g+2G, entry of g+3G
        int32_t ccn[RPF];
        VT vvn[RPF];
        double rjn = 0.0;
        data(q1, b1, e1, o1, rjn, ccn, vvn);
        Grp q2 = group_decode(t2, n, my, false);
        int64_t b2 = 0, e2 = 0;
        int32_t o2 = 0;
        bounds(q2, b2, e2, o2);
        const int4 t3 = group_entry(g + 3 * G, ngroups, gt, n, rows_per_group);
        if (!rows) {                                  // block-wide group (block-uniform branch)
            if (q.kind == GK_COMBINE) {
                if (threadIdx.x == 0) {
                    const XT sum = combine_parts(q, part, spin_limit, status);
                    zreset[j] = sentinel<XT>();
                    st_pub(y + j, to_x<XT>(rhs[operm[j]]) - sum);
                }
            } else {
                const XT sum = block_part<false, VT, XT>(q, rp[j], rp[j + 1], ci, v, y, red, spin_limit, status);
                if (threadIdx.x == 0) {
                    if (q.kind == GK_CHUNK) {
                        st_pub(part + q.slot, sum);
                    } else {
                        zreset[j] = sentinel<XT>();
                        st_pub(y + j, to_x<XT>(rhs[operm[j]]) - sum);
                    }
                }
            }
            __syncthreads();
        } else if (j >= 0) {
            XT acc = 0;
            const int64_t h = head_len<SKIP ? 0 : TAIL>(e - b);
            bool ok = finish_chunk<VT, XT>(y, cc, vv, xx, acc, spin_limit, status);
            if (ok && h > (int64_t)RPF * S)
                ok = dot_ready<false, VT, XT>(b, b + h, sl + RPF * S, S, ci, v, y, acc, spin_limit, status);
            if (h > 0) {
#pragma unroll
                for (int off = S / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(smask, acc, off);
            }
            if (sl == 0) {
                if (ok && !SKIP) ok = tail_sum<false, VT, XT>(b, e, ci, v, y, acc, spin_limit, status);
                zreset[j] = sentinel<XT>();
                st_pub(y + j, to_x<XT>(rj) - acc);
            }
            if (!ok) set_status(status, ST_TIMEOUT);
        }
        g += G;
        q = q1; b = b1; e = e1; rj = rjn;
#pragma unroll
        for (int r = 0; r < RPF; ++r) { cc[r] = ccn[r]; vv[r] = vvn[r]; }
        q1 = q2; b1 = b2; e1 = e2; o1 = o2;
        t2 = t3;
    }
}

// Backward: z[j] = y[j] Dinv[j] - sum_{i>j} F(i,j) z[i] over CSC column j, in
// decreasing position order, walking each column from its last entry (whose
// unknown was published first); writes zout[operm[j]], resets y[j] to the
// sentinel, and accumulates r_orig . z into the block partial.  Loads are
// pipelined as in the forward solve.
template <int S, typename VT, typename XT, bool SKIP>
__global__ void k_trsv_bwd(int32_t n, const int64_t *cp, const int32_t *ri, const VT *v, const double *Dinv,
                           const int32_t *operm, XT *y, XT *z, double *zout, const double *r_orig, double *partial,
                           const int4 *gt, int32_t ngs, XT *part, const PcgState *st, long long spin_limit,
                           int32_t *status, const int32_t *skip)
{
    __shared__ XT red[32];
    if (st && st->done) return;
    const unsigned lane = threadIdx.x & 31;
    const int sub = lane / S, sl = lane % S;
    const unsigned smask = (S == 32) ? FULL : (((1u << S) - 1u) << (sub * S));
    const int rows_per_group = (blockDim.x / 32) * (32 / S);
    const int my = (threadIdx.x >> 5) * (32 / S) + sub;
    const int64_t ngroups = gt ? (int64_t)ngs : ((int64_t)n + rows_per_group - 1) / rows_per_group;
    const int64_t G = gridDim.x;
    double dotacc = 0.0;
    auto bounds = [&](Grp &r, int64_t &bb, int64_t &ee, int32_t &o) {
        if constexpr (SKIP) r.aux = skip[r.aux];
        if (r.kind == GK_ROWS && r.j >= 0) {
            bb = cp[r.j]; ee = cp[r.j + 1];
            if (sl == 0) o = operm[r.j];
        }
    };
    auto data = [&](Grp &r, int64_t bb, int64_t ee, int32_t o, XT &yv, double &dv, double &rv,
                    int32_t (&c)[RPF], VT (&w)[RPF]) {
        if constexpr (SKIP)
            if (r.aux) { r.kind = GK_ROWS; r.j = -1; }
        if (r.kind == GK_ROWS && r.j >= 0) {
            if (sl == 0) {
                yv = y[r.j]; dv = Dinv[r.j];
                rv = r_orig ? r_orig[o] : 0.0;
            }
            fetch_chunk<S, true, VT>(ee - head_len<SKIP ? 0 : TAIL>(ee - bb), ee, sl, ri, v, c, w);
        }
    };
    // finish column j with the sum of its terms (thread / lane that owns it)
    auto publish = [&](int64_t jj, XT yv, double dv, int32_t ov, double rv, XT sum) {
        const XT zj = to_x<XT>((double)yv * dv) - sum;
        y[jj] = sentinel<XT>();
        st_pub(z + jj, zj);
        zout[ov] = (double)zj;
        dotacc += rv * (double)zj;
    };
    int64_t g = blockIdx.x;
    Grp q = group_decode(group_entry(g, ngroups, gt, n, rows_per_group), n, my, true);
    Grp q1 = group_decode(group_entry(g + G, ngroups, gt, n, rows_per_group), n, my, true);
    int4 t2 = group_entry(g + 2 * G, ngroups, gt, n, rows_per_group);
    int64_t b = 0, e = 0, b1 = 0, e1 = 0;
    int32_t o = 0, o1 = 0;
    XT yj = 0;
    double dj = 0.0, rj = 0.0;
    int32_t cc[RPF];
    VT vv[RPF];
    XT xx[RPF];
    bounds(q, b, e, o);
    bounds(q1, b1, e1, o1);
    data(q, b, e, o, yj, dj, rj, cc, vv);
    while (g < ngroups) {
        const int64_t j = q.j;
        const bool rows = q.kind == GK_ROWS;
        if (rows && j >= 0) issue_x(z, cc, xx);
        int32_t ccn[RPF];
        VT vvn[RPF];
        XT yjn = 0;
        double djn = 0.0, rjn = 0.0;
        data(q1, b1, e1, o1, yjn, djn, rjn, ccn, vvn);
        Grp q2 = group_decode(t2, n, my, true);
        int64_t b2 = 0, e2 = 0;
        int32_t o2 = 0;
        bounds(q2, b2, e2, o2);
        const int4 t3 = group_entry(g + 3 * G, ngroups, gt, n, rows_per_group);
        if (!rows) {                                  // block-wide group (block-uniform branch)
            XT sum = 0;
            if (q.kind == GK_COMBINE) {
                if (threadIdx.x == 0) sum = combine_parts(q, part, spin_limit, status);
            } else {
                sum = block_part<true, VT, XT>(q, cp[j], cp[j + 1], ri, v, z, red, spin_limit, status);
            }
            if (threadIdx.x == 0) {
                if (q.kind == GK_CHUNK) {
                    st_pub(part + q.slot, sum);
                } else {
                    const int32_t os = operm[j];
                    publish(j, y[j], Dinv[j], os, r_orig ? r_orig[os] : 0.0, sum);
                }
            }
            __syncthreads();
        } else if (j >= 0) {
            XT acc = 0;
            const int64_t h = head_len<SKIP ? 0 : TAIL>(e - b);
            bool ok = finish_chunk<VT, XT>(z, cc, vv, xx, acc, spin_limit, status);
            if (ok && h > (int64_t)RPF * S)
                ok = dot_ready<true, VT, XT>(e - h, e, sl + RPF * S, S, ri, v, z, acc, spin_limit, status);
            if (h > 0) {
#pragma unroll
                for (int off = S / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(smask, acc, off);
            }
            if (sl == 0) {
                if (ok && !SKIP) ok = tail_sum<true, VT, XT>(b, e, ri, v, z, acc, spin_limit, status);
                publish(j, yj, dj, o, rj, acc);
            }
            if (!ok) set_status(status, ST_TIMEOUT);
        }
        g += G;
        q = q1; b = b1; e = e1; o = o1; yj = yjn; dj = djn; rj = rjn;
#pragma unroll
        for (int r = 0; r < RPF; ++r) { cc[r] = ccn[r]; vv[r] = vvn[r]; }
        q1 = q2; b1 = b2; e1 = e2; o1 = o2;
        t2 = t3;
    }
    if (partial) {
        const double s = block_sum(dotacc);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------- hybrid solves
// Measured on a 128^3 grid (per-row publication times): two thirds of a
// warp-per-row solve went to the wide dependency levels (thousands of rows,
// most of them short), where one row per warp makes the warps' row
// throughput the limit -- a warp spends ~460 instructions on a row -- and one
// third to hundreds of narrow levels of a few long rows each, where the
// latency from a row's last dependency to its publication is the limit.  So
// each level is handled by the form that suits it: a table lists, in level
// order, runs of up to 32 rows of a wide level (one lane per row: lane l of
// the warp takes the run's l-th row, fetches its entries PF at a time, waits
// for their unknowns and adds the products in entry order) and the single
// rows of the narrow levels (one warp per row: lanes sum the head entries in
// lane-strided order and reduce them, lane 0 adds the tail, see tail_sum).
// Rows of more than TPR_LONG entries inside a run are taken by the whole warp
// the same way, one after another.  Entry c goes to warp c mod W; a run never
// crosses a level, so no row waits on a row of its own entry, and every
// dependency sits in an earlier entry: with the grid fully co-resident the
// smallest unfinished entry never waits on an unfinished entry.  The bounds
// and right-hand side of the warp's next entry are loaded before the waits,
// its first indices and values prefetched to L2.
constexpr int TPR_LONG = 64;

// Bring a row's first indices and values towards L2 ahead of use.
template <typename VT>
__device__ __forceinline__ void prefetch_l2(const int32_t *idx, const VT *val)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(idx));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(val));
}

// One row [b, e) of the solve done by the whole warp; the sum is valid in lane 0.
template <bool REV, typename VT, typename XT>
__device__ __forceinline__ XT warp_row(int64_t b, int64_t e, int lane, const int32_t *idx, const VT *v, const XT *x,
                                       long long spin_limit, int32_t *status)
{
    const int64_t h = head_len(e - b);
    XT acc = 0;
    bool ok = true;
    if (h > 0) {
        ok = REV ? dot_ready<true, VT, XT>(e - h, e, lane, 32, idx, v, x, acc, spin_limit, status)
                 : dot_ready<false, VT, XT>(b, b + h, lane, 32, idx, v, x, acc, spin_limit, status);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    }
    if (lane == 0 && ok) ok = tail_sum<REV, VT, XT>(b, e, idx, v, x, acc, spin_limit, status);
    if (!ok) set_status(status, ST_TIMEOUT);
    return acc;
}

// Table entry (schedule.h, hybrid_table): {first position, rows | sys <<
// HY_SYS_SHIFT} for a run of a wide level, {position, 0 | sys << ...} for a
// row of a narrow level.  SKIP: entries of systems whose stop flag is set are
// skipped (the flag is read when the entry is prefetched).
struct HyEntry {
    int64_t j;      // this lane's position (its run row, or the warp's row)
    int32_t cnt;    // rows of the run; 0: one row for the whole warp
    bool has;       // this lane has work in the entry
};

template <bool SKIP>
__device__ __forceinline__ HyEntry hy_decode(int64_t c, int32_t nt, const int2 *tab, bool rev, int lane,
                                             const int32_t *skip)
{
    HyEntry h{0, 0, false};
    if (c >= nt) return h;
    const int2 t = __ldg(tab + (rev ? nt - 1 - c : c));
    h.cnt = t.y & HY_COUNT_MASK;
    if constexpr (SKIP)
        if (__ldg(skip + (t.y >> HY_SYS_SHIFT))) return h;     // a stopped system: nothing to do
    h.j = (int64_t)t.x + (h.cnt > 0 ? lane : 0);
    h.has = h.cnt == 0 || lane < h.cnt;
    return h;
}

template <typename VT, typename XT, bool SKIP>
__global__ void __launch_bounds__(256) k_trsv_fwd_h(const int2 *tab, int32_t nt, const int64_t *rp,
                                                    const int32_t *ci, const VT *v, const int32_t *operm,
                                                    const double *rhs, XT *y, XT *zreset, const PcgState *st,
                                                    long long spin_limit, int32_t *status, const int32_t *skip)
{
    if (st && st->done) return;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    HyEntry h = hy_decode<SKIP>(c, nt, tab, false, lane, skip);
    int64_t b = 0, e = 0;
    double rj = 0.0;
    if (h.has) { b = rp[h.j]; e = rp[h.j + 1]; rj = rhs[operm[h.j]]; }
    for (; c < nt; c += W) {
        const HyEntry hn = hy_decode<SKIP>(c + W, nt, tab, false, lane, skip);
        int64_t bn = 0, en = 0;
        double rn = 0.0;
        if (hn.has) {
            bn = rp[hn.j]; en = rp[hn.j + 1]; rn = rhs[operm[hn.j]];
            if (hn.cnt > 0 || lane == 0) prefetch_l2(ci + bn, v + bn);
        }
        const XT rx = to_x<XT>(rj);                      // converted before any wait
        if (h.has && h.cnt == 0) {                        // a narrow level's row: the whole warp
            const XT acc = warp_row<false, VT, XT>(b, e, lane, ci, v, y, spin_limit, status);
            if (lane == 0) {
                zreset[h.j] = sentinel<XT>();
                st_pub(y + h.j, rx - acc);
            }
        } else if (h.cnt > 0) {                           // a run of a wide level: a lane per row
            const bool lng = h.has && e - b > TPR_LONG;
            if (h.has && !lng) {
                XT acc = 0;
                if (!dot_ready<false, VT, XT>(b, e, 0, 1, ci, v, y, acc, spin_limit, status))
                    set_status(status, ST_TIMEOUT);
                zreset[h.j] = sentinel<XT>();
                st_pub(y + h.j, rx - acc);
            }
            for (unsigned lm = __ballot_sync(FULL, lng); lm; lm &= lm - 1) {
                const int src = __ffs(lm) - 1;
                const int64_t bb = __shfl_sync(FULL, b, src), ee = __shfl_sync(FULL, e, src);
                XT acc = warp_row<false, VT, XT>(bb, ee, lane, ci, v, y, spin_limit, status);
                acc = __shfl_sync(FULL, acc, 0);
                if (lane == src) {
                    zreset[h.j] = sentinel<XT>();
                    st_pub(y + h.j, rx - acc);
                }
            }
        }
        h = hn; b = bn; e = en; rj = rn;
    }
}

// Backward solve over the same table from its end: z[j] = RN(y[j] Dinv[j]) -
// sum_{i>j} F(i,j) z[i], each column walked from its last entry (whose unknown
// was published first); writes zout[operm[j]] and resets y[j] to the sentinel.
template <typename VT, typename XT, bool SKIP>
__global__ void __launch_bounds__(256) k_trsv_bwd_h(const int2 *tab, int32_t nt, const int64_t *cp,
                                                    const int32_t *ri, const VT *v, const double *Dinv,
                                                    const int32_t *operm, XT *y, XT *z, double *zout,
                                                    const PcgState *st, long long spin_limit, int32_t *status,
                                                    const int32_t *skip)
{
    if (st && st->done) return;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    HyEntry h = hy_decode<SKIP>(c, nt, tab, true, lane, skip);
    int64_t b = 0, e = 0;
    int32_t o = 0;
    XT yj = 0;
    double dj = 0.0;
    if (h.has) { b = cp[h.j]; e = cp[h.j + 1]; o = operm[h.j]; yj = y[h.j]; dj = Dinv[h.j]; }
    for (; c < nt; c += W) {
        const HyEntry hn = hy_decode<SKIP>(c + W, nt, tab, true, lane, skip);
        int64_t bn = 0, en = 0;
        int32_t on = 0;
        XT yn = 0;
        double dn = 0.0;
        if (hn.has) {
            bn = cp[hn.j]; en = cp[hn.j + 1]; on = operm[hn.j]; yn = y[hn.j]; dn = Dinv[hn.j];
            if ((hn.cnt > 0 || lane == 0) && en > bn) prefetch_l2(ri + en - 1, v + en - 1);
        }
        const XT sj = to_x<XT>((double)yj * dj);         // D^+ y, rounded, before any wait
        if (h.has && h.cnt == 0) {
            const XT acc = warp_row<true, VT, XT>(b, e, lane, ri, v, z, spin_limit, status);
            if (lane == 0) {
                const XT zj = sj - acc;
                y[h.j] = sentinel<XT>();
                st_pub(z + h.j, zj);
                zout[o] = (double)zj;
            }
        } else if (h.cnt > 0) {
            const bool lng = h.has && e - b > TPR_LONG;
            if (h.has && !lng) {
                XT acc = 0;
                if (!dot_ready<true, VT, XT>(b, e, 0, 1, ri, v, z, acc, spin_limit, status))
                    set_status(status, ST_TIMEOUT);
                const XT zj = sj - acc;
                y[h.j] = sentinel<XT>();
                st_pub(z + h.j, zj);
                zout[o] = (double)zj;
            }
            for (unsigned lm = __ballot_sync(FULL, lng); lm; lm &= lm - 1) {
                const int src = __ffs(lm) - 1;
                const int64_t bb = __shfl_sync(FULL, b, src), ee = __shfl_sync(FULL, e, src);
                XT acc = warp_row<true, VT, XT>(bb, ee, lane, ri, v, z, spin_limit, status);
                acc = __shfl_sync(FULL, acc, 0);
                if (lane == src) {
                    const XT zj = sj - acc;
                    y[h.j] = sentinel<XT>();
                    st_pub(z + h.j, zj);
                    zout[o] = (double)zj;
                }
            }
        }
        h = hn; b = bn; e = en; o = on; yj = yn; dj = dn;
    }
}

inline int vec_grid(int32_t n, int maxb)
{
    int b = (int)(((int64_t)n + VEC_THREADS - 1) / VEC_THREADS);
    if (b < 1) b = 1;
    return b < maxb ? b : maxb;
}

template <int S>
cudaError_t spmv_t(const SolveArgs &A, const double *x, double *y, double *partial, const PcgState *st, int blocks,
                   cudaStream_t s)
{
    k_spmv<S><<<blocks, VEC_THREADS, 0, s>>>(A.n, A.Lp, A.Li, A.Lv, x, y, partial, st); count_launches(1);
    return cudaGetLastError();
}

cudaError_t spmv(const SolveArgs &A, const double *x, double *y, double *partial, const PcgState *st, int blocks,
                 cudaStream_t s)
{
    switch (A.lanes_spmv) {
    case 4: return spmv_t<4>(A, x, y, partial, st, blocks, s);
    case 8: return spmv_t<8>(A, x, y, partial, st, blocks, s);
    case 16: return spmv_t<16>(A, x, y, partial, st, blocks, s);
    default: return spmv_t<32>(A, x, y, partial, st, blocks, s);
    }
}

template <int S, typename VT, typename XT>
cudaError_t apply_t(const SolveArgs &A, const VT *vr, const VT *vc, XT *y, XT *z, const double *r, double *zout,
                    double *partial, const PcgState *st, cudaStream_t s)
{
    const int threads = A.trsv_warps * 32;
    // a group table is built for the launch's rows per group (trsv_warps * 32 / S)
    const int4 *gf = A.gt_f, *gb = A.gt_b;
    if constexpr (S == 32) {
        if (A.skip) {                 // per-system stop flags (batched solves, one row per warp)
            k_trsv_fwd<S, VT, XT, true><<<A.trsv_blocks, threads, 0, s>>>(
                A.n, A.Frp, A.Fcol, vr, A.operm, r, y, z, gf, A.ng_f, (XT *)A.part_f, st, A.spin_limit, A.status,
                A.skip);
            k_trsv_bwd<S, VT, XT, true><<<A.trsv_blocks, threads, 0, s>>>(
                A.n, A.Fcp, A.Frow, vc, A.Dinv, A.operm, y, z, zout, partial ? r : nullptr, partial, gb, A.ng_b,
                (XT *)A.part_b, st, A.spin_limit, A.status, A.skip);
            count_launches(2);
            return cudaGetLastError();
        }
    }
    k_trsv_fwd<S, VT, XT, false><<<A.trsv_blocks, threads, 0, s>>>(A.n, A.Frp, A.Fcol, vr, A.operm, r, y, z, gf,
                                                                    A.ng_f, (XT *)A.part_f, st, A.spin_limit,
                                                                    A.status, nullptr);
    count_launches(1);
    k_trsv_bwd<S, VT, XT, false><<<A.trsv_blocks, threads, 0, s>>>(A.n, A.Fcp, A.Frow, vc, A.Dinv, A.operm, y, z,
                                                                    zout, partial ? r : nullptr, partial, gb, A.ng_b,
                                                                    (XT *)A.part_b, st, A.spin_limit, A.status,
                                                                    nullptr);
    count_launches(1);
    return cudaGetLastError();
}

template <int S>
cudaError_t apply_s(const SolveArgs &A, const PcgBuffers &B, const double *r, double *zout, double *partial,
                    const PcgState *st, cudaStream_t s)
{
    if (A.prec == 32) return apply_t<S, float, float>(A, A.Fvalr32, A.Fval32, B.yl32, B.zl32, r, zout, partial, st, s);
    return apply_t<S, double, double>(A, A.Fvalr64, A.Fval64, B.yl64, B.zl64, r, zout, partial, st, s);
}

template <typename VT, typename XT, bool SKIP>
cudaError_t apply_tpr(const SolveArgs &A, const VT *vr, const VT *vc, XT *y, XT *z, const double *r, double *zout,
                      const PcgState *st, cudaStream_t s)
{
    k_trsv_fwd_h<VT, XT, SKIP><<<A.tpr_blocks, TPR_THREADS, 0, s>>>(A.tpr_chunks, A.ntpr, A.Frp, A.Fcol, vr, A.operm,
                                                                    r, y, z, st, A.spin_limit, A.status, A.skip);
    k_trsv_bwd_h<VT, XT, SKIP><<<A.tpr_blocks, TPR_THREADS, 0, s>>>(A.tpr_chunks, A.ntpr, A.Fcp, A.Frow, vc, A.Dinv,
                                                                    A.operm, y, z, zout, st, A.spin_limit, A.status,
                                                                    A.skip);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t apply(const SolveArgs &A, const PcgBuffers &B, const double *r, double *zout, double *partial,
                  const PcgState *st, cudaStream_t s)
{
    if (A.tpr_blocks > 0 && A.tpr_chunks && !A.gt_f && !partial) {
        if (A.skip) {
            if (A.prec == 32) return apply_tpr<float, float, true>(A, A.Fvalr32, A.Fval32, B.yl32, B.zl32, r, zout, st, s);
            return apply_tpr<double, double, true>(A, A.Fvalr64, A.Fval64, B.yl64, B.zl64, r, zout, st, s);
        }
        if (A.prec == 32) return apply_tpr<float, float, false>(A, A.Fvalr32, A.Fval32, B.yl32, B.zl32, r, zout, st, s);
        return apply_tpr<double, double, false>(A, A.Fvalr64, A.Fval64, B.yl64, B.zl64, r, zout, st, s);
    }
    switch (A.lanes_trsv) {
    case 4: return apply_s<4>(A, B, r, zout, partial, st, s);
    case 8: return apply_s<8>(A, B, r, zout, partial, st, s);
    case 16: return apply_s<16>(A, B, r, zout, partial, st, s);
    default: return apply_s<32>(A, B, r, zout, partial, st, s);
    }
}

cudaError_t fill_sentinels(const SolveArgs &A, const PcgBuffers &B, cudaStream_t s)
{
    const int g = vec_grid(A.n, 4096);
    if (A.prec == 32) k_fill_sentinel<float><<<g, VEC_THREADS, 0, s>>>(A.n, B.yl32, B.zl32);
    else k_fill_sentinel<double><<<g, VEC_THREADS, 0, s>>>(A.n, B.yl64, B.zl64);
    count_launches(1);
    if (A.gt_f && (A.nslot_f > 0 || A.nslot_b > 0)) {      // split-row partials start unpublished
        const int32_t m = A.nslot_f > A.nslot_b ? A.nslot_f : A.nslot_b;
        if (A.prec == 32) k_fill_part<float><<<vec_grid(m, 64), VEC_THREADS, 0, s>>>((float *)A.part_f, A.nslot_f, (float *)A.part_b, A.nslot_b);
        else k_fill_part<double><<<vec_grid(m, 64), VEC_THREADS, 0, s>>>((double *)A.part_f, A.nslot_f, (double *)A.part_b, A.nslot_b);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace

// the SpMV, the preconditioner apply and the sentinel reset, for the batched
// PCG (batch.cu); st gates the launches (st->done: nothing to do)
cudaError_t solve_spmv(const SolveArgs &A, const double *x, double *y, const PcgState *st, int blocks, cudaStream_t s)
{
    return spmv(A, x, y, nullptr, st, blocks, s);
}

cudaError_t solve_apply(const SolveArgs &A, const PcgBuffers &B, const double *r, double *z, const PcgState *st,
                        cudaStream_t s)
{
    return apply(A, B, r, z, nullptr, st, s);
}

cudaError_t solve_fill_sentinels(const SolveArgs &A, const PcgBuffers &B, cudaStream_t s)
{
    return fill_sentinels(A, B, s);
}

size_t pcg_state_bytes() { return sizeof(PcgState); }

cudaError_t set_poll_backoff(unsigned max_ns)
{
    // written only when it changes, per device (the copy is synchronous and
    // would otherwise serialise concurrent solves)
    static std::mutex mu;
    static unsigned last[NOALLOC_MAX_DEVICES] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < NOALLOC_MAX_DEVICES && last[dev] == max_ns) return cudaSuccess;
    e = cudaMemcpyToSymbol(g_poll_max_ns, &max_ns, sizeof max_ns);
    if (e == cudaSuccess && dev >= 0 && dev < NOALLOC_MAX_DEVICES) last[dev] = max_ns;
    return e;
}

int trsv_configure(int lanes, int warps, int *blocks_per_sm, int prec, bool skip)
{
    cudaError_t e;
    const int threads = warps * 32;
    switch (lanes) {
    case 4:
        e = prec == 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<4, float, float, false>, threads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<4, double, double, false>, threads, 0);
        break;
    case 8:
        e = prec == 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<8, float, float, false>, threads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<8, double, double, false>, threads, 0);
        break;
    case 16:
        e = prec == 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<16, float, float, false>, threads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<16, double, double, false>, threads, 0);
        break;
    default:
        e = prec == 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<32, float, float, false>, threads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trsv_fwd<32, double, double, false>, threads, 0);
    }
    int b2 = 0;
    // the backward kernel must fit the same grid
    switch (lanes) {
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, prec == 32 ? (const void *)k_trsv_bwd<4, float, float, false> : (const void *)k_trsv_bwd<4, double, double, false>, threads, 0); break;
    case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, prec == 32 ? (const void *)k_trsv_bwd<8, float, float, false> : (const void *)k_trsv_bwd<8, double, double, false>, threads, 0); break;
    case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, prec == 32 ? (const void *)k_trsv_bwd<16, float, float, false> : (const void *)k_trsv_bwd<16, double, double, false>, threads, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, prec == 32 ? (const void *)k_trsv_bwd<32, float, float, false> : (const void *)k_trsv_bwd<32, double, double, false>, threads, 0);
    }
    if (b2 < *blocks_per_sm) *blocks_per_sm = b2;
    if (skip) {                       // the per-system stop-flag solves (one row per warp) are launched instead
        int a = 0, c = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, prec == 32 ? (const void *)k_trsv_fwd<32, float, float, true> : (const void *)k_trsv_fwd<32, double, double, true>, threads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, prec == 32 ? (const void *)k_trsv_bwd<32, float, float, true> : (const void *)k_trsv_bwd<32, double, double, true>, threads, 0);
        *blocks_per_sm = std::min(a, c);
    }
    return e == cudaSuccess ? 0 : -1;
}

int tpr_blocks_per_sm(int prec)
{
    int a = 0, b = 0;
    if (prec == 32) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_trsv_fwd_h<float, float, false>, TPR_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trsv_bwd_h<float, float, false>, TPR_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_trsv_fwd_h<double, double, false>, TPR_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trsv_bwd_h<double, double, false>, TPR_THREADS, 0);
    }
    return std::min(a, b);
}

cudaError_t precond_apply(const SolveArgs &A, const PcgBuffers &B, const double *r, double *z, cudaStream_t st)
{
    cudaError_t e = fill_sentinels(A, B, st);
    if (e != cudaSuccess) return e;
    return apply(A, B, r, z, nullptr, nullptr, st);
}

// ---------------------------------------------------------------- allocation-free apply
// Work space of parac_precond_apply_noalloc: the forward and backward
// unknowns of the two triangular solves (two n-vectors, FP64 or FP32), held
// in a fixed array that every device loading the library keeps until exit.
// All calls share it; its contents are the last call's, and every call
// resets the part it uses before reading it.
static __device__ __align__(256) double g_noalloc_work[2 * (size_t)NOALLOC_MAX_N];

// Device address of g_noalloc_work on the current device.  The name is only a
// host-side stand-in in host code, so the address is looked up once per
// device (with that device current) and cached.
static cudaError_t noalloc_work_ptr(double **out)
{
    static std::mutex mu;
    static double *ptrs[NOALLOC_MAX_DEVICES] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_work);
        if (e != cudaSuccess) return e;
        ptrs[dev] = (double *)p;
    }
    *out = ptrs[dev];
    return cudaSuccess;
}

cudaError_t precond_apply_noalloc(const SolveArgs &A, const double *r, double *z, cudaStream_t st)
{
    if (A.n > NOALLOC_MAX_N) return cudaErrorInvalidValue;
    double *work = nullptr;
    cudaError_t e = noalloc_work_ptr(&work);
    if (e != cudaSuccess) return e;
    PcgBuffers B{};
    if (A.prec == 32) {
        B.yl32 = (float *)work;
        B.zl32 = (float *)work + A.n;
    } else {
        B.yl64 = work;
        B.zl64 = work + A.n;
    }
    e = fill_sentinels(A, B, st);     // the unknowns must start as "not yet published"
    if (e != cudaSuccess) return e;
    return apply(A, B, r, z, nullptr, nullptr, st);
}

cudaError_t pcg_init(const SolveArgs &A, const PcgBuffers &B, double tol, int32_t maxit, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    double *p_bb = B.partials, *p_rz = B.partials + B.pstride;
    k_init_vectors<<<nb, VEC_THREADS, 0, s>>>(A.n, B.b, B.x, B.r, p_bb); count_launches(1);
    cudaError_t e = fill_sentinels(A, B, s);
    if (e != cudaSuccess) return e;
    e = apply(A, B, B.r, B.z, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    k_dot<<<nb, VEC_THREADS, 0, s>>>(A.n, B.r, B.z, p_rz, nullptr); count_launches(1);
    k_init_scalars<<<1, 256, 0, s>>>(B.state, p_bb, nb, p_rz, nb, tol, maxit); count_launches(1);
    k_copy<<<nb, VEC_THREADS, 0, s>>>(A.n, B.z, B.p); count_launches(1);
    return cudaGetLastError();
}

cudaError_t pcg_iteration(const SolveArgs &A, const PcgBuffers &B, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    double *p_pq = B.partials, *p_rr = B.partials + B.pstride, *p_rz = B.partials + 2 * B.pstride;
    cudaError_t e = spmv(A, B.p, B.q, p_pq, B.state, nb, s);
    if (e != cudaSuccess) return e;
    k_alpha<<<1, 256, 0, s>>>(B.state, p_pq, nb); count_launches(1);
    k_update_xr<<<nb, VEC_THREADS, 0, s>>>(A.n, B.x, B.r, B.p, B.q, p_rr, B.state); count_launches(1);
    k_check<<<1, 256, 0, s>>>(B.state, p_rr, nb); count_launches(1);
    e = apply(A, B, B.r, B.z, nullptr, B.state, s);
    if (e != cudaSuccess) return e;
    k_dot<<<nb, VEC_THREADS, 0, s>>>(A.n, B.r, B.z, p_rz, B.state); count_launches(1);
    k_beta<<<1, 256, 0, s>>>(B.state, p_rz, nb); count_launches(1);
    k_update_p<<<nb, VEC_THREADS, 0, s>>>(A.n, B.p, B.z, B.state); count_launches(1);
    return cudaGetLastError();
}

// resume after a recurrence convergence that the true residual rejected:
// precondition the current residual and update p, then clear `done`.
__global__ void k_clear_done(PcgState *st) { st->done = 0; st->converged = 0; }

cudaError_t pcg_clear_done(const PcgBuffers &B, cudaStream_t s)
{
    k_clear_done<<<1, 1, 0, s>>>(B.state); count_launches(1);
    return cudaGetLastError();
}

cudaError_t pcg_resume(const SolveArgs &A, const PcgBuffers &B, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    double *p_rz = B.partials + 2 * B.pstride;
    cudaError_t e = apply(A, B, B.r, B.z, nullptr, B.state, s);
    if (e != cudaSuccess) return e;
    k_dot<<<nb, VEC_THREADS, 0, s>>>(A.n, B.r, B.z, p_rz, B.state); count_launches(1);
    k_beta<<<1, 256, 0, s>>>(B.state, p_rz, nb); count_launches(1);
    k_update_p<<<nb, VEC_THREADS, 0, s>>>(A.n, B.p, B.z, B.state); count_launches(1);
    return cudaGetLastError();
}

cudaError_t pcg_true_residual(const SolveArgs &A, const PcgBuffers &B, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    cudaError_t e = spmv(A, B.x, B.q, nullptr, nullptr, nb, s);
    if (e != cudaSuccess) return e;
    k_resid_sq<<<nb, VEC_THREADS, 0, s>>>(A.n, B.b, B.q, B.partials); count_launches(1);
    k_true_rr<<<1, 256, 0, s>>>(B.state, B.partials, nb); count_launches(1);
    return cudaGetLastError();
}

cudaError_t pcg_read_state(const PcgBuffers &B, PcgHostState *h, cudaStream_t s)
{
    PcgState hs;
    cudaError_t e = cudaMemcpyAsync(&hs, B.state, sizeof(PcgState), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    h->done = hs.done; h->iters = hs.iters; h->rr = hs.rr; h->bb = hs.bb; h->true_rr = hs.true_rr; h->maxit = hs.maxit;
    return cudaSuccess;
}

}  // namespace parac
