// block.cu -- PCG (Sec. V) for several right-hand sides at once.  The
// blocks X, R, Z, P, Q are row-major n x nrhs, so a warp that owns one row
// reads and writes the nrhs values of that row as one coalesced segment, one
// lane per right-hand side.  SpMM with L, the forward and backward triangular
// solves with F (SpTRSM: the sync-free level-ordered scheme of solve.cu, the
// lane of column j polling only its own unknowns), and per-column scalars:
// every column runs its own CG recurrence and stops on its own residual; the
// launches are the same for all columns.
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace parac {

struct BlockState {
    double rz[32], alpha[32], beta[32], bb[32], rr[32], true_rr[32], tol2bb[32];
    int32_t done[32], iters[32], converged[32];
    int32_t all_done, maxit, nrhs, pad;
};

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BT = 256;                       // threads per block of the block kernels (8 warps)

__device__ __forceinline__ double sentinel64() { return __longlong_as_double((long long)0xfff7ffffffffffffull); }
__device__ __forceinline__ float sentinel32() { return __int_as_float((int)0xffbfffffu); }
__device__ __forceinline__ bool is_sent(double x) { return __double_as_longlong(x) == (long long)0xfff7ffffffffffffull; }
__device__ __forceinline__ bool is_sent(float x) { return __float_as_int(x) == (int)0xffbfffffu; }
template <typename T> __device__ __forceinline__ T sent();
template <> __device__ __forceinline__ double sent<double>() { return sentinel64(); }
template <> __device__ __forceinline__ float sent<float>() { return sentinel32(); }
__device__ __forceinline__ double ldp(const double *p) { return ld_relaxed_f64(p); }
__device__ __forceinline__ float ldp(const float *p) { return ld_relaxed_f32(p); }
__device__ __forceinline__ void stp(double *p, double v) { st_relaxed_f64(p, v); }
__device__ __forceinline__ void stp(float *p, float v) { st_relaxed_f32(p, v); }
template <typename XT> __device__ __forceinline__ XT tox(double v);
template <> __device__ __forceinline__ double tox<double>(double v) { return v; }
template <> __device__ __forceinline__ float tox<float>(double v) { return __double2float_rn(v); }

// per-column block partial: lane j of every warp holds a value for column j;
// the block's sum for column j goes to partial[blockIdx.x * 32 + j]
__device__ void block_colsum(double v, double *partial)
{
    __shared__ double ws[32][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ws[w][lane] = v;
    __syncthreads();
    if (w == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i][lane];
        partial[blockIdx.x * 32 + lane] = s;
    }
    __syncthreads();
}

// Column sums of nb block partials, partial[b * 32 + j]: out[j] (shared) for
// j < 32, by all 1024 threads of the block in a fixed reduction tree (thread
// (q, j) adds blocks q, q+32, ... of column j, then warp j adds the 32 results
// by shuffles); deterministic.
constexpr int ST = 1024;     // threads of the scalar kernels

__device__ void colsums(const double *partial, int nb, double *out)
{
    __shared__ double s[32][33];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    double a = 0.0;
    for (int b = w; b < nb; b += 32) a += partial[b * 32 + l];
    s[w][l] = a;
    __syncthreads();
    double v = s[l][w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if (l == 0) out[w] = v;
    __syncthreads();
}

__global__ void k_bpack(int32_t n, int nrhs, const double *B, int64_t ldb, double *Bt)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * nrhs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nrhs, j = e % nrhs;
        Bt[e] = B[j * ldb + i];
    }
}

__global__ void k_bunpack(int32_t n, int nrhs, const double *Xt, double *X, int64_t ldx)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * nrhs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nrhs, j = e % nrhs;
        X[j * ldx + i] = Xt[e];
    }
}

// Q = L P (warp per row, lane = column) and per-column partial p.q
__global__ void k_bspmm(int32_t n, int nrhs, const int64_t *Lp, const int32_t *Li, const double *Lv, const double *P,
                        double *Q, double *partial, const BlockState *st)
{
    if (st && st->all_done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool col = lane < nrhs;
    double dot = 0.0;
    for (int64_t i = w0; i < n; i += nw) {
        double acc = 0.0;
        for (int64_t t = Lp[i]; t < Lp[i + 1]; ++t) {
            const int32_t c = __ldg(Li + t);
            const double v = __ldg(Lv + t);
            if (col) acc += v * P[(int64_t)c * nrhs + lane];
        }
        if (col) {
            Q[i * nrhs + lane] = acc;
            dot += acc * P[i * nrhs + lane];
        }
    }
    if (partial) block_colsum(dot, partial);
}

__global__ void k_binit(int32_t n, int nrhs, const double *B, double *X, double *R, double *partial_bb)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    if (lane < nrhs)
        for (int64_t i = w0; i < n; i += nw) {
            const double b = B[i * nrhs + lane];
            X[i * nrhs + lane] = 0.0;
            R[i * nrhs + lane] = b;
            acc += b * b;
        }
    block_colsum(acc, partial_bb);
}

__global__ void k_bupdate_xr(int32_t n, int nrhs, double *X, double *R, const double *P, const double *Q,
                             double *partial_rr, const BlockState *st)
{
    if (st->all_done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    if (lane < nrhs) {
        const bool act = !st->done[lane];
        const double a = st->alpha[lane];
        for (int64_t i = w0; i < n; i += nw) {
            const int64_t e = i * nrhs + lane;
            double r = R[e];
            if (act) {
                X[e] += a * P[e];
                r -= a * Q[e];
                R[e] = r;
            }
            acc += r * r;
        }
    }
    block_colsum(acc, partial_rr);
}

// per-column partials of r . z (warp per row, lane = column) over a grid that
// depends only on n, so the rounding does not depend on the solves' launch shape
__global__ void k_bdot(int32_t n, int nrhs, const double *R, const double *Z, double *partial, const BlockState *st)
{
    if (st && st->all_done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    if (lane < nrhs)
        for (int64_t i = w0; i < n; i += nw) acc += R[i * nrhs + lane] * Z[i * nrhs + lane];
    block_colsum(acc, partial);
}

__global__ void k_bupdate_p(int32_t n, int nrhs, double *P, const double *Z, const BlockState *st)
{
    if (st->all_done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (lane >= nrhs || st->done[lane]) return;
    const double bt = st->beta[lane];
    for (int64_t i = w0; i < n; i += nw) {
        const int64_t e = i * nrhs + lane;
        P[e] = Z[e] + bt * P[e];
    }
}

__global__ void k_bcopy(int64_t m, const double *a, double *b)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = a[e];
}

template <typename T>
__global__ void k_bfill_sentinel(int64_t m, T *a, T *b)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        a[e] = sent<T>();
        b[e] = sent<T>();
    }
}

// ---------------------------------------------------------------- scalar kernels (one block of ST threads)
__device__ void update_all_done(BlockState *st)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < st->nrhs; ++q) all &= st->done[q];
        st->all_done = all;
    }
}

__global__ void k_binit_scalars(BlockState *st, int nrhs, const double *pbb, int nbb, const double *prz, int nrz,
                                double tol, int32_t maxit)
{
    __shared__ double bbs[32], rzs[32];
    colsums(pbb, nbb, bbs);
    colsums(prz, nrz, rzs);
    const int j = threadIdx.x;
    if (j < 32) {
        const bool col = j < nrhs;
        const double bb = col ? bbs[j] : 0.0, rz = col ? rzs[j] : 0.0;
        st->bb[j] = bb; st->rz[j] = rz; st->rr[j] = bb; st->tol2bb[j] = tol * tol * bb;
        st->alpha[j] = st->beta[j] = 0.0; st->true_rr[j] = 0.0;
        st->iters[j] = 0;
        st->converged[j] = col && bb == 0.0;
        st->done[j] = !col || bb == 0.0 || maxit <= 0;
    }
    if (j == 0) { st->maxit = maxit; st->nrhs = nrhs; }
    update_all_done(st);
}

__global__ void k_balpha(BlockState *st, const double *ppq, int nb)
{
    __shared__ double pq[32];
    if (st->all_done) return;
    colsums(ppq, nb, pq);
    const int j = threadIdx.x;
    if (j < st->nrhs && !st->done[j]) st->alpha[j] = st->rz[j] / pq[j];
}

__global__ void k_bcheck(BlockState *st, const double *prr, int nb)
{
    __shared__ double rrs[32];
    if (st->all_done) return;
    colsums(prr, nb, rrs);
    const int j = threadIdx.x;
    if (j < st->nrhs && !st->done[j]) {
        const double rr = rrs[j];
        st->rr[j] = rr;
        st->iters[j] += 1;
        if (rr <= st->tol2bb[j]) { st->done[j] = 1; st->converged[j] = 1; }
        else if (st->iters[j] >= st->maxit) st->done[j] = 1;
    }
    update_all_done(st);
}

__global__ void k_bbeta(BlockState *st, const double *prz, int nb)
{
    __shared__ double rzs[32];
    if (st->all_done) return;
    colsums(prz, nb, rzs);
    const int j = threadIdx.x;
    if (j < st->nrhs && !st->done[j]) {
        st->beta[j] = rzs[j] / st->rz[j];
        st->rz[j] = rzs[j];
    }
}

__global__ void k_btrue(BlockState *st, const double *p, int nb)
{
    __shared__ double t[32];
    colsums(p, nb, t);
    const int j = threadIdx.x;
    if (j < st->nrhs) st->true_rr[j] = t[j];
}

__global__ void k_bresid(int32_t n, int nrhs, const double *B, const double *LX, double *partial)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    if (lane < nrhs)
        for (int64_t i = w0; i < n; i += nw) {
            const double d = B[i * nrhs + lane] - LX[i * nrhs + lane];
            acc += d * d;
        }
    block_colsum(acc, partial);
}

// reopen the columns whose true residual failed the test (recurrence drift)
__global__ void k_breopen(BlockState *st)
{
    const int j = threadIdx.x;
    if (j < st->nrhs && st->converged[j] && !(st->true_rr[j] <= st->tol2bb[j]) && st->iters[j] < st->maxit) {
        st->converged[j] = 0;
        st->done[j] = 0;
    }
    __syncthreads();
    if (j == 0) {
        int all = 1;
        for (int q = 0; q < st->nrhs; ++q) all &= st->done[q];
        st->all_done = all;
    }
}

// ---------------------------------------------------------------- SpTRSM
// Rows (positions) are handed out in groups, in position order (ascending for
// the forward solve, descending for the backward one), round-robin over a
// co-resident grid as in solve.cu.  A group is either up to one row per warp
// of the block, or a single long row (more than LONG_ROW_BLOCK entries) that all
// warps of the block share: the rows at the end of the elimination order
// collect the most fill and form a chain of long rows, which one warp would
// walk alone, 32 entries at a time for every column.
//
// Within a warp, lane = column.  Entries are staged 32 at a time in the
// warp's shared-memory slot (one coalesced load); each lane issues the loads
// of up to PF unknowns of its column at once and the warp consumes them in
// entry order, waiting together (a vote, then one back-off for the warp)
// until the current entry is published in every column and re-polling all
// its still-unpublished entries each round.  Entries sit in ascending
// position order, so the early ones -- long published -- are summed while the
// late ones are awaited.  Two accumulators (even / odd entries of a stage) and
// a fixed cross-warp order for shared rows keep the result deterministic.
constexpr int MAXW = 32;         // warps per block, at most

// Entries u in [u0, u_end), in stages of 32 starting every `stride`, of the
// row [b, b+len): entry u is b+u, or b+len-1-u when REV (the backward solve
// walks a column from its last entry, whose unknown was published first).
template <bool REV, typename VT, typename XT>
__device__ __forceinline__ bool brow_dot(int64_t b, int64_t len, int64_t u0, int64_t u_end, int64_t stride, int lane,
                                         int nrhs, const int32_t *idx, const VT *v, const XT *x, XT &acc0, XT &acc1,
                                         long long spin_limit, const int32_t *status, int32_t *s_c, VT *s_v)
{
    constexpr int PF = 16;
    const bool col = lane < nrhs;
    bool ok = true;
    long long spins = 0;
    for (int64_t base = u0; base < u_end && ok; base += stride) {
        const int64_t u = base + lane;
        const int64_t t = REV ? b + len - 1 - u : b + u;
        __syncwarp();
        s_c[lane] = u < u_end ? __ldg(idx + t) : -1;
        s_v[lane] = u < u_end ? v[t] : (VT)0;
        __syncwarp();
        const int cnt = (int)(u_end - base < 32 ? u_end - base : 32);
        for (int sub = 0; sub < cnt && ok; sub += PF) {
            const int m = cnt - sub < PF ? cnt - sub : PF;
            XT xx[PF];
#pragma unroll
            for (int r = 0; r < PF; ++r)
                xx[r] = (col && r < m) ? ldp(x + (int64_t)s_c[sub + r] * nrhs + lane) : (XT)0;
            unsigned ns = 16;
#pragma unroll
            for (int r = 0; r < PF; ++r) {
                if (r < m && ok) {
                    while (!__all_sync(FULL, !col || !is_sent(xx[r]))) {
                        ++spins;
                        if ((spins & 127) == 0 &&
                            __any_sync(FULL, spins > spin_limit || read_status(status) != ST_OK)) {
                            ok = false;
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 256) ns <<= 1;
#pragma unroll
                        for (int q = r; q < PF; ++q)
                            if (col && q < m && is_sent(xx[q])) xx[q] = ldp(x + (int64_t)s_c[sub + q] * nrhs + lane);
                    }
                    if (col) {
                        const XT term = (XT)s_v[sub + r] * xx[r];
                        if (r & 1) acc1 += term;
                        else acc0 += term;
                    }
                }
            }
        }
    }
    return ok;
}

// Block-wide part of a row of length len at b: the whole row (GK_SHARED) or
// chunk `arg` (GK_CHUNK); every warp takes stages of 32 entries, the warps'
// sums are added in warp order.  Valid for warp 0, lane = column.
template <bool REV, typename VT, typename XT>
__device__ __forceinline__ XT block_row_part(const int4 q, int64_t b, int64_t len, int lane, int my, int nw, int nrhs,
                                             const int32_t *idx, const VT *v, const XT *x, long long spin_limit,
                                             int32_t *status, int32_t *s_c, VT *s_v, XT (*red)[32])
{
    int64_t u0 = 0, u1 = len;
    if (q.y == GK_CHUNK) {
        u0 = (int64_t)q.z * CHUNK_BLOCK;
        u1 = u0 + CHUNK_BLOCK < len ? u0 + CHUNK_BLOCK : len;
    }
    XT a0 = 0, a1 = 0;
    if (!brow_dot<REV, VT, XT>(b, len, u0 + 32 * my, u1, 32 * nw, lane, nrhs, idx, v, x, a0, a1, spin_limit, status,
                               s_c, s_v))
        set_status(status, ST_TIMEOUT);
    red[my][lane] = a0 + a1;
    __syncthreads();
    XT acc = 0;
    if (my == 0)
        for (int w = 0; w < nw; ++w) acc += red[w][lane];
    return acc;
}

// GK_COMBINE, warp 0: the row's chunk partials (lane = column) summed in
// chunk order, each awaited and then reset to the sentinel.
template <typename XT>
__device__ __forceinline__ XT block_combine(const int4 q, int lane, int nrhs, XT *part, long long spin_limit,
                                            int32_t *status)
{
    XT acc = 0;
    if (lane < nrhs) {
        for (int c = 0; c < q.z; ++c) {
            XT *p = part + (int64_t)(q.w + c) * 32 + lane;
            XT x = ldp(p);
            long long spins = 0;
            unsigned ns = 16;
            while (is_sent(x)) {
                ++spins;
                if ((spins & 127) == 0 && (spins > spin_limit || read_status(status) != ST_OK)) {
                    set_status(status, ST_TIMEOUT);
                    x = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
                x = ldp(p);
            }
            acc += x;
            *p = sent<XT>();
        }
    }
    return acc;
}

// Forward: y[j] = rhs[operm[j]] - sum_c F(j,c) y[c] over CSR row j (all
// columns); also resets the backward unknowns z[j] to the sentinel.
template <typename VT, typename XT>
__global__ void k_btrsm_fwd(int32_t n, int nrhs, const int64_t *rp, const int32_t *ci, const VT *v,
                            const int32_t *operm, const double *rhs, XT *y, XT *zreset, const int4 *gt,
                            int32_t ngroups, XT *part, const BlockState *st, long long spin_limit, int32_t *status)
{
    __shared__ int32_t s_c[MAXW][32];
    __shared__ VT s_v[MAXW][32];
    __shared__ XT red[MAXW][32];
    if (st && st->all_done) return;
    const int lane = threadIdx.x & 31, my = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool col = lane < nrhs;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int4 q = gt[g];
        if (q.y != GK_ROWS) {                                   // block-wide group (block-uniform)
            const int64_t j = q.x;
            XT acc = 0;
            if (q.y == GK_COMBINE) {
                if (my == 0) acc = block_combine(q, lane, nrhs, part, spin_limit, status);
            } else {
                acc = block_row_part<false, VT, XT>(q, rp[j], rp[j + 1] - rp[j], lane, my, nw, nrhs, ci, v, y,
                                                    spin_limit, status, s_c[my], s_v[my], red);
            }
            if (my == 0 && col) {
                if (q.y == GK_CHUNK) {
                    stp(part + (int64_t)q.w * 32 + lane, acc);
                } else {
                    zreset[j * nrhs + lane] = sent<XT>();
                    stp(y + j * nrhs + lane, tox<XT>(rhs[(int64_t)operm[j] * nrhs + lane]) - acc);
                }
            }
            __syncthreads();
            continue;
        }
        if (my >= q.z) continue;
        const int64_t j = (int64_t)q.x + my;
        const int64_t b = rp[j], e = rp[j + 1];
        const double rj = col ? rhs[(int64_t)operm[j] * nrhs + lane] : 0.0;
        XT a0 = 0, a1 = 0;
        if (!brow_dot<false, VT, XT>(b, e - b, 0, e - b, 32, lane, nrhs, ci, v, y, a0, a1, spin_limit, status,
                                     s_c[my], s_v[my]))
            set_status(status, ST_TIMEOUT);
        if (col) {
            zreset[j * nrhs + lane] = sent<XT>();
            stp(y + j * nrhs + lane, tox<XT>(rj) - (a0 + a1));
        }
    }
}

// Backward: z[j] = D^+[j] y[j] - sum_r F(r,j) z[r] over CSC column j, scattered
// to zout[operm[j]]; resets y[j] to the sentinel and accumulates the
// per-column partial r_orig . z.  The groups run over kk = n-1-j.
template <typename VT, typename XT>
__global__ void k_btrsm_bwd(int32_t n, int nrhs, const int64_t *cp, const int32_t *ri, const VT *v,
                            const double *Dinv, const int32_t *operm, XT *y, XT *z, double *zout,
                            const double *r_orig, double *partial, const int4 *gt, int32_t ngroups, XT *part,
                            const BlockState *st, long long spin_limit, int32_t *status)
{
    __shared__ int32_t s_c[MAXW][32];
    __shared__ VT s_v[MAXW][32];
    __shared__ XT red[MAXW][32];
    if (st && st->all_done) return;
    const int lane = threadIdx.x & 31, my = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool col = lane < nrhs;
    double dot = 0.0;
    auto publish = [&](int64_t j, XT acc) {
        const int32_t o = operm[j];
        const XT yj = y[j * nrhs + lane];
        const XT zj = tox<XT>((double)yj * Dinv[j]) - acc;
        y[j * nrhs + lane] = sent<XT>();
        stp(z + j * nrhs + lane, zj);
        zout[(int64_t)o * nrhs + lane] = (double)zj;
        if (r_orig) dot += r_orig[(int64_t)o * nrhs + lane] * (double)zj;
    };
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int4 q = gt[g];
        if (q.y != GK_ROWS) {                                   // block-wide group (block-uniform)
            const int64_t j = (int64_t)n - 1 - q.x;
            XT acc = 0;
            if (q.y == GK_COMBINE) {
                if (my == 0) acc = block_combine(q, lane, nrhs, part, spin_limit, status);
            } else {
                acc = block_row_part<true, VT, XT>(q, cp[j], cp[j + 1] - cp[j], lane, my, nw, nrhs, ri, v, z,
                                                   spin_limit, status, s_c[my], s_v[my], red);
            }
            if (my == 0 && col) {
                if (q.y == GK_CHUNK) stp(part + (int64_t)q.w * 32 + lane, acc);
                else publish(j, acc);
            }
            __syncthreads();
            continue;
        }
        if (my >= q.z) continue;
        const int64_t j = (int64_t)n - 1 - ((int64_t)q.x + my);
        const int64_t b = cp[j], e = cp[j + 1];
        XT a0 = 0, a1 = 0;
        if (!brow_dot<true, VT, XT>(b, e - b, 0, e - b, 32, lane, nrhs, ri, v, z, a0, a1, spin_limit, status,
                                    s_c[my], s_v[my]))
            set_status(status, ST_TIMEOUT);
        if (col) publish(j, a0 + a1);
    }
    if (partial) block_colsum(dot, partial);
}

inline int grid_for(int64_t m, int maxb)
{
    int64_t b = (m + BT - 1) / BT;
    if (b < 1) b = 1;
    return (int)(b < maxb ? b : maxb);
}

}  // namespace

size_t block_state_bytes() { return sizeof(BlockState); }

// resident blocks per SM of the two SpTRSM kernels at `warps` warps per block
// (the static row schedule needs the whole grid co-resident)
int btrsm_blocks_per_sm(int warps, int prec)
{
    int a = 0, b = 0;
    const int t = warps * 32;
    if (prec == 32) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_btrsm_fwd<float, float>, t, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_btrsm_bwd<float, float>, t, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_btrsm_fwd<double, double>, t, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_btrsm_bwd<double, double>, t, 0);
    }
    return a < b ? a : b;
}

cudaError_t bpack(int32_t n, int nrhs, const double *B, int64_t ldb, double *Bt, cudaStream_t s)
{
    k_bpack<<<grid_for((int64_t)n * nrhs, 4096), BT, 0, s>>>(n, nrhs, B, ldb, Bt);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t bunpack(int32_t n, int nrhs, const double *Xt, double *X, int64_t ldx, cudaStream_t s)
{
    k_bunpack<<<grid_for((int64_t)n * nrhs, 4096), BT, 0, s>>>(n, nrhs, Xt, X, ldx);
    count_launches(1);
    return cudaGetLastError();
}

namespace {

template <typename VT, typename XT>
cudaError_t bapply_t(const SolveArgs &A, const BlockBuffers &B, const VT *vr, const VT *vc, XT *y, XT *z,
                     const double *r, double *zout, double *partial, const BlockState *st, cudaStream_t s)
{
    const int threads = A.trsv_warps * 32;
    const int gf = B.ng_f < A.trsv_blocks ? B.ng_f : A.trsv_blocks;
    const int gb = B.ng_b < A.trsv_blocks ? B.ng_b : A.trsv_blocks;
    k_btrsm_fwd<VT, XT><<<gf, threads, 0, s>>>(A.n, B.nrhs, A.Frp, A.Fcol, vr, A.operm, r, y, z, B.gt_f, B.ng_f,
                                               (XT *)B.part_f, st, A.spin_limit, A.status);
    count_launches(1);
    k_btrsm_bwd<VT, XT><<<gb, threads, 0, s>>>(A.n, B.nrhs, A.Fcp, A.Frow, vc, A.Dinv, A.operm, y, z, zout,
                                               partial ? r : nullptr, partial, B.gt_b, B.ng_b, (XT *)B.part_b, st,
                                               A.spin_limit, A.status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t bapply(const SolveArgs &A, const BlockBuffers &B, const double *r, double *zout, double *partial,
                   const BlockState *st, cudaStream_t s)
{
    if (A.prec == 32)
        return bapply_t<float, float>(A, B, A.Fvalr32, A.Fval32, B.yl32, B.zl32, r, zout, partial, st, s);
    return bapply_t<double, double>(A, B, A.Fvalr64, A.Fval64, B.yl64, B.zl64, r, zout, partial, st, s);
}

cudaError_t bfill(const SolveArgs &A, const BlockBuffers &B, cudaStream_t s)
{
    const int64_t m = (int64_t)A.n * B.nrhs;
    if (A.prec == 32) k_bfill_sentinel<float><<<grid_for(m, 4096), BT, 0, s>>>(m, B.yl32, B.zl32);
    else k_bfill_sentinel<double><<<grid_for(m, 4096), BT, 0, s>>>(m, B.yl64, B.zl64);
    count_launches(1);
    const int64_t mf = (int64_t)B.nslot_f * 32, mb = (int64_t)B.nslot_b * 32;
    if (mf > 0 || mb > 0) {          // split-row partials start unpublished
        if (A.prec == 32) {
            k_bfill_sentinel<float><<<grid_for(mf, 4096), BT, 0, s>>>(mf, (float *)B.part_f, (float *)B.part_f);
            k_bfill_sentinel<float><<<grid_for(mb, 4096), BT, 0, s>>>(mb, (float *)B.part_b, (float *)B.part_b);
        } else {
            k_bfill_sentinel<double><<<grid_for(mf, 4096), BT, 0, s>>>(mf, (double *)B.part_f, (double *)B.part_f);
            k_bfill_sentinel<double><<<grid_for(mb, 4096), BT, 0, s>>>(mb, (double *)B.part_b, (double *)B.part_b);
        }
        count_launches(2);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t bpcg_init(const SolveArgs &A, const BlockBuffers &B, double tol, int32_t maxit, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    double *p_bb = B.partials, *p_rz = B.partials + 32 * (size_t)B.pstride;
    k_binit<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.b, B.x, B.r, p_bb);
    count_launches(1);
    cudaError_t e = bfill(A, B, s);
    if (e != cudaSuccess) return e;
    e = bapply(A, B, B.r, B.z, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    k_bdot<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.r, B.z, p_rz, nullptr);
    count_launches(1);
    k_binit_scalars<<<1, ST, 0, s>>>(B.state, B.nrhs, p_bb, nb, p_rz, nb, tol, maxit);
    k_bcopy<<<grid_for((int64_t)A.n * B.nrhs, 4096), BT, 0, s>>>((int64_t)A.n * B.nrhs, B.z, B.p);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t bpcg_iteration(const SolveArgs &A, const BlockBuffers &B, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    double *p_pq = B.partials, *p_rr = B.partials + 32 * (size_t)B.pstride,
           *p_rz = B.partials + 64 * (size_t)B.pstride;
    k_bspmm<<<nb, BT, 0, s>>>(A.n, B.nrhs, A.Lp, A.Li, A.Lv, B.p, B.q, p_pq, B.state);
    k_balpha<<<1, ST, 0, s>>>(B.state, p_pq, nb);
    k_bupdate_xr<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.x, B.r, B.p, B.q, p_rr, B.state);
    k_bcheck<<<1, ST, 0, s>>>(B.state, p_rr, nb);
    count_launches(4);
    cudaError_t e = bapply(A, B, B.r, B.z, nullptr, B.state, s);
    if (e != cudaSuccess) return e;
    k_bdot<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.r, B.z, p_rz, B.state);
    count_launches(1);
    k_bbeta<<<1, ST, 0, s>>>(B.state, p_rz, nb);
    k_bupdate_p<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.p, B.z, B.state);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t bpcg_true_residual(const SolveArgs &A, const BlockBuffers &B, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    k_bspmm<<<nb, BT, 0, s>>>(A.n, B.nrhs, A.Lp, A.Li, A.Lv, B.x, B.q, nullptr, nullptr);
    k_bresid<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.b, B.q, B.partials);
    k_btrue<<<1, ST, 0, s>>>(B.state, B.partials, nb);
    count_launches(3);
    return cudaGetLastError();
}

// After a true-residual check: reopen drifted columns and, if any reopened,
// precondition their residual and update their search direction.
cudaError_t bpcg_reopen(const SolveArgs &A, const BlockBuffers &B, cudaStream_t s)
{
    const int nb = B.vec_blocks;
    k_breopen<<<1, 32, 0, s>>>(B.state);
    count_launches(1);
    double *p_rz = B.partials + 64 * (size_t)B.pstride;
    cudaError_t e = bapply(A, B, B.r, B.z, nullptr, B.state, s);
    if (e != cudaSuccess) return e;
    k_bdot<<<nb, BT, 0, s>>>(A.n, B.nrhs, B.r, B.z, p_rz, B.state);
    count_launches(1);
    k_bbeta<<<1, ST, 0, s>>>(B.state, p_rz, nb);
    k_bupdate_p<<<B.vec_blocks, BT, 0, s>>>(A.n, B.nrhs, B.p, B.z, B.state);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t bpcg_read_state(const BlockBuffers &B, BlockHostState *h, cudaStream_t s)
{
    BlockState hs;
    cudaError_t e = cudaMemcpyAsync(&hs, B.state, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    h->all_done = hs.all_done;
    for (int j = 0; j < 32; ++j) {
        h->iters[j] = hs.iters[j]; h->bb[j] = hs.bb[j]; h->true_rr[j] = hs.true_rr[j];
        h->converged[j] = hs.converged[j]; h->done[j] = hs.done[j];
    }
    return cudaSuccess;
}

}  // namespace parac
