// batch.cu -- PCG (Sec. V) on many factored systems at once, one right-hand
// side each (the batched form of the solve).  The systems' matrices, factors
// and vectors are concatenated; the shared SpMV and triangular-solve kernels
// run once per step over all of them (the solves' schedule interleaves the
// systems' rows by dependency level, so one launch advances every system's
// chain, and its groups of stopped systems are skipped through per-system
// stop flags).  Each system keeps its own CG scalars and stopping test.  Every dot
// product is reduced over fixed row chunks that never straddle two systems,
// then per system over its chunks in order: deterministic, and independent of
// the launch shape.
#include "common.cuh"
#include "kernels.h"

namespace parac {

namespace {

constexpr int BT = 256;

__device__ double bsum(double v)
{
    __shared__ double ws[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
    __syncthreads();
    return s;
}

// chunk c's partial of a . b
__global__ void k_cdot(int32_t nchunks, const int64_t *clo, const double *a, const double *b, double *partial,
                       const BatchState *st)
{
    if (st && st->gate.done) return;
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        double acc = 0.0;
        for (int64_t i = clo[c] + threadIdx.x; i < clo[c + 1]; i += blockDim.x) acc += a[i] * b[i];
        const double s = bsum(acc);
        if (threadIdx.x == 0) partial[c] = s;
    }
}

__global__ void k_cinit(int32_t nchunks, const int64_t *clo, const double *b, double *x, double *r, double *pbb)
{
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        double acc = 0.0;
        for (int64_t i = clo[c] + threadIdx.x; i < clo[c + 1]; i += blockDim.x) {
            const double bi = b[i];
            x[i] = 0.0;
            r[i] = bi;
            acc += bi * bi;
        }
        const double s = bsum(acc);
        if (threadIdx.x == 0) pbb[c] = s;
    }
}

// x += alpha_s p, r -= alpha_s q for the systems still running; chunk partials of r . r
__global__ void k_cupdate_xr(int32_t nchunks, const int64_t *clo, const int32_t *csys, const SysState *sys,
                             double *x, double *r, const double *p, const double *q, double *prr, const BatchState *st)
{
    if (st->gate.done) return;
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const SysState &y = sys[csys[c]];
        const bool act = !y.done;
        const double a = y.alpha;
        double acc = 0.0;
        for (int64_t i = clo[c] + threadIdx.x; i < clo[c + 1]; i += blockDim.x) {
            double ri = r[i];
            if (act) {
                x[i] += a * p[i];
                ri -= a * q[i];
                r[i] = ri;
            }
            acc += ri * ri;
        }
        const double s = bsum(acc);
        if (threadIdx.x == 0) prr[c] = s;
    }
}

__global__ void k_cupdate_p(int32_t nchunks, const int64_t *clo, const int32_t *csys, const SysState *sys, double *p,
                            const double *z, const BatchState *st)
{
    if (st->gate.done) return;
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const SysState &y = sys[csys[c]];
        if (y.done) continue;
        const double bt = y.beta;
        for (int64_t i = clo[c] + threadIdx.x; i < clo[c + 1]; i += blockDim.x) p[i] = z[i] + bt * p[i];
    }
}

__global__ void k_ccopy(int64_t n, const double *a, double *b)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_cresid(int32_t nchunks, const int64_t *clo, const double *b, const double *Lx, double *partial)
{
    for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        double acc = 0.0;
        for (int64_t i = clo[c] + threadIdx.x; i < clo[c + 1]; i += blockDim.x) {
            const double d = b[i] - Lx[i];
            acc += d * d;
        }
        const double s = bsum(acc);
        if (threadIdx.x == 0) partial[c] = s;
    }
}

// ---------------------------------------------------------------- per-system scalars (thread per system)
__device__ __forceinline__ double sys_sum(const double *partial, const int32_t *c0, int s)
{
    double acc = 0.0;
    for (int32_t c = c0[s]; c < c0[s + 1]; ++c) acc += partial[c];
    return acc;
}

__global__ void k_sinit(int32_t count, const int32_t *c0, SysState *sys, int32_t *stop, const double *pbb,
                        const double *prz, double tol, int32_t maxit)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        SysState &y = sys[s];
        const double bb = sys_sum(pbb, c0, s), rz = sys_sum(prz, c0, s);
        y.bb = bb; y.rz = rz; y.rr = bb; y.tol2bb = tol * tol * bb;
        y.alpha = y.beta = 0.0; y.true_rr = 0.0;
        y.iters = 0;
        y.converged = bb == 0.0;
        y.done = bb == 0.0 || maxit <= 0;
        stop[s] = y.done;
    }
}

__global__ void k_salpha(int32_t count, const int32_t *c0, SysState *sys, const double *ppq, const BatchState *st)
{
    if (st->gate.done) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        SysState &y = sys[s];
        if (!y.done) y.alpha = y.rz / sys_sum(ppq, c0, s);
    }
}

__global__ void k_scheck(int32_t count, const int32_t *c0, SysState *sys, int32_t *stop, const double *prr,
                         const BatchState *st)
{
    if (st->gate.done) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        SysState &y = sys[s];
        if (y.done) continue;
        const double rr = sys_sum(prr, c0, s);
        y.rr = rr;
        y.iters += 1;
        if (rr <= y.tol2bb) { y.done = 1; y.converged = 1; }
        else if (y.iters >= st->maxit) y.done = 1;
        stop[s] = y.done;
    }
}

__global__ void k_sbeta(int32_t count, const int32_t *c0, SysState *sys, const double *prz, const BatchState *st)
{
    if (st->gate.done) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        SysState &y = sys[s];
        if (y.done) continue;
        const double rz = sys_sum(prz, c0, s);
        y.beta = rz / y.rz;
        y.rz = rz;
    }
}

__global__ void k_strue(int32_t count, const int32_t *c0, SysState *sys, const double *p)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x)
        sys[s].true_rr = sys_sum(p, c0, s);
}

// reopen the systems whose true residual failed the test (recurrence drift)
__global__ void k_sreopen(int32_t count, SysState *sys, int32_t *stop, const BatchState *st)
{
    const int32_t maxit = st->maxit;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        SysState &y = sys[s];
        if (y.converged && !(y.true_rr <= y.tol2bb) && y.iters < maxit) { y.converged = 0; y.done = 0; stop[s] = 0; }
    }
}

// gate.done = every system stopped (one block)
__global__ void k_sall(int32_t count, const SysState *sys, BatchState *st)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int mine = 0;
    for (int s = threadIdx.x; s < count; s += blockDim.x) mine |= !sys[s].done;
    if (mine) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) st->gate.done = any ? 0 : 1;
}

__global__ void k_sstate(BatchState *st, int32_t count, int32_t maxit)
{
    st->count = count;
    st->maxit = maxit;
    st->gate.done = 0;
}

inline int sgrid(int32_t count) { return (count + BT - 1) / BT > 0 ? (count + BT - 1) / BT : 1; }
inline int cgrid(int32_t nchunks) { return nchunks < 65535 ? (nchunks > 0 ? nchunks : 1) : 65535; }

}  // namespace

size_t batch_state_bytes() { return sizeof(BatchState); }

cudaError_t spcg_init(const SolveArgs &A, const BatchBuffers &B, double tol, int32_t maxit, cudaStream_t s)
{
    double *pbb = B.partials, *prz = B.partials + B.nchunks;
    k_sstate<<<1, 1, 0, s>>>(B.st, B.count, maxit);
    cudaError_t e0 = cudaMemsetAsync(B.stop, 0, sizeof(int32_t) * (size_t)B.count, s);
    if (e0 != cudaSuccess) return e0;
    k_cinit<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.b, B.x, B.r, pbb);
    count_launches(2);
    cudaError_t e = solve_fill_sentinels(A, B.solve, s);
    if (e != cudaSuccess) return e;
    e = solve_apply(A, B.solve, B.r, B.z, nullptr, s);
    if (e != cudaSuccess) return e;
    k_cdot<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.r, B.z, prz, nullptr);
    k_sinit<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys_c0, B.sys, B.stop, pbb, prz, tol, maxit);
    k_sall<<<1, BT, 0, s>>>(B.count, B.sys, B.st);
    k_ccopy<<<cgrid(B.nchunks), BT, 0, s>>>(A.n, B.z, B.p);
    count_launches(4);
    return cudaGetLastError();
}

cudaError_t spcg_iteration(const SolveArgs &A, const BatchBuffers &B, cudaStream_t s)
{
    double *ppq = B.partials, *prr = B.partials + B.nchunks, *prz = B.partials + 2 * (size_t)B.nchunks;
    const PcgState *gate = &B.st->gate;
    cudaError_t e = solve_spmv(A, B.p, B.q, gate, B.spmv_blocks, s);
    if (e != cudaSuccess) return e;
    k_cdot<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.p, B.q, ppq, B.st);
    k_salpha<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys_c0, B.sys, ppq, B.st);
    k_cupdate_xr<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.csys, B.sys, B.x, B.r, B.p, B.q, prr, B.st);
    k_scheck<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys_c0, B.sys, B.stop, prr, B.st);
    k_sall<<<1, BT, 0, s>>>(B.count, B.sys, B.st);
    count_launches(5);
    e = solve_apply(A, B.solve, B.r, B.z, gate, s);
    if (e != cudaSuccess) return e;
    k_cdot<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.r, B.z, prz, B.st);
    k_sbeta<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys_c0, B.sys, prz, B.st);
    k_cupdate_p<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.csys, B.sys, B.p, B.z, B.st);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t spcg_true_residual(const SolveArgs &A, const BatchBuffers &B, cudaStream_t s)
{
    cudaError_t e = solve_spmv(A, B.x, B.q, nullptr, B.spmv_blocks, s);
    if (e != cudaSuccess) return e;
    k_cresid<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.b, B.q, B.partials);
    k_strue<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys_c0, B.sys, B.partials);
    count_launches(2);
    return cudaGetLastError();
}

// after a true-residual check: reopen the systems whose recurrence converged
// but whose true residual did not, precondition the residual and update their
// search directions
cudaError_t spcg_reopen(const SolveArgs &A, const BatchBuffers &B, cudaStream_t s)
{
    double *prz = B.partials + 2 * (size_t)B.nchunks;
    k_sreopen<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys, B.stop, B.st);
    k_sall<<<1, BT, 0, s>>>(B.count, B.sys, B.st);
    count_launches(2);
    cudaError_t e = solve_apply(A, B.solve, B.r, B.z, &B.st->gate, s);
    if (e != cudaSuccess) return e;
    k_cdot<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.r, B.z, prz, B.st);
    k_sbeta<<<sgrid(B.count), BT, 0, s>>>(B.count, B.sys_c0, B.sys, prz, B.st);
    k_cupdate_p<<<cgrid(B.nchunks), BT, 0, s>>>(B.nchunks, B.clo, B.csys, B.sys, B.p, B.z, B.st);
    count_launches(3);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- concatenation
namespace {

template <typename T>
__global__ void k_cat(const CatSeg *seg, int32_t nseg, T *dst)
{
    for (int32_t k = blockIdx.y; k < nseg; k += gridDim.y) {
        const CatSeg q = seg[k];
        const T *src = (const T *)q.src;
        const T add = (T)q.add;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q.count; i += (int64_t)gridDim.x * blockDim.x)
            dst[q.dst + i] = src[i] + add;
    }
}

// dst_k[i] = src[q.src + i] + q.add for every segment k (the inverse of k_cat)
template <typename T>
__global__ void k_split(const SplitSeg *seg, int32_t nseg, const T *src)
{
    for (int32_t k = blockIdx.y; k < nseg; k += gridDim.y) {
        const SplitSeg q = seg[k];
        T *dst = (T *)q.dst;
        const T add = (T)q.add;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q.count; i += (int64_t)gridDim.x * blockDim.x)
            dst[i] = src[q.src + i] + add;
    }
}

__global__ void k_gather_ends(const int64_t *const *ptr, const int64_t *idx, int32_t m, int64_t *out)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) out[i] = ptr[i][idx[i]];
}

__global__ void k_seg_max(int64_t n, const int32_t *val, const int32_t *seg_of, int32_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicMax(out + seg_of[i], val[i]);
}

__global__ void k_seg_hist(int64_t n, const int32_t *val, const int32_t *seg_of, const int64_t *seg_off, int32_t *hist)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(hist + seg_off[seg_of[i]] + val[i], 1);
}

inline int grid1(int64_t n)
{
    int64_t b = (n + BT - 1) / BT;
    return (int)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

}  // namespace

cudaError_t launch_split(const SplitSeg *seg, int32_t nseg, int64_t max_count, int elem, bool is_float,
                         const void *src, cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t bx = (max_count + BT - 1) / BT;
    bx = bx < 1 ? 1 : bx > 64 ? 64 : bx;
    const dim3 grid((unsigned)bx, (unsigned)(nseg < 65535 ? nseg : 65535));
    if (elem == 8 && is_float) k_split<double><<<grid, BT, 0, s>>>(seg, nseg, (const double *)src);
    else if (elem == 8) k_split<int64_t><<<grid, BT, 0, s>>>(seg, nseg, (const int64_t *)src);
    else if (is_float) k_split<float><<<grid, BT, 0, s>>>(seg, nseg, (const float *)src);
    else k_split<int32_t><<<grid, BT, 0, s>>>(seg, nseg, (const int32_t *)src);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_ends(const int64_t *const *ptr, const int64_t *idx, int32_t m, int64_t *out, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_gather_ends<<<grid1(m), BT, 0, s>>>(ptr, idx, m, out); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_seg_max(int64_t n, const int32_t *val, const int32_t *seg_of, int32_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_seg_max<<<grid1(n), BT, 0, s>>>(n, val, seg_of, out); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_seg_hist(int64_t n, const int32_t *val, const int32_t *seg_of, const int64_t *seg_off,
                            int32_t *hist, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_seg_hist<<<grid1(n), BT, 0, s>>>(n, val, seg_of, seg_off, hist); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cat(const CatSeg *seg, int32_t nseg, int64_t max_count, int elem, bool is_float, void *dst,
                       cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t bx = (max_count + BT - 1) / BT;
    bx = bx < 1 ? 1 : bx > 64 ? 64 : bx;
    const dim3 grid((unsigned)bx, (unsigned)(nseg < 65535 ? nseg : 65535));
    if (elem == 8 && is_float) k_cat<double><<<grid, BT, 0, s>>>(seg, nseg, (double *)dst);
    else if (elem == 8) k_cat<int64_t><<<grid, BT, 0, s>>>(seg, nseg, (int64_t *)dst);
    else if (is_float) k_cat<float><<<grid, BT, 0, s>>>(seg, nseg, (float *)dst);
    else k_cat<int32_t><<<grid, BT, 0, s>>>(seg, nseg, (int32_t *)dst);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace parac
