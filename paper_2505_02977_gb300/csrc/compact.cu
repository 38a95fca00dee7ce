// compact.cu -- factor compaction (the step between the elimination and the
// solve; the paper's GPU "Total" counts the solver's analysis here, Sec. V-B):
// per-pivot columns written anywhere in the factor workspace become CSC(F)
// with F(u,k) = -w_u / D_k (Sec. IV scaled form), ground rows/columns
// removed (Sec. V SDDM handling), plus CSR(F) by transposition for the
// forward triangular solve and optional FP32 copies.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace parac {

namespace {

inline int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

__global__ void k_out_of_label_single(int32_t nl, int32_t n, int32_t *o)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x)
        o[l] = l < n ? (int32_t)l : -1;
}

__global__ void k_out_of_label_batch(int32_t nl, const int32_t *sys_of_label, const int32_t *sys_lbase,
                                     const int32_t *sys_obase, const int32_t *sys_n, int32_t *o)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = sys_of_label[l];
        const int32_t loc = (int32_t)l - sys_lbase[s];
        o[l] = loc < sys_n[s] ? sys_obase[s] + loc : -1;
    }
}

__global__ void k_sys_of_label(int32_t S, const int32_t *sys_lbase, int32_t nl, int32_t *sys_of_label)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = sys_lbase[s], e = (s + 1 < S) ? sys_lbase[s + 1] : nl;
        for (int32_t l = b; l < e; ++l) sys_of_label[l] = (int32_t)s;
    }
}

// output column length: the pivot's merged count, minus its ground row (the
// largest label of its system, hence last in row order) when present
__global__ void k_out_len(int32_t nl, const int32_t *out_of_label, const int64_t *f_start, const int32_t *f_len,
                          const int32_t *f_row, int32_t *olen)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = out_of_label[l];
        if (o < 0) continue;
        int32_t len = f_len[l];
        if (len > 0 && out_of_label[f_row[f_start[l] + len - 1]] < 0) --len;
        olen[o] = len;
    }
}

// one warp per label column
__global__ void k_gather_factor(int32_t nl, const int32_t *out_of_label, const int64_t *f_start,
                                const int32_t *f_row, const double *f_val, const double *D, const int64_t *fcp,
                                int32_t *Frow, double *Fval, double *Dout)
{
    const unsigned lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = w0; l < nl; l += nw) {
        const int32_t o = out_of_label[l];
        if (o < 0) continue;
        const int64_t dst = fcp[o];
        const int64_t len = fcp[o + 1] - dst;
        const int64_t src = f_start[l];
        const double Dk = D[l];
        for (int64_t i = lane; i < len; i += 32) {
            Frow[dst + i] = out_of_label[f_row[src + i]];
            Fval[dst + i] = __ddiv_rn(-f_val[src + i], Dk);
        }
        if (lane == 0) Dout[o] = Dk;
    }
}

__global__ void k_row_count(int64_t nnz, const int32_t *rows, int32_t *cnt)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + rows[t], 1);
}

// one warp per column of CSC: entries go to their rows in CSR
__global__ void k_transpose_scatter(int32_t n, const int64_t *cp, const int32_t *rows, const double *vals,
                                    const int64_t *rp, int32_t *cursor, int32_t *cols_out, double *vals_out)
{
    const unsigned lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < n; c += nw) {
        for (int64_t t = cp[c] + lane; t < cp[c + 1]; t += 32) {
            const int32_t r = rows[t];
            const int64_t at = rp[r] + atomicAdd(cursor + r, 1);
            cols_out[at] = (int32_t)c;
            vals_out[at] = vals[t];
        }
    }
}

// Sort each CSR row by column (one warp per row, rows of up to SORT_STAGE
// entries staged in shared memory; an entry's slot is the number of entries
// with a smaller column).  Longer rows keep the scatter order, which only
// changes the summation order of the forward solve.
constexpr int SORT_STAGE = 256;

__global__ void k_sort_rows(int32_t n, const int64_t *rp, int32_t *cols, double *vals)
{
    __shared__ int32_t sc[8][SORT_STAGE];
    __shared__ double sv[8][SORT_STAGE];
    const unsigned lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw) {
        const int64_t b = rp[r], len = rp[r + 1] - b;
        if (len <= 1 || len > SORT_STAGE) continue;
        for (int64_t i = lane; i < len; i += 32) { sc[wib][i] = cols[b + i]; sv[wib][i] = vals[b + i]; }
        __syncwarp();
        for (int64_t i = lane; i < len; i += 32) {
            const int32_t c = sc[wib][i];
            int64_t rank = 0;
            for (int64_t q = 0; q < len; ++q) rank += sc[wib][q] < c;
            cols[b + rank] = c;
            vals[b + rank] = sv[wib][i];
        }
        __syncwarp();
    }
}

__global__ void k_scatter_levels(int32_t nl, const int32_t *out_of_label, const int32_t *lvl, int32_t *lev_out)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = out_of_label[l];
        if (o >= 0) lev_out[o] = lvl[l];
    }
}

__global__ void k_max_i32(const int32_t *a, int64_t n, int32_t *mx)
{
    int32_t m = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = max(m, a[t]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// ---------------------------------------------------------------- stable radix sort (key, value) pairs
// One 8-bit digit per pass, least significant first; every pass is stable, so
// after the passes the pairs are ordered by key and, within a key, keep their
// input order.  A tile of RADIX_TILE pairs per block: the per-tile digit
// histograms (digit-major) are scanned into each (digit, tile)'s output
// offset, and each tile scatters its pairs in input order: RADIX_TILE / 256
// rounds of 256 pairs, a pair's rank among its round's equal digits found from
// its warp's match mask plus the counts of the warps before it.
constexpr int RADIX_THREADS = 256, RADIX_ROUNDS = 8, RADIX_TILE = RADIX_THREADS * RADIX_ROUNDS;

__global__ void __launch_bounds__(RADIX_THREADS) k_radix_hist(int32_t n, const int32_t *keys, int shift, int32_t ntiles,
                                                              int32_t *hist)
{
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        const int64_t i = base + r * RADIX_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RADIX_THREADS) k_radix_scatter(int32_t n, const int32_t *keys, const int32_t *vals,
                                                                 int shift, int32_t ntiles, const int64_t *offs,
                                                                 int32_t *keys_out, int32_t *vals_out)
{
    __shared__ int32_t run[256];                  // pairs of each digit placed by earlier rounds
    __shared__ int32_t wcnt[RADIX_THREADS / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    run[threadIdx.x] = 0;
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        for (int w = 0; w < RADIX_THREADS / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + r * RADIX_THREADS + threadIdx.x;
        const bool in = i < n;
        const int32_t k = in ? keys[i] : 0;
        const int d = in ? (k >> shift) & 255 : 256;           // 256: no pair
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (in && (peers & lt) == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (in) {
            int32_t rank = run[d] + __popc(peers & lt);
            for (int w = 0; w < warp; ++w) rank += wcnt[w][d];
            const int64_t at = offs[(int64_t)d * ntiles + blockIdx.x] + rank;
            keys_out[at] = k;
            vals_out[at] = vals[i];
        }
        __syncthreads();
        int32_t add = 0;
        for (int w = 0; w < RADIX_THREADS / 32; ++w) add += wcnt[w][threadIdx.x];
        run[threadIdx.x] += add;
    }
}

__global__ void k_copy_i32(int64_t n, const int32_t *a, int32_t *b)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = a[t];
}

// Sort rows of more than SORT_STAGE and at most SORT_LONG entries by column,
// one block per row staged in shared memory (rank = entries with a smaller
// column; the columns of a row are distinct).
constexpr int SORT_LONG = 2048;

__global__ void __launch_bounds__(256) k_sort_long_rows(int32_t n, const int64_t *rp, int32_t *cols, double *vals)
{
    __shared__ int32_t sc[SORT_LONG];
    __shared__ double sv[SORT_LONG];
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t b = rp[r], len = rp[r + 1] - b;
        if (len <= SORT_STAGE || len > SORT_LONG) continue;
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) { sc[i] = cols[b + i]; sv[i] = vals[b + i]; }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
            const int32_t c = sc[i];
            int64_t rank = 0;
            for (int64_t q = 0; q < len; ++q) rank += sc[q] < c;
            cols[b + rank] = c;
            vals[b + rank] = sv[i];
        }
        __syncthreads();
    }
}

__global__ void k_inverse_perm(int32_t n, const int32_t *order, int32_t *posof)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        posof[order[t]] = (int32_t)t;
}

__global__ void k_relabel_lengths(int32_t n, const int32_t *order, const int64_t *cp, int32_t *len)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = order[t];
        len[t] = (int32_t)(cp[c + 1] - cp[c]);
    }
}

// one warp per new column j: old column order[j], rows mapped to positions
__global__ void k_relabel_gather(int32_t n, const int32_t *order, const int32_t *posof, const int64_t *cp,
                                 const int32_t *rows, const double *vals, const int64_t *ncp, int32_t *nrows,
                                 double *nvals)
{
    const unsigned lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w0; j < n; j += nw) {
        const int32_t c = order[j];
        const int64_t src = cp[c], len = cp[c + 1] - src, dst = ncp[j];
        for (int64_t i = lane; i < len; i += 32) {
            nrows[dst + i] = posof[rows[src + i]];
            nvals[dst + i] = vals[src + i];
        }
    }
}

__global__ void k_gather_i32(int32_t n, const int32_t *idx, const int32_t *src, int32_t *dst)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[idx[t]];
}

__global__ void k_gather_f64(int32_t n, const int32_t *idx, const double *src, double *dst)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[idx[t]];
}

__global__ void k_to_f32(const double *in, float *out, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = __double2float_rn(in[t]);
}

__global__ void k_dinv(int32_t n, const double *D, double *Dinv)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        Dinv[t] = D[t] > 0.0 ? 1.0 / D[t] : 0.0;
}

// ---------------------------------------------------------------- solve group tables on the device
// The group table of row_groups (schedule.cpp) built by scans: walk position
// kk takes row j = kk (or n - 1 - kk descending) of `ptr`.  A row longer than
// long_row is "long"; a maximal run of short positions is cut into groups of
// `warps` consecutive positions from the run's start; a long row emits one
// shared group, or (above split_row) nch = ceil(len / chunk) chunk groups
// followed by their combine, with nch partial slots.  Groups are emitted at
// their first position, in walk order.
__global__ void k_rg_mark(const int64_t *ptr, int64_t n, int desc, int long_row, int split_row, int chunk,
                          int32_t *islong, int32_t *cntL, int32_t *slots)
{
    for (int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kk < n; kk += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = desc ? n - 1 - kk : kk;
        const int64_t len = ptr[j + 1] - ptr[j];
        const bool lng = len > long_row;
        const int32_t nch = (int32_t)((len + chunk - 1) / chunk);
        islong[kk] = lng ? 1 : 0;
        cntL[kk] = lng ? (len > split_row ? nch + 1 : 1) : 0;
        slots[kk] = lng && len > split_row ? nch : 0;
    }
}

__global__ void k_rg_longpos(int64_t n, const int32_t *islong, const int64_t *lrank, int64_t *longpos)
{
    for (int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kk < n; kk += (int64_t)gridDim.x * blockDim.x)
        if (islong[kk]) longpos[lrank[kk]] = kk;
}

// groups emitted at each position (cntL for long rows, 1 where a short group starts)
__global__ void k_rg_count(int64_t n, int warps, const int32_t *islong, const int64_t *lrank, const int64_t *longpos,
                           int32_t *cnt)
{
    for (int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kk < n; kk += (int64_t)gridDim.x * blockDim.x) {
        if (islong[kk]) continue;
        const int64_t r = lrank[kk];
        const int64_t prev = r > 0 ? longpos[r - 1] : -1;
        cnt[kk] = ((kk - prev - 1) % warps) == 0 ? 1 : 0;
    }
}

__global__ void k_rg_write(const int64_t *ptr, int64_t n, int desc, int warps, int split_row, int chunk,
                           const int32_t *islong, const int64_t *lrank, const int64_t *longpos, const int64_t *goff,
                           const int64_t *soff, int32_t *g)
{
    for (int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kk < n; kk += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g0 = goff[kk];
        if (!islong[kk]) {
            if (goff[kk + 1] == g0) continue;                // no group starts here
            const int64_t r = lrank[kk], nlong = lrank[n];
            const int64_t next = r < nlong ? longpos[r] : n;
            const int64_t rows = next - kk < warps ? next - kk : warps;
            int32_t *e = g + 4 * g0;
            e[0] = (int32_t)kk; e[1] = GK_ROWS; e[2] = (int32_t)rows; e[3] = 0;
            continue;
        }
        const int64_t j = desc ? n - 1 - kk : kk;
        const int64_t len = ptr[j + 1] - ptr[j];
        if (len > split_row) {
            const int32_t nch = (int32_t)((len + chunk - 1) / chunk);
            const int32_t s0 = (int32_t)soff[kk];
            for (int32_t c = 0; c < nch; ++c) {
                int32_t *e = g + 4 * (g0 + c);
                e[0] = (int32_t)kk; e[1] = GK_CHUNK; e[2] = c; e[3] = s0 + c;
            }
            int32_t *e = g + 4 * (g0 + nch);
            e[0] = (int32_t)kk; e[1] = GK_COMBINE; e[2] = nch; e[3] = s0;
        } else {
            int32_t *e = g + 4 * g0;
            e[0] = (int32_t)kk; e[1] = GK_SHARED; e[2] = 0; e[3] = 0;
        }
    }
}

// ---------------------------------------------------------------- rows above SORT_LONG entries
// Rows longer than the shared-memory row sort are sorted by column as one
// segmented sort: their entries gathered into one buffer (segment = the
// row's rank among them), stably sorted by column, then stably by segment,
// and written back into their rows.
__global__ void k_huge_flags(int32_t n, const int64_t *rp, int lim, int32_t *flag, int32_t *len)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = rp[r + 1] - rp[r];
        flag[r] = l > lim ? 1 : 0;
        len[r] = l > lim ? (int32_t)l : 0;
    }
}

// one block per row (grid-stride over rows); seg_start[s] / seg_row[s]: the
// segment's first buffer position and its row's first CSR position
__global__ void k_huge_gather(int32_t n, const int64_t *rp, const int32_t *flag, const int64_t *hrank,
                              const int64_t *hoff, const int32_t *cols, const double *vals, int32_t *key,
                              int32_t *idx, int32_t *seg_of, int32_t *tcol, double *tval, int64_t *seg_start,
                              int64_t *seg_row)
{
    for (int32_t r = blockIdx.x; r < n; r += gridDim.x) {
        if (!flag[r]) continue;
        const int64_t s = hrank[r], base = hoff[r], start = rp[r], len = rp[r + 1] - start;
        if (threadIdx.x == 0) { seg_start[s] = base; seg_row[s] = start; }
        for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
            const int32_t c = cols[start + t];
            key[base + t] = c; idx[base + t] = (int32_t)(base + t); seg_of[base + t] = (int32_t)s;
            tcol[base + t] = c; tval[base + t] = vals[start + t];
        }
    }
}

__global__ void k_huge_segkeys(int64_t e, const int32_t *idx, const int32_t *seg_of, int32_t *key)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < e; t += (int64_t)gridDim.x * blockDim.x)
        key[t] = seg_of[idx[t]];
}

__global__ void k_huge_scatter(int64_t e, const int32_t *idx, const int32_t *seg, const int64_t *seg_start,
                               const int64_t *seg_row, const int32_t *tcol, const double *tval, int32_t *cols,
                               double *vals)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < e; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = seg[t], src = idx[t];
        const int64_t pos = seg_row[s] + (t - seg_start[s]);
        cols[pos] = tcol[src];
        vals[pos] = tval[src];
    }
}

}  // namespace

cudaError_t launch_out_of_label_single(int32_t nl, int32_t n, int32_t *o, cudaStream_t st)
{
    if (nl == 0) return cudaSuccess;
    k_out_of_label_single<<<grid_for(nl, 256), 256, 0, st>>>(nl, n, o); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_out_of_label_batch(int32_t nl, const int32_t *sys_of_label, const int32_t *sys_lbase,
                                      const int32_t *sys_obase, const int32_t *sys_n, int32_t *o, cudaStream_t st)
{
    if (nl == 0) return cudaSuccess;
    k_out_of_label_batch<<<grid_for(nl, 256), 256, 0, st>>>(nl, sys_of_label, sys_lbase, sys_obase, sys_n, o); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sys_of_label(int32_t S, const int32_t *sys_lbase, int32_t nl, int32_t *sys_of_label, cudaStream_t st)
{
    if (S == 0) return cudaSuccess;
    k_sys_of_label<<<grid_for(S, 64), 64, 0, st>>>(S, sys_lbase, nl, sys_of_label); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_out_len(int32_t nl, const int32_t *out_of_label, const int64_t *f_start, const int32_t *f_len,
                           const int32_t *f_row, int32_t *olen, cudaStream_t st)
{
    if (nl == 0) return cudaSuccess;
    k_out_len<<<grid_for(nl, 256), 256, 0, st>>>(nl, out_of_label, f_start, f_len, f_row, olen); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_factor(int32_t nl, const int32_t *out_of_label, const int64_t *f_start,
                                 const int32_t *f_row, const double *f_val, const double *D, const int64_t *fcp,
                                 int32_t *Frow, double *Fval, double *Dout, cudaStream_t st)
{
    if (nl == 0) return cudaSuccess;
    k_gather_factor<<<grid_for((int64_t)nl * 32, 256), 256, 0, st>>>(nl, out_of_label, f_start, f_row, f_val, D,
                                                                     fcp, Frow, Fval, Dout); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_row_count(int64_t nnz, const int32_t *rows, int32_t *cnt, cudaStream_t st)
{
    if (nnz == 0) return cudaSuccess;
    k_row_count<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, rows, cnt); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transpose_scatter(int32_t n, const int64_t *cp, const int32_t *rows, const double *vals,
                                     const int64_t *rp, int32_t *cursor, int32_t *cols_out, double *vals_out,
                                     cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_transpose_scatter<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, cp, rows, vals, rp, cursor, cols_out,
                                                                         vals_out); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sort_rows(int32_t n, const int64_t *rp, int32_t *cols, double *vals, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_sort_rows<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, rp, cols, vals); count_launches(1);
    return cudaGetLastError();
}

size_t radix_tmp_bytes(int64_t n)
{
    const int64_t ntiles = (n + RADIX_TILE - 1) / RADIX_TILE;
    const int64_t nh = 256 * std::max<int64_t>(ntiles, 1);
    return 8 * (size_t)n + 4 * (size_t)nh + 8 * (size_t)(nh + 1) + scan_tmp_bytes(nh + 1) + 512;
}

cudaError_t stable_sort_pairs(int32_t n, int32_t *keys, int32_t *vals, int key_bits, void *tmp, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    const int32_t ntiles = (int32_t)((n + RADIX_TILE - 1) / RADIX_TILE);
    const int64_t nh = 256 * (int64_t)ntiles;
    char *p = (char *)tmp;
    int32_t *k2 = (int32_t *)p; p += 4 * (size_t)n;
    int32_t *v2 = (int32_t *)p; p += 4 * (size_t)n;
    int32_t *hist = (int32_t *)p; p += 4 * (size_t)nh;
    p = (char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    int64_t *offs = (int64_t *)p; p += 8 * (size_t)(nh + 1);
    void *stmp = (void *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    int32_t *ki = keys, *vi = vals, *ko = k2, *vo = v2;
    int passes = 0;
    for (int shift = 0; shift < std::max(key_bits, 1); shift += 8, ++passes) {
        k_radix_hist<<<ntiles, RADIX_THREADS, 0, st>>>(n, ki, shift, ntiles, hist); count_launches(1);
        cudaError_t e = scan_i32_to_i64(hist, offs, nh, stmp, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<ntiles, RADIX_THREADS, 0, st>>>(n, ki, vi, shift, ntiles, offs, ko, vo); count_launches(1);
        std::swap(ki, ko); std::swap(vi, vo);
    }
    if (passes & 1) {            // the sorted pairs are in the scratch arrays
        k_copy_i32<<<grid_for(n, 256), 256, 0, st>>>(n, ki, keys); count_launches(1);
        k_copy_i32<<<grid_for(n, 256), 256, 0, st>>>(n, vi, vals); count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort_long_rows(int32_t n, const int64_t *rp, int32_t *cols, double *vals, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_sort_long_rows<<<std::min(n, 1024), 256, 0, st>>>(n, rp, cols, vals); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scatter_levels(int32_t nl, const int32_t *out_of_label, const int32_t *lvl, int32_t *lev_out,
                                  cudaStream_t st)
{
    if (nl == 0) return cudaSuccess;
    k_scatter_levels<<<grid_for(nl, 256), 256, 0, st>>>(nl, out_of_label, lvl, lev_out); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_max_i32(const int32_t *a, int64_t n, int32_t *mx, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_max_i32<<<grid_for(n, 256) < 1024 ? grid_for(n, 256) : 1024, 256, 0, st>>>(a, n, mx); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_inverse_perm(int32_t n, const int32_t *order, int32_t *posof, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_inverse_perm<<<grid_for(n, 256), 256, 0, st>>>(n, order, posof);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_relabel_lengths(int32_t n, const int32_t *order, const int64_t *cp, int32_t *len, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_relabel_lengths<<<grid_for(n, 256), 256, 0, st>>>(n, order, cp, len);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_relabel_gather(int32_t n, const int32_t *order, const int32_t *posof, const int64_t *cp,
                                  const int32_t *rows, const double *vals, const int64_t *ncp, int32_t *nrows,
                                  double *nvals, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_relabel_gather<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, order, posof, cp, rows, vals, ncp, nrows,
                                                                      nvals);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_i32(int32_t n, const int32_t *idx, const int32_t *src, int32_t *dst, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_gather_i32<<<grid_for(n, 256), 256, 0, st>>>(n, idx, src, dst);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_f64(int32_t n, const int32_t *idx, const double *src, double *dst, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_gather_f64<<<grid_for(n, 256), 256, 0, st>>>(n, idx, src, dst);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double *in, float *out, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_to_f32<<<grid_for(n, 256), 256, 0, st>>>(in, out, n); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dinv(int32_t n, const double *D, double *Dinv, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_dinv<<<grid_for(n, 256), 256, 0, st>>>(n, D, Dinv); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- solve group tables on the device
size_t row_groups_tmp_bytes(int64_t n)
{
    const size_t n1 = (size_t)n + 1;
    return 3 * 4 * n1 + 4 * 8 * n1 + scan_tmp_bytes(n + 1) + 1024;
}

// First pass: counts (ngroups, nslots), read back to the host (one small copy).
cudaError_t row_groups_count(const int64_t *ptr, int64_t n, bool descending, int warps, int long_row, int split_row,
                             int chunk, void *tmp, int64_t *ngroups, int64_t *nslots, cudaStream_t st)
{
    *ngroups = 0; *nslots = 0;
    if (n <= 0) return cudaSuccess;
    const size_t n1 = (size_t)n + 1;
    unsigned char *t = (unsigned char *)tmp;
    int32_t *islong = (int32_t *)t, *cnt = islong + n1, *slots = cnt + n1;
    int64_t *lrank = (int64_t *)(((uintptr_t)(slots + n1) + 15) & ~(uintptr_t)15);
    int64_t *longpos = lrank + n1, *goff = longpos + n1, *soff = goff + n1;
    void *stmp = (void *)(((uintptr_t)(soff + n1) + 255) & ~(uintptr_t)255);
    const int gr = grid_for(n, 256);
    k_rg_mark<<<gr, 256, 0, st>>>(ptr, n, descending ? 1 : 0, long_row, split_row, chunk, islong, cnt, slots);
    count_launches(1);
    cudaError_t e = scan_i32_to_i64(islong, lrank, n, stmp, st);
    if (e != cudaSuccess) return e;
    k_rg_longpos<<<gr, 256, 0, st>>>(n, islong, lrank, longpos); count_launches(1);
    k_rg_count<<<gr, 256, 0, st>>>(n, warps, islong, lrank, longpos, cnt); count_launches(1);
    e = scan_i32_to_i64(cnt, goff, n, stmp, st);
    if (e != cudaSuccess) return e;
    e = scan_i32_to_i64(slots, soff, n, stmp, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(ngroups, goff + n, 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(nslots, soff + n, 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

// Second pass: the table (4 ints per group) from the first pass's scans in tmp.
cudaError_t row_groups_write(const int64_t *ptr, int64_t n, bool descending, int warps, int split_row, int chunk,
                             const void *tmp, int32_t *table, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const size_t n1 = (size_t)n + 1;
    const unsigned char *t = (const unsigned char *)tmp;
    const int32_t *islong = (const int32_t *)t, *slots = islong + 2 * n1;
    const int64_t *lrank = (const int64_t *)(((uintptr_t)(slots + n1) + 15) & ~(uintptr_t)15);
    const int64_t *longpos = lrank + n1, *goff = longpos + n1, *soff = goff + n1;
    k_rg_write<<<grid_for(n, 256), 256, 0, st>>>(ptr, n, descending ? 1 : 0, warps, split_row, chunk, islong, lrank,
                                                  longpos, goff, soff, table);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- rows above SORT_LONG entries
size_t huge_rows_tmp_bytes(int64_t n)
{
    const size_t n1 = (size_t)n + 1;
    return 2 * 4 * n1 + 2 * 8 * n1 + scan_tmp_bytes(n + 1) + 512;
}

cudaError_t huge_rows_count(int32_t n, const int64_t *rp, void *tmp, int64_t *nrows, int64_t *entries,
                            cudaStream_t st)
{
    *nrows = 0; *entries = 0;
    if (n <= 0) return cudaSuccess;
    const size_t n1 = (size_t)n + 1;
    int32_t *flag = (int32_t *)tmp, *len = flag + n1;
    int64_t *hrank = (int64_t *)(((uintptr_t)(len + n1) + 15) & ~(uintptr_t)15), *hoff = hrank + n1;
    void *stmp = (void *)(((uintptr_t)(hoff + n1) + 255) & ~(uintptr_t)255);
    k_huge_flags<<<grid_for(n, 256), 256, 0, st>>>(n, rp, SORT_LONG, flag, len); count_launches(1);
    cudaError_t e = scan_i32_to_i64(flag, hrank, n, stmp, st);
    if (e != cudaSuccess) return e;
    e = scan_i32_to_i64(len, hoff, n, stmp, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(nrows, hrank + n, 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(entries, hoff + n, 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

size_t huge_rows_sort_bytes(int64_t nrows, int64_t entries)
{
    const size_t e = (size_t)entries;
    return 4 * 4 * e + 8 * e + 2 * 8 * (size_t)nrows + radix_tmp_bytes(entries) + 1024;
}

cudaError_t huge_rows_sort(int32_t n, const int64_t *rp, int32_t *cols, double *vals, const void *tmp, int64_t nrows,
                           int64_t entries, void *work, cudaStream_t st)
{
    if (nrows <= 0 || entries <= 0) return cudaSuccess;
    const size_t n1 = (size_t)n + 1, e = (size_t)entries;
    const int32_t *flag = (const int32_t *)tmp, *len = flag + n1;
    const int64_t *hrank = (const int64_t *)(((uintptr_t)(len + n1) + 15) & ~(uintptr_t)15), *hoff = hrank + n1;
    unsigned char *w = (unsigned char *)work;
    int32_t *key = (int32_t *)w, *idx = key + e, *seg_of = idx + e, *tcol = seg_of + e;
    double *tval = (double *)(((uintptr_t)(tcol + e) + 15) & ~(uintptr_t)15);
    int64_t *seg_start = (int64_t *)(tval + e), *seg_row = seg_start + nrows;
    void *rtmp = (void *)(((uintptr_t)(seg_row + nrows) + 255) & ~(uintptr_t)255);
    k_huge_gather<<<std::min(n, 4096), 256, 0, st>>>(n, rp, flag, hrank, hoff, cols, vals, key, idx, seg_of, tcol, tval,
                                                     seg_start, seg_row);
    count_launches(1);
    int cbits = 1, sbits = 1;
    while (cbits < 31 && ((int64_t)1 << cbits) < (int64_t)n) ++cbits;
    while (sbits < 31 && ((int64_t)1 << sbits) < nrows) ++sbits;
    cudaError_t er = stable_sort_pairs((int32_t)entries, key, idx, cbits, rtmp, st);   // by column
    if (er != cudaSuccess) return er;
    k_huge_segkeys<<<grid_for(entries, 256), 256, 0, st>>>(entries, idx, seg_of, key); count_launches(1);
    er = stable_sort_pairs((int32_t)entries, key, idx, sbits, rtmp, st);                // then by row
    if (er != cudaSuccess) return er;
    k_huge_scatter<<<grid_for(entries, 256), 256, 0, st>>>(entries, idx, key, seg_start, seg_row, tcol, tval, cols, vals);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace parac
