// ingest.cu -- input preprocessing on the device (Sec. V conventions, Sec. III
// counter initialisation, Alg. 4 lines 1-2): ordering -> labels, validation,
// SDDM row excess -> ground-node edges, strict-lower CSC in label order,
// initial dependency counters and ready queue; plus the exclusive scan used
// throughout.
#include "common.cuh"
#include "kernels.h"

namespace parac {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// block-wide inclusive scan of one int64 per thread
__device__ int64_t block_scan_incl(int64_t x, int64_t *warp_tot)
{
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if ((int)lane >= off) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, off);
            if ((int)lane >= off) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (w > 0) x += warp_tot[w - 1];
    __syncthreads();
    return x;
}

__global__ void k_scan_reduce(const int32_t *in, int64_t n, int64_t *tile_sums)
{
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    const int64_t incl = block_scan_incl(s, wt);
    if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = incl;
}

// single block: exclusive scan of the tile sums in place, total to *total
__global__ void k_scan_top(int64_t *tile_sums, int64_t ntiles, int64_t *total)
{
    __shared__ int64_t wt[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < ntiles ? tile_sums[i] : 0;
        const int64_t incl = block_scan_incl(v, wt);
        if (i < ntiles) tile_sums[i] = carry + incl - v;
        if (threadIdx.x == blockDim.x - 1) wt[0] = incl;
        __syncthreads();
        carry += wt[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_down(const int32_t *in, int64_t n, const int64_t *tile_off, int64_t *out)
{
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    const int64_t incl = block_scan_incl(s, wt);
    int64_t run = tile_off[blockIdx.x] + incl - s;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
}

__global__ void k_set_total(int64_t *out, int64_t n, const int64_t *total) { out[n] = *total; }

// ---------------------------------------------------------------- labels
__global__ void k_iperm(int64_t n, const int32_t *ord, const int32_t *label_of_k, int32_t *iperm, int32_t *status)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ord[k];
        if (v < 0 || v >= n) { atomicOr(status, INGEST_BAD_INDEX); continue; }
        const int32_t lab = label_of_k ? label_of_k[k] : (int32_t)k;
        if (atomicExch(iperm + v, lab) != -1) atomicOr(status, INGEST_BAD_INDEX);
    }
}

__global__ void k_identity(int64_t n, int32_t *p)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = (int32_t)k;
}

__device__ __forceinline__ int32_t ground_of(const IngestArgs &a, int64_t j)
{
    if (!a.sys_of_orig) return a.single_ground;
    return a.sys_ground[a.sys_of_orig[j]];
}

// One thread per original column j: validation, row excess (sequential sum of
// the stored entries in stored order, diagonal included), ground edge,
// strict-lower count of label column iperm[j], counter increments.
__global__ void k_ingest_count(IngestArgs a)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = a.n;
        if (a.sys_of_orig) {
            const int32_t s = a.sys_of_orig[j];
            lo = a.sys_obase[s]; hi = lo + a.sys_n[s];
        }
        const int32_t lj = a.iperm[j];
        double e = 0.0, dg = 0.0;
        int32_t cnt = 0;
        bool bad = false, notsdd = false;
        for (int64_t t = a.colptr[j]; t < a.colptr[j + 1]; ++t) {
            const int32_t i = a.rowind[t];
            const double v = a.val[t];
            if (i < lo || i >= hi) { bad = true; continue; }
            if (i == j) dg = __dadd_rn(dg, v);
            else if (v > 0.0) notsdd = true;
            e = __dadd_rn(e, v);
            if (i != j && v != 0.0) {
                const int32_t li = a.iperm[i];
                if (li > lj) { ++cnt; atomicAdd(a.dp + li, 1); }
            }
        }
        double gw = 0.0;
        bool kindbad = false;
        if (!bad && !notsdd) {
            if (e < -1e-12 * dg || (e < 0.0 && dg <= 0.0)) notsdd = true;
            else if (e > 1e-12 * dg) {
                const int32_t gl = ground_of(a, j);
                if (a.kind == 1 || gl < 0) kindbad = true; // Laplacian requested but excess present
                else { gw = e; ++cnt; atomicAdd(a.dp + gl, 1); }
            }
        }
        if (bad) atomicOr(a.status, INGEST_BAD_INDEX);
        if (notsdd) atomicOr(a.status, INGEST_NOT_SDD);
        if (kindbad) atomicOr(a.status, INGEST_KIND);
        a.gw[j] = gw;
        a.lcnt[lj] = cnt;
    }
}

// One warp per original column: compact the strict-lower entries (stored
// order) into label column iperm[j], ground edge last.
__global__ void k_ingest_scatter(IngestArgs a, const int64_t *lcp, int32_t *lrow, double *lw)
{
    const unsigned lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp0; j < a.n; j += nwarps) {
        const int32_t lj = a.iperm[j];
        int64_t pos = lcp[lj];
        for (int64_t t0 = a.colptr[j]; t0 < a.colptr[j + 1]; t0 += 32) {
            const int64_t t = t0 + lane;
            bool take = false;
            int32_t li = 0;
            double v = 0.0;
            if (t < a.colptr[j + 1]) {
                const int32_t i = a.rowind[t];
                v = a.val[t];
                if (i != j && v != 0.0) { li = a.iperm[i]; take = li > lj; }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int64_t at = pos + __popc(bal & ((1u << lane) - 1u));
                lrow[at] = li;
                lw[at] = -v;
            }
            pos += __popc(bal);
        }
        if (lane == 0 && a.gw[j] > 0.0) {
            lrow[pos] = ground_of(a, j);
            lw[pos] = a.gw[j];
        }
    }
}

__global__ void k_queue_init(int32_t nl, const int32_t *dp, int32_t *queue, uint32_t *q_tail)
{
    const unsigned lane = threadIdx.x & 31;
    for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x) & ~31ll; i0 < nl; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + (threadIdx.x & ~31u) + lane;
        const bool ready = i < nl && dp[i] == 0;
        const unsigned bal = __ballot_sync(0xffffffffu, ready);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            uint32_t b = 0;
            if ((int)lane == leader) b = atomicAdd(q_tail, (uint32_t)__popc(bal));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (ready) queue[b + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
        }
    }
}

__global__ void k_add_off_i32(const int32_t *in, int32_t *out, int64_t n, int32_t off)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = in[k] + off;
}

__global__ void k_add_off_i64(const int64_t *in, int64_t *out, int64_t n, int64_t off)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = in[k] + off;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = v;
}

__global__ void k_iota_i32(int32_t *p, int64_t n, int32_t base)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = base + (int32_t)k;
}

// ---------------------------------------------------------------- NNZ-sorted ordering
// Sec. V's "NNZ-sorted" ordering (the paper's recommendation for the GPU):
// vertices by ascending count of stored entries in their column; ties by a
// seeded key, then by vertex index.  The key of local vertex v is the top 31
// bits of the (v+1)-th output of the splitmix64 generator started from state
// `seed` (Steele, Lea, Flood: "Fast splittable pseudorandom number
// generators", OOPSLA 2014).
__device__ __forceinline__ uint64_t splitmix64_output(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_order_keys(int64_t n, const int64_t *colptr, const int32_t *sys_of_v, const int32_t *sys_obase,
                             uint64_t seed, int32_t *tie, int32_t *deg, int32_t *ord)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lv = sys_of_v ? v - sys_obase[sys_of_v[v]] : v;
        tie[v] = (int32_t)(splitmix64_output(seed, (uint64_t)lv + 1) >> 33);
        const int64_t d = colptr[v + 1] - colptr[v];
        deg[v] = (int32_t)(d < 0x7fffffff ? d : 0x7fffffff);
        ord[v] = (int32_t)v;
    }
}

__global__ void k_gather_keys(int64_t n, const int32_t *src, const int32_t *ord, int32_t *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[ord[i]];
}

inline int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

}  // namespace

size_t scan_tmp_bytes(int64_t n)
{
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE + 1;
    return (size_t)(tiles + 1) * sizeof(int64_t);
}

cudaError_t scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t st)
{
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t *ts = (int64_t *)tmp;
    int64_t *total = ts + tiles + 1;
    if (tiles > 0) {
        k_scan_reduce<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, ts); count_launches(1);
        k_scan_top<<<1, 1024, 0, st>>>(ts, tiles, total); count_launches(1);
        k_scan_down<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, ts, out); count_launches(1);
    } else {
        cudaMemsetAsync(total, 0, sizeof(int64_t), st);
    }
    k_set_total<<<1, 1, 0, st>>>(out, n, total); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_iperm(int64_t n, const int32_t *ord, const int32_t *label_of_k, int32_t *iperm,
                         int32_t *status, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_iperm<<<grid_for(n, 256), 256, 0, st>>>(n, ord, label_of_k, iperm, status); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_identity_iperm(int64_t n, int32_t *iperm, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_identity<<<grid_for(n, 256), 256, 0, st>>>(n, iperm); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ingest_count(const IngestArgs &a, cudaStream_t st)
{
    if (a.n == 0) return cudaSuccess;
    k_ingest_count<<<grid_for(a.n, 128), 128, 0, st>>>(a); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ingest_scatter(const IngestArgs &a, const int64_t *lcp, int32_t *lrow, double *lw, cudaStream_t st)
{
    if (a.n == 0) return cudaSuccess;
    k_ingest_scatter<<<grid_for(a.n * 32, 256), 256, 0, st>>>(a, lcp, lrow, lw); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_queue_init(int32_t nl, const int32_t *dp, int32_t *queue, uint32_t *q_tail, cudaStream_t st)
{
    if (nl == 0) return cudaSuccess;
    k_queue_init<<<grid_for(nl, 256), 256, 0, st>>>(nl, dp, queue, q_tail); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_add_offset_i32(const int32_t *in, int32_t *out, int64_t n, int32_t off, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_add_off_i32<<<grid_for(n, 256), 256, 0, st>>>(in, out, n, off); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_add_offset_i64(const int64_t *in, int64_t *out, int64_t n, int64_t off, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_add_off_i64<<<grid_for(n, 256), 256, 0, st>>>(in, out, n, off); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_fill_i32<<<grid_for(n, 256), 256, 0, st>>>(p, n, v); count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_iota_i32(int32_t *p, int64_t n, int32_t base, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_iota_i32<<<grid_for(n, 256), 256, 0, st>>>(p, n, base); count_launches(1);
    return cudaGetLastError();
}

size_t nnz_order_tmp_bytes(int64_t n) { return 12 * (size_t)n + radix_tmp_bytes(n) + 256; }

cudaError_t nnz_sorted_order(int64_t n, const int64_t *colptr, const int32_t *sys_of_v, const int32_t *sys_obase,
                             int32_t nsys, uint64_t seed, int32_t *ord, void *tmp, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    int32_t *tie = (int32_t *)tmp, *deg = tie + n, *key = deg + n;
    void *rtmp = (void *)(((uintptr_t)(key + n) + 255) & ~(uintptr_t)255);
    const int g = grid_for(n, 256);
    k_order_keys<<<g, 256, 0, st>>>(n, colptr, sys_of_v, sys_obase, seed, tie, deg, ord); count_launches(1);
    // stable passes from the least significant key: tie, then degree, then system
    cudaError_t e = stable_sort_pairs((int32_t)n, tie, ord, 31, rtmp, st);
    if (e != cudaSuccess) return e;
    k_gather_keys<<<g, 256, 0, st>>>(n, deg, ord, key); count_launches(1);
    e = stable_sort_pairs((int32_t)n, key, ord, 31, rtmp, st);
    if (e != cudaSuccess || !sys_of_v) return e;
    int bits = 0;
    while (bits < 31 && ((nsys - 1) >> bits) != 0) ++bits;
    k_gather_keys<<<g, 256, 0, st>>>(n, sys_of_v, ord, key); count_launches(1);
    return stable_sort_pairs((int32_t)n, key, ord, bits, rtmp, st);
}

}  // namespace parac
