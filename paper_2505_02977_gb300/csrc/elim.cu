// elim.cu -- persistent randomized-elimination kernel (rchol's SampleClique per
// pivot, Alg. 2; scheduled by ParAC's dependency counters, Sec. III; one
// persistent launch for the whole factorisation as in Alg. 4 / Sec. IV-C).
//
// Worker = one warp.  A worker claims ready-queue slots with one atomicAdd per
// `queue_chunk` slots, waits (bounded) until a slot is published, and then
// eliminates that vertex k:
//   gather     original strict-lower column k + every fill entry appended to
//              column k (inline slab + overflow levels)
//   sort       by (row, weight bits), bitonic network over the padded length
//   merge      each equal-row run summed left to right -> (u, w_u, m_u)
//   store      row-ordered (u, w_u) into the factor workspace (F values are
//              -w_u / D_k, formed later by the compaction kernel)
//   sort       by (weight bits, row), carrying m_u
//   scan       canonical suffix sums S (32-lane Hillis-Steele tiles over the
//              reversed weights, serial tile carries) and their exact
//              running maximum M; D_k = S[0]
//   sample     slot p = 1..d-1: v from Philox4x64-10 counter (k, p, sys, 0),
//              R = S[p] v, pick the largest j with M[j] >= R (equivalently
//              S[j] >= R), weight c = (S[p] w_{p-1}) / D_k; append
//              (max(u,v), c) to column min(u,v) and increment its counter
//   release    fence, then every neighbour's counter drops by m_u; a
//              positive-to-zero transition publishes the vertex on the queue.
// Working sets up to `warp_cap` entries live in the warp's shared memory, up
// to `block_cap` in one per-CTA shared buffer (taken under a CTA lock), larger
// ones in a global scratch arena.
#include "common.cuh"
#include "kernels.h"

namespace parac {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int32_t ROW_SENTINEL = 0x7fffffff;

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

struct View {           // per-vertex working set
    double *w;          // weights
    double *S;          // suffix sums
    double *M;          // running maximum of S from the right
    int32_t *row;
    int32_t *mult;
};

__device__ __forceinline__ View make_view(unsigned char *base, int cap)
{
    View v;
    v.w = (double *)base;
    v.S = (double *)(base + 8 * (size_t)cap);
    v.M = (double *)(base + 16 * (size_t)cap);
    v.row = (int32_t *)(base + 24 * (size_t)cap);
    v.mult = (int32_t *)(base + 28 * (size_t)cap);
    return v;
}

__device__ __forceinline__ int next_pow2(int x)
{
    return x <= 1 ? 1 : 1 << (32 - __clz(x - 1));
}

// Bitonic sort of P (power of two) entries by (row, weight bits).
__device__ void sort_row_bits(View v, int P)
{
    const unsigned lane = lane_id();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < (P >> 1); t += 32) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const int l = i + j;
                const bool asc = (i & kk) == 0;
                const int32_t ri = v.row[i], rl = v.row[l];
                const double wi = v.w[i], wl = v.w[l];
                const bool gt = (ri > rl) || (ri == rl && dbits(wi) > dbits(wl));
                if (gt == asc) {
                    v.row[i] = rl; v.row[l] = ri;
                    v.w[i] = wl; v.w[l] = wi;
                }
            }
            __syncwarp();
        }
    }
}

// Bitonic sort of P entries by (weight bits, row), carrying the multiplicity.
__device__ void sort_bits_row(View v, int P)
{
    const unsigned lane = lane_id();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < (P >> 1); t += 32) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const int l = i + j;
                const bool asc = (i & kk) == 0;
                const double wi = v.w[i], wl = v.w[l];
                const int32_t ri = v.row[i], rl = v.row[l];
                const unsigned long long bi = dbits(wi), bl = dbits(wl);
                const bool gt = (bi > bl) || (bi == bl && ri > rl);
                if (gt == asc) {
                    const int32_t mi = v.mult[i], ml = v.mult[l];
                    v.row[i] = rl; v.row[l] = ri;
                    v.w[i] = wl; v.w[l] = wi;
                    v.mult[i] = ml; v.mult[l] = mi;
                }
            }
            __syncwarp();
        }
    }
}

// Bounded wait until *slot is non-zero.  Returns the value, or 0 on timeout /
// abort (status set by someone).
__device__ __forceinline__ uint32_t wait_nonzero(const uint32_t *slot, const ElimArgs &a)
{
    long long spins = 0;
    uint32_t g;
    while ((g = ld_acquire_u32(slot)) == 0u) {
        if (read_status(a.status) != ST_OK) return 0u;
        if (++spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); return 0u; }
        __nanosleep(64);
    }
    return g;
}

struct WarpState {
    unsigned long long fcur, fend;     // factor-workspace chunk owned by this warp
    unsigned long long sbase, scap;    // global scratch owned by this warp (bytes)
    unsigned long long n_warp, n_block, n_global, n_fill;
    int fchunk;
};

// Eliminate pivot k with the warp.  Returns false if the kernel must stop.
__device__ bool eliminate(const ElimArgs &a, int32_t k, unsigned char *wbuf, unsigned char *bbuf,
                          int *block_lock, WarpState &ws)
{
    const unsigned lane = lane_id();
    const unsigned lt_mask = (1u << lane) - 1u;

    // ---------------------------------------------------------------- gather sizes
    const int64_t o0 = __ldg(a.lcp + k), o1 = __ldg(a.lcp + k + 1);
    const int32_t norig = (int32_t)(o1 - o0);
    const uint32_t cnt = __ldcg(a.fcnt + k);
    const int g = norig + (int)cnt;
    const int P = next_pow2(g);

    // ---------------------------------------------------------------- choose working set
    View v;
    bool block_held = false;
    int path;
    if (P <= a.warp_cap) {
        v = make_view(wbuf, a.warp_cap);
        path = 0;
    } else if (P <= a.block_cap) {
        int got = 0;
        if (lane == 0) {
            long long spins = 0;
            while (!(got = (atomicCAS(block_lock, 0, 1) == 0))) {
                if (read_status(a.status) != ST_OK) break;
                if (++spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); break; }
                __nanosleep(64);
            }
            __threadfence_block();
        }
        got = __shfl_sync(FULL, got, 0);
        if (!got || read_status(a.status) != ST_OK) {
            if (got && lane == 0) atomicExch(block_lock, 0);
            return false;
        }
        block_held = true;
        v = make_view(bbuf, a.block_cap);
        path = 1;
    } else {
        const unsigned long long need = (unsigned long long)P * ENTRY_BYTES;
        if (ws.scap < need) {
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(a.scratch_top, (need + 255ull) & ~255ull);
                if (base + need > a.scratch_cap) set_status(a.status, ST_POOL);
            }
            base = __shfl_sync(FULL, base, 0);
            if (read_status(a.status) != ST_OK) return false;
            ws.sbase = base; ws.scap = need;
        }
        v = make_view(a.scratch + ws.sbase, P);
        path = 2;
    }

    // ---------------------------------------------------------------- gather
    for (int i = lane; i < norig; i += 32) {
        v.row[i] = __ldg(a.lrow + o0 + i);
        v.w[i] = __ldg(a.lw + o0 + i);
    }
    {
        const int ninl = cnt < (uint32_t)FILL_C0 ? (int)cnt : FILL_C0;
        const size_t ib = (size_t)k * FILL_C0;
        for (int i = lane; i < ninl; i += 32) {
            v.row[norig + i] = __ldcg(a.in_row + ib + i);
            v.w[norig + i] = __ldcg(a.in_w + ib + i);
        }
        for (int j = 1; j <= FILL_LEVELS; ++j) {
            const uint32_t start = fill_level_start(j);
            if (cnt <= start) break;
            const uint32_t capj = fill_level_cap(j);
            const uint32_t len = (cnt - start) < capj ? (cnt - start) : capj;
            const uint32_t gidx = __ldcg(a.dir + (size_t)k * FILL_LEVELS + (j - 1));
            if (gidx == 0u || gidx == 0xffffffffu) {   // never published: give up rather than read wild memory
                set_status(a.status, ST_INVAL);
                if (block_held && lane == 0) atomicExch(block_lock, 0);
                return false;
            }
            const unsigned long long pb = (unsigned long long)(gidx - 1u) * FILL_GRANULE;
            for (uint32_t i = lane; i < len; i += 32) {
                v.row[norig + start + i] = __ldcg(a.pool_row + pb + i);
                v.w[norig + start + i] = __ldcg(a.pool_w + pb + i);
            }
        }
    }
    for (int i = g + lane; i < P; i += 32) { v.row[i] = ROW_SENTINEL; v.w[i] = 0.0; }
    __syncwarp();

    // ---------------------------------------------------------------- sort + merge (in place)
    sort_row_bits(v, P);
    int d = 0;
    for (int base = 0; base < g; base += 32) {
        const int i = base + lane;
        bool head = false;
        int32_t r = 0, len = 0;
        double sum = 0.0;
        if (i < g) {
            r = v.row[i];
            head = (i == 0) || (v.row[i - 1] != r);
            if (head) {
                sum = v.w[i]; len = 1;
                while (i + len < g && v.row[i + len] == r) { sum = __dadd_rn(sum, v.w[i + len]); ++len; }
            }
        }
        const unsigned bal = __ballot_sync(FULL, head);
        const int rank = d + __popc(bal & lt_mask);
        __syncwarp();
        if (head) { v.row[rank] = r; v.w[rank] = sum; v.mult[rank] = len; }
        d += __popc(bal);
        __syncwarp();
    }

    // ---------------------------------------------------------------- store row-ordered column
    unsigned long long fpos = 0;
    if (d > 0) {
        if (ws.fcur + (unsigned long long)d > ws.fend) {
            const unsigned long long sz = d > ws.fchunk ? (unsigned long long)d : (unsigned long long)ws.fchunk;
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(a.f_top, sz);
                if (base + sz > a.f_cap) set_status(a.status, ST_POOL);
            }
            base = __shfl_sync(FULL, base, 0);
            if (read_status(a.status) != ST_OK) {
                if (block_held && lane == 0) atomicExch(block_lock, 0);
                return false;
            }
            ws.fcur = base; ws.fend = base + sz;
        }
        fpos = ws.fcur;
        ws.fcur += (unsigned long long)d;
        for (int i = lane; i < d; i += 32) {
            a.f_row[fpos + i] = v.row[i];
            a.f_val[fpos + i] = v.w[i];
        }
    }
    if (lane == 0) { a.f_start[k] = (int64_t)fpos; a.f_len[k] = d; }
    if (d == 0) {
        if (lane == 0) a.D[k] = 0.0;
        if (block_held) { __syncwarp(); if (lane == 0) { __threadfence_block(); atomicExch(block_lock, 0); } }
        if (path == 0) ++ws.n_warp; else if (path == 1) ++ws.n_block; else ++ws.n_global;
        return true;
    }

    // ---------------------------------------------------------------- weight sort
    const int P2 = next_pow2(d);
    for (int i = d + lane; i < P2; i += 32) {
        v.row[i] = ROW_SENTINEL;
        v.w[i] = __longlong_as_double((long long)0xffffffffffffffffull);
        v.mult[i] = 0;
    }
    __syncwarp();
    sort_bits_row(v, P2);

    // ---------------------------------------------------------------- canonical suffix scan
    {
        double carry = 0.0, mcarry = 0.0;
        for (int base = 0; base < d; base += 32) {
            const int t = base + lane;
            double x = (t < d) ? v.w[d - 1 - t] : 0.0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double y = __shfl_up_sync(FULL, x, off);
                if ((int)lane >= off) x = __dadd_rn(x, y);
            }
            x = __dadd_rn(x, carry);
            double m = x;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double y = __shfl_up_sync(FULL, m, off);
                if ((int)lane >= off) m = fmax(m, y);
            }
            m = fmax(m, mcarry);
            if (t < d) { v.S[d - 1 - t] = x; v.M[d - 1 - t] = m; }
            carry = __shfl_sync(FULL, x, 31);
            mcarry = __shfl_sync(FULL, m, 31);
        }
    }
    __syncwarp();
    const double Dk = v.S[0];
    if (lane == 0) a.D[k] = Dk;

    // ---------------------------------------------------------------- sample clique tree + append
    uint64_t klocal = (uint64_t)k, sys = 0;
    if (a.sys_of) {
        const int32_t s = __ldg(a.sys_of + k);
        sys = (uint64_t)s;
        klocal = (uint64_t)(k - __ldg(a.sys_base + s));
    }
    bool ok = true;
    for (int pb = 1; pb < d; pb += 32) {
        const int p = pb + lane;
        const bool act = p < d;
        int32_t lo = 0, hi = 0;
        double c = 0.0;
        uint32_t idx = 0;
        if (act) {
            const int32_t u = v.row[p - 1];
            const double wu = v.w[p - 1];
            const double Sp = v.S[p];
            const double R = __dmul_rn(Sp, slot_uniform(a.seed, klocal, (uint64_t)p, sys));
            int lo_j = p, hi_j = d - 1;            // largest j with M[j] >= R; M[p] >= R
            while (lo_j < hi_j) {
                const int mid = lo_j + ((hi_j - lo_j + 1) >> 1);
                if (v.M[mid] >= R) lo_j = mid; else hi_j = mid - 1;
            }
            const int32_t x = v.row[lo_j];
            c = __ddiv_rn(__dmul_rn(Sp, wu), Dk);
            lo = u < x ? u : x;
            hi = u < x ? x : u;
            idx = atomicAdd(a.fcnt + lo, 1u);
            if (idx < (uint32_t)FILL_C0) {
                a.in_row[(size_t)lo * FILL_C0 + idx] = hi;
                a.in_w[(size_t)lo * FILL_C0 + idx] = c;
            } else {
                const int j = fill_level(idx);
                if (j > FILL_LEVELS) {
                    set_status(a.status, ST_POOL);      // column exceeds the directory's reach
                } else if (idx == fill_level_start(j)) {  // this lane opens level j of column lo
                    const uint32_t capj = fill_level_cap(j);
                    const unsigned long long pbase = atomicAdd(a.pool_top, (unsigned long long)capj);
                    uint32_t *slot = a.dir + (size_t)lo * FILL_LEVELS + (j - 1);
                    if (pbase + capj > a.pool_cap) {
                        set_status(a.status, ST_POOL);
                        st_release_u32(slot, 0xffffffffu);
                    } else {
                        st_release_u32(slot, (uint32_t)(pbase / FILL_GRANULE) + 1u);
                    }
                }
            }
            red_add_relaxed(a.dp + hi, 1);
        }
        __syncwarp();
        if (act && idx >= (uint32_t)FILL_C0) {
            const int j = fill_level(idx);
            const uint32_t gi = j > FILL_LEVELS ? 0u : wait_nonzero(a.dir + (size_t)lo * FILL_LEVELS + (j - 1), a);
            if (gi == 0u || gi == 0xffffffffu) {
                ok = false;
            } else {
                const unsigned long long at = (unsigned long long)(gi - 1u) * FILL_GRANULE + (idx - fill_level_start(j));
                a.pool_row[at] = hi;
                a.pool_w[at] = c;
            }
        }
        if (__any_sync(FULL, !ok)) {
            if (block_held && lane == 0) atomicExch(block_lock, 0);
            return false;
        }
    }
    ws.n_fill += (unsigned long long)(d - 1);

    // ---------------------------------------------------------------- release, then decrements
    __threadfence();
    __syncwarp();
    __threadfence();
    for (int ib = 0; ib < d; ib += 32) {
        const int i = ib + lane;
        bool ready = false;
        int32_t u = 0;
        if (i < d) {
            u = v.row[i];
            const int32_t m = v.mult[i];
            const int32_t r = atomicSub(a.dp + u, m);
            ready = (r == m);
        }
        const unsigned bal = __ballot_sync(FULL, ready);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            uint32_t qb = 0;
            if ((int)lane == leader) qb = atomicAdd(a.q_tail, (uint32_t)__popc(bal));
            qb = __shfl_sync(FULL, qb, leader);
            if (ready) {
                const uint32_t at = qb + __popc(bal & lt_mask);
                if (at < (uint32_t)a.nl) {
                    fence_acq_rel();
                    st_release(a.queue + at, u);
                } else {
                    set_status(a.status, ST_INVAL);    // a vertex became ready twice: counters are corrupt
                }
            }
        }
    }
    __syncwarp();
    if (block_held && lane == 0) { __threadfence_block(); atomicExch(block_lock, 0); }
    if (path == 0) ++ws.n_warp; else if (path == 1) ++ws.n_block; else ++ws.n_global;
    return true;
}

__global__ void __launch_bounds__(512) elim_kernel(ElimArgs a, int fchunk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int block_lock;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned lane = lane_id();
    if (threadIdx.x == 0) block_lock = 0;
    __syncthreads();

    unsigned char *wbuf = smem + (size_t)warp * a.warp_cap * ENTRY_BYTES;
    unsigned char *bbuf = smem + (size_t)nw * a.warp_cap * ENTRY_BYTES;

    WarpState ws;
    ws.fcur = ws.fend = 0; ws.sbase = 0; ws.scap = 0;
    ws.n_warp = ws.n_block = ws.n_global = ws.n_fill = 0;
    ws.fchunk = fchunk;
    unsigned long long spins_total = 0;

    const uint32_t nl = (uint32_t)a.nl;
    bool run = true;
    while (run) {
        uint32_t s = 0;
        if (lane == 0) s = atomicAdd(a.q_head, (uint32_t)a.queue_chunk);
        s = __shfl_sync(FULL, s, 0);
        if (s >= nl) break;
        const uint32_t e = (s + (uint32_t)a.queue_chunk) < nl ? s + (uint32_t)a.queue_chunk : nl;
        for (uint32_t slot = s; slot < e; ++slot) {
            int32_t k;
            long long spins = 0;
            uint32_t seen_tail = 0;
            // The watchdog counts polls without global progress: the count
            // restarts whenever the queue tail has moved since the last look.
            while ((k = ld_acquire(a.queue + slot)) < 0) {
                if (read_status(a.status) != ST_OK) { run = false; break; }
                if ((++spins & 255) == 0) {
                    const uint32_t t = *(volatile const uint32_t *)a.q_tail;
                    if (t != seen_tail) { seen_tail = t; spins_total += (unsigned long long)spins; spins = 0; }
                }
                if (spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); run = false; break; }
                __nanosleep(100);
            }
            spins_total += (unsigned long long)spins;
            if (__any_sync(FULL, !run)) { run = false; break; }
            if (!eliminate(a, k, wbuf, bbuf, &block_lock, ws)) { run = false; break; }
        }
    }
    if (lane == 0 && a.stats) {
        atomicAdd(a.stats + 0, ws.n_warp);
        atomicAdd(a.stats + 1, ws.n_block);
        atomicAdd(a.stats + 2, ws.n_global);
        atomicAdd(a.stats + 3, ws.n_fill);
        atomicAdd(a.stats + 4, spins_total);
    }
}

}  // namespace

size_t elim_smem_bytes(int warps_per_block, int warp_cap, int block_cap)
{
    return (size_t)(warps_per_block * warp_cap + block_cap) * ENTRY_BYTES;
}

cudaError_t elim_configure(int warps_per_block, int warp_cap, int block_cap, int *blocks_per_sm)
{
    const size_t smem = elim_smem_bytes(warps_per_block, warp_cap, block_cap);
    cudaError_t e = cudaFuncSetAttribute(elim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, elim_kernel, warps_per_block * 32, smem);
}

cudaError_t elim_launch(const ElimArgs &a, int blocks, int warps_per_block, int fchunk, cudaStream_t st)
{
    const size_t smem = elim_smem_bytes(warps_per_block, a.warp_cap, a.block_cap);
    elim_kernel<<<blocks, warps_per_block * 32, smem, st>>>(a, fchunk);
    return cudaGetLastError();
}

}  // namespace parac
