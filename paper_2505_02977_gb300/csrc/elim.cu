// elim.cu -- persistent randomized-elimination kernel (rchol's SampleClique per
// pivot, Alg. 2; scheduled by ParAC's dependency counters, Sec. III; one
// persistent launch for the whole factorisation as in Alg. 4 / Sec. IV-C).
//
// Worker = one warp.  A free worker claims a ready-queue slot (one atomicAdd
// per `queue_chunk` slots) and waits, bounded, until it is published; a
// worker that has just made vertices ready keeps one of them and eliminates
// it next without a queue round trip (the others are published).  Eliminating
// vertex k:
//   gather     original strict-lower column k + every fill entry appended to
//              column k (inline slab + overflow levels)
//   sort       by (row, weight bits)
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
//              positive-to-zero transition makes the vertex ready.
// Working sets of up to 32 entries live in registers (one entry per lane,
// shuffle networks), up to `warp_cap` in the warp's shared memory, up to
// `block_cap` in one per-CTA shared buffer (taken under a CTA lock), larger
// ones in a global scratch arena.
#include "common.cuh"
#include "kernels.h"

namespace parac {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int32_t ROW_SENTINEL = 0x7fffffff;
constexpr unsigned long long WBITS_SENTINEL = 0xffffffffffffffffull;

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

struct View {           // per-vertex working set in shared or global memory
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

// Register bitonic networks: lane i holds entry i; only the first P lanes
// (P a power of two, warp-uniform) carry entries, the rest hold sentinels
// that sort last, so the stages with block size above P are skipped.  For
// the pair (i, i^j) the lower lane keeps the smaller key when the block is
// ascending.
__device__ __forceinline__ void reg_sort_row_bits(int32_t &row, double &w, int P)
{
    const unsigned lane = lane_id();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t ro = __shfl_xor_sync(FULL, row, j);
            const double wo = __shfl_xor_sync(FULL, w, j);
            const bool lower = (lane & j) == 0, asc = (lane & k) == 0;
            const unsigned long long b = dbits(w), bo = dbits(wo);
            const bool self_gt = (row > ro) || (row == ro && b > bo);
            const bool other_gt = (ro > row) || (ro == row && bo > b);
            const bool take = lower == asc ? self_gt : other_gt;
            if (take) { row = ro; w = wo; }
        }
    }
}

__device__ __forceinline__ void reg_sort_bits_row(int32_t &row, double &w, int32_t &m, int P)
{
    const unsigned lane = lane_id();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t ro = __shfl_xor_sync(FULL, row, j);
            const double wo = __shfl_xor_sync(FULL, w, j);
            const int32_t mo = __shfl_xor_sync(FULL, m, j);
            const bool lower = (lane & j) == 0, asc = (lane & k) == 0;
            const unsigned long long b = dbits(w), bo = dbits(wo);
            const bool self_gt = (b > bo) || (b == bo && row > ro);
            const bool other_gt = (bo > b) || (bo == b && ro > row);
            const bool take = lower == asc ? self_gt : other_gt;
            if (take) { row = ro; w = wo; m = mo; }
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
        ++spins;
        if ((spins & 63) == 0) {           // the shared status word is read only now and then
            if (read_status(a.status) != ST_OK) return 0u;
            if (spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); return 0u; }
        }
        if (spins > 32) __nanosleep(32);
    }
    return g;
}

struct WarpState {
    unsigned long long fcur, fend;     // factor-workspace chunk owned by this warp
    unsigned long long sbase, scap;    // global scratch owned by this warp (bytes)
    unsigned long long n_reg, n_warp, n_block, n_global, n_fill, n_handoff;
    unsigned long long cyc[16];        // per-phase cycles (profiling runs only)
    long long t_mark;
    int fchunk;
};

// Per-phase cycle accounting, active only when the launch asks for it:
// 0 queue wait, 1 gather, 2 sort + merge, 3 store (+ weight sort + scan on
// the shared-memory path), 4 sampling + append, 5 levels + release +
// decrements, 6 register weight sort, 7 register scan; cooperative path (as
// seen by the requesting warp): 8 join, 9 gather, 10 row sort, 11 merge +
// store, 12 weight sort, 13 scan, 14 sampling + append, 15 release.
__device__ __forceinline__ void prof_mark(const ElimArgs &a, WarpState &ws, int phase)
{
    if (a.profile) {
        long long t;
        asm volatile("mov.u64 %0, %%clock64;" : "=l"(t) : : "memory");   // memory ops stay on their side
        if (phase >= 0) ws.cyc[phase] += (unsigned long long)(t - ws.t_mark);
        ws.t_mark = t;
    }
}

// Reserve d factor-workspace entries from the warp's chunk.  Warp-uniform.
__device__ __forceinline__ bool reserve_factor(const ElimArgs &a, WarpState &ws, int d, unsigned long long &pos)
{
    if (ws.fcur + (unsigned long long)d > ws.fend) {
        const unsigned long long sz = d > ws.fchunk ? (unsigned long long)d : (unsigned long long)ws.fchunk;
        unsigned long long base = 0;
        if (lane_id() == 0) {
            base = atomicAdd(a.f_top, sz);
            if (base + sz > a.f_cap) set_status(a.status, ST_POOL);
        }
        base = __shfl_sync(FULL, base, 0);
        if (read_status(a.status) != ST_OK) return false;
        ws.fcur = base; ws.fend = base + sz;
    }
    pos = ws.fcur;
    ws.fcur += (unsigned long long)d;
    return true;
}

// Append fill entry (row hi, weight c) to column lo and count the new edge in
// dp[hi]; lanes with act == false only join the warp-wide steps.  The lane
// that takes the first index of an overflow level allocates that level's slab
// and publishes it; the other lanes of the level wait for it.  Warp-uniform
// result; false means the kernel must stop.
constexpr unsigned long long W_MAX_PROBE = 1ull << 16;   // probes before an insert counts as overflow

__device__ bool append_fill(const ElimArgs &a, bool act, int32_t lo, int32_t hi, double c)
{
    if (a.hash_store) {
        // hashmap W (Sec. IV-C): probe from step fill_count(lo) of lo's sequence
        // (see w_stride) for a free slot, claim it (free -> busy), write the
        // entry, publish the tag
        bool ok = true;
        if (act) {
            const uint32_t idx = atomicAdd(a.fcnt + lo, 1u);
            const unsigned long long stride = w_stride(lo, a.wcap);
            unsigned long long i = w_slot(w_base(lo, a.wcap), stride, idx, a.wcap);
            const unsigned long long lim = a.wcap < W_MAX_PROBE ? a.wcap : W_MAX_PROBE;
            bool placed = false;
            for (unsigned long long step = 0; step < lim; ++step) {
                if (*(volatile const int32_t *)(a.wcol + i) == W_FREE && atomicCAS(a.wcol + i, W_FREE, W_BUSY) == W_FREE) {
                    a.wrow[i] = hi;
                    a.ww[i] = c;
                    __threadfence();
                    st_release(a.wcol + i, lo);
                    placed = true;
                    break;
                }
                i = (i + stride) & (a.wcap - 1);
            }
            if (!placed) { set_status(a.status, ST_POOL); ok = false; }
            red_add_relaxed(a.dp + hi, 1);
        }
        return !__any_sync(FULL, !ok);
    }
    uint32_t idx = 0;
    if (act) {
        idx = atomicAdd(a.fcnt + lo, 1u);
        if (idx < (uint32_t)FILL_C0) {
            a.in_row[(size_t)lo * FILL_C0 + idx] = hi;
            a.in_w[(size_t)lo * FILL_C0 + idx] = c;
        } else {
            const int j = fill_level(idx);
            if (j > FILL_LEVELS) {
                set_status(a.status, ST_POOL);        // column exceeds the directory's reach
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
    bool ok = true;
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
    return !__any_sync(FULL, !ok);
}

// Counter decrements of one group of up to 32 merged neighbours (lane holds
// u, m when valid).  A positive-to-zero transition makes u ready: the first
// such vertex is kept in `keep` when it is -1 (empty; -2 means never keep)
// for this warp, the others are published on the queue.
// Counter decrements of one group of up to 32 merged neighbours (lane holds
// u, m when valid).  A positive-to-zero transition makes u ready: the first
// such vertex is kept in `keep` when it is -1 (empty; -2 means never keep)
// for this warp, the others are published on the queue.
__device__ void decrement_group(const ElimArgs &a, int32_t pivot, bool valid, int32_t u, int32_t m, int32_t &keep)
{
    const unsigned lane = lane_id();
    bool ready = false;
    if (valid) {
        const int32_t r = atomicSub(a.dp + u, m);
        ready = (r == m);
        if (ready && a.trace) { a.trace[4 * (size_t)u] = global_ns(); a.trace_parent[u] = pivot; }
    }
    unsigned bal = __ballot_sync(FULL, ready);
    if (!bal) return;
    if (keep == -1) {
        const int kl = __ffs(bal) - 1;
        keep = __shfl_sync(FULL, u, kl);
        bal &= ~(1u << kl);
        if ((int)lane == kl) ready = false;
    }
    if (!bal) return;
    const int leader = __ffs(bal) - 1;
    uint32_t qb = 0;
    if ((int)lane == leader) qb = atomicAdd(a.q_tail, (uint32_t)__popc(bal));
    qb = __shfl_sync(FULL, qb, leader);
    if (ready) {
        const uint32_t at = qb + __popc(bal & ((1u << lane) - 1u));
        if (at < (uint32_t)a.nl) {
            fence_acq_rel();
            st_release(a.queue + at, u);
        } else {
            set_status(a.status, ST_INVAL);    // a vertex became ready twice: counters are corrupt
        }
    }
}

__device__ __forceinline__ void sys_of(const ElimArgs &a, int32_t k, uint64_t &klocal, uint64_t &sys)
{
    klocal = (uint64_t)k; sys = 0;
    if (a.sys_of) {
        const int32_t s = __ldg(a.sys_of + k);
        sys = (uint64_t)s;
        klocal = (uint64_t)(k - __ldg(a.sys_base + s));
    }
}

// Fill entries of column k from the hashmap W: the warp scans k's probe
// sequence, 32 slots at a time, until all cnt entries tagged k are found.
// Every entry of k was published (release) before k became ready, so a busy
// slot is never k's.  put(pos, row, w) receives the entry of scan rank pos;
// the slot is freed for reuse.  false if the scan wrapped the whole table.
template <typename Put>
__device__ __forceinline__ bool warp_hash_gather(const ElimArgs &a, int32_t k, uint32_t cnt, Put &&put)
{
    const unsigned lane = lane_id();
    const unsigned long long base = w_base(k, a.wcap), stride = w_stride(k, a.wcap);
    uint32_t found = 0;
    unsigned long long off = 0;
    while (found < cnt) {
        if (off >= a.wcap) return false;
        const unsigned long long i = w_slot(base, stride, off + lane, a.wcap);
        const bool mine = off + lane < a.wcap && ld_acquire(a.wcol + i) == k;
        const unsigned bal = __ballot_sync(FULL, mine);
        if (mine) {
            put(found + __popc(bal & ((1u << lane) - 1u)), a.wrow[i], a.ww[i]);
            st_release(a.wcol + i, W_FREE);          // after the entry was read
        }
        found += __popc(bal);
        off += 32;
    }
    return true;
}

// Pivot k whose working set fits in registers (g <= 32).  Returns the vertex
// this warp keeps for itself (-1: none), or -2 if the kernel must stop.
// FP64 is slow on this part, so only the canonical arithmetic runs in FP64
// (run sums, suffix sums, the sampling product and the weight quotient); the
// running maximum and the sampling search compare bit patterns, which order
// non-negative doubles exactly as their values.
__device__ int32_t eliminate_small(const ElimArgs &a, int32_t k, int64_t o0, int32_t norig, uint32_t cnt,
                                   WarpState &ws)
{
    const unsigned lane = lane_id();
    const int g = norig + (int)cnt;

    // gather: lane i holds gathered entry i
    int32_t row = ROW_SENTINEL;
    double w = 0.0;
    bool bad = false;
    if ((int)lane < norig) {
        row = __ldg(a.lrow + o0 + lane);
        w = __ldg(a.lw + o0 + lane);
    }
    if (a.hash_store) {
        // fill entries from W to lanes norig.. (scan rank order): each round, the
        // lane of the p-th entry found hands it to lane norig + found + p
        const unsigned long long base = w_base(k, a.wcap), stride = w_stride(k, a.wcap);
        uint32_t found = 0;
        unsigned long long off = 0;
        while (found < cnt) {
            if (off >= a.wcap) { bad = true; break; }
            const unsigned long long i = w_slot(base, stride, off + lane, a.wcap);
            const bool mine = off + lane < a.wcap && ld_acquire(a.wcol + i) == k;
            const unsigned bal = __ballot_sync(FULL, mine);
            int32_t fr = 0;
            double fw = 0.0;
            if (mine) {
                fr = a.wrow[i]; fw = a.ww[i];
                st_release(a.wcol + i, W_FREE);          // after the entry was read
            }
            const int nb = __popc(bal);
            const int p = (int)lane - norig - (int)found;
            int src = 0;
            if (p >= 0 && p < nb) {                       // lane of the (p+1)-th set bit
                int blo = 0, bhi = 31;
                while (blo < bhi) {
                    const int mid = (blo + bhi) >> 1;
                    if (__popc(bal & ((2u << mid) - 1u)) >= p + 1) bhi = mid; else blo = mid + 1;
                }
                src = blo;
            }
            const int32_t rr = __shfl_sync(FULL, fr, src);
            const double wv = __shfl_sync(FULL, fw, src);
            if (p >= 0 && p < nb) { row = rr; w = wv; }
            found += (uint32_t)nb;
            off += 32;
        }
    } else if ((int)lane < g && (int)lane >= norig) {
        const uint32_t f = lane - (uint32_t)norig;       // fill index
        if (f < (uint32_t)FILL_C0) {
            row = __ldcg(a.in_row + (size_t)k * FILL_C0 + f);
            w = __ldcg(a.in_w + (size_t)k * FILL_C0 + f);
        } else {                                         // level 1 of the overflow directory
            const uint32_t gidx = __ldcg(a.dir + (size_t)k * FILL_LEVELS);
            if (gidx == 0u || gidx == 0xffffffffu) {
                bad = true;
            } else {
                const unsigned long long pb = (unsigned long long)(gidx - 1u) * FILL_GRANULE + (f - FILL_C0);
                row = __ldcg(a.pool_row + pb);
                w = __ldcg(a.pool_w + pb);
            }
        }
    }
    // the uniform of slot p = lane depends only on (seed, k, p, sys): draw it
    // while the gathered entries are in flight
    uint64_t klocal, sys;
    sys_of(a, k, klocal, sys);
    const double vrand = (lane >= 1 && (int)lane < g) ? slot_uniform(a.seed, klocal, (uint64_t)lane, sys) : 1.0;
    if (__any_sync(FULL, bad)) {            // never published: give up rather than read wild memory
        if (lane == 0) set_status(a.status, ST_INVAL);
        return -2;
    }
    prof_mark(a, ws, 1);

    // sort by (row, weight bits), merge runs left to right
    reg_sort_row_bits(row, w, next_pow2(g));
    const int32_t prow = __shfl_up_sync(FULL, row, 1);
    const bool head = ((int)lane < g) && (lane == 0 || prow != row);
    const unsigned hb = __ballot_sync(FULL, head);
    const unsigned rest = lane == 31 ? 0u : (hb >> (lane + 1));
    const int len = head ? (rest ? __ffs(rest) : g - (int)lane) : 0;
    const int maxlen = (int)__reduce_max_sync(FULL, (unsigned)len);
    double sum = w;
    for (int off = 1; off < maxlen; ++off) {
        const double nv = __shfl_down_sync(FULL, w, off);
        if (head && off < len) sum = __dadd_rn(sum, nv);
    }
    const int d = __popc(hb);
    // lane r < d takes the r-th run head: the smallest lane i with r+1 heads in 0..i
    int src = 0;
    if ((int)lane < d) {
        int blo = 0, bhi = 31;
        while (blo < bhi) {
            const int mid = (blo + bhi) >> 1;
            if (__popc(hb & ((2u << mid) - 1u)) >= (int)lane + 1) bhi = mid; else blo = mid + 1;
        }
        src = blo;
    }
    int32_t mrow = __shfl_sync(FULL, row, src);
    double mw = __shfl_sync(FULL, sum, src);
    int32_t mm = __shfl_sync(FULL, len, src);
    const bool valid = (int)lane < d;
    prof_mark(a, ws, 2);

    // store the row-ordered column
    unsigned long long fpos = 0;
    if (d > 0 && !reserve_factor(a, ws, d, fpos)) return -2;
    if (valid) {
        a.f_row[fpos + lane] = mrow;
        a.f_val[fpos + lane] = mw;
    }
    if (lane == 0) { a.f_start[k] = (int64_t)fpos; a.f_len[k] = d; }
    if (d == 0) {
        if (lane == 0) a.D[k] = 0.0;
        ++ws.n_reg;
        return -1;
    }
    prof_mark(a, ws, 3);

    // sort by (weight bits, row)
    if (!valid) { mrow = ROW_SENTINEL; mw = __longlong_as_double((long long)WBITS_SENTINEL); mm = 0; }
    reg_sort_bits_row(mrow, mw, mm, next_pow2(d));
    prof_mark(a, ws, 6);

    // canonical suffix sums: lane t holds S[d-1-t] (one tile).  Hillis-Steele
    // offsets >= d add nothing to lanes below d, so they are skipped.
    double x = __shfl_sync(FULL, mw, (int)lane < d ? d - 1 - (int)lane : 0);
    if ((int)lane >= d) x = 0.0;
    for (int off = 1; off < d; off <<= 1) {
        const double y = __shfl_up_sync(FULL, x, off);
        if ((int)lane >= off) x = __dadd_rn(x, y);
    }
    x = __dadd_rn(x, 0.0);                 // carry of the (empty) preceding tiles
    unsigned long long mx = dbits(x);      // running maximum, as bit patterns
    for (int off = 1; off < d; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, mx, off);
        if ((int)lane >= off && y > mx) mx = y;
    }
    const double Dk = __shfl_sync(FULL, x, d - 1);
    if (lane == 0) a.D[k] = Dk;
    prof_mark(a, ws, 7);

    // sample the clique tree: lane p handles slot p (1 <= p <= d-1)
    const int p = (int)lane;
    const bool act = p >= 1 && p < d;
    const double Sp = __shfl_sync(FULL, x, act ? d - 1 - p : 0);
    const int32_t u = __shfl_sync(FULL, mrow, act ? p - 1 : 0);
    const double wu = __shfl_sync(FULL, mw, act ? p - 1 : 0);
    const unsigned long long Rb = act ? dbits(__dmul_rn(Sp, vrand)) : 0ull;
    int lo_j = act ? p : 0, hi_j = act ? d - 1 : 0;        // largest j with M[j] >= R
    const int steps = d > 1 ? 32 - __clz(d - 1) : 0;
    for (int it = 0; it < steps; ++it) {
        const int mid = lo_j + ((hi_j - lo_j + 1) >> 1);
        const unsigned long long Mm = __shfl_sync(FULL, mx, (d - 1 - mid) & 31);
        if (lo_j < hi_j) {
            if (Mm >= Rb) lo_j = mid; else hi_j = mid - 1;
        }
    }
    const int32_t xv = __shfl_sync(FULL, mrow, lo_j & 31);
    double c = 0.0;
    int32_t lo = 0, hi = 0;
    if (act) {
        c = __ddiv_rn(__dmul_rn(Sp, wu), Dk);
        if (a.samples > 1) c = __ddiv_rn(c, (double)a.samples);
        lo = u < xv ? u : xv;
        hi = u < xv ? xv : u;
    }
    if (!append_fill(a, act, lo, hi, c)) return -2;
    // further samples of every slot (MS(k)): own uniforms, the same weight
    for (int q = 1; q < a.samples; ++q) {
        const unsigned long long Rq = act ? dbits(__dmul_rn(Sp, slot_uniform(a.seed, klocal, (uint64_t)p, sys,
                                                                                (uint64_t)q))) : 0ull;
        int qlo = act ? p : 0, qhi = act ? d - 1 : 0;
        for (int it = 0; it < steps; ++it) {
            const int mid = qlo + ((qhi - qlo + 1) >> 1);
            const unsigned long long Mm = __shfl_sync(FULL, mx, (d - 1 - mid) & 31);
            if (qlo < qhi) {
                if (Mm >= Rq) qlo = mid; else qhi = mid - 1;
            }
        }
        const int32_t xq = __shfl_sync(FULL, mrow, qlo & 31);
        if (act) { lo = u < xq ? u : xq; hi = u < xq ? xq : u; }
        if (!append_fill(a, act, lo, hi, c)) return -2;
    }
    ws.n_fill += (unsigned long long)(d - 1) * (unsigned long long)a.samples;
    prof_mark(a, ws, 4);

    // dependency levels, release, decrements
    const int32_t lk = __ldcg(a.lvl + k) + 1;
    if (valid) red_max_relaxed(a.lvl + mrow, lk);
    __syncwarp();
    __threadfence();
    int32_t keep = -1;
    decrement_group(a, k, valid, mrow, mm, keep);
    ++ws.n_reg;
    prof_mark(a, ws, 5);
    return keep;
}

// Pivot k with a larger working set (shared or global memory).
__device__ int32_t eliminate_big(const ElimArgs &a, int32_t k, int64_t o0, int32_t norig, uint32_t cnt,
                                 unsigned char *wbuf, unsigned char *bbuf, int *block_lock, WarpState &ws)
{
    const unsigned lane = lane_id();
    const unsigned lt_mask = (1u << lane) - 1u;
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
                if ((++spins & 63) == 0) {
                    if (read_status(a.status) != ST_OK) break;
                    if (spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); break; }
                }
                __nanosleep(64);
            }
            __threadfence_block();
        }
        got = __shfl_sync(FULL, got, 0);
        if (!got || read_status(a.status) != ST_OK) {
            if (got && lane == 0) atomicExch(block_lock, 0);
            return -2;
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
            if (read_status(a.status) != ST_OK) return -2;
            ws.sbase = base; ws.scap = need;
        }
        v = make_view(a.scratch + ws.sbase, P);
        path = 2;
    }
    auto release_block = [&]() {
        if (block_held) {
            __syncwarp();
            if (lane == 0) { __threadfence_block(); atomicExch(block_lock, 0); }
        }
    };

    // ---------------------------------------------------------------- gather
    for (int i = lane; i < norig; i += 32) {
        v.row[i] = __ldg(a.lrow + o0 + i);
        v.w[i] = __ldg(a.lw + o0 + i);
    }
    if (a.hash_store) {
        if (!warp_hash_gather(a, k, cnt, [&](uint32_t pos, int32_t r, double x) {
                v.row[norig + pos] = r; v.w[norig + pos] = x; })) {
            set_status(a.status, ST_INVAL);
            release_block();
            return -2;
        }
    } else {
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
                release_block();
                return -2;
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
    prof_mark(a, ws, 1);

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

    prof_mark(a, ws, 2);

    // ---------------------------------------------------------------- store row-ordered column
    unsigned long long fpos = 0;
    if (d > 0 && !reserve_factor(a, ws, d, fpos)) { release_block(); return -2; }
    for (int i = lane; i < d; i += 32) {
        a.f_row[fpos + i] = v.row[i];
        a.f_val[fpos + i] = v.w[i];
    }
    if (lane == 0) { a.f_start[k] = (int64_t)fpos; a.f_len[k] = d; }
    if (d == 0) {
        if (lane == 0) a.D[k] = 0.0;
        release_block();
        if (path == 0) ++ws.n_warp; else if (path == 1) ++ws.n_block; else ++ws.n_global;
        return -1;
    }

    // ---------------------------------------------------------------- weight sort
    const int P2 = next_pow2(d);
    for (int i = d + lane; i < P2; i += 32) {
        v.row[i] = ROW_SENTINEL;
        v.w[i] = __longlong_as_double((long long)WBITS_SENTINEL);
        v.mult[i] = 0;
    }
    __syncwarp();
    sort_bits_row(v, P2);

    // ---------------------------------------------------------------- canonical suffix scan
    {
        double carry = 0.0;
        unsigned long long mcarry = 0ull;
        for (int base = 0; base < d; base += 32) {
            const int t = base + lane;
            double x = (t < d) ? v.w[d - 1 - t] : 0.0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double y = __shfl_up_sync(FULL, x, off);
                if ((int)lane >= off) x = __dadd_rn(x, y);
            }
            x = __dadd_rn(x, carry);
            unsigned long long m = dbits(x);      // running maximum, as bit patterns
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL, m, off);
                if ((int)lane >= off && y > m) m = y;
            }
            if (mcarry > m) m = mcarry;
            if (t < d) { v.S[d - 1 - t] = x; v.M[d - 1 - t] = __longlong_as_double((long long)m); }
            carry = __shfl_sync(FULL, x, 31);
            mcarry = __shfl_sync(FULL, m, 31);
        }
    }
    __syncwarp();
    const double Dk = v.S[0];
    if (lane == 0) a.D[k] = Dk;
    prof_mark(a, ws, 3);

    // ---------------------------------------------------------------- sample clique tree + append
    uint64_t klocal, sys;
    sys_of(a, k, klocal, sys);
    for (int q = 0; q < a.samples; ++q) {                // sample q of every slot (q > 0: MS(k))
        for (int pb = 1; pb < d; pb += 32) {
            const int p = pb + lane;
            const bool act = p < d;
            int32_t lo = 0, hi = 0;
            double c = 0.0;
            if (act) {
                const int32_t u = v.row[p - 1];
                const double wu = v.w[p - 1];
                const double Sp = v.S[p];
                const double R = __dmul_rn(Sp, slot_uniform(a.seed, klocal, (uint64_t)p, sys, (uint64_t)q));
                const unsigned long long Rb = dbits(R);
                int lo_j = p, hi_j = d - 1;            // largest j with M[j] >= R; M[p] >= R
                while (lo_j < hi_j) {
                    const int mid = lo_j + ((hi_j - lo_j + 1) >> 1);
                    if (dbits(v.M[mid]) >= Rb) lo_j = mid; else hi_j = mid - 1;
                }
                const int32_t x = v.row[lo_j];
                c = __ddiv_rn(__dmul_rn(Sp, wu), Dk);
                if (a.samples > 1) c = __ddiv_rn(c, (double)a.samples);
                lo = u < x ? u : x;
                hi = u < x ? x : u;
            }
            if (!append_fill(a, act, lo, hi, c)) { release_block(); return -2; }
        }
    }
    ws.n_fill += (unsigned long long)(d - 1) * (unsigned long long)a.samples;
    prof_mark(a, ws, 4);

    // ---------------------------------------------------------------- levels, release, decrements
    {
        const int32_t lk = __ldcg(a.lvl + k) + 1;
        for (int i = lane; i < d; i += 32) red_max_relaxed(a.lvl + v.row[i], lk);
    }
    __syncwarp();
    __threadfence();
    int32_t keep = -1;
    for (int ib = 0; ib < d; ib += 32) {
        const int i = ib + lane;
        const bool valid = i < d;
        decrement_group(a, k, valid, valid ? v.row[i] : 0, valid ? v.mult[i] : 0, keep);
    }
    release_block();
    if (path == 0) ++ws.n_warp; else if (path == 1) ++ws.n_block; else ++ws.n_global;
    prof_mark(a, ws, 5);
    return keep;
}

// ---------------------------------------------------------------- CTA-cooperative path
// A vertex whose working set exceeds a warp's shared buffer is eliminated by
// all warps of its CTA together: the warp that popped it posts a request,
// every other warp of the CTA joins at its next poll point, and the block runs
// the same steps with block-wide networks.  One request at a time per CTA;
// all barriers are bounded software barriers over the CTA's warps.
struct CoopShared {
    int k;                       // vertex being eliminated cooperatively (-1: none)
    int gen;                     // bumped for every request
    int req_warp;                // warp that posted the request
    int arrive;                  // barrier arrivals (monotonic)
    int d, ntile, abort;
    int hcount[32];              // per-warp head counts of the merge
    int nbig;                    // sample sort: buckets above a warp's slice
    unsigned long long fpos;
    unsigned long long sbase, scap;   // CTA scratch (global), reused across requests
    long long spin_limit;
    GhTask *gt;                  // grid help: the step being posted (in the CTA's global scratch)
    uint32_t gh_gen;             // last generation posted on the board
    int gh;                      // this vertex holds the board
    int gh_req;                  // the posted request asks for grid help
};
// Static shared memory stays small: two CTAs of 8 warps (98,824 bytes of
// dynamic shared memory each) fit the SM's 196 KB shared-memory carve-out
// only with at most 504 bytes of static shared memory per CTA; beyond it the
// 228 KB carve-out halves the L1 cache (measured: the whole elimination ~9%
// slower).
static_assert(sizeof(CoopShared) <= 320, "static shared memory of the elimination kernel");

__device__ __forceinline__ volatile int &vol(int &x) { return *(volatile int *)&x; }

constexpr int GH_COARSE = 512;   // coarse entries of the sampling search (one 4 KB warp slice)
constexpr long long GH_GRACE_NS = 3000;   // the owner's warps leave a step's chunks to the helpers this long

// Bytes of a CTA's global working set of P entries: the entries, the scan
// tiles, bucket offsets / merged counts / oversized list; with grid help
// also the tile maxima, splitters (rows, weight bits), bucket counters,
// compacted offsets and the coarse search table.
__device__ __forceinline__ unsigned long long coop_scratch_bytes(int P, int cap, bool gh)
{
    const unsigned long long p = (unsigned long long)P, c = (unsigned long long)cap;
    unsigned long long need = p * ENTRY_BYTES + (p / 32 + 1) * 8 + 16ull + 4ull * (3ull * c + 3ull);
    if (gh) need += 16ull + sizeof(GhTask) + (p / 32 + 1) * 8 + 12ull * c + 4ull * (3ull * c + 1ull) + 16ull + 8ull * GH_COARSE;
    return need;
}

// Bounded barrier over the CTA's warps; false if it gave up (status set).
__device__ bool cta_barrier(CoopShared &cs, const ElimArgs &a)
{
    const int nw = blockDim.x >> 5;
    __syncwarp();
    int ok = 1;
    if (lane_id() == 0) {
        __threadfence_block();
        const int old = atomicAdd(&cs.arrive, 1);
        const int target = (old / nw + 1) * nw;
        long long spins = 0;
        while (vol(cs.arrive) < target) {
            ++spins;
            if ((spins & 63) == 0) {
                if (read_status(a.status) != ST_OK) { ok = 0; break; }
                if (spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); ok = 0; break; }
            }
            if (spins > 64) __nanosleep(32);
        }
        __threadfence_block();
    }
    return __shfl_sync(FULL, ok, 0) != 0;
}

// One compare-exchange of the bitonic network: entries i < l = i + j of
// direction asc (ascending when (i & block) == 0).  KEY 0 orders by (row,
// weight bits), KEY 1 by (weight bits, row) and carries the multiplicity.
template <int KEY>
__device__ __forceinline__ void cex(View v, int i, int l, bool asc)
{
    const int32_t ri = v.row[i], rl = v.row[l];
    const double wi = v.w[i], wl = v.w[l];
    const unsigned long long bi = dbits(wi), bl = dbits(wl);
    const bool gt = KEY == 0 ? ((ri > rl) || (ri == rl && bi > bl)) : ((bi > bl) || (bi == bl && ri > rl));
    if (gt == asc) {
        v.row[i] = rl; v.row[l] = ri; v.w[i] = wl; v.w[l] = wi;
        if (KEY == 1) { const int32_t mi = v.mult[i], ml = v.mult[l]; v.mult[i] = ml; v.mult[l] = mi; }
    }
}

// Block-wide bitonic sort of P entries of v (a power of two).  When v lives
// in global memory and P exceeds the shared tile (T entries, a power of two),
// the stages with stride below T run on T-entry tiles staged in shared
// memory: tiles are sorted first, then every merge block of size kk > T runs
// its strides >= T on global memory and its strides < T tile by tile.  This
// is the same network (the direction of an exchange depends on the global
// index), so the result is identical; it only moves fewer bytes.
template <int KEY>
__device__ void coop_sort(View v, int P, View tile, int T)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (T <= 0 || P <= T) {
        for (int kk = 2; kk <= P; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int t = tid; t < (P >> 1); t += nt) {
                    const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                    cex<KEY>(v, i, i + j, (i & kk) == 0);
                }
                __syncthreads();
            }
        }
        return;
    }
    // strides below T of merge blocks up to kk_hi, on shared tiles
    auto tile_pass = [&](int kk_lo, int kk_hi) {
        for (int base = 0; base < P; base += T) {
            for (int i = tid; i < T; i += nt) {
                tile.row[i] = v.row[base + i];
                tile.w[i] = v.w[base + i];
                if (KEY == 1) tile.mult[i] = v.mult[base + i];
            }
            __syncthreads();
            for (int kk = kk_lo; kk <= kk_hi; kk <<= 1) {
                for (int j = (kk >> 1) < T ? (kk >> 1) : (T >> 1); j > 0; j >>= 1) {
                    for (int t = tid; t < (T >> 1); t += nt) {
                        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                        cex<KEY>(tile, i, i + j, ((base + i) & kk) == 0);
                    }
                    __syncthreads();
                }
            }
            for (int i = tid; i < T; i += nt) {
                v.row[base + i] = tile.row[i];
                v.w[base + i] = tile.w[i];
                if (KEY == 1) v.mult[base + i] = tile.mult[i];
            }
            __syncthreads();
        }
    };
    tile_pass(2, T);                                  // every tile sorted (direction by global index)
    for (int kk = 2 * T; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j >= T; j >>= 1) {      // large strides on global memory
            for (int t = tid; t < (P >> 1); t += nt) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                cex<KEY>(v, i, i + j, (i & kk) == 0);
            }
            __syncthreads();
        }
        tile_pass(kk, kk);                            // strides below T of this merge block
    }
}

// ---------------------------------------------------------------- sample sort
// Sorting a working set that lives in global memory (more entries than the
// CTA's shared buffer): a sorted sample in shared memory (8 entries per
// bucket, 256 to cap entries) gives B-1 splitters, every entry is counted into
// its bucket and scattered to the temporary arrays (weights in v.S, row |
// mult << 32 in v.M), and each bucket is sorted -- by one warp when it fits
// the warp's slice of the buffer (in registers up to 256 entries), else by the
// whole CTA.  Bucket boundaries are a deterministic
// function of the keys and every bucket is fully sorted, so the result is the
// sorted sequence itself, as from any other exact sort.  The bucket offsets
// and merged counts live in global scratch (gbo[B+1], gbd[B]).

// Exclusive scan of n ints by the CTA (a and out may be the same array).
__device__ int block_excl_scan(const int *a, int n, int *out, CoopShared &cs)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int c = (n + nt - 1) / nt;
    const int lo = tid * c < n ? tid * c : n, hi = lo + c < n ? lo + c : n;
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += a[i];
    int x = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(FULL, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) cs.hcount[warp] = x;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) { const int h = cs.hcount[w]; if (w < warp) before += h; total += h; }
    int run = before + x - sum;
    for (int i = lo; i < hi; ++i) { const int ai = a[i]; out[i] = run; run += ai; }
    __syncthreads();
    return total;
}

// Bucket of a key: the number of splitters strictly below it, splitter b
// (b = 1..B-1) being sample entry b*stride (stride = SS/B, both powers of two).  KEY 0 compares rows only (every
// entry of a row falls in one bucket), KEY 1 the full (weight bits, row) key.
template <int KEY>
__device__ __forceinline__ int bucket_of(const View &smp, int stride, int B, int32_t r, unsigned long long wb)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int si = mid * stride;
        const int32_t sr = smp.row[si];
        bool below;
        if (KEY == 0) {
            below = sr < r;
        } else {
            const unsigned long long sw = dbits(smp.w[si]);
            below = sw < wb || (sw == wb && sr < r);
        }
        if (below) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shared part of both sorts: sample, count, bucket offsets, scatter.  n >
// cap entries (row, w, mult) of v are moved to the temporaries in bucket
// order; gbo[0..B] receives the bucket offsets and gbig[0..cs.nbig) the
// buckets larger than a warp's slice.  Returns B.
template <int KEY>
__device__ int sample_partition(View v, int n, View tile, int cap, int wcap, CoopShared &cs, int *gbo, int *gbig)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    // B a power of two, buckets half a warp's slice on average; 8 samples per
    // bucket (at least 256, at most cap: a power of two), so at least 4
    int B = next_pow2((2 * n + wcap - 1) / wcap);
    if (B > cap / 4) B = cap / 4;
    if (B < 1) B = 1;
    int SS = 8 * B;
    if (SS < 256) SS = 256;
    if (SS > cap) SS = cap;
    const int lg = __ffs(SS) - 1;
    for (int s2 = tid; s2 < SS; s2 += nt) {
        const int i = (int)(((long long)s2 * n) >> lg);
        tile.row[s2] = v.row[i];
        tile.w[s2] = v.w[i];
        if (KEY == 1) tile.mult[s2] = v.mult[i];
    }
    __syncthreads();
    coop_sort<KEY>(tile, SS, tile, 0);
    const int stride = SS / B;
    int *cnt = (int *)tile.S, *cur = (int *)tile.S + cap, *off = (int *)tile.M;
    for (int b = tid; b < B; b += nt) { cnt[b] = 0; cur[b] = 0; }
    if (tid == 0) cs.nbig = 0;
    __syncthreads();
    for (int i0 = tid; i0 < n; i0 += 4 * nt) {
        int32_t r[4];
        unsigned long long wb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * nt;
            r[q] = i < n ? v.row[i] : 0;
            wb[q] = KEY == 1 && i < n ? dbits(v.w[i]) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (i0 + q * nt < n) atomicAdd(cnt + bucket_of<KEY>(tile, stride, B, r[q], wb[q]), 1);
    }
    __syncthreads();
    for (int b = tid; b < B; b += nt)
        if (cnt[b] > wcap) gbig[atomicAdd(&cs.nbig, 1)] = b;
    block_excl_scan(cnt, B, off, cs);
    if (tid == 0) off[B] = n;
    __syncthreads();
    unsigned long long *tM = (unsigned long long *)v.M;
    for (int i0 = tid; i0 < n; i0 += 4 * nt) {
        int32_t r[4], m[4];
        double w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * nt;
            r[q] = i < n ? v.row[i] : 0;
            w[q] = i < n ? v.w[i] : 0.0;
            m[q] = KEY == 1 && i < n ? v.mult[i] : 0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i0 + q * nt >= n) continue;
            const int b = bucket_of<KEY>(tile, stride, B, r[q], KEY == 1 ? dbits(w[q]) : 0ull);
            const int pos = off[b] + atomicAdd(cur + b, 1);
            v.S[pos] = w[q];
            tM[pos] = (unsigned long long)(uint32_t)r[q] | ((unsigned long long)(uint32_t)m[q] << 32);
        }
    }
    for (int b = tid; b <= B; b += nt) gbo[b] = off[b];
    __syncthreads();
    return B;
}

// Sort one oversized bucket (temporaries [o, o + cb)) with the whole CTA: in
// the shared buffer when it fits, else in v[0, P) (free once the entries are
// scattered) with the tiled network.  Returns the view holding the sorted
// bucket at [0, cb).
template <int KEY>
__device__ View sort_big_bucket(View v, View tile, int cap, int o, int cb)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const double *tS = v.S;
    const unsigned long long *tM = (const unsigned long long *)v.M;
    const int Pb = next_pow2(cb);
    const View w = Pb <= cap ? tile : v;
    const double wpad = KEY == 0 ? 0.0 : __longlong_as_double((long long)WBITS_SENTINEL);
    for (int i = tid; i < Pb; i += nt) {
        if (i < cb) {
            const unsigned long long rm = tM[o + i];
            const double x = tS[o + i];
            w.row[i] = (int32_t)(uint32_t)rm; w.w[i] = x;
            if (KEY == 1) w.mult[i] = (int32_t)(rm >> 32);
        } else {
            w.row[i] = ROW_SENTINEL; w.w[i] = wpad;
            if (KEY == 1) w.mult[i] = 0;
        }
    }
    __syncthreads();
    coop_sort<KEY>(w, Pb, tile, Pb <= cap ? 0 : cap);
    return w;
}

// Buckets of up to 256 entries are sorted by one warp with a rank sort: the
// keys go to the warp's shared slice, and every entry's place is the number
// of entries with a smaller key, counted against all of them (equal keys,
// i.e. identical (row, weight) entries, by their index).  The places form a
// permutation that sorts the bucket, the same sorted list as any exact sort;
// a lane holds entries lane + 32e, e < E.
template <int KEY>
__device__ __forceinline__ bool key_lt(int32_t ra, unsigned long long ba, int32_t rb, unsigned long long bb)
{
    return KEY == 0 ? (ra < rb || (ra == rb && ba < bb)) : (ba < bb || (ba == bb && ra < rb));
}

// Buckets of 65 to 256 entries go through a bitonic network in registers
// instead (lane l holds positions lE .. lE + E - 1 of the list padded to 32E
// entries; stages with stride j < E compare two slots of a lane, the others
// pair lane l with lane l ^ (j / E) through shuffles): its cost grows with
// log^2 of the size where the rank sort's grows with the square.
template <int KEY>
__device__ __forceinline__ bool key_gt(int32_t ra, unsigned long long ba, int32_t rb, unsigned long long bb)
{
    return KEY == 0 ? (ra > rb || (ra == rb && ba > bb)) : (ba > bb || (ba == bb && ra > rb));
}

// Stages with stride J < E: slots e and e + J of one lane.
template <int KEY, int E, int J>
__device__ __forceinline__ void reg_bucket_intra(int32_t (&r)[E], unsigned long long (&b)[E], int32_t (&m)[E],
                                                 int lane, int kk)
{
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (e & J) continue;
        const bool asc = ((lane * E + e) & kk) == 0;
        if (key_gt<KEY>(r[e], b[e], r[e + J], b[e + J]) == asc) {
            const int32_t rt = r[e]; r[e] = r[e + J]; r[e + J] = rt;
            const unsigned long long bt = b[e]; b[e] = b[e + J]; b[e + J] = bt;
            if (KEY == 1) { const int32_t mt = m[e]; m[e] = m[e + J]; m[e + J] = mt; }
        }
    }
}

// The stage loops stay loops (only the slots of one stage are unrolled):
// the network runs rarely on any one SM, so its code is kept small.
template <int KEY, int E>
__device__ __forceinline__ void reg_bucket_net(int32_t (&r)[E], unsigned long long (&b)[E], int32_t (&m)[E])
{
    const int lane = (int)lane_id();
#pragma unroll 1
    for (int kk = 2; kk <= 32 * E; kk <<= 1) {
#pragma unroll 1
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const bool asc = ((lane * E + e) & kk) == 0;
                    const int32_t ro = __shfl_xor_sync(FULL, r[e], lj);
                    const unsigned long long bo = __shfl_xor_sync(FULL, b[e], lj);
                    const int32_t mo = KEY == 1 ? __shfl_xor_sync(FULL, m[e], lj) : 0;
                    const bool take = lower == asc ? key_gt<KEY>(r[e], b[e], ro, bo) : key_gt<KEY>(ro, bo, r[e], b[e]);
                    if (take) { r[e] = ro; b[e] = bo; if (KEY == 1) m[e] = mo; }
                }
            } else if (j == 1) {
                if (E > 1) reg_bucket_intra<KEY, E, (E > 1 ? 1 : 0)>(r, b, m, lane, kk);
            } else if (j == 2) {
                if (E > 2) reg_bucket_intra<KEY, E, (E > 2 ? 2 : 0)>(r, b, m, lane, kk);
            } else {
                if (E > 4) reg_bucket_intra<KEY, E, (E > 4 ? 4 : 0)>(r, b, m, lane, kk);
            }
        }
    }
}

// Load bucket [o, o + cb) of the temporaries (weights tS, row | mult << 32 in
// tM) into the lanes' slots, sentinels past cb.
template <int KEY, int E>
__device__ __forceinline__ void reg_bucket_load(const double *tS, const unsigned long long *tM, int o, int cb,
                                                int32_t (&r)[E], unsigned long long (&b)[E], int32_t (&m)[E])
{
    const int lane = (int)lane_id();
    unsigned long long rm[E], wb[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane * E + e;
        rm[e] = i < cb ? __ldcg(tM + o + i) : (unsigned long long)(uint32_t)ROW_SENTINEL;
        wb[e] = i < cb ? dbits(__ldcg(tS + o + i)) : (KEY == 0 ? 0ull : WBITS_SENTINEL);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) { r[e] = (int32_t)(uint32_t)rm[e]; m[e] = (int32_t)(rm[e] >> 32); b[e] = wb[e]; }
}

// Load bucket [o, o + cb) of the temporaries (weights tS, row | mult << 32 in
// tM), put its keys in sv and return every held entry's place.
template <int KEY, int E>
__device__ __forceinline__ void rank_bucket(const double *tS, const unsigned long long *tM, int o, int cb, View sv,
                                            int32_t (&r)[E], unsigned long long (&b)[E], int32_t (&m)[E],
                                            int (&place)[E])
{
    const int lane = (int)lane_id();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        const unsigned long long rm = i < cb ? __ldcg(tM + o + i) : 0ull;
        b[e] = i < cb ? dbits(__ldcg(tS + o + i)) : 0ull;
        r[e] = (int32_t)(uint32_t)rm;
        m[e] = (int32_t)(rm >> 32);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < cb) { sv.row[i] = r[e]; sv.w[i] = __longlong_as_double((long long)b[e]); }
        place[e] = 0;
    }
    __syncwarp();
    for (int j = 0; j < cb; ++j) {
        const int32_t rj = sv.row[j];
        const unsigned long long bj = dbits(sv.w[j]);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane + 32 * e;
            place[e] += (key_lt<KEY>(rj, bj, r[e], b[e]) || (rj == r[e] && bj == b[e] && j < i)) ? 1 : 0;
        }
    }
    __syncwarp();
}

// Row phase: sort the bucket by (row, weight bits) into [0, cb) of the warp's
// shared slice, for the run merge.
template <int E>
__device__ __noinline__ void reg_bucket_rows(const double *tS, const unsigned long long *tM, int o, int cb, View sv)
{
    int32_t r[E], m[E];
    unsigned long long b[E];
    if (E >= 4) {                                         // network: lane l holds positions lE + e
        reg_bucket_load<0, E>(tS, tM, o, cb, r, b, m);
        reg_bucket_net<0, E>(r, b, m);
        const int lane = (int)lane_id();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane * E + e;
            if (i < cb) { sv.row[i] = r[e]; sv.w[i] = __longlong_as_double((long long)b[e]); }
        }
        __syncwarp();
        return;
    }
    int place[E];
    rank_bucket<0, E>(tS, tM, o, cb, sv, r, b, m, place);
    const int lane = (int)lane_id();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (lane + 32 * e < cb) { sv.row[place[e]] = r[e]; sv.w[place[e]] = __longlong_as_double((long long)b[e]); }
    }
    __syncwarp();
}

// Weight phase: sort the bucket by (weight bits, row) into [o, o + cb) of v
// (sv is the warp's shared slice for the keys).
template <int E>
__device__ __noinline__ void reg_bucket_weights(const double *tS, const unsigned long long *tM, int o, int cb, View sv,
                                                View v)
{
    int32_t r[E], m[E];
    unsigned long long b[E];
    if (E >= 4) {
        reg_bucket_load<1, E>(tS, tM, o, cb, r, b, m);
        reg_bucket_net<1, E>(r, b, m);
        const int lane = (int)lane_id();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane * E + e;
            if (i < cb) { v.row[o + i] = r[e]; v.w[o + i] = __longlong_as_double((long long)b[e]); v.mult[o + i] = m[e]; }
        }
        return;
    }
    int place[E];
    rank_bucket<1, E>(tS, tM, o, cb, sv, r, b, m, place);
    const int lane = (int)lane_id();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (lane + 32 * e < cb) {
            const int q = o + place[e];
            v.row[q] = r[e]; v.w[q] = __longlong_as_double((long long)b[e]); v.mult[q] = m[e];
        }
    }
    __syncwarp();
}

constexpr int REG_BUCKET_MAX = 256;

// Merge the sorted runs of a bucket held in a shared view (rows, weights in
// [0, cb)), writing (sum, row | len << 32) to [o, o + d_b) of the temporaries
// by one warp; returns d_b.  Runs are summed left to right.
__device__ __forceinline__ int warp_merge_bucket(View sv, int cb, double *tS, unsigned long long *tM, int o)
{
    const unsigned lane = lane_id();
    int db = 0;
    for (int base = 0; base < cb; base += 32) {
        const int i = base + (int)lane;
        bool head = false;
        int32_t r = 0;
        int len = 0;
        double sum = 0.0;
        if (i < cb) {
            r = sv.row[i];
            head = (i == 0) || (sv.row[i - 1] != r);
            if (head) {
                sum = sv.w[i]; len = 1;
                while (i + len < cb && sv.row[i + len] == r) { sum = __dadd_rn(sum, sv.w[i + len]); ++len; }
            }
        }
        const unsigned bal = __ballot_sync(FULL, head);
        if (head) {
            const int rank = db + __popc(bal & ((1u << lane) - 1u));
            tS[o + rank] = sum;
            tM[o + rank] = (unsigned long long)(uint32_t)r | ((unsigned long long)(uint32_t)len << 32);
        }
        db += __popc(bal);
    }
    return db;
}

// Row phase on a global working set: sort (row, weight bits), merge runs,
// compact in bucket order into v[0, d) (row, w, mult) and store the F column
// rows / merged weights.  Returns d, or -2 on abort.
__device__ int coop_row_phase(const ElimArgs &a, CoopShared &cs, View v, int g, unsigned char *bbuf, int cap,
                              int *gbo, int *gbd, int *gbig, int32_t k)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int wcap = cap / nw;
    const View tile = make_view(bbuf, cap);
    const int B = sample_partition<0>(v, g, tile, cap, wcap, cs, gbo, gbig);
    double *tS = v.S;
    unsigned long long *tM = (unsigned long long *)v.M;
    // oversized buckets first, by the whole CTA (their work space may be v itself)
    const int nbig = cs.nbig;
    for (int q = 0; q < nbig; ++q) {
        const int b = gbig[q];
        const int o = gbo[b], cb = gbo[b + 1] - o;
        const View w = sort_big_bucket<0>(v, tile, cap, o, cb);
        if (warp == 0) {
            const int db = warp_merge_bucket(w, cb, tS, tM, o);
            if (lane == 0) gbd[b] = db;
        }
        __syncthreads();
    }
    // the others: one warp each, in the warp's slice of the shared buffer
    const View sv = make_view(bbuf + (size_t)warp * wcap * ENTRY_BYTES, wcap);
    for (int b = warp; b < B; b += nw) {
        const int o = gbo[b], cb = gbo[b + 1] - o;
        if (cb > wcap) continue;
        int db = 0;
        if (cb > 0) {
            const int Pb = next_pow2(cb);
            if (Pb <= REG_BUCKET_MAX) {
                if (Pb <= 32) reg_bucket_rows<1>(tS, tM, o, cb, sv);
                else if (Pb == 64) reg_bucket_rows<2>(tS, tM, o, cb, sv);
                else if (Pb == 128) reg_bucket_rows<4>(tS, tM, o, cb, sv);
                else reg_bucket_rows<8>(tS, tM, o, cb, sv);
            } else {
                for (int i = lane; i < Pb; i += 32) {
                    if (i < cb) { sv.row[i] = (int32_t)(uint32_t)tM[o + i]; sv.w[i] = tS[o + i]; }
                    else { sv.row[i] = ROW_SENTINEL; sv.w[i] = 0.0; }
                }
                __syncwarp();
                sort_row_bits(sv, Pb);
            }
            db = warp_merge_bucket(sv, cb, tS, tM, o);
            __syncwarp();
        }
        if (lane == 0) gbd[b] = db;
    }
    __syncthreads();
    // compaction in bucket order, with the F column store
    int *pd = (int *)bbuf;
    for (int b = tid; b < B; b += nt) pd[b] = gbd[b];
    __syncthreads();
    const int d = block_excl_scan(pd, B, pd, cs);
    if (tid == 0) {
        const unsigned long long base = d > 0 ? atomicAdd(a.f_top, (unsigned long long)d) : 0ull;
        if (d > 0 && base + d > a.f_cap) set_status(a.status, ST_POOL);
        cs.fpos = base;
    }
    if (__syncthreads_or(read_status(a.status) != ST_OK)) return -2;
    const unsigned long long fpos = cs.fpos;
    for (int b = warp; b < B; b += nw) {
        const int o = gbo[b], db = gbd[b], p0 = pd[b];
        for (int i = lane; i < db; i += 32) {
            const unsigned long long rm = tM[o + i];
            const int32_t r = (int32_t)(uint32_t)rm;
            const double w = tS[o + i];
            v.row[p0 + i] = r; v.w[p0 + i] = w; v.mult[p0 + i] = (int32_t)(rm >> 32);
            a.f_row[fpos + p0 + i] = r; a.f_val[fpos + p0 + i] = w;
        }
    }
    if (tid == 0) { a.f_start[k] = (int64_t)fpos; a.f_len[k] = d; }
    __syncthreads();
    return d;
}

// Weight phase on a global working set: sort v[0, d) by (weight bits, row)
// carrying the multiplicity.
__device__ void coop_weight_phase(View v, int d, unsigned char *bbuf, int cap, CoopShared &cs, int *gbo, int *gbig)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int wcap = cap / nw;
    const View tile = make_view(bbuf, cap);
    if (d <= cap) {                                   // one tile
        const int Pd = next_pow2(d);
        for (int i = tid; i < Pd; i += nt) {
            if (i < d) { tile.row[i] = v.row[i]; tile.w[i] = v.w[i]; tile.mult[i] = v.mult[i]; }
            else { tile.row[i] = ROW_SENTINEL; tile.w[i] = __longlong_as_double((long long)WBITS_SENTINEL); tile.mult[i] = 0; }
        }
        __syncthreads();
        coop_sort<1>(tile, Pd, tile, 0);
        for (int i = tid; i < d; i += nt) { v.row[i] = tile.row[i]; v.w[i] = tile.w[i]; v.mult[i] = tile.mult[i]; }
        __syncthreads();
        return;
    }
    const int B = sample_partition<1>(v, d, tile, cap, wcap, cs, gbo, gbig);
    double *tS = v.S;
    unsigned long long *tM = (unsigned long long *)v.M;
    // oversized buckets first, sorted back into the temporaries (v may be their work space)
    const int nbig = cs.nbig;
    for (int q = 0; q < nbig; ++q) {
        const int b = gbig[q];
        const int o = gbo[b], cb = gbo[b + 1] - o;
        const View w = sort_big_bucket<1>(v, tile, cap, o, cb);
        for (int i = tid; i < cb; i += nt) {
            tS[o + i] = w.w[i];
            tM[o + i] = (unsigned long long)(uint32_t)w.row[i] | ((unsigned long long)(uint32_t)w.mult[i] << 32);
        }
        __syncthreads();
    }
    // every bucket to its final place: small ones sorted by one warp each, big ones copied
    const View sv = make_view(bbuf + (size_t)warp * wcap * ENTRY_BYTES, wcap);
    for (int b = warp; b < B; b += nw) {
        const int o = gbo[b], cb = gbo[b + 1] - o;
        if (cb == 0) continue;
        if (cb > wcap) {
            for (int i = lane; i < cb; i += 32) {
                const unsigned long long rm = tM[o + i];
                v.row[o + i] = (int32_t)(uint32_t)rm; v.mult[o + i] = (int32_t)(rm >> 32); v.w[o + i] = tS[o + i];
            }
            continue;
        }
        const int Pb = next_pow2(cb);
        if (Pb <= REG_BUCKET_MAX) {
            if (Pb <= 32) reg_bucket_weights<1>(tS, tM, o, cb, sv, v);
            else if (Pb == 64) reg_bucket_weights<2>(tS, tM, o, cb, sv, v);
            else if (Pb == 128) reg_bucket_weights<4>(tS, tM, o, cb, sv, v);
            else reg_bucket_weights<8>(tS, tM, o, cb, sv, v);
            continue;
        }
        for (int i = lane; i < Pb; i += 32) {
            if (i < cb) {
                const unsigned long long rm = tM[o + i];
                sv.row[i] = (int32_t)(uint32_t)rm; sv.mult[i] = (int32_t)(rm >> 32); sv.w[i] = tS[o + i];
            } else {
                sv.row[i] = ROW_SENTINEL; sv.mult[i] = 0; sv.w[i] = __longlong_as_double((long long)WBITS_SENTINEL);
            }
        }
        __syncwarp();
        sort_bits_row(sv, Pb);
        for (int i = lane; i < cb; i += 32) { v.row[o + i] = sv.row[i]; v.w[o + i] = sv.w[i]; v.mult[o + i] = sv.mult[i]; }
        __syncwarp();
    }
    __syncthreads();
}

// ---------------------------------------------------------------- grid help
// A vertex whose working set lives in global scratch is eliminated by its
// CTA, but every data-parallel step of it (gather, bucket counts, scatter,
// bucket sorts, compaction, scan tiles, sampling, decrements) is posted on a
// global board and cut into chunks that any idle warp of the grid may claim.
// The owning CTA claims chunks too and waits (bounded) until every claimed
// chunk is done; the serial steps between them (the sample of splitters,
// bucket scans, the carry chains) stay with the owner.  Only who computes a
// chunk changes, never what it computes, so the factor is the same.
//
// Board: gh_word = generation << 48 | chunks << 32 | next chunk.  A claim is
// an atomicAdd of 1; it is valid when the old next is below the old chunk
// count, for the generation it shows, whose descriptor stays in place until
// all its chunks are done.  A helper releases its writes (fence) before it
// counts its chunk done; the owner acquires the done count before the next
// step.  Data that other SMs wrote are read through L2 (ld.cg).
enum : int32_t {
    // numbered as in the step profile of the statistics (2 and 3 are unused)
    GH_GATHER = 1, GH_SCATTER0 = 4, GH_SCATTER1, GH_ROWB, GH_COMPACT, GH_WB, GH_TILES, GH_CARRYMAX, GH_SAMPLE,
    GH_DECR
};
static_assert(sizeof(GhTask) % 16 == 0, "task descriptors are copied in 16-byte units");

// Compact view of a warp's slice for a bucket of up to 256 entries: weights,
// then rows (3 KB).
__device__ __forceinline__ View slice_view(unsigned char *slice)
{
    View v;
    v.w = (double *)slice;
    v.row = (int32_t *)(slice + 8 * REG_BUCKET_MAX);
    v.S = v.M = nullptr;
    v.mult = nullptr;
    return v;
}

// Bucket of an entry among splitters sr/sw[1 .. B-1] (in the warp's slice, or
// in global memory when they do not fit): as bucket_of.
template <int KEY>
__device__ __forceinline__ int gh_bucket(const int32_t *sr, const unsigned long long *sw, int B, bool glob,
                                         int32_t r, unsigned long long wb)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int32_t s = glob ? __ldcg(sr + mid) : sr[mid];
        bool below;
        if (KEY == 0) {
            below = s < r;
        } else {
            const unsigned long long w = glob ? __ldcg(sw + mid) : sw[mid];
            below = w < wb || (w == wb && s < r);
        }
        if (below) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Splitters 1..B-1 of the posted sample sort into the warp's slice when they
// fit (rows from the slice's start, weight bits from byte 2048), a lane's
// loads in flight together.  Returns true when they stay in global memory.
template <int KEY>
__device__ __forceinline__ bool gh_stage(const GhTask &t, unsigned char *slice, const int32_t *&sr,
                                         const unsigned long long *&sw)
{
    sr = t.spl_row; sw = t.spl_wb;
    if (!t.spl_shared) return true;
    const int lane = (int)lane_id();
    int32_t *lr = (int32_t *)slice;
    unsigned long long *lw = (unsigned long long *)(slice + 8 * REG_BUCKET_MAX);
    for (int b0 = 0; b0 < t.B; b0 += 256) {
        int32_t x[8];
        unsigned long long y[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = b0 + 32 * q + lane;
            x[q] = b < t.B ? __ldcg(t.spl_row + b) : 0;
            y[q] = KEY == 1 && b < t.B ? __ldcg(t.spl_wb + b) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = b0 + 32 * q + lane;
            if (b < t.B) { lr[b] = x[q]; if (KEY == 1) lw[b] = y[q]; }
        }
    }
    __syncwarp();
    sr = lr; sw = lw;
    return false;
}

// Count Q entries per lane (ok[q]: the entry exists) into their buckets:
// one atomic per bucket and warp step, all in flight together.
template <int KEY, int Q>
__device__ __forceinline__ void gh_count(const GhTask &t, const int32_t *sr, const unsigned long long *sw, bool glob,
                                         const int32_t (&r)[Q], const unsigned long long (&wb)[Q], const bool (&ok)[Q])
{
    const int lane = (int)lane_id();
    int bk[Q];
    unsigned grp[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        bk[q] = ok[q] ? gh_bucket<KEY>(sr, sw, t.B, glob, r[q], wb[q]) : -1;
        grp[q] = __match_any_sync(FULL, bk[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (bk[q] >= 0 && lane == __ffs(grp[q]) - 1) atomicAdd(t.cnt_b + bk[q], __popc(grp[q]));
}

// Entry i of column k's gathered list: its original lower entries, then its
// fill by append index (inline slab, then the overflow levels; gi is the
// level's directory entry, loaded beforehand).
__device__ __forceinline__ uint32_t gh_fill_dir(const ElimArgs &a, int32_t k, int norig, int g, int i)
{
    const uint32_t f = (uint32_t)(i - norig);
    if (i < norig || i >= g || f < (uint32_t)FILL_C0) return 0u;
    const int j = fill_level(f);
    return j <= FILL_LEVELS ? __ldcg(a.dir + (size_t)k * FILL_LEVELS + (j - 1)) : 0u;
}

__device__ __forceinline__ void gh_src_entry(const ElimArgs &a, int32_t k, int norig, int g, int64_t o0, int i,
                                             uint32_t gi, int32_t &r, double &w)
{
    r = ROW_SENTINEL; w = 0.0;
    if (i < norig) {
        r = __ldg(a.lrow + o0 + i); w = __ldg(a.lw + o0 + i);
    } else if (i < g) {
        const uint32_t f = (uint32_t)(i - norig);
        if (f < (uint32_t)FILL_C0) {
            r = __ldcg(a.in_row + (size_t)k * FILL_C0 + f); w = __ldcg(a.in_w + (size_t)k * FILL_C0 + f);
        } else if (gi == 0u || gi == 0xffffffffu) {
            set_status(a.status, ST_INVAL);
        } else {
            const unsigned long long at = (unsigned long long)(gi - 1u) * FILL_GRANULE + (f - fill_level_start(fill_level(f)));
            r = __ldcg(a.pool_row + at); w = __ldcg(a.pool_w + at);
        }
    }
}

// Scatter one chunk of entries into their buckets (positions from the
// bucket offsets and per-bucket cursors).
template <int KEY>
__device__ void gh_scatter_chunk(const GhTask &t, int lo, int hi, unsigned char *slice)
{
    const int lane = (int)lane_id();
    const View v = make_view(t.vbase, t.cap);
    const int32_t *sr;
    const unsigned long long *sw;
    const bool glob = gh_stage<KEY>(t, slice, sr, sw);
    double *tS = v.S;
    unsigned long long *tM = (unsigned long long *)v.M;
    for (int i0 = lo; i0 < hi; i0 += 8 * 32) {
        int32_t r[8], m[8], bk[8];
        double w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + 32 * q + lane;
            r[q] = i < hi ? __ldcg(v.row + i) : 0;
            w[q] = i < hi ? __ldcg(v.w + i) : 0.0;
            m[q] = KEY == 1 && i < hi ? __ldcg(v.mult + i) : 0;
        }
        unsigned grp[8];
        int base[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + 32 * q + lane;
            bk[q] = i < hi ? gh_bucket<KEY>(sr, sw, t.B, glob, r[q], KEY == 1 ? dbits(w[q]) : 0ull) : -1;
            grp[q] = __match_any_sync(FULL, bk[q]);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {                      // all of the batch's atomics in flight together
            const int leader = __ffs(grp[q]) - 1;
            base[q] = 0;
            if (bk[q] >= 0 && lane == leader) base[q] = atomicAdd(t.cur_b + bk[q], __popc(grp[q]));
        }
        {
            int off[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) off[q] = bk[q] >= 0 ? __ldcg(t.gbo + bk[q]) : 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int bq = __shfl_sync(FULL, base[q], __ffs(grp[q]) - 1);
                if (bk[q] >= 0) {
                    const int pos = off[q] + bq + __popc(grp[q] & ((1u << lane) - 1u));
                    tS[pos] = w[q];
                    tM[pos] = (unsigned long long)(uint32_t)r[q] | ((unsigned long long)(uint32_t)m[q] << 32);
                }
            }
        }
    }
    __syncwarp();
}

// One chunk of a posted step, by one warp.  keep: as decrement_group.
// Returns false when the kernel must stop.
__device__ __noinline__ bool gh_do(const ElimArgs &a, const GhTask &t, int idx, unsigned char *slice, int32_t &keep)
{
    const int lane = (int)lane_id();
    if (idx < 0 || idx >= t.nch || (long long)idx * t.chunk >= (long long)t.n) {
        set_status(a.status, ST_INVAL);
        return false;
    }
    const int lo = idx * t.chunk, hi = lo + t.chunk < t.n ? lo + t.chunk : t.n;
    const View v = make_view(t.vbase, t.cap);
    double *tS = v.S;
    unsigned long long *tM = (unsigned long long *)v.M;
    const int d = t.d;
    switch (t.op) {
    case GH_GATHER: {                                         // gather, and count the row sort's buckets
        const int32_t *sr;
        const unsigned long long *sw;
        const bool glob = gh_stage<0>(t, slice, sr, sw);
        const int k = t.k, norig = t.norig, g = t.norig + (int)t.cnt;
        for (int base = lo; base < hi; base += 128) {
            uint32_t gi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = base + 32 * q + lane;
                gi[q] = i < hi ? gh_fill_dir(a, k, norig, g, i) : 0u;
            }
            int32_t r[4];
            double w[4];
            unsigned long long wb[4];
            bool ok[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = base + 32 * q + lane;
                gh_src_entry(a, k, norig, g, t.o0, i < hi ? i : g, gi[q], r[q], w[q]);
                wb[q] = 0ull;
                ok[q] = i < hi && i < g;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = base + 32 * q + lane;
                if (i < hi) { v.row[i] = r[q]; v.w[i] = w[q]; }
            }
            gh_count<0, 4>(t, sr, sw, glob, r, wb, ok);
        }
        __syncwarp();
        return true;
    }
    case GH_SCATTER0: gh_scatter_chunk<0>(t, lo, hi, slice); return true;
    case GH_SCATTER1: gh_scatter_chunk<1>(t, lo, hi, slice); return true;
    case GH_ROWB: {
        const View sv = slice_view(slice);
        for (int b = lo; b < hi; ++b) {
            const int o = __ldcg(t.gbo + b), cb = __ldcg(t.gbo + b + 1) - o;
            if (cb > t.bmax) continue;                       // sorted and merged by the owner
            int db = 0;
            if (cb > 0) {
                const int Pb = next_pow2(cb);
                if (Pb <= 32) reg_bucket_rows<1>(tS, tM, o, cb, sv);
                else if (Pb == 64) reg_bucket_rows<2>(tS, tM, o, cb, sv);
                else if (Pb == 128) reg_bucket_rows<4>(tS, tM, o, cb, sv);
                else reg_bucket_rows<8>(tS, tM, o, cb, sv);
                db = warp_merge_bucket(sv, cb, tS, tM, o);
                __syncwarp();
            }
            if (lane == 0) t.gbd[b] = db;
        }
        return true;
    }
    case GH_COMPACT: {                                        // compaction + F store (+ the weight sort's counts)
        const int32_t *sr = nullptr;
        const unsigned long long *sw = nullptr;
        const bool count = t.B > 0;
        const bool glob = count ? gh_stage<1>(t, slice, sr, sw) : true;
        for (int b = lo; b < hi; ++b) {
            const int o = __ldcg(t.gbo + b), db = __ldcg(t.gbd + b), p0 = __ldcg(t.pd + b);
            for (int i0 = 0; i0 < db; i0 += 128) {
                unsigned long long rm[4];
                double x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = i0 + 32 * q + lane;
                    rm[q] = i < db ? __ldcg(tM + o + i) : 0ull;
                    x[q] = i < db ? __ldcg(tS + o + i) : 0.0;
                }
                int32_t r[4];
                unsigned long long wb[4];
                bool ok[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = i0 + 32 * q + lane;
                    r[q] = (int32_t)(uint32_t)rm[q];
                    wb[q] = dbits(x[q]);
                    ok[q] = i < db;
                    if (i >= db) continue;
                    v.row[p0 + i] = r[q]; v.w[p0 + i] = x[q]; v.mult[p0 + i] = (int32_t)(rm[q] >> 32);
                    a.f_row[t.fpos + p0 + i] = r[q]; a.f_val[t.fpos + p0 + i] = x[q];
                }
                if (count) gh_count<1, 4>(t, sr, sw, glob, r, wb, ok);
            }
        }
        __syncwarp();
        return true;
    }
    case GH_WB: {
        for (int b = lo; b < hi; ++b) {
            const int o = __ldcg(t.gbo + b), cb = __ldcg(t.gbo + b + 1) - o;
            if (cb == 0) continue;
            if (cb > t.bmax) {                               // sorted by the owner: to its place
                for (int i = lane; i < cb; i += 32) {
                    const unsigned long long rm = __ldcg(tM + o + i);
                    v.row[o + i] = (int32_t)(uint32_t)rm; v.mult[o + i] = (int32_t)(rm >> 32);
                    v.w[o + i] = __ldcg(tS + o + i);
                }
                continue;
            }
            const int Pb = next_pow2(cb);
            const View sv = slice_view(slice);
            if (Pb <= 32) reg_bucket_weights<1>(tS, tM, o, cb, sv, v);
            else if (Pb == 64) reg_bucket_weights<2>(tS, tM, o, cb, sv, v);
            else if (Pb == 128) reg_bucket_weights<4>(tS, tM, o, cb, sv, v);
            else reg_bucket_weights<8>(tS, tM, o, cb, sv, v);
        }
        return true;
    }
    case GH_TILES: {                                          // scan of each 32-entry tile of the reversed weights
        for (int j0 = lo; j0 < hi; j0 += 4) {
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int tt = 32 * (j0 + q) + lane;
                x[q] = j0 + q < hi && tt < d ? __ldcg(v.w + (d - 1 - tt)) : 0.0;
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double y = __shfl_up_sync(FULL, x[q], off);
                    if (lane >= off) x[q] = __dadd_rn(x[q], y);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (j0 + q >= hi) continue;
                const int tt = 32 * (j0 + q) + lane;
                if (tt < d) v.S[d - 1 - tt] = x[q];
                if (lane == 31) t.tiles[j0 + q] = x[q];
            }
        }
        return true;
    }
    case GH_CARRYMAX: {                                       // tile carry, then the tile's running maximum
        for (int j0 = lo; j0 < hi; j0 += 4) {
            double sv[4], c[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int tt = 32 * (j0 + q) + lane;
                const bool in = j0 + q < hi && tt < d;
                c[q] = j0 + q < hi ? __ldcg(t.tiles + j0 + q) : 0.0;
                sv[q] = in ? __ldcg(v.S + (d - 1 - tt)) : 0.0;
            }
            unsigned long long m[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int tt = 32 * (j0 + q) + lane;
                const bool in = j0 + q < hi && tt < d;
                if (in) { sv[q] = __dadd_rn(sv[q], c[q]); v.S[d - 1 - tt] = sv[q]; }
                m[q] = in ? dbits(sv[q]) : 0ull;
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned long long y = __shfl_up_sync(FULL, m[q], off);
                    if (lane >= off && y > m[q]) m[q] = y;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (j0 + q >= hi) continue;
                const int tt = 32 * (j0 + q) + lane;
                if (tt < d) v.M[d - 1 - tt] = __longlong_as_double((long long)m[q]);
                if (lane == 31) t.tmax[j0 + q] = m[q];
            }
        }
        return true;
    }
    case GH_SAMPLE: {
        // levels of the merged rows, then slots p = i >= 1, two per lane with
        // their searches interleaved.  M_final[j] = max(M[j], running maximum
        // of the tiles before j's tile) is non-increasing; the largest j in
        // [p, d) with M_final[j] >= R is sampled: first among the coarse
        // entries coarse[c] = M_final[c * cstride] (staged in the slice),
        // then within that stride.
        bool ok = true;
        for (int i = lo + lane; i < hi; i += 32) red_max_relaxed(a.lvl + __ldcg(v.row + i), t.lk);
        unsigned long long *co = (unsigned long long *)slice;
        const int nco = t.nco, cst = t.cstride;
        for (int c0 = 0; c0 < nco; c0 += 256) {
            unsigned long long x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) { const int c = c0 + 32 * q + lane; x[q] = c < nco ? __ldcg(t.coarse + c) : 0ull; }
#pragma unroll
            for (int q = 0; q < 8; ++q) { const int c = c0 + 32 * q + lane; if (c < nco) co[c] = x[q]; }
        }
        __syncwarp();
        const int samples = a.samples;
        for (int base = lo; base < hi && ok; base += 64)
        for (int q = 0; q < samples && ok; ++q) {
            int p[2], jl[2], jh[2];
            unsigned long long Rb[2];
            double Sp[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                p[s] = base + 32 * s + lane;
                const bool act = p[s] >= 1 && p[s] < hi;
                Sp[s] = act ? __ldcg(v.S + p[s]) : 0.0;
                Rb[s] = act ? dbits(__dmul_rn(Sp[s], slot_uniform(a.seed, t.klocal, (uint64_t)p[s], t.sys, (uint64_t)q))) : 0ull;
                jl[s] = 0; jh[s] = 0;
                if (act) {                                   // largest coarse c with coarse[c] >= R (c = p / cst qualifies)
                    int clo = p[s] / cst, chi = nco - 1;
                    while (clo < chi) {
                        const int mid = clo + ((chi - clo + 1) >> 1);
                        if (co[mid] >= Rb[s]) clo = mid; else chi = mid - 1;
                    }
                    jl[s] = clo * cst > p[s] ? clo * cst : p[s];
                    jh[s] = (clo + 1) * cst - 1 < d - 1 ? (clo + 1) * cst - 1 : d - 1;
                }
            }
            while (jl[0] < jh[0] || jl[1] < jh[1]) {
                unsigned long long mv[2] = {0ull, 0ull}, tv[2] = {0ull, 0ull};
                int mid[2];
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    mid[s] = jl[s] + ((jh[s] - jl[s] + 1) >> 1);
                    if (jl[s] < jh[s]) {
                        mv[s] = dbits(__ldcg(v.M + mid[s]));
                        tv[s] = __ldcg(t.tmax + ((d - 1 - mid[s]) >> 5));
                    }
                }
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    if (jl[s] < jh[s]) {
                        const unsigned long long mf = mv[s] > tv[s] ? mv[s] : tv[s];
                        if (mf >= Rb[s]) jl[s] = mid[s]; else jh[s] = mid[s] - 1;
                    }
                }
            }
            int32_t u[2], x[2];
            double wu[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const bool act = p[s] >= 1 && p[s] < hi;
                u[s] = act ? __ldcg(v.row + p[s] - 1) : 0;
                wu[s] = act ? __ldcg(v.w + p[s] - 1) : 0.0;
                x[s] = act ? __ldcg(v.row + jl[s]) : 0;
            }
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const bool act = p[s] >= 1 && p[s] < hi;
                double c = 0.0;
                if (act) {
                    c = __ddiv_rn(__dmul_rn(Sp[s], wu[s]), t.Dk);
                    if (samples > 1) c = __ddiv_rn(c, (double)samples);
                }
                const int32_t lo_v = u[s] < x[s] ? u[s] : x[s], hi_v = u[s] < x[s] ? x[s] : u[s];
                if (!append_fill(a, act, lo_v, hi_v, c)) ok = false;
            }
        }
        __syncwarp();
        return ok;
    }
    case GH_DECR: {
        for (int ib = lo; ib < hi; ib += 128) {
            int32_t u[4], m[4], r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = ib + 32 * q + lane;
                u[q] = i < hi ? __ldcg(v.row + i) : 0;
                m[q] = i < hi ? __ldcg(v.mult + i) : 0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = ib + 32 * q + lane < hi ? atomicSub(a.dp + u[q], m[q]) : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                bool ready = ib + 32 * q + lane < hi && r[q] == m[q];
                if (ready && a.trace) { a.trace[4 * (size_t)u[q]] = global_ns(); a.trace_parent[u[q]] = t.k; }
                unsigned bal = __ballot_sync(FULL, ready);      // as decrement_group, after its atomic
                if (!bal) continue;
                if (keep == -1) {
                    const int kl = __ffs(bal) - 1;
                    keep = __shfl_sync(FULL, u[q], kl);
                    bal &= ~(1u << kl);
                    if (lane == kl) ready = false;
                }
                if (!bal) continue;
                const int leader = __ffs(bal) - 1;
                uint32_t qb = 0;
                if (lane == leader) qb = atomicAdd(a.q_tail, (uint32_t)__popc(bal));
                qb = __shfl_sync(FULL, qb, leader);
                if (ready) {
                    const uint32_t at = qb + __popc(bal & ((1u << lane) - 1u));
                    if (at < (uint32_t)a.nl) { fence_acq_rel(); st_release(a.queue + at, u[q]); }
                    else set_status(a.status, ST_INVAL);
                }
            }
        }
        return true;
    }
    default:
        set_status(a.status, ST_INVAL);
        return false;
    }
}

// Claim and run chunks of generation gen (any generation when gen < 0) until
// none is left.  Warp-uniform; returns the number of chunks run.
__device__ __noinline__ int gh_claim_loop(const ElimArgs &a, const GhTask *own, int gen, unsigned char *slice, int32_t &keep,
                                          int *seen_gen = nullptr)
{
    const int lane = (int)lane_id();
    int runs = 0;
    GhTask t;
    for (;;) {
        unsigned long long old = 0;
        if (lane == 0) {
            // a plain read first: once a step's chunks are all claimed, the
            // late helpers do not queue atomics in front of the real claims
            const unsigned long long cur = *(volatile const unsigned long long *)a.gh_word;
            const bool open = (uint32_t)cur < (uint32_t)((cur >> 32) & 0xffffull) && (gen < 0 || (int)(cur >> 48) == gen);
            old = open ? atomicAdd(a.gh_word, 1ull) : cur | 0xffffffffull;
        }
        old = __shfl_sync(FULL, old, 0);
        const int g = (int)(old >> 48);
        const uint32_t nch = (uint32_t)((old >> 32) & 0xffffull), idx = (uint32_t)old;   // unsigned: a closed step reads 0xffffffff
        if (seen_gen) *seen_gen = g;
        if (idx >= nch || (gen >= 0 && g != gen)) break;
        const int slot = g & (GH_RING - 1);
        const GhTask *tp = own;
        if (!own) {
            fence_acq_rel();                              // acquire: the post precedes the chunk's reads
            const uint4 *src = (const uint4 *)(a.gh_task + slot);
            uint4 *dst = (uint4 *)&t;
#pragma unroll
            for (int i = 0; i < (int)(sizeof(GhTask) / 16); ++i) dst[i] = __ldcg(src + i);
            tp = &t;
        }
        bool ok = tp->gen == g;
        if (!ok) set_status(a.status, ST_INVAL);
        else if (idx >= (uint32_t)tp->nch) { set_status(a.status, ST_INVAL); ok = false; }
        else {
            const long long c0 = a.profile && !own ? clock64() : 0;
            ok = gh_do(a, *tp, (int)idx, slice, keep);
            if (a.profile && !own && lane == 0 && a.stats && tp->op >= 1 && tp->op <= 12) {
                const unsigned long long dc = (unsigned long long)(clock64() - c0);
                atomicAdd(a.stats + 80 + tp->op, dc);
                atomicAdd(a.stats + 96 + tp->op, 1ull);
                if (runs > 0) { atomicAdd(a.stats + 112 + tp->op, dc); atomicAdd(a.stats + 128 + tp->op, 1ull); }
            }
        }
        __threadfence();                                  // release the chunk's writes
        __syncwarp();
        if (lane == 0) atomicAdd(a.gh_done + 32 * slot, 1u);
        ++runs;
        if (!ok || read_status(a.status) != ST_OK) break;
    }
    return runs;
}

// Helper side, from an idle worker's poll loop: the hint is read inline, the
// claims run out of line only when a post was seen.
__device__ __noinline__ int gh_help(const ElimArgs &a, unsigned char *slice, int *seen_gen)
{
    int32_t keep = -2;
    const int runs = gh_claim_loop(a, nullptr, -1, slice, keep, seen_gen);
    if (a.stats && lane_id() == 0 && runs > 0) atomicAdd(a.stats + 25, (unsigned long long)runs);
    return runs;
}

__device__ __forceinline__ int gh_serve(const ElimArgs &a, unsigned char *slice, uint32_t &seen, uint32_t h)
{
    if (h == 0u || h == seen) return 0;
    int g = -1;
    const int runs = gh_help(a, slice, &g);
    if (g == (int)(h & 0xffffu)) seen = h;     // the word had reached the hinted step (else look again)
    return runs;
}

// Owner side: post step `op` over n items in chunks of `chunk` (from the
// task in cs.gt), run chunks with every warp of the CTA, wait for the rest.
// false: the kernel must stop.
__device__ __noinline__ bool gh_phase(const ElimArgs &a, CoopShared &cs, int op, int n, int chunk, unsigned char *slice,
                         int32_t &keep)
{
    const int tid = threadIdx.x;
    if (n <= 0) return true;
    if ((n + chunk - 1) / chunk > 0xffff) chunk = (n + 0xfffe) / 0xffff;
    const int nch = (n + chunk - 1) / chunk;
    const long long c0 = a.profile ? clock64() : 0;
    if (tid == 0) {
        const int gen = (int)((cs.gh_gen + 1u) & 0xffffu);
        cs.gh_gen = (uint32_t)gen;
        GhTask &t = *cs.gt;
        t.gen = gen; t.op = op; t.n = n; t.chunk = chunk; t.nch = nch;
        const int slot = gen & (GH_RING - 1);
        const uint4 *src = (const uint4 *)&t;
        uint4 *dst = (uint4 *)(a.gh_task + slot);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(GhTask) / 16); ++i) dst[i] = src[i];
        a.gh_done[32 * slot] = 0u;
        __threadfence();                                  // release: the step's inputs and descriptor
        atomicExch(a.gh_word, ((unsigned long long)gen << 48) | ((unsigned long long)nch << 32));
        // relaxed hints: a helper that sees one before the word counts the
        // step as seen only once the word shows its generation
        for (int h = 0; h < GH_HINTS; ++h) *(volatile uint32_t *)(a.gh_hint + 32 * h) = (uint32_t)gen | 0x10000u;
    }
    __syncthreads();
    const int gen = (int)cs.gh_gen;
    const long long c1 = a.profile ? clock64() : 0;
    // the helpers take the chunks; the owner's warps claim only what is still
    // unclaimed GH_GRACE_NS after the post (so a step never depends on helpers)
    {
        const long long t0 = global_ns();
        for (;;) {
            unsigned long long cur = 0;
            if (lane_id() == 0) cur = *(volatile const unsigned long long *)a.gh_word;
            cur = __shfl_sync(FULL, cur, 0);
            if ((uint32_t)cur >= (uint32_t)nch || read_status(a.status) != ST_OK) break;
            if (global_ns() - t0 > GH_GRACE_NS) break;
            __nanosleep(100);
        }
    }
    const int runs = gh_claim_loop(a, cs.gt, gen, slice, keep);
    if (a.stats && lane_id() == 0 && runs > 0) atomicAdd(a.stats + 26, (unsigned long long)runs);
    const long long c2 = a.profile ? clock64() : 0;
    if (tid == 0) {
        const uint32_t *done = a.gh_done + 32 * (gen & (GH_RING - 1));
        long long spins = 0;
        while (ld_acquire_u32(done) < (uint32_t)nch) {
            ++spins;
            if ((spins & 63) == 0) {
                if (read_status(a.status) != ST_OK) break;
                if (spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); break; }
            }
            if (spins > 256) __nanosleep(32);
        }
        fence_acq_rel();                                  // acquire: the helpers' results
        if (a.profile && a.stats && op >= 1 && op <= 12) {
            unsigned long long *ps = a.stats + 32 + 4 * (op - 1);
            atomicAdd(ps + 0, (unsigned long long)(c1 - c0));
            atomicAdd(ps + 1, (unsigned long long)(c2 - c1));
            atomicAdd(ps + 2, (unsigned long long)(clock64() - c2));
            atomicAdd(ps + 3, 1ull);
        }
    }
    return !__syncthreads_or(read_status(a.status) != ST_OK);
}

// Splitters of a sample sort posted for helpers: SS evenly spaced entries of
// the n to be sorted, sorted in the CTA's shared tile, every stride-th one
// kept; zeroes the bucket counters.  The entries are read from v (SRC 0),
// from the column's sources before the gather (SRC 1: original entries, then
// fill by append index), or from the merged row buckets before compaction
// (SRC 2: entry i lies in the last bucket b with pd[b] <= i, at gbo[b] + i -
// pd[b] of the temporaries).  Returns B.
template <int KEY, int SRC>
__device__ __noinline__ int gh_splitters(const ElimArgs &a, const GhTask &t, View v, int n, View tile, int cap, int wcap,
                                         int slice_bytes, CoopShared &cs, int nrow = 0)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    int B = next_pow2((2 * n + wcap - 1) / wcap);
    if (B > cap / 4) B = cap / 4;
    if (B < 1) B = 1;
    int SS = 8 * B;
    if (SS < 256) SS = 256;
    if (SS > cap) SS = cap;
    const int lg = __ffs(SS) - 1;
    int *spd = (int *)tile.S, *sbo = (int *)tile.M;       // SRC 2: bucket offsets staged in unused tile arrays
    if (SRC == 2) {
        for (int b = tid; b < nrow; b += nt) { spd[b] = t.pd[b]; sbo[b] = t.gbo[b]; }
        __syncthreads();
    }
    for (int s2 = tid; s2 < SS; s2 += nt) {
        const int i = (int)(((long long)s2 * n) >> lg);
        if (SRC == 0) {
            tile.row[s2] = __ldcg(v.row + i);
            tile.w[s2] = __ldcg(v.w + i);
            if (KEY == 1) tile.mult[s2] = __ldcg(v.mult + i);
        } else if (SRC == 1) {
            const int g = t.norig + (int)t.cnt;
            int32_t r;
            double w;
            gh_src_entry(a, t.k, t.norig, g, t.o0, i, gh_fill_dir(a, t.k, t.norig, g, i), r, w);
            tile.row[s2] = r; tile.w[s2] = w;
            if (KEY == 1) tile.mult[s2] = 1;
        } else {
            int lo = 0, hi = nrow - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (spd[mid] <= i) lo = mid; else hi = mid - 1;
            }
            const int pos = sbo[lo] + (i - spd[lo]);
            const unsigned long long rm = __ldcg((const unsigned long long *)v.M + pos);
            tile.row[s2] = (int32_t)(uint32_t)rm;
            tile.w[s2] = __ldcg(v.S + pos);
            if (KEY == 1) tile.mult[s2] = (int32_t)(rm >> 32);
        }
    }
    __syncthreads();
    coop_sort<KEY>(tile, SS, tile, 0);
    const int stride = SS / B;
    for (int b = tid; b < B; b += nt) {
        t.spl_row[b] = tile.row[b * stride];
        t.spl_wb[b] = dbits(tile.w[b * stride]);
        t.cnt_b[b] = 0;
        t.cur_b[b] = 0;
    }
    if (tid == 0) {
        cs.gt->B = B;
        cs.gt->spl_shared = (KEY == 0 ? 4 * B : 12 * B) <= slice_bytes && B <= 2 * REG_BUCKET_MAX ? 1 : 0;
    }
    __syncthreads();
    return B;
}

// Bucket offsets from the counts (gbo[0..B]), the oversized buckets (gbig)
// listed in cs.nbig.
__device__ __noinline__ void gh_bucket_scan(const GhTask &t, int n, int B, int bmax, int *gbig, CoopShared &cs)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) cs.nbig = 0;
    __syncthreads();
    for (int b = tid; b < B; b += nt) {
        const int c = __ldcg(t.cnt_b + b);          // counted by other SMs: read through L2
        t.gbo[b] = c;
        if (c > bmax) gbig[atomicAdd(&cs.nbig, 1)] = b;
    }
    __syncthreads();
    block_excl_scan(t.gbo, B, t.gbo, cs);
    if (tid == 0) t.gbo[B] = n;
    __syncthreads();
}

// Cooperative elimination of a vertex offered to the grid (the CTA holds the
// board's lock).  Same results as coop_eliminate's global-memory path.
__device__ __noinline__ int32_t gh_eliminate(const ElimArgs &a, CoopShared &cs, unsigned char *bbuf, WarpState &ws,
                                             long long &tp)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    // the working set and its arrays in the CTA's scratch, laid out as by coop_eliminate
    const int32_t k = cs.k;
    const int64_t o0 = __ldg(a.lcp + k);
    const int32_t norig = (int32_t)(__ldg(a.lcp + k + 1) - o0);
    const uint32_t cnt = __ldcg(a.fcnt + k);
    const int P = next_pow2(norig + (int)cnt);
    const View v = make_view(a.scratch + cs.sbase, P);
    double *tiles = (double *)(a.scratch + cs.sbase + (size_t)P * ENTRY_BYTES);
    int *gbo = (int *)(((uintptr_t)(tiles + (P / 32 + 1)) + 15) & ~(uintptr_t)15);
    int *gbd = gbo + a.block_cap + 1;
    int *gbig = gbd + a.block_cap + 1;
    unsigned char *ghx = (unsigned char *)(((uintptr_t)(gbig + a.block_cap + 1) + 15) & ~(uintptr_t)15);
    const bool requester = warp == cs.req_warp;
    auto mark = [&](int phase) {
        if (!requester) return;
        prof_mark(a, ws, phase);
        if (a.trace_phase && lane == 0) {
            const long long t = clock64();
            a.trace_phase[8 * (size_t)k + (phase - 8)] = (int32_t)(t - tp);
            tp = t;
        }
    };
    const int cap = a.block_cap, wcap = cap / nw;
    const int slice_bytes = a.warp_cap * ENTRY_BYTES;
    unsigned char *slice = bbuf - (size_t)(nw - warp) * slice_bytes;
    const View tile = make_view(bbuf, cap);
    const int g = norig + (int)cnt;
    int32_t keep = requester ? -1 : -2;
    // extra scratch: tile maxima, splitters, bucket counters, compacted offsets
    const int ntile_cap = P / 32 + 1;
    GhTask *gtask = (GhTask *)ghx;
    unsigned long long *tmax = (unsigned long long *)(ghx + sizeof(GhTask));
    unsigned long long *spl_wb = tmax + ntile_cap;
    int32_t *spl_row = (int32_t *)(spl_wb + cap);
    int32_t *cnt_b = spl_row + cap, *cur_b = cnt_b + cap, *pd = cur_b + cap;
    unsigned long long *coarse = (unsigned long long *)(((uintptr_t)(pd + cap) + 15) & ~(uintptr_t)15);
    if (tid == 0) cs.gt = gtask;
    __syncthreads();
    if (tid == 0) {
        GhTask &t = *cs.gt;
        t.k = k; t.d = 0; t.cap = P; t.norig = norig; t.cnt = cnt; t.o0 = o0;
        t.bmax = wcap < REG_BUCKET_MAX ? wcap : REG_BUCKET_MAX;
        t.slice = slice_bytes; t.lk = 0; t.fpos = 0; t.Dk = 0.0; t.klocal = 0; t.sys = 0;
        t.vbase = (unsigned char *)v.w; t.tiles = tiles; t.tmax = tmax;
        t.gbo = gbo; t.gbd = gbd; t.pd = pd; t.cnt_b = cnt_b; t.cur_b = cur_b; t.spl_row = spl_row; t.spl_wb = spl_wb;
        t.coarse = coarse; t.nco = 0; t.cstride = 1;
        t.B = 0; t.spl_shared = 0;
    }
    if (tid == 0 && a.stats) atomicAdd(a.stats + 24, 1ull);
    __syncthreads();
    const int bmax = cs.gt->bmax;
    auto fail = [&]() -> int32_t {
        __syncthreads();
        if (tid == 0) { __threadfence(); atomicExch(a.gh_lock, 0); cs.k = -1; }
        return -2;
    };
    double *tS = v.S;
    unsigned long long *tM = (unsigned long long *)v.M;

    // ---------------------------------------------------------------- gather, with the row sort's counts
    // (its splitters sampled from the column's sources)
    const int wcap_gh = wcap < 128 ? wcap : 128;          // buckets of ~64 entries for the helpers' rank sorts
    int B = gh_splitters<0, 1>(a, *cs.gt, v, g, tile, cap, wcap_gh, slice_bytes, cs);
    if (!gh_phase(a, cs, GH_GATHER, P, 128, slice, keep)) return fail();
    mark(9);

    // ---------------------------------------------------------------- rows: sort, merge, compact, store
    gh_bucket_scan(*cs.gt, g, B, bmax, gbig, cs);
    if (!gh_phase(a, cs, GH_SCATTER0, g, 128, slice, keep)) return fail();
    for (int q = 0; q < cs.nbig; ++q) {                     // oversized buckets: the whole CTA
        const int b = gbig[q];
        const int o = gbo[b], cb = gbo[b + 1] - o;
        const View w = sort_big_bucket<0>(v, tile, cap, o, cb);
        if (warp == 0) {
            const int db = warp_merge_bucket(w, cb, tS, tM, o);
            if (lane == 0) gbd[b] = db;
        }
        __syncthreads();
    }
    if (!gh_phase(a, cs, GH_ROWB, B, 1, slice, keep)) return fail();
    for (int b = tid; b < B; b += nt) pd[b] = __ldcg(gbd + b);
    __syncthreads();
    const int d = block_excl_scan(pd, B, pd, cs);
    if (tid == 0) {
        const unsigned long long base = d > 0 ? atomicAdd(a.f_top, (unsigned long long)d) : 0ull;
        if (d > 0 && base + d > a.f_cap) set_status(a.status, ST_POOL);
        cs.gt->fpos = base; cs.gt->d = d;
    }
    if (__syncthreads_or(read_status(a.status) != ST_OK)) return fail();
    if (tid == 0) { a.f_start[k] = (int64_t)cs.gt->fpos; a.f_len[k] = d; }
    if (d == 0) {
        mark(10); mark(11);
        if (tid == 0) a.D[k] = 0.0;
        __syncthreads();
        if (tid == 0) { __threadfence(); atomicExch(a.gh_lock, 0); cs.k = -1; }
        return -1;
    }
    const bool small_d = d <= (cap < 1024 ? cap : 1024);
    const int Brow = B;
    if (small_d) {                                         // compaction alone
        if (tid == 0) cs.gt->B = 0;
        __syncthreads();
    } else {                                               // the weight sort's splitters, sampled from the row buckets
        B = gh_splitters<1, 2>(a, *cs.gt, v, d, tile, cap, wcap_gh, slice_bytes, cs, Brow);
    }
    if (!gh_phase(a, cs, GH_COMPACT, Brow, 1, slice, keep)) return fail();
    mark(10); mark(11);

    // ---------------------------------------------------------------- weights
    if (small_d) {                                         // one shared tile
        const int Pd = next_pow2(d);
        for (int i = tid; i < Pd; i += nt) {
            if (i < d) { tile.row[i] = __ldcg(v.row + i); tile.w[i] = __ldcg(v.w + i); tile.mult[i] = __ldcg(v.mult + i); }
            else { tile.row[i] = ROW_SENTINEL; tile.w[i] = __longlong_as_double((long long)WBITS_SENTINEL); tile.mult[i] = 0; }
        }
        __syncthreads();
        coop_sort<1>(tile, Pd, tile, 0);
        for (int i = tid; i < d; i += nt) { v.row[i] = tile.row[i]; v.w[i] = tile.w[i]; v.mult[i] = tile.mult[i]; }
        __syncthreads();
    } else {
        gh_bucket_scan(*cs.gt, d, B, bmax, gbig, cs);
        if (!gh_phase(a, cs, GH_SCATTER1, d, 128, slice, keep)) return fail();
        for (int q = 0; q < cs.nbig; ++q) {
            const int b = gbig[q];
            const int o = gbo[b], cb = gbo[b + 1] - o;
            const View w = sort_big_bucket<1>(v, tile, cap, o, cb);
            for (int i = tid; i < cb; i += nt) {
                tS[o + i] = w.w[i];
                tM[o + i] = (unsigned long long)(uint32_t)w.row[i] | ((unsigned long long)(uint32_t)w.mult[i] << 32);
            }
            __syncthreads();
        }
        if (!gh_phase(a, cs, GH_WB, B, 1, slice, keep)) return fail();
    }
    mark(12);

    // ---------------------------------------------------------------- canonical suffix scan, running maximum
    const int ntile = (d + 31) / 32;
    if (!gh_phase(a, cs, GH_TILES, ntile, 4, slice, keep)) return fail();
    if (tid == 0) {            // serial carry chain over the tile totals
        double carry = 0.0;
        for (int j0 = 0; j0 < ntile; j0 += 8) {
            double tot[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) tot[q] = j0 + q < ntile ? __ldcg(tiles + j0 + q) : 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < ntile) { tiles[j0 + q] = carry; carry = __dadd_rn(tot[q], carry); }
        }
    }
    __syncthreads();
    if (!gh_phase(a, cs, GH_CARRYMAX, ntile, 4, slice, keep)) return fail();
    if (tid == 0) {            // running maximum over the tiles before each tile
        unsigned long long run = 0ull;
        for (int j0 = 0; j0 < ntile; j0 += 8) {
            unsigned long long tm[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) tm[q] = j0 + q < ntile ? __ldcg(tmax + j0 + q) : 0ull;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < ntile) { tmax[j0 + q] = run; if (tm[q] > run) run = tm[q]; }
        }
        const double Dk = __ldcg(v.S);
        a.D[k] = Dk;
        cs.gt->Dk = Dk;
        cs.gt->lk = __ldcg(a.lvl + k) + 1;
        uint64_t klocal, sys;
        sys_of(a, k, klocal, sys);
        cs.gt->klocal = klocal; cs.gt->sys = sys;
        const int cst = (d + GH_COARSE - 1) / GH_COARSE;
        cs.gt->cstride = cst; cs.gt->nco = (d + cst - 1) / cst;
    }
    __syncthreads();
    {                          // coarse copy of M_final for the sampling searches
        const int cst = cs.gt->cstride, nco = cs.gt->nco;
        for (int c = tid; c < nco; c += nt) {
            const int j = c * cst;
            const unsigned long long m = dbits(__ldcg(v.M + j)), tm = tmax[(d - 1 - j) >> 5];
            coarse[c] = m > tm ? m : tm;
        }
    }
    __syncthreads();
    mark(13);

    // ---------------------------------------------------------------- sampling, fill, levels
    if (!gh_phase(a, cs, GH_SAMPLE, d, 32, slice, keep)) return fail();
    if (tid == 0) ws.n_fill += (unsigned long long)(d - 1) * (unsigned long long)a.samples;
    mark(14);

    // ---------------------------------------------------------------- decrements (every append is done and released)
    if (!gh_phase(a, cs, GH_DECR, d, 64, slice, keep)) return fail();
    __syncthreads();
    if (tid == 0) { __threadfence(); atomicExch(a.gh_lock, 0); cs.k = -1; }
    mark(15);
    return requester ? (keep >= 0 ? keep : -1) : -1;
}

// Cooperative elimination of cs.k by every warp of the CTA (the callers have
// all reached this function).  __syncthreads() is used only after the bounded
// join barrier has seen every warp arrive.  Returns, for the requesting warp,
// the vertex it keeps (-1: none); -2 if the kernel must stop.
__device__ __noinline__ int32_t coop_eliminate(const ElimArgs &a, CoopShared &cs, unsigned char *bbuf,
                                               WarpState &ws)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    long long tp = 0;
    if (a.trace_phase) tp = clock64();
    if (!cta_barrier(cs, a)) return -2;                  // join: every warp is here
    __syncthreads();
    const int32_t k = cs.k;
    const bool requester = warp == cs.req_warp;
    // phase accounting of the requesting warp (profile counters, per-vertex trace)
    auto mark = [&](int phase) {
        if (!requester) return;
        prof_mark(a, ws, phase);
        if (a.trace_phase && lane == 0) {
            const long long t = clock64();
            a.trace_phase[8 * (size_t)k + (phase - 8)] = (int32_t)(t - tp);
            tp = t;
        }
    };
    mark(8);
    const int64_t o0 = __ldg(a.lcp + k), o1 = __ldg(a.lcp + k + 1);
    const int32_t norig = (int32_t)(o1 - o0);
    const uint32_t cnt = __ldcg(a.fcnt + k);
    const int g = norig + (int)cnt;
    const int P = next_pow2(g);

    // ---------------------------------------------------------------- working set
    View v;
    double *tiles;
    if (P <= a.block_cap) {
        v = make_view(bbuf, a.block_cap);
        tiles = (double *)(bbuf + (size_t)a.block_cap * ENTRY_BYTES);
    } else {
        const unsigned long long need = coop_scratch_bytes(P, a.block_cap, false);
        if (tid == 0 && cs.scap < need) {
            const unsigned long long base = atomicAdd(a.scratch_top, (need + 255ull) & ~255ull);
            if (base + need > a.scratch_cap) set_status(a.status, ST_POOL);
            cs.sbase = base; cs.scap = need;
        }
        if (__syncthreads_or(read_status(a.status) != ST_OK)) { __syncthreads(); if (tid == 0) cs.k = -1; return -2; }
        v = make_view(a.scratch + cs.sbase, P);
        tiles = (double *)(a.scratch + cs.sbase + (size_t)P * ENTRY_BYTES);
    }
    // bucket offsets and merged counts of the sample sort (global working sets)
    int *gbo = (int *)(((uintptr_t)(tiles + (P / 32 + 1)) + 15) & ~(uintptr_t)15);
    int *gbd = gbo + a.block_cap + 1;
    int *gbig = gbd + a.block_cap + 1;


    // ---------------------------------------------------------------- gather
    for (int i = tid; i < norig; i += nt) { v.row[i] = __ldg(a.lrow + o0 + i); v.w[i] = __ldg(a.lw + o0 + i); }
    if (a.hash_store) {
        // fill from W: the CTA scans k's probe sequence, nt slots a round
        const unsigned long long base = w_base(k, a.wcap), stride = w_stride(k, a.wcap);
        uint32_t found = 0;
        unsigned long long off = 0;
        while (found < cnt) {
            if (off >= a.wcap) { if (tid == 0) set_status(a.status, ST_INVAL); break; }
            const unsigned long long i = w_slot(base, stride, off + tid, a.wcap);
            const bool mine = off + tid < a.wcap && ld_acquire(a.wcol + i) == k;
            const unsigned bal = __ballot_sync(FULL, mine);
            if (lane == 0) cs.hcount[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w2 = 0; w2 < nw; ++w2) { const int c2 = cs.hcount[w2]; if (w2 < warp) before += c2; total += c2; }
            if (mine) {
                const uint32_t pos = found + before + __popc(bal & ((1u << lane) - 1u));
                v.row[norig + pos] = a.wrow[i];
                v.w[norig + pos] = a.ww[i];
                st_release(a.wcol + i, W_FREE);          // after the entry was read
            }
            found += (uint32_t)total;
            off += (unsigned long long)nt;
            __syncthreads();
        }
    } else {
        const int ninl = cnt < (uint32_t)FILL_C0 ? (int)cnt : FILL_C0;
        for (int i = tid; i < ninl; i += nt) {
            v.row[norig + i] = __ldcg(a.in_row + (size_t)k * FILL_C0 + i);
            v.w[norig + i] = __ldcg(a.in_w + (size_t)k * FILL_C0 + i);
        }
        uint32_t gl[FILL_LEVELS];               // directory entries of the used levels, loaded together
#pragma unroll
        for (int j = 1; j <= FILL_LEVELS; ++j)
            gl[j - 1] = cnt > fill_level_start(j) ? __ldcg(a.dir + (size_t)k * FILL_LEVELS + (j - 1)) : 0u;
        for (int j = 1; j <= FILL_LEVELS; ++j) {
            const uint32_t start = fill_level_start(j);
            if (cnt <= start) break;
            const uint32_t capj = fill_level_cap(j);
            const uint32_t len = (cnt - start) < capj ? (cnt - start) : capj;
            const uint32_t gidx = gl[j - 1];
            if (gidx == 0u || gidx == 0xffffffffu) {          // never published
                if (tid == 0) set_status(a.status, ST_INVAL);
                break;
            }
            const unsigned long long pb = (unsigned long long)(gidx - 1u) * FILL_GRANULE;
            for (uint32_t i = tid; i < len; i += nt) {
                v.row[norig + start + i] = __ldcg(a.pool_row + pb + i);
                v.w[norig + start + i] = __ldcg(a.pool_w + pb + i);
            }
        }
    }
    for (int i = g + tid; i < P; i += nt) { v.row[i] = ROW_SENTINEL; v.w[i] = 0.0; }
    if (__syncthreads_or(read_status(a.status) != ST_OK)) { __syncthreads(); if (tid == 0) cs.k = -1; return -2; }
    mark(9);

    // ---------------------------------------------------------------- sort + merge
    const bool global_ws = P > a.block_cap;
    const View tile = make_view(bbuf, a.block_cap);
    int d = -1;
    const bool sample = global_ws && a.sample_sort && a.block_cap >= 256;
    if (sample) {
        d = coop_row_phase(a, cs, v, g, bbuf, a.block_cap, gbo, gbd, gbig, k);
        if (d == -2) { __syncthreads(); if (tid == 0) cs.k = -1; return -2; }
        mark(10); mark(11);
    }
    if (d < 0) {                                   // bitonic network, merge in place, store
        coop_sort<0>(v, P, tile, global_ws ? a.block_cap : 0);
        mark(10);
        d = 0;
        for (int base = 0; base < g; base += nt) {
            const int i = base + tid;
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
            if (lane == 0) cs.hcount[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w2 = 0; w2 < nw; ++w2) { const int c = cs.hcount[w2]; if (w2 < warp) before += c; total += c; }
            const int rank = d + before + __popc(bal & ((1u << lane) - 1u));
            __syncthreads();                                   // every read of this chunk is done
            if (head) { v.row[rank] = r; v.w[rank] = sum; v.mult[rank] = len; }
            d += total;
            __syncthreads();
        }
        // store the row-ordered column
        if (tid == 0) {
            const unsigned long long base = d > 0 ? atomicAdd(a.f_top, (unsigned long long)d) : 0ull;
            if (d > 0 && base + d > a.f_cap) set_status(a.status, ST_POOL);
            cs.fpos = base;
        }
        if (__syncthreads_or(read_status(a.status) != ST_OK)) { __syncthreads(); if (tid == 0) cs.k = -1; return -2; }
        const unsigned long long fpos = cs.fpos;
        for (int i = tid; i < d; i += nt) { a.f_row[fpos + i] = v.row[i]; a.f_val[fpos + i] = v.w[i]; }
        if (tid == 0) { a.f_start[k] = (int64_t)fpos; a.f_len[k] = d; }
        mark(11);
    }
    if (d == 0) {
        if (tid == 0) a.D[k] = 0.0;
        __syncthreads();
        if (tid == 0) cs.k = -1;
        return -1;
    }

    // ---------------------------------------------------------------- weight sort
    __syncthreads();
    if (sample) {
        coop_weight_phase(v, d, bbuf, a.block_cap, cs, gbo, gbig);
    } else {
        const int P2 = next_pow2(d);
        for (int i = d + tid; i < P2; i += nt) {
            v.row[i] = ROW_SENTINEL; v.w[i] = __longlong_as_double((long long)WBITS_SENTINEL); v.mult[i] = 0;
        }
        __syncthreads();
        coop_sort<1>(v, P2, tile, global_ws ? a.block_cap : 0);
    }
    mark(12);

    // ---------------------------------------------------------------- canonical suffix scan
    // each 32-lane tile of the reversed weights: Hillis-Steele within the tile
    // (all warps in parallel), then the serial carry chain over tiles, then
    // every lane adds its tile's carry -- the pairings of the canonical scan
    const int ntile = (d + 31) / 32;
    for (int j = warp; j < ntile; j += nw) {
        const int t = 32 * j + lane;
        double x = (t < d) ? v.w[d - 1 - t] : 0.0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x = __dadd_rn(x, y);
        }
        if (t < d) v.S[d - 1 - t] = x;
        if (lane == 31) tiles[j] = x;
    }
    __syncthreads();
    if (tid == 0) {            // serial carry chain; the tile totals are loaded 8 at a time
        double carry = 0.0;
        for (int j0 = 0; j0 < ntile; j0 += 8) {
            double tot[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) tot[q] = j0 + q < ntile ? tiles[j0 + q] : 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < ntile) { tiles[j0 + q] = carry; carry = __dadd_rn(tot[q], carry); }
        }
    }
    __syncthreads();
    for (int t = tid; t < d; t += nt) v.S[d - 1 - t] = __dadd_rn(v.S[d - 1 - t], tiles[t >> 5]);
    __syncthreads();
    // running maximum from the right, on bit patterns (exact in any order)
    for (int j = warp; j < ntile; j += nw) {
        const int t = 32 * j + lane;
        unsigned long long m = t < d ? dbits(v.S[d - 1 - t]) : 0ull;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, m, off);
            if (lane >= off && y > m) m = y;
        }
        if (t < d) v.M[d - 1 - t] = __longlong_as_double((long long)m);
        if (lane == 31) tiles[j] = __longlong_as_double((long long)m);
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0ull;
        for (int j0 = 0; j0 < ntile; j0 += 8) {
            unsigned long long tm[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) tm[q] = j0 + q < ntile ? dbits(tiles[j0 + q]) : 0ull;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < ntile) { tiles[j0 + q] = __longlong_as_double((long long)run); if (tm[q] > run) run = tm[q]; }
        }
    }
    __syncthreads();
    for (int t = tid; t < d; t += nt) {
        const unsigned long long c = dbits(tiles[t >> 5]), m = dbits(v.M[d - 1 - t]);
        if (c > m) v.M[d - 1 - t] = __longlong_as_double((long long)c);
    }
    __syncthreads();
    const double Dk = v.S[0];
    if (tid == 0) a.D[k] = Dk;
    mark(13);

    // ---------------------------------------------------------------- sample clique tree + append
    // For a working set in global memory, a coarse copy of M (every
    // stride-th value) in shared memory narrows each search to one stride of
    // global values.  M is non-increasing and M[p] >= R, so the largest j
    // with M[j] >= R over the whole list is the one searched for in [p, d).
    int stride = 1, ncoarse = 0;
    unsigned long long *coarse = (unsigned long long *)tile.w;
    if (global_ws) {
        stride = (d + a.block_cap - 1) / a.block_cap;
        ncoarse = (d + stride - 1) / stride;
        for (int c = tid; c < ncoarse; c += nt) coarse[c] = dbits(v.M[c * stride]);
        __syncthreads();
    }
    uint64_t klocal, sys;
    sys_of(a, k, klocal, sys);
    bool ok = true;
    for (int q = 0; q < a.samples && ok; ++q)             // sample q of every slot (q > 0: MS(k))
    for (int pb = 1; pb < d; pb += nt) {
        const int p = pb + tid;
        const bool act = p < d;
        int32_t lo = 0, hi = 0;
        double c = 0.0;
        if (act) {
            const int32_t u = v.row[p - 1];
            const double wu = v.w[p - 1];
            const double Sp = v.S[p];
            const unsigned long long Rb = dbits(__dmul_rn(Sp, slot_uniform(a.seed, klocal, (uint64_t)p, sys,
                                                                           (uint64_t)q)));
            int lo_j = p, hi_j = d - 1;
            if (global_ws) {                       // largest coarse index c with M[c * stride] >= R
                int clo = 0, chi = ncoarse - 1;
                while (clo < chi) {
                    const int mid = clo + ((chi - clo + 1) >> 1);
                    if (coarse[mid] >= Rb) clo = mid; else chi = mid - 1;
                }
                const int jl = clo * stride, jh = (clo + 1) * stride - 1 < d - 1 ? (clo + 1) * stride - 1 : d - 1;
                lo_j = jl > p ? jl : p;
                hi_j = jh;
            }
            while (lo_j < hi_j) {
                const int mid = lo_j + ((hi_j - lo_j + 1) >> 1);
                if (dbits(v.M[mid]) >= Rb) lo_j = mid; else hi_j = mid - 1;
            }
            const int32_t x = v.row[lo_j];
            c = __ddiv_rn(__dmul_rn(Sp, wu), Dk);
            if (a.samples > 1) c = __ddiv_rn(c, (double)a.samples);
            lo = u < x ? u : x;
            hi = u < x ? x : u;
        }
        if (!append_fill(a, act, lo, hi, c)) { ok = false; break; }
    }
    if (tid == 0) ws.n_fill += (unsigned long long)(d - 1) * (unsigned long long)a.samples;
    mark(14);

    // ---------------------------------------------------------------- levels, release, decrements
    {
        const int32_t lk = __ldcg(a.lvl + k) + 1;
        for (int i = tid; i < d; i += nt) red_max_relaxed(a.lvl + v.row[i], lk);
    }
    __threadfence();
    if (!cta_barrier(cs, a)) ok = false;                  // every append is done and fenced
    if (__syncthreads_or(!ok)) { __syncthreads(); if (tid == 0) cs.k = -1; return -2; }
    __threadfence();
    int32_t keep = requester ? -1 : -2;
    for (int ib = 0; ib < d; ib += nt) {
        const int i = ib + tid;
        const bool valid = i < d;
        decrement_group(a, k, valid, valid ? v.row[i] : 0, valid ? v.mult[i] : 0, keep);
    }
    __syncthreads();
    if (tid == 0) cs.k = -1;
    mark(15);
    return requester ? (keep >= 0 ? keep : -1) : -1;
}

// A cooperative request flagged for grid help: join as coop_eliminate does,
// take the board (else eliminate the vertex in the CTA alone), set up the
// larger working set and run gh_eliminate.
__device__ __noinline__ int32_t gh_entry(const ElimArgs &a, CoopShared &cs, unsigned char *bbuf, WarpState &ws)
{
    const int tid = threadIdx.x;
    long long tp = 0;
    if (a.trace_phase) tp = clock64();
    if (!cta_barrier(cs, a)) return -2;
    __syncthreads();
    if (tid == 0) {
        cs.gh = atomicCAS(a.gh_lock, 0, 1) == 0 ? 1 : 0;
        if (cs.gh) { fence_acq_rel(); cs.gh_gen = (uint32_t)(__ldcg(a.gh_word) >> 48); }
    }
    __syncthreads();
    if (!cs.gh) return coop_eliminate(a, cs, bbuf, ws);     // every warp; it joins again
    const int32_t k = cs.k;
    const int warp = tid >> 5, lane = tid & 31;
    if (warp == cs.req_warp) {
        prof_mark(a, ws, 8);
        if (a.trace_phase && lane == 0) {
            const long long t = clock64();
            a.trace_phase[8 * (size_t)k] = (int32_t)(t - tp);
            tp = t;
        }
    }
    const int P = next_pow2((int)(__ldg(a.lcp + k + 1) - __ldg(a.lcp + k)) + (int)__ldcg(a.fcnt + k));
    const unsigned long long need = coop_scratch_bytes(P, a.block_cap, true);
    if (tid == 0 && cs.scap < need) {
        const unsigned long long base = atomicAdd(a.scratch_top, (need + 255ull) & ~255ull);
        if (base + need > a.scratch_cap) set_status(a.status, ST_POOL);
        cs.sbase = base; cs.scap = need;
    }
    if (__syncthreads_or(read_status(a.status) != ST_OK)) {
        __syncthreads();
        if (tid == 0) { __threadfence(); atomicExch(a.gh_lock, 0); cs.k = -1; }
        return -2;
    }
    return gh_eliminate(a, cs, bbuf, ws, tp);
}

// Dispatch of a joined cooperative request.
__device__ __forceinline__ int32_t coop_dispatch(const ElimArgs &a, CoopShared &cs, unsigned char *bbuf, WarpState &ws)
{
    return vol(cs.gh_req) ? gh_entry(a, cs, bbuf, ws) : coop_eliminate(a, cs, bbuf, ws);
}

// Join a pending cooperative request of this CTA, if there is one this warp
// has not served yet.  Returns -3 if there was none, else coop_eliminate's
// result for a helper (-1, or -2 on abort).
template <bool GH>
__device__ __forceinline__ int32_t serve_help(const ElimArgs &a, CoopShared &cs, int &seen_gen, unsigned char *bbuf,
                                              WarpState &ws)
{
    const int g = vol(cs.gen);
    if (g == seen_gen) return -3;
    seen_gen = g;
    ++ws.n_block;
    return GH ? coop_dispatch(a, cs, bbuf, ws) : coop_eliminate(a, cs, bbuf, ws);
}

// GH: the instantiation with grid help (idle warps serve the board, large
// working sets are offered to it); the other one has none of that code.
template <bool GH>
__global__ void __launch_bounds__(256, 2) elim_kernel(ElimArgs a, int fchunk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int block_lock;
    __shared__ CoopShared cs;
    __shared__ uint32_t gh_seen[8];        // grid help: last posting hint each warp has served
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned lane = lane_id();
    if (threadIdx.x < 8) gh_seen[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        block_lock = 0;
        cs.k = -1; cs.gen = 0; cs.req_warp = -1; cs.arrive = 0; cs.sbase = 0; cs.scap = 0;
    }
    __syncthreads();

    unsigned char *wbuf = smem + (size_t)warp * a.warp_cap * ENTRY_BYTES;
    unsigned char *bbuf = smem + (size_t)nw * a.warp_cap * ENTRY_BYTES;

    WarpState ws;
    ws.fcur = ws.fend = 0; ws.sbase = 0; ws.scap = 0;
    ws.n_reg = ws.n_warp = ws.n_block = ws.n_global = ws.n_fill = ws.n_handoff = 0;
    for (int i = 0; i < 16; ++i) ws.cyc[i] = 0;
    ws.t_mark = 0;
    ws.fchunk = fchunk;
    prof_mark(a, ws, -1);
    unsigned long long spins_total = 0;
    int seen_gen = 0;

    const uint32_t nl = (uint32_t)a.nl;
    uint32_t slot = 0, slot_end = 0;       // claimed, not yet consumed queue slots
    bool claims_done = false;              // every queue slot has been claimed
    int32_t next = -1;                     // vertex handed to this warp by its last pivot
    for (;;) {
        if (a.coop) {
            const int32_t h = serve_help<GH>(a, cs, seen_gen, bbuf, ws);
            if (h == -2) break;
        }
        int32_t k;
        if (next >= 0) {
            k = next;
            next = -1;
            ++ws.n_handoff;
            fence_acq_rel();               // acquire: the counter transition precedes the column reads
        } else {
            if (slot == slot_end && !claims_done) {
                uint32_t s = 0;
                if (lane == 0) s = atomicAdd(a.q_head, (uint32_t)a.queue_chunk);
                s = __shfl_sync(FULL, s, 0);
                if (s >= nl) claims_done = true;
                else {
                    slot = s;
                    slot_end = (s + (uint32_t)a.queue_chunk) < nl ? s + (uint32_t)a.queue_chunk : nl;
                }
            }
            long long spins = 0;
            uint32_t seen_tail = 0, seen_done = 0;
            bool stop = false;
            // Wait for the claimed slot (or, once every slot is claimed, for
            // the end), serving cooperative requests of this CTA meanwhile.
            // The watchdog counts polls without global progress.  Slots past
            // the last publication stay empty (vertices handed over directly
            // never enter the queue): the wait ends when every vertex has
            // been eliminated.
            k = -1;
            // grid help: one warp in gh_mask + 1 reads the posting hint, in
            // the same round trip as its queue slot
            const int gwarp = (int)blockIdx.x * nw + warp;
            const bool gh_on = GH && a.grid_help > 0 && (gwarp & a.gh_mask) == 0;
            for (;;) {
                uint32_t hint = 0u;
                if (!claims_done) k = *(volatile const int32_t *)(a.queue + slot);
                if (gh_on && lane == 0) hint = *(volatile const uint32_t *)(a.gh_hint + 32 * (gwarp & (GH_HINTS - 1)));
                if (!claims_done) {
                    if (__shfl_sync(FULL, k, 0) >= 0) { k = __shfl_sync(FULL, k, 0); break; }
                }
                if (a.coop) {
                    const int32_t h = serve_help<GH>(a, cs, seen_gen, bbuf, ws);
                    if (h == -2) { stop = true; break; }
                    if (h != -3) spins = 0;
                }
                if (GH && gh_on && gh_serve(a, wbuf, gh_seen[warp], __shfl_sync(FULL, hint, 0)) > 0) spins = 0;
                if ((++spins & 63) == 0) {
                    if (read_status(a.status) != ST_OK) { stop = true; break; }
                    const uint32_t t = *(volatile const uint32_t *)a.q_tail;
                    const uint32_t dn = *(volatile const uint32_t *)a.done;
                    if (dn >= nl) { stop = true; break; }
                    if (t != seen_tail || dn != seen_done) {
                        seen_tail = t; seen_done = dn; spins_total += (unsigned long long)spins; spins = 0;
                    }
                }
                if (spins > a.spin_limit) { set_status(a.status, ST_TIMEOUT); stop = true; break; }
                // idle workers back off so that their polls do not crowd the
                // memory pipeline of the warps doing eliminations
                if (spins > 4) __nanosleep(spins < 64 ? 64u : (unsigned)a.idle_ns);
            }
            spins_total += (unsigned long long)spins;
            if (__any_sync(FULL, stop)) break;
            fence_acq_rel();               // acquire once the slot is seen (the polls are relaxed)
            ++slot;
        }
        prof_mark(a, ws, 0);
        const long long t_start = a.trace ? global_ns() : 0;
        const int64_t o0 = __ldg(a.lcp + k), o1 = __ldg(a.lcp + k + 1);
        const int32_t norig = (int32_t)(o1 - o0);
        const uint32_t cnt = __ldcg(a.fcnt + k);
        const int g = norig + (int)cnt;
        int32_t r;
        if (g <= 32) {
            r = eliminate_small(a, k, o0, norig, cnt, ws);
        } else if (!a.coop || next_pow2(g) <= a.warp_cap) {
            r = eliminate_big(a, k, o0, norig, cnt, wbuf, bbuf, &block_lock, ws);
        } else {
            // post the request (or help the one already posted, then retry)
            r = -3;
            prof_mark(a, ws, 1);
            while (r == -3) {
                int posted = 0;
                if (lane == 0 && atomicCAS(&cs.k, -1, k) == -1) {
                    cs.req_warp = warp;
                    // grid help for working sets in global scratch (large enough)
                    cs.gh_req = GH && a.grid_help > 0 && g >= a.grid_help && next_pow2(g) > a.block_cap &&
                                a.sample_sort && a.block_cap >= 256 && !a.hash_store;
                    __threadfence_block();
                    posted = atomicAdd(&cs.gen, 1) + 1;
                }
                posted = __shfl_sync(FULL, posted, 0);
                if (posted) {
                    seen_gen = posted;
                    r = GH ? coop_dispatch(a, cs, bbuf, ws) : coop_eliminate(a, cs, bbuf, ws);
                    ++ws.n_global;
                } else {
                    const int32_t h = serve_help<GH>(a, cs, seen_gen, bbuf, ws);
                    if (h == -2) { r = -2; break; }
                    if (h == -3) __nanosleep(32);
                }
            }
        }
        if (r == -2) break;
        if (a.trace && lane == 0) {
            a.trace[4 * (size_t)k + 1] = t_start;
            a.trace[4 * (size_t)k + 2] = global_ns();
            a.trace[4 * (size_t)k + 3] = ((long long)g << 32) | (unsigned)a.f_len[k];
        }
        if (lane == 0) atomicAdd(a.done, 1u);
        // keep the handed-over vertex only while no claimed slot is pending
        if (r >= 0) {
            if (slot == slot_end) {
                next = r;
            } else {
                uint32_t qb = 0;
                if (lane == 0) {
                    qb = atomicAdd(a.q_tail, 1u);
                    if (qb < nl) { fence_acq_rel(); st_release(a.queue + qb, r); }
                    else set_status(a.status, ST_INVAL);
                }
                __syncwarp();
            }
        }
    }
    if (lane == 0 && a.stats) {
        atomicAdd(a.stats + 0, ws.n_warp + ws.n_reg);
        atomicAdd(a.stats + 1, ws.n_block);
        atomicAdd(a.stats + 2, ws.n_global);
        atomicAdd(a.stats + 3, ws.n_fill);
        atomicAdd(a.stats + 4, spins_total);
        atomicAdd(a.stats + 5, ws.n_reg);
        atomicAdd(a.stats + 6, ws.n_handoff);
        for (int i = 0; i < 16; ++i) atomicAdd(a.stats + 8 + i, ws.cyc[i]);
    }
}

}  // namespace

size_t elim_smem_bytes(int warps_per_block, int warp_cap, int block_cap)
{
    // per-warp buffers, then the CTA buffer and its scan-tile array
    return (size_t)(warps_per_block * warp_cap + block_cap) * ENTRY_BYTES + ((size_t)block_cap / 32 + 1) * 8;
}

cudaError_t elim_configure(int warps_per_block, int warp_cap, int block_cap, int *blocks_per_sm)
{
    const size_t smem = elim_smem_bytes(warps_per_block, warp_cap, block_cap);
    cudaError_t e = cudaFuncSetAttribute(elim_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(elim_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int b0 = 0, b1 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, elim_kernel<false>, warps_per_block * 32, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, elim_kernel<true>, warps_per_block * 32, smem);
    *blocks_per_sm = b0 < b1 ? b0 : b1;
    return e;
}

cudaError_t elim_launch(const ElimArgs &a, int blocks, int warps_per_block, int fchunk, cudaStream_t st)
{
    const size_t smem = elim_smem_bytes(warps_per_block, a.warp_cap, a.block_cap);
    if (a.grid_help > 0) elim_kernel<true><<<blocks, warps_per_block * 32, smem, st>>>(a, fchunk);
    else elim_kernel<false><<<blocks, warps_per_block * 32, smem, st>>>(a, fchunk);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace parac
