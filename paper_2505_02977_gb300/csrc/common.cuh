// common.cuh -- device primitives and shared structures of libparac (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace parac {

// ---------------------------------------------------------------- status words
// Device status word values (the first non-zero one written wins).
enum : int32_t {
    ST_OK = 0,
    ST_POOL = 1,       // fill / factor / scratch workspace overflow
    ST_TIMEOUT = 2,    // a bounded wait gave up
    ST_NOT_SDD = 3,    // positive off-diagonal / negative excess
    ST_INVAL = 4,      // malformed input (bad index, not a permutation, kind mismatch)
};

__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ int32_t read_status(const int32_t *status)
{
    return *(volatile const int32_t *)status;
}

// ---------------------------------------------------------------- memory ordering
__device__ __forceinline__ int32_t ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int32_t v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double ld_relaxed_f64(const double *p)
{
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_f64(double *p, double v)
{
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_i32(int32_t *p, int32_t v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float ld_relaxed_f32(const float *p)
{
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_f32(float *p, float v)
{
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void red_add_relaxed(int32_t *p, int32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_max_relaxed(int32_t *p, int32_t v)
{
    asm volatile("red.relaxed.gpu.global.max.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t) : : "memory");
    return t;
}

// ---------------------------------------------------------------- Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11), 4 words x 64 bits, 10
// rounds.  Round: two 64x64->128 products of words 0 and 2 with the round
// multipliers; the new words are (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2),
// hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)); the key advances by the Weyl constants
// between rounds.
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    U64x4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Uniform in (0, 1] for sample q of sampling slot p of pivot k (local label)
// of system sys (q > 0 only with several samples per slot, MS(k)): the top 53
// bits of the first output word, plus one, times 2^-53.
__device__ __forceinline__ double slot_uniform(uint64_t seed, uint64_t k, uint64_t p, uint64_t sys,
                                               uint64_t q = 0ull)
{
    const U64x4 o = philox4x64_10(k, p, sys, q, seed, 0ull);
    return (double)((o.v[0] >> 11) + 1ull) * 0x1.0p-53;
}

// ---------------------------------------------------------------- hashmap fill store
// Base slot of column c in W: a fixed bijective mix of the label (a
// pseudo-random permutation of 32-bit labels, independent of the elimination
// order) scaled to the table.
constexpr int32_t W_FREE = -1, W_BUSY = -2;

__host__ __device__ __forceinline__ unsigned long long w_base(int32_t c, unsigned long long wcap)
{
    uint32_t x = (uint32_t)c;
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return ((unsigned long long)x * wcap) >> 32;
}

// Probe stride of column c: odd, so that over the power-of-two table every
// column's probe sequence base, base + s, base + 2s, ... visits every slot.
// With one stride for all columns (plain linear probing) a hub column's
// hundreds of thousands of fill entries form one run of occupied slots, and
// any column whose base lands in it probes through the whole run; with a
// stride per column the columns' sequences cross only at single slots.
__host__ __device__ __forceinline__ unsigned long long w_stride(int32_t c, unsigned long long wcap)
{
    uint32_t x = (uint32_t)c * 0x9e3779b9u;
    x ^= x >> 15; x *= 0x2c1b3c6du;
    x ^= x >> 12;
    return (((unsigned long long)x * wcap) >> 32) | 1ull;
}

// Slot of step m of column c's probe sequence (wcap a power of two).
__host__ __device__ __forceinline__ unsigned long long w_slot(unsigned long long base, unsigned long long stride,
                                                             unsigned long long m, unsigned long long wcap)
{
    return (base + m * stride) & (wcap - 1);
}

// ---------------------------------------------------------------- fill store geometry
// Column c's fill entries: indices [0, C0) live in an inline slab of the
// column; index i >= C0 lives in overflow level j = 1 + floor(log4(i / C0)),
// covering [C0 4^(j-1), C0 4^j) (capacity 3 C0 4^(j-1)), allocated from the
// pool on first use.  The directory keeps one granule index per level.
constexpr int FILL_C0 = 16;
constexpr int FILL_LEVELS = 12;          // up to 16 * 4^12 = 2^28 entries per column
constexpr int FILL_GRANULE = 16;         // directory unit (entries)

__host__ __device__ __forceinline__ int fill_level(uint32_t i)
{
    // i >= FILL_C0
    const uint32_t q = i / FILL_C0;       // >= 1
#ifdef __CUDA_ARCH__
    const int lg = 31 - __clz(q);
#else
    const int lg = 31 - __builtin_clz(q);
#endif
    return lg / 2 + 1;
}

__host__ __device__ __forceinline__ uint32_t fill_level_start(int j) { return (uint32_t)FILL_C0 << (2 * (j - 1)); }
__host__ __device__ __forceinline__ uint32_t fill_level_cap(int j) { return 3u * ((uint32_t)FILL_C0 << (2 * (j - 1))); }

// ---------------------------------------------------------------- grid help
// One step of a large vertex's elimination posted for idle warps: the items
// [0, n) cut into nch chunks of `chunk`, claimed one at a time.
constexpr int GH_RING = 4;       // task descriptors / done counters in flight
constexpr int GH_HINTS = 16;     // copies of the posting hint (one 128-byte line each)
struct __align__(16) GhTask {
    int32_t gen, op, k, n;            // generation, step, vertex, items
    int32_t chunk, nch, B, d;         // items per chunk, chunks, buckets, merged entries
    int32_t cap, norig, bmax, lk;     // working-set capacity, original entries, helper bucket limit, level + 1
    uint32_t cnt;                     // fill entries of k
    int32_t spl_shared, slice, nco;   // splitters staged in the warp slice; slice bytes; coarse entries
    int64_t o0;                       // first original entry of k
    unsigned long long fpos;          // F column position
    double Dk;
    uint64_t klocal, sys;
    unsigned char *vbase;             // working set: make_view(vbase, cap)
    double *tiles;                    // suffix-scan tile totals, then carries
    unsigned long long *tmax;         // tile maxima of S, then their running maxima
    int32_t *gbo, *gbd, *pd;          // bucket offsets, merged counts, compacted offsets
    int32_t *cnt_b, *cur_b;           // bucket counts and scatter cursors
    int32_t *spl_row;                 // splitters b = 1 .. B-1
    unsigned long long *spl_wb;
    unsigned long long *coarse;       // running maximum at every cstride-th position (sampling)
    int32_t cstride, pad0, pad1, pad2;
};

// ---------------------------------------------------------------- elimination arguments
struct ElimArgs {
    int32_t nl;                    // labels (all systems, ground labels included)
    const int64_t *lcp;            // strict-lower CSC of the input [nl+1]
    const int32_t *lrow;
    const double *lw;
    const int32_t *sys_of;         // label -> system (nullptr: single system 0)
    const int32_t *sys_base;       // system -> first label
    uint64_t seed;

    int32_t *dp;                   // dependency counters [nl]
    int32_t *queue;                // ready queue [nl], -1 = empty slot
    uint32_t *q_head;              // claim counter
    uint32_t *q_tail;              // push counter
    uint32_t *done;                // vertices eliminated so far

    uint32_t *fcnt;                // fill entries appended per column [nl]
    int32_t *in_row;               // inline slabs [nl * FILL_C0]
    double *in_w;
    uint32_t *dir;                 // overflow directory [nl * FILL_LEVELS] (granule + 1, 0 = none)
    int32_t *pool_row;             // overflow pool
    double *pool_w;
    unsigned long long *pool_top;  // entries used
    unsigned long long pool_cap;

    int32_t *f_row;                // factor columns, as written by the pivots
    double *f_val;
    unsigned long long *f_top;
    unsigned long long f_cap;
    int64_t *f_start;              // [nl]
    int32_t *f_len;                // [nl]
    double *D;                     // [nl]
    int32_t *lvl;                  // [nl] dependency level (longest chain of pivots reaching the vertex)

    unsigned char *scratch;        // big-vertex scratch arena
    unsigned long long *scratch_top;
    unsigned long long scratch_cap;

    int32_t *status;
    long long spin_limit;
    unsigned long long *stats;     // [16] counters (see elim.cu)
    int32_t warp_cap;              // per-warp shared-memory entries (power of two)
    int32_t block_cap;             // per-CTA shared big-vertex buffer entries (power of two, 0 = none)
    int32_t queue_chunk;
    int32_t profile;               // nonzero: accumulate per-phase cycle counts into stats[8..15]
    int32_t idle_ns;               // sleep between polls of an idle worker (ns)
    int32_t coop;                  // nonzero: working sets above warp_cap use the CTA-cooperative path
    long long *trace;              // optional per-vertex trace [nl * 4]: ready, start, end (ns), g << 32 | d
    int32_t *trace_parent;         // optional: pivot whose decrement made the vertex ready
    int32_t *trace_phase;          // optional: cycles of the cooperative path's 8 phases [nl * 8]
    int32_t sample_sort;           // cooperative path: sample sort for working sets in global memory
    int32_t samples;               // samples per clique-tree slot (MS(k)); 1: Alg. 2
    // hashmap fill store (Sec. IV-C): slot state / column tag, entry row and weight
    int32_t hash_store;            // 1: fill goes to the hashmap W instead of slabs
    int32_t *wcol;                 // [wcap] -1 free, -2 busy, else the column the entry belongs to
    int32_t *wrow;
    double *ww;
    unsigned long long wcap;
    // grid help: idle warps take chunks of a large vertex's data-parallel steps
    int32_t grid_help;             // gathered entries from which a vertex is offered (0: never)
    int32_t gh_mask;               // warps with (grid index & gh_mask) == 0 serve as helpers
    unsigned long long *gh_word;   // generation << 48 | chunks << 32 | next chunk
    uint32_t *gh_hint;             // GH_HINTS copies, one per 128-byte line: generation | 1 << 16
    uint32_t *gh_done;             // GH_RING done counters, one per 128-byte line
    int32_t *gh_lock;              // 0 free, 1 held by the vertex being helped
    GhTask *gh_task;               // GH_RING task descriptors
};

// Bytes of shared/scratch memory per entry of the per-vertex working set:
// sort key row (4) + weight (8) + multiplicity (4) + suffix sum (8) + envelope (8).
constexpr int ENTRY_BYTES = 32;

}  // namespace parac
