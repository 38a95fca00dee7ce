// api.cu -- the C ABI of libparac (declared in include/parac.h): argument
// checks, host/device marshalling, workspace sizing and regrowth, and the
// orchestration of ingest -> persistent elimination -> compaction -> solve.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/parac.h"
#include "common.cuh"
#include "kernels.h"

using namespace parac;

namespace parac {
static unsigned long long g_launches = 0;
// launches recorded into a graph being captured by this thread are counted
// here instead, and added to the total at each replay
static thread_local unsigned long long *t_capture_count = nullptr;
void count_launches(unsigned n)
{
    if (t_capture_count) *t_capture_count += n;
    else __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED);
}
void count_graph_launches(unsigned long long n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }
void capture_launch_counts(unsigned long long *acc) { t_capture_count = acc; }
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
}  // namespace parac

namespace {

thread_local std::string g_err;

void set_err(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

struct CudaFail {
    cudaError_t e;
    const char *where;
};

#define CK(call)                                                                \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) throw CudaFail{e_, #call};                       \
    } while (0)

struct StatusFail {
    parac_status s;
};

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory the given device can use directly: memory allocated on it,
// or managed memory.
bool on_device(const void *p, int device)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

// Stream-ordered device buffer.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DBuf() = default;
    DBuf(size_t b, cudaStream_t s) { alloc(b, s); }
    void alloc(size_t b, cudaStream_t s)
    {
        release();
        st = s;
        bytes = b;
        if (b) {
            cudaError_t e = cudaMallocAsync(&p, b, s);
            if (e != cudaSuccess) { p = nullptr; cudaGetLastError(); throw StatusFail{PARAC_ENOMEM}; }
        }
    }
    void release()
    {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    ~DBuf() { release(); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), bytes(o.bytes), st(o.st) { o.p = nullptr; o.bytes = 0; }
    DBuf &operator=(DBuf &&o) noexcept
    {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; st = o.st; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    template <typename T> T *as() const { return (T *)p; }
};

template <typename T>
DBuf dalloc(size_t count, cudaStream_t s) { return DBuf(count * sizeof(T), s); }

// A device view of a caller array: the caller's pointer if it is device memory,
// else a stream-ordered copy.
template <typename T>
struct DView {
    const T *p = nullptr;
    DBuf own;
    void set(const T *src, size_t count, cudaStream_t s)
    {
        if (!src || count == 0) { p = src; return; }
        if (is_device_ptr(src)) { p = src; return; }
        own.alloc(count * sizeof(T), s);
        CK(cudaMemcpyAsync(own.p, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
        p = own.as<T>();
    }
};

void copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (!bytes) return;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

// Device memory size, queried once per device (a per-call cudaMemGetInfo
// would add a device-wide query to every factorisation).
unsigned long long device_memory_bytes()
{
    static std::atomic<unsigned long long> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    unsigned long long v = cache[dev].load();
    if (v == 0) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) v = (unsigned long long)p.totalGlobalMem;
        else cudaGetLastError();
        cache[dev].store(v);
    }
    return v;
}

int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

void set_mempool_keep()
{
    static bool done = false;
    if (done) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done = true;
}

int lanes_for(double avg)
{
    if (avg <= 6.0) return 4;
    if (avg <= 12.0) return 8;
    if (avg <= 24.0) return 16;
    return 32;
}

}  // namespace

// ------------------------------------------------------------------ handle
struct SolveCache {
    int32_t n = -1;
    DBuf x, r, z, p, q, b, y64, zl64, y32, zl32, partials, state;
    PcgBuffers B{};
};

// Buffers of the block (several right-hand sides) PCG: row-major n x nrhs.
struct BlockCache {
    int32_t n = -1, nrhs = 0, prec = 0, pstride = 0;
    DBuf x, r, z, p, q, b, y, zl, partials, state;
    DBuf gt_f, gt_b;                 // SpTRSM group tables (depend on the factor and the warps per block)
    int32_t ng_f = 0, ng_b = 0, g_warps = 0;
    DBuf part_f, part_b;             // partial sums of split rows, 32 columns per slot
    int32_t nslot_f = 0, nslot_b = 0;
    BlockBuffers B{};
};

// A captured CUDA graph of `check_every` PCG iterations, replayed until the
// run stops.  The key holds every pointer and scalar baked into the captured
// launches; any change re-captures.
struct GraphCache {
    static constexpr int KEY = 24;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;     // kernel launches in one replay
    uint64_t key[KEY] = {0};
    GraphCache() = default;
    GraphCache(const GraphCache &) = delete;
    GraphCache &operator=(const GraphCache &) = delete;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        launches = 0;
    }
    ~GraphCache() { reset(); }
};

// The solves run on a stream of the library's own (joined to the handle's
// stream by events), so that graph capture never touches a caller's or the
// legacy default stream.
struct SolveStream {
    cudaStream_t s = nullptr;
    cudaEvent_t in = nullptr, out = nullptr, h = nullptr;
    SolveStream() = default;
    SolveStream(const SolveStream &) = delete;
    SolveStream &operator=(const SolveStream &) = delete;
    ~SolveStream()
    {
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
        if (in) cudaEventDestroy(in);
        if (out) cudaEventDestroy(out);
        if (h) cudaEventDestroy(h);
    }
};

struct parac_factor_s {
    int device = 0;
    int64_t n = 0;
    int64_t nnzF = 0;
    int32_t prec = 64;
    long long spin_limit = 0;
    int32_t sptrsv = 0;
    int32_t check_every = 8;
    int32_t trsv_blocks = 0, poll_ns = 64;             // solve schedule (parac_opts)
    int32_t pcg_graph = 0, pcg_many = 0, pcg_workers = 4;
    bool host_tables = false;                          // solve group tables built on the host (reference builder)
    cudaStream_t stream = nullptr;
    DBuf perm, Fcp, Frow, Fval, D, Lp, Li, Lv;          // label space (export) and the matrix
    DBuf Lev;                                          // dependency level of each column
    // solve arrays: F relabelled into dependency-level order (positions)
    DBuf Scp, Srow, Sval, Sval32, Srp, Scol, Svalr, Svalr32, Sdinv, Sperm;
    int32_t depth = 0;
    std::vector<int64_t> lstart;                       // first position of each level (depth + 1)
    int64_t nnzL = 0;
    std::string stats;
    SolveCache cache;
    int32_t max_row = 0;                               // longest row / column of F
    DBuf tpr_chunks;                                   // table of the hybrid solves (int2), built lazily
    int32_t ntpr = 0;
    bool tpr_tried = false;
    DBuf sgt_f, sgt_b;                                 // group tables of the one-row-per-warp solves
    int32_t sng_f = 0, sng_b = 0;
    DBuf spart_f, spart_b;                             // partial sums of their split rows
    int32_t snslot_f = 0, snslot_b = 0;
    BlockCache bcache;
    DBuf status;
    SolveStream sstream;
    GraphCache graph;
};

namespace {

struct Opts {
    parac_opts o;
    cudaStream_t st;
};

Opts read_opts(const parac_opts *in)
{
    Opts r;
    parac_opts_default(&r.o);
    if (in) r.o = *in;
    if (r.o.pool_mult < 0) r.o.pool_mult = 0.0;        // 0: chosen from the input (run_factor)
    if (r.o.max_pool_regrow < 0) r.o.max_pool_regrow = 0;
    if (r.o.spin_limit <= 0) r.o.spin_limit = 1ll << 24;
    if (r.o.warps_per_block <= 0) r.o.warps_per_block = 8;
    if (r.o.warps_per_block > 8) r.o.warps_per_block = 8;     // the elimination kernel's launch bound
    if (r.o.queue_chunk <= 0) r.o.queue_chunk = 1;
    if (r.o.check_every <= 0) r.o.check_every = 8;
    if (r.o.g_precision != 32) r.o.g_precision = 64;
    if (r.o.samples <= 0) r.o.samples = 1;
    if (r.o.fill_store != 1) r.o.fill_store = 0;
    if (r.o.order != PARAC_ORDER_NNZ) r.o.order = PARAC_ORDER_GIVEN;
    if (r.o.idle_ns < 0) r.o.idle_ns = 0;
    if (r.o.grid_help_min < 0) r.o.grid_help_min = 0;
    if (r.o.host_tables != PARAC_ON) r.o.host_tables = PARAC_DEFAULT;
    if (r.o.trsv_blocks < 0) r.o.trsv_blocks = 0;
    r.o.poll_ns = r.o.poll_ns <= 0 ? 64 : std::max(16, std::min(100000, r.o.poll_ns));
    r.o.pcg_workers = r.o.pcg_workers <= 0 ? 4 : std::min(64, r.o.pcg_workers);
    r.st = (cudaStream_t)r.o.stream;
    return r;
}

// ---------------------------------------------------------------- factor job
struct SysDesc {
    int64_t n;
    int64_t obase, lbase;
    int32_t ground;   // label or -1
};

struct FactorOut {
    // output-space (N) arrays
    DBuf Fcp, Frow, Fval, D, Lev;
    int64_t nnzF = 0;
    int64_t nl = 0, nnz_low = 0;
    unsigned long long stats[160] = {0};
    unsigned long long pool_used = 0, f_used = 0, scratch_used = 0;
    int32_t max_lower_column = 0;
    int32_t samples = 1, fill_store = 0;
    int regrows = 0;
    double t_ingest = 0, t_elim = 0, t_compact = 0;
    int blocks = 0, warps = 0;
};

parac_status map_status(int32_t s)
{
    switch (s) {
    case ST_OK: return PARAC_OK;
    case ST_POOL: return PARAC_EPOOL;
    case ST_TIMEOUT: return PARAC_ETIMEOUT;
    case ST_NOT_SDD: return PARAC_ENOT_SDD;
    default: return PARAC_EINVAL;
    }
}

struct EvTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on;
    cudaStream_t st;
    EvTimer(bool on_, cudaStream_t s) : on(on_), st(s)
    {
        if (on) { cudaEventCreate(&a); cudaEventCreate(&b); cudaEventRecord(a, st); }
    }
    double stop()
    {
        if (!on) return 0.0;
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~EvTimer() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
};

// Factor a (possibly block-diagonal) system already on the device.
//   N, colptr/rowind/val: concatenated input (global row indices)
//   ord_global / label_of_k: position q -> original vertex / label (nullptr: identity)
//   systems: per-system ranges (size 1 for a single matrix)
void run_factor(int64_t N, const int64_t *colptr, const int32_t *rowind, const double *val,
                const int32_t *ord_global, const int32_t *label_of_k, const std::vector<SysDesc> &systems,
                int32_t kind, uint64_t seed, const Opts &O, FactorOut &out)
{
    cudaStream_t st = O.st;
    const int S = (int)systems.size();
    const bool batch = S > 1;
    int64_t nl = 0;
    for (auto &s : systems) nl = std::max<int64_t>(nl, s.lbase + s.n + (s.ground >= 0 ? 1 : 0));
    out.nl = nl;
    if (nl >= 0x7fffffffLL) throw StatusFail{PARAC_EINVAL};

    EvTimer t_in(O.o.timing != 0, st);
    // per-system device descriptors (batch only)
    DBuf d_sys_of_orig, d_sys_obase, d_sys_n, d_sys_ground, d_sys_lbase, d_sys_of_label;
    if (batch) {
        std::vector<int32_t> obase(S), nn(S), gr(S), lb(S);
        for (int s = 0; s < S; ++s) {
            obase[s] = (int32_t)systems[s].obase; nn[s] = (int32_t)systems[s].n;
            gr[s] = systems[s].ground; lb[s] = (int32_t)systems[s].lbase;
        }
        d_sys_obase = dalloc<int32_t>(S, st); d_sys_n = dalloc<int32_t>(S, st);
        d_sys_ground = dalloc<int32_t>(S, st); d_sys_lbase = dalloc<int32_t>(S, st);
        CK(cudaMemcpyAsync(d_sys_obase.p, obase.data(), 4 * S, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_sys_n.p, nn.data(), 4 * S, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_sys_ground.p, gr.data(), 4 * S, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_sys_lbase.p, lb.data(), 4 * S, cudaMemcpyHostToDevice, st));
        d_sys_of_orig = dalloc<int32_t>(N, st);
        d_sys_of_label = dalloc<int32_t>(nl, st);
        for (int s = 0; s < S; ++s)
            CK(launch_fill_i32(d_sys_of_orig.as<int32_t>() + systems[s].obase, systems[s].n, s, st));
        CK(launch_sys_of_label(S, d_sys_lbase.as<int32_t>(), (int32_t)nl, d_sys_of_label.as<int32_t>(), st));
    }

    DBuf flags = dalloc<int32_t>(1, st);
    CK(cudaMemsetAsync(flags.p, 0, 4, st));
    DBuf iperm = dalloc<int32_t>(N, st);
    if (ord_global) {
        CK(cudaMemsetAsync(iperm.p, 0xff, 4 * N, st));
        CK(launch_iperm(N, ord_global, label_of_k, iperm.as<int32_t>(), flags.as<int32_t>(), st));
    } else {
        CK(launch_identity_iperm(N, iperm.as<int32_t>(), st));
    }
    DBuf lcnt = dalloc<int32_t>(nl, st), dp0 = dalloc<int32_t>(nl, st), gw = dalloc<double>(N, st);
    CK(cudaMemsetAsync(lcnt.p, 0, 4 * nl, st));
    CK(cudaMemsetAsync(dp0.p, 0, 4 * nl, st));
    IngestArgs ia{};
    ia.n = N; ia.colptr = colptr; ia.rowind = rowind; ia.val = val;
    ia.sys_of_orig = batch ? d_sys_of_orig.as<int32_t>() : nullptr;
    ia.sys_obase = batch ? d_sys_obase.as<int32_t>() : nullptr;
    ia.sys_n = batch ? d_sys_n.as<int32_t>() : nullptr;
    ia.sys_ground = batch ? d_sys_ground.as<int32_t>() : nullptr;
    ia.single_ground = systems[0].ground;
    ia.kind = kind;
    ia.iperm = iperm.as<int32_t>(); ia.lcnt = lcnt.as<int32_t>(); ia.dp = dp0.as<int32_t>(); ia.gw = gw.as<double>();
    ia.status = flags.as<int32_t>();
    // the count kernel reads iperm; a bad ordering must be reported before
    int32_t hflags = 0;
    CK(cudaMemcpyAsync(&hflags, flags.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hflags & INGEST_BAD_INDEX) { set_err("ordering is not a permutation"); throw StatusFail{PARAC_EINVAL}; }
    CK(launch_ingest_count(ia, st));
    DBuf lcp = dalloc<int64_t>(nl + 1, st);
    DBuf scan_tmp(scan_tmp_bytes(std::max<int64_t>(nl, N) + 1), st);
    CK(scan_i32_to_i64(lcnt.as<int32_t>(), lcp.as<int64_t>(), nl, scan_tmp.p, st));
    int64_t nnz_low = 0;
    CK(cudaMemcpyAsync(&hflags, flags.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&nnz_low, lcp.as<int64_t>() + nl, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hflags & INGEST_BAD_INDEX) { set_err("row index out of range"); throw StatusFail{PARAC_EINVAL}; }
    if (hflags & INGEST_NOT_SDD) { set_err("positive off-diagonal entry or negative row excess"); throw StatusFail{PARAC_ENOT_SDD}; }
    if (hflags & INGEST_KIND) { set_err("matrix has row excess but kind is LAPLACIAN"); throw StatusFail{PARAC_EINVAL}; }
    out.nnz_low = nnz_low;
    DBuf lrow = dalloc<int32_t>(std::max<int64_t>(nnz_low, 1), st), lw = dalloc<double>(std::max<int64_t>(nnz_low, 1), st);
    CK(launch_ingest_scatter(ia, lcp.as<int64_t>(), lrow.as<int32_t>(), lw.as<double>(), st));
    out.t_ingest = t_in.stop();

    // ---------------------------------------------------------------- elimination
    EvTimer t_el(O.o.timing != 0, st);
    const int warps = O.o.warps_per_block;
    // CTA buffer of the cooperative path: 2048 entries while two CTAs still
    // fit an SM, else 1024
    int warp_cap = 128, block_cap = 2048;
    if (O.o.big_threshold > 0) {
        int b = 32;
        while (b < O.o.big_threshold && b < 4096) b <<= 1;
        warp_cap = b;
        block_cap = 1024;
        if (block_cap < 2 * warp_cap) block_cap = 2 * warp_cap;
    }
    if (O.o.block_cap > 0) {
        int b = 256;
        while (b < O.o.block_cap && b < 8192) b <<= 1;
        block_cap = std::max(b, 2 * warp_cap);
    }
    int bps = 0;
    CK(elim_configure(warps, warp_cap, block_cap, &bps));
    if (bps < 2 && block_cap > 1024 && block_cap > 2 * warp_cap) {
        block_cap = std::max(1024, 2 * warp_cap);
        CK(elim_configure(warps, warp_cap, block_cap, &bps));
    }
    if (bps < 1) { block_cap = 0; CK(elim_configure(warps, warp_cap, block_cap, &bps)); }
    if (bps < 1) { set_err("elimination kernel does not fit on an SM"); throw StatusFail{PARAC_EINVAL}; }
    int blocks = num_sms() * bps;
    if (O.o.blocks > 0) blocks = std::min(blocks, O.o.blocks);
    out.blocks = blocks; out.warps = warps;
    const int total_warps = blocks * warps;
    const int fchunk = 256;

    DBuf dp = dalloc<int32_t>(nl, st), queue = dalloc<int32_t>(nl, st), ctrs = dalloc<uint32_t>(3, st);
    DBuf fcnt = dalloc<uint32_t>(nl, st), in_row = dalloc<int32_t>((size_t)nl * FILL_C0, st),
         in_w = dalloc<double>((size_t)nl * FILL_C0, st), dir = dalloc<uint32_t>((size_t)nl * FILL_LEVELS, st);
    DBuf f_start = dalloc<int64_t>(nl, st), f_len = dalloc<int32_t>(nl, st), Dl = dalloc<double>(nl, st);
    DBuf lvl = dalloc<int32_t>(nl, st);
    DBuf tops = dalloc<unsigned long long>(3, st), status = dalloc<int32_t>(1, st), stats = dalloc<unsigned long long>(160, st);
    // grid-help board: word, hints and done counters one 128-byte line each, lock, task ring
    constexpr size_t GH_WORD = 0, GH_HINT = 128, GH_DONE = GH_HINT + 128 * GH_HINTS, GH_LOCK = GH_DONE + 128 * GH_RING,
                     GH_TASK = GH_LOCK + 128, GH_BYTES = GH_TASK + sizeof(GhTask) * GH_RING;
    DBuf ghb(GH_BYTES, st);

    // optional per-vertex trace, written to the file opts->trace_path names
    const char *trace_path = O.o.trace_path;
    DBuf trace_buf, trace_par, trace_ph;
    if (trace_path) {
        trace_buf = dalloc<long long>((size_t)nl * 4, st);
        trace_par = dalloc<int32_t>((size_t)nl, st);
        CK(cudaMemsetAsync(trace_buf.p, 0, 32 * (size_t)nl, st));
        CK(cudaMemsetAsync(trace_par.p, 0xff, 4 * (size_t)nl, st));
        trace_ph = dalloc<int32_t>((size_t)nl * 8, st);
        CK(cudaMemsetAsync(trace_ph.p, 0, 32 * (size_t)nl, st));
    }
    double mult = O.o.pool_mult;                        // set below when 0 (automatic)
    // Global scratch of the cooperative (CTA-per-vertex) path: every CTA may
    // hold a working set of next_pow2(gather) entries, and a vertex's gather
    // is its original lower column plus the fill it receives.  Sized from the
    // longest lower column (x4 for fill, x2 for the arena's growth by
    // doubling), at most a quarter of the free device memory.
    unsigned long long scratch_cap = 256ull << 20;
    {
        DBuf mx = dalloc<int32_t>(1, st);
        CK(cudaMemsetAsync(mx.p, 0, 4, st));
        if (nl > 0) CK(launch_max_i32(lcnt.as<int32_t>(), nl, mx.as<int32_t>(), st));
        int32_t maxlow = 0;
        CK(cudaMemcpyAsync(&maxlow, mx.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        unsigned long long p2 = 1;
        while (p2 < 4ull * (unsigned long long)maxlow + 64ull) p2 <<= 1;
        const unsigned long long want = (unsigned long long)blocks * 2ull * (ENTRY_BYTES + 1) * p2 + (256ull << 20);
        scratch_cap = std::max(scratch_cap, std::min<unsigned long long>(want, device_memory_bytes() / 8));
        out.max_lower_column = maxlow;
        // Fill workspace: bounded-degree inputs (grids) use ~3.5x their lower
        // entries, power-law graphs ~8x (hub columns' overflow slabs); an
        // overflow reruns the whole elimination, so hub-dominated inputs start at 10x.
        if (mult <= 0.0) {
            const double avg = nl > 0 ? (double)nnz_low / (double)nl : 0.0;
            mult = (double)maxlow > 16.0 * std::max(avg, 1.0) ? 10.0 : 5.0;
        }
    }
    DBuf pool_row, pool_w, f_row, f_val, scratch, w_col, w_row, w_w;
    for (int attempt = 0;; ++attempt) {
        // per-slot multi-sampling MS(k): k fill edges per slot, and the neighbour
        // lists of later pivots grow with them -- MS(2) on 3D grids has 10-30x
        // the fill of Alg. 2
        const double ks = O.o.samples > 1 ? 4.0 * (double)O.o.samples * (double)O.o.samples : 1.0;
        const unsigned long long pool_cap = (unsigned long long)std::ceil(mult * ks * (double)nnz_low) + 4096ull;
        const unsigned long long f_cap = (unsigned long long)std::ceil(std::max(mult, 4.0) * ks * (double)nnz_low) +
                                         (unsigned long long)nl + (unsigned long long)total_warps * fchunk + 4096ull;
        // load factor at most 1/2 of the slab estimate; a power of two, so that
        // every odd probe stride reaches every slot (w_stride)
        unsigned long long wcap = 2;
        while (wcap < 2ull * pool_cap) wcap <<= 1;
        if (O.o.fill_store == 1) {                // hashmap W (Sec. IV-C)
            pool_row = dalloc<int32_t>(1, st); pool_w = dalloc<double>(1, st);
            w_col = dalloc<int32_t>(wcap, st); w_row = dalloc<int32_t>(wcap, st);
            w_w = dalloc<double>(wcap, st);
            CK(cudaMemsetAsync(w_col.p, 0xff, 4 * (size_t)wcap, st));      // every slot free (-1)
        } else {
            pool_row = dalloc<int32_t>(pool_cap, st); pool_w = dalloc<double>(pool_cap, st);
        }
        f_row = dalloc<int32_t>(f_cap, st); f_val = dalloc<double>(f_cap, st);
        scratch.alloc(scratch_cap, st);
        CK(cudaMemcpyAsync(dp.p, dp0.p, 4 * nl, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(queue.p, 0xff, 4 * nl, st));
        CK(cudaMemsetAsync(ctrs.p, 0, 12, st));
        CK(cudaMemsetAsync(fcnt.p, 0, 4 * nl, st));
        CK(cudaMemsetAsync(dir.p, 0, 4 * (size_t)nl * FILL_LEVELS, st));
        CK(cudaMemsetAsync(tops.p, 0, 24, st));
        CK(cudaMemsetAsync(status.p, 0, 4, st));
        CK(cudaMemsetAsync(stats.p, 0, 1280, st));
        CK(cudaMemsetAsync(lvl.p, 0, 4 * nl, st));
        CK(cudaMemsetAsync(ghb.p, 0, GH_BYTES, st));
        CK(launch_queue_init((int32_t)nl, dp.as<int32_t>(), queue.as<int32_t>(), ctrs.as<uint32_t>() + 1, st));

        ElimArgs a{};
        a.nl = (int32_t)nl; a.lcp = lcp.as<int64_t>(); a.lrow = lrow.as<int32_t>(); a.lw = lw.as<double>();
        a.sys_of = batch ? d_sys_of_label.as<int32_t>() : nullptr;
        a.sys_base = batch ? d_sys_lbase.as<int32_t>() : nullptr;
        a.seed = seed;
        a.dp = dp.as<int32_t>(); a.queue = queue.as<int32_t>();
        a.q_head = ctrs.as<uint32_t>(); a.q_tail = ctrs.as<uint32_t>() + 1; a.done = ctrs.as<uint32_t>() + 2;
        a.fcnt = fcnt.as<uint32_t>(); a.in_row = in_row.as<int32_t>(); a.in_w = in_w.as<double>();
        a.dir = dir.as<uint32_t>(); a.pool_row = pool_row.as<int32_t>(); a.pool_w = pool_w.as<double>();
        a.pool_top = tops.as<unsigned long long>(); a.pool_cap = pool_cap;
        a.f_row = f_row.as<int32_t>(); a.f_val = f_val.as<double>();
        a.f_top = tops.as<unsigned long long>() + 1; a.f_cap = f_cap;
        a.f_start = f_start.as<int64_t>(); a.f_len = f_len.as<int32_t>(); a.D = Dl.as<double>();
        a.lvl = lvl.as<int32_t>();
        a.scratch = scratch.as<unsigned char>(); a.scratch_top = tops.as<unsigned long long>() + 2;
        a.scratch_cap = scratch_cap;
        a.status = status.as<int32_t>(); a.spin_limit = O.o.spin_limit;
        a.stats = stats.as<unsigned long long>();
        a.warp_cap = warp_cap; a.block_cap = block_cap; a.queue_chunk = O.o.queue_chunk;
        a.profile = O.o.timing >= 2 ? 1 : 0;
        a.trace = trace_buf.as<long long>();
        a.trace_parent = trace_par.as<int32_t>();
        a.trace_phase = trace_ph.as<int32_t>();
        a.idle_ns = 512;
        a.coop = 1;
        if (O.o.coop == PARAC_OFF) a.coop = 0;
        a.samples = O.o.samples;
        a.hash_store = O.o.fill_store == 1 ? 1 : 0;
        a.wcol = w_col.as<int32_t>(); a.wrow = w_row.as<int32_t>(); a.ww = w_w.as<double>();
        a.wcap = O.o.fill_store == 1 ? wcap : 0;
        out.samples = O.o.samples;
        out.fill_store = O.o.fill_store;
        a.sample_sort = 1;
        {
            unsigned char *gb = ghb.as<unsigned char>();
            a.gh_word = (unsigned long long *)(gb + GH_WORD);
            a.gh_hint = (uint32_t *)(gb + GH_HINT);
            a.gh_done = (uint32_t *)(gb + GH_DONE);
            a.gh_lock = (int32_t *)(gb + GH_LOCK);
            a.gh_task = (GhTask *)(gb + GH_TASK);
            // default: only for hub-dominated inputs (longest lower column above 16x the
            // average, as for the fill workspace), whose late vertices gather thousands of entries
            const double avg_low = nl > 0 ? (double)nnz_low / (double)nl : 0.0;
            const bool hubs = (double)out.max_lower_column > 16.0 * std::max(avg_low, 1.0);
            const bool gh = O.o.grid_help == PARAC_ON || (O.o.grid_help == PARAC_DEFAULT && hubs);
            a.grid_help = !gh || warp_cap < 128 ? 0 : std::max(1, O.o.grid_help_min);
            a.gh_mask = 3;                                  // one warp in four
        }
        if (O.o.sample_sort == PARAC_OFF) a.sample_sort = 0;
        if (O.o.idle_ns > 0) a.idle_ns = std::max(32, std::min(1000000, O.o.idle_ns));
        if (nl > 0) CK(elim_launch(a, blocks, warps, fchunk, st));
        int32_t hst = 0;
        unsigned long long htops[3];
        CK(cudaMemcpyAsync(&hst, status.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(htops, tops.p, 24, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(out.stats, stats.p, 1280, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        out.pool_used = htops[0]; out.f_used = htops[1]; out.scratch_used = htops[2];
        if (hst == ST_OK) break;
        // which workspace ran out: every reservation bumps its top, also past the end
        const bool over_pool = htops[0] > pool_cap || htops[1] > f_cap, over_scratch = htops[2] > scratch_cap;
        if (hst == ST_POOL && attempt < O.o.max_pool_regrow) {
            if (over_pool || !over_scratch) mult *= 2.0;
            if (over_scratch) scratch_cap *= 4;
            out.regrows++;
            continue;
        }
        if (hst == ST_POOL)
            set_err("%s workspace overflow (raise pool_mult or max_pool_regrow)",
                    over_scratch ? "cooperative-path scratch" : "fill");
        else
            set_err("device wait exceeded spin_limit");
        throw StatusFail{map_status(hst)};
    }
    scratch.release(); pool_row.release(); pool_w.release(); w_col.release(); w_row.release(); w_w.release();
    out.t_elim = t_el.stop();
    if (trace_path) {
        std::vector<long long> tr((size_t)nl * 4);
        std::vector<int32_t> par((size_t)nl), lv((size_t)nl);
        CK(cudaMemcpyAsync(tr.data(), trace_buf.p, 32 * (size_t)nl, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(par.data(), trace_par.p, 4 * (size_t)nl, cudaMemcpyDeviceToHost, st));
        std::vector<int32_t> ph((size_t)nl * 8);
        CK(cudaMemcpyAsync(ph.data(), trace_ph.p, 32 * (size_t)nl, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(lv.data(), lvl.p, 4 * (size_t)nl, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (FILE *f = fopen(trace_path, "wb")) {
            const long long nn = nl;
            fwrite(&nn, 8, 1, f);
            fwrite(tr.data(), 8, tr.size(), f);
            fwrite(par.data(), 4, par.size(), f);
            fwrite(lv.data(), 4, lv.size(), f);
            fwrite(ph.data(), 4, ph.size(), f);
            fclose(f);
        }
    }

    // ---------------------------------------------------------------- compaction
    EvTimer t_cp(O.o.timing != 0, st);
    DBuf out_of_label = dalloc<int32_t>(nl, st);
    if (batch)
        CK(launch_out_of_label_batch((int32_t)nl, d_sys_of_label.as<int32_t>(), d_sys_lbase.as<int32_t>(),
                                     d_sys_obase.as<int32_t>(), d_sys_n.as<int32_t>(), out_of_label.as<int32_t>(), st));
    else
        CK(launch_out_of_label_single((int32_t)nl, (int32_t)N, out_of_label.as<int32_t>(), st));
    DBuf olen = dalloc<int32_t>(std::max<int64_t>(N, 1), st);
    CK(launch_out_len((int32_t)nl, out_of_label.as<int32_t>(), f_start.as<int64_t>(), f_len.as<int32_t>(),
                      f_row.as<int32_t>(), olen.as<int32_t>(), st));
    out.Fcp = dalloc<int64_t>(N + 1, st);
    CK(scan_i32_to_i64(olen.as<int32_t>(), out.Fcp.as<int64_t>(), N, scan_tmp.p, st));
    int64_t nnzF = 0;
    CK(cudaMemcpyAsync(&nnzF, out.Fcp.as<int64_t>() + N, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out.nnzF = nnzF;
    out.Frow = dalloc<int32_t>(std::max<int64_t>(nnzF, 1), st);
    out.Fval = dalloc<double>(std::max<int64_t>(nnzF, 1), st);
    out.D = dalloc<double>(std::max<int64_t>(N, 1), st);
    out.Lev = dalloc<int32_t>(std::max<int64_t>(N, 1), st);
    CK(launch_scatter_levels((int32_t)nl, out_of_label.as<int32_t>(), lvl.as<int32_t>(), out.Lev.as<int32_t>(), st));
    CK(launch_gather_factor((int32_t)nl, out_of_label.as<int32_t>(), f_start.as<int64_t>(), f_row.as<int32_t>(),
                            f_val.as<double>(), Dl.as<double>(), out.Fcp.as<int64_t>(), out.Frow.as<int32_t>(),
                            out.Fval.as<double>(), out.D.as<double>(), st));
    out.t_compact = t_cp.stop();
}

std::string stats_json(const parac_factor_s *h, const FactorOut &fo, int sys_index);

// Group tables of the one-row-per-warp solves for a factor with rows longer
// than 4 x LONG_ROW_SINGLE entries (a host pass over the relabelled factor's
// row and column pointers).
// CSR rows of more than 2,048 entries sorted by column as well (the shorter
// ones are sorted by launch_sort_rows / launch_sort_long_rows), so that the
// solve arrays are the same on every run.
void sort_huge_rows(int64_t n, int64_t *rp, int32_t *cols, double *vals, cudaStream_t st)
{
    DBuf tmp(huge_rows_tmp_bytes(n), st);
    int64_t nrows = 0, entries = 0;
    CK(huge_rows_count((int32_t)n, rp, tmp.p, &nrows, &entries, st));
    if (nrows == 0) return;
    DBuf work(huge_rows_sort_bytes(nrows, entries), st);
    CK(huge_rows_sort((int32_t)n, rp, cols, vals, tmp.p, nrows, entries, work.p, st));
}

void build_group_tables(parac_factor_s *h, cudaStream_t st)
{
    const int64_t n = h->n;
    if (!h->host_tables) {                 // built on the device by scans (row_groups_count / _write)
        DBuf tmp(row_groups_tmp_bytes(n), st);
        int64_t ngf = 0, nsf = 0, ngb = 0, nsb = 0;
        CK(row_groups_count(h->Srp.as<int64_t>(), n, false, SOLVE_WARPS, LONG_ROW_SINGLE, SPLIT_ROW_SINGLE, CHUNK_SINGLE,
                            tmp.p, &ngf, &nsf, st));
        h->sgt_f = dalloc<int32_t>((size_t)(4 * ngf), st);
        CK(row_groups_write(h->Srp.as<int64_t>(), n, false, SOLVE_WARPS, SPLIT_ROW_SINGLE, CHUNK_SINGLE, tmp.p,
                            h->sgt_f.as<int32_t>(), st));
        CK(row_groups_count(h->Scp.as<int64_t>(), n, true, SOLVE_WARPS, LONG_ROW_SINGLE, SPLIT_ROW_SINGLE, CHUNK_SINGLE,
                            tmp.p, &ngb, &nsb, st));
        h->sgt_b = dalloc<int32_t>((size_t)(4 * ngb), st);
        CK(row_groups_write(h->Scp.as<int64_t>(), n, true, SOLVE_WARPS, SPLIT_ROW_SINGLE, CHUNK_SINGLE, tmp.p,
                            h->sgt_b.as<int32_t>(), st));
        h->spart_f = dalloc<double>((size_t)std::max<int64_t>(nsf, 1), st);
        h->spart_b = dalloc<double>((size_t)std::max<int64_t>(nsb, 1), st);
        CK(cudaStreamSynchronize(st));     // tmp is released on return
        h->sng_f = (int32_t)ngf; h->sng_b = (int32_t)ngb;
        h->snslot_f = (int32_t)nsf; h->snslot_b = (int32_t)nsb;
        return;
    }
    std::vector<int64_t> rp((size_t)n + 1), cp((size_t)n + 1);
    CK(cudaMemcpyAsync(rp.data(), h->Srp.p, 8 * ((size_t)n + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(cp.data(), h->Scp.p, 8 * ((size_t)n + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const GroupTable gf = row_groups(rp, false, SOLVE_WARPS, LONG_ROW_SINGLE, SPLIT_ROW_SINGLE, CHUNK_SINGLE),
                     gb = row_groups(cp, true, SOLVE_WARPS, LONG_ROW_SINGLE, SPLIT_ROW_SINGLE, CHUNK_SINGLE);
    h->sgt_f = dalloc<int32_t>(gf.g.size(), st);
    h->sgt_b = dalloc<int32_t>(gb.g.size(), st);
    CK(cudaMemcpyAsync(h->sgt_f.p, gf.g.data(), 4 * gf.g.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->sgt_b.p, gb.g.data(), 4 * gb.g.size(), cudaMemcpyHostToDevice, st));
    h->spart_f = dalloc<double>((size_t)std::max(gf.nslots, 1), st);
    h->spart_b = dalloc<double>((size_t)std::max(gb.nslots, 1), st);
    CK(cudaStreamSynchronize(st));
    h->sng_f = gf.ngroups; h->sng_b = gb.ngroups;
    h->snslot_f = gf.nslots; h->snslot_b = gb.nslots;
}

// Build the solve-side arrays of a handle from its label-space CSC(F): sort
// the columns by dependency level, relabel F into that order (positions),
// and build the CSR of the relabelled factor for the forward solve.
void finish_handle(parac_factor_s *h, int64_t n, int64_t nnzF, const Opts &O)
{
    cudaStream_t st = O.st;
    const size_t n1 = (size_t)std::max<int64_t>(n, 1), z1 = (size_t)std::max<int64_t>(nnzF, 1);
    DBuf order = dalloc<int32_t>(n1, st);
    h->depth = 0;
    if (n > 0) {
        DBuf mx = dalloc<int32_t>(1, st);
        CK(cudaMemsetAsync(mx.p, 0, 4, st));
        CK(launch_max_i32(h->Lev.as<int32_t>(), n, mx.as<int32_t>(), st));
        int32_t hmax = 0;
        CK(cudaMemcpyAsync(&hmax, mx.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        h->depth = hmax + 1;
        DBuf hist = dalloc<int32_t>((size_t)hmax + 1, st), lstart = dalloc<int64_t>((size_t)hmax + 2, st);
        CK(cudaMemsetAsync(hist.p, 0, 4 * ((size_t)hmax + 1), st));
        CK(launch_row_count(n, h->Lev.as<int32_t>(), hist.as<int32_t>(), st));
        DBuf tmp2(scan_tmp_bytes(hmax + 2), st);
        CK(scan_i32_to_i64(hist.as<int32_t>(), lstart.as<int64_t>(), hmax + 1, tmp2.p, st));
        h->lstart.assign((size_t)hmax + 2, 0);
        CK(cudaMemcpyAsync(h->lstart.data(), lstart.p, 8 * ((size_t)hmax + 2), cudaMemcpyDeviceToHost, st));
        // positions: columns sorted by level, stably (a level's columns in
        // label order), so that the solve arrays are the same on every run
        DBuf keys = dalloc<int32_t>(n1, st), rtmp(radix_tmp_bytes(n), st);
        CK(cudaMemcpyAsync(keys.p, h->Lev.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
        CK(launch_iota_i32(order.as<int32_t>(), n, 0, st));
        int bits = 0;
        while (bits < 31 && (hmax >> bits) != 0) ++bits;
        CK(stable_sort_pairs((int32_t)n, keys.as<int32_t>(), order.as<int32_t>(), bits, rtmp.p, st));
    }
    DBuf posof = dalloc<int32_t>(n1, st), len = dalloc<int32_t>(n1, st);
    CK(launch_inverse_perm((int32_t)n, order.as<int32_t>(), posof.as<int32_t>(), st));
    CK(launch_relabel_lengths((int32_t)n, order.as<int32_t>(), h->Fcp.as<int64_t>(), len.as<int32_t>(), st));
    DBuf tmp(scan_tmp_bytes(n + 1), st);
    h->Scp = dalloc<int64_t>((size_t)n + 1, st);
    CK(scan_i32_to_i64(len.as<int32_t>(), h->Scp.as<int64_t>(), n, tmp.p, st));
    h->Srow = dalloc<int32_t>(z1, st);
    h->Sval = dalloc<double>(z1, st);
    CK(launch_relabel_gather((int32_t)n, order.as<int32_t>(), posof.as<int32_t>(), h->Fcp.as<int64_t>(),
                             h->Frow.as<int32_t>(), h->Fval.as<double>(), h->Scp.as<int64_t>(), h->Srow.as<int32_t>(),
                             h->Sval.as<double>(), st));
    // CSR of the relabelled factor
    h->Srp = dalloc<int64_t>((size_t)n + 1, st);
    h->Scol = dalloc<int32_t>(z1, st);
    h->Svalr = dalloc<double>(z1, st);
    DBuf cnt = dalloc<int32_t>(n1, st);
    CK(cudaMemsetAsync(cnt.p, 0, 4 * n1, st));
    CK(launch_row_count(nnzF, h->Srow.as<int32_t>(), cnt.as<int32_t>(), st));
    CK(scan_i32_to_i64(cnt.as<int32_t>(), h->Srp.as<int64_t>(), n, tmp.p, st));
    // longest row (forward) or column (backward) of the solves
    DBuf mxlen = dalloc<int32_t>(1, st);
    CK(cudaMemsetAsync(mxlen.p, 0, 4, st));
    CK(launch_max_i32(cnt.as<int32_t>(), n, mxlen.as<int32_t>(), st));
    CK(launch_max_i32(len.as<int32_t>(), n, mxlen.as<int32_t>(), st));
    int32_t maxlen = 0;
    CK(cudaMemcpyAsync(&maxlen, mxlen.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(cnt.p, 0, 4 * n1, st));
    CK(launch_transpose_scatter((int32_t)n, h->Scp.as<int64_t>(), h->Srow.as<int32_t>(), h->Sval.as<double>(),
                                h->Srp.as<int64_t>(), cnt.as<int32_t>(), h->Scol.as<int32_t>(), h->Svalr.as<double>(), st));
    CK(launch_sort_rows((int32_t)n, h->Srp.as<int64_t>(), h->Scol.as<int32_t>(), h->Svalr.as<double>(), st));
    CK(launch_sort_long_rows((int32_t)n, h->Srp.as<int64_t>(), h->Scol.as<int32_t>(), h->Svalr.as<double>(), st));
    sort_huge_rows(n, h->Srp.as<int64_t>(), h->Scol.as<int32_t>(), h->Svalr.as<double>(), st);
    // pivots and original indices by position
    DBuf Dpos = dalloc<double>(n1, st);
    CK(launch_gather_f64((int32_t)n, order.as<int32_t>(), h->D.as<double>(), Dpos.as<double>(), st));
    h->Sdinv = dalloc<double>(n1, st);
    CK(launch_dinv((int32_t)n, Dpos.as<double>(), h->Sdinv.as<double>(), st));
    h->Sperm = dalloc<int32_t>(n1, st);
    CK(launch_gather_i32((int32_t)n, order.as<int32_t>(), h->perm.as<int32_t>(), h->Sperm.as<int32_t>(), st));
    if (h->prec == 32) {
        h->Sval32 = dalloc<float>(z1, st);
        h->Svalr32 = dalloc<float>(z1, st);
        CK(launch_to_f32(h->Sval.as<double>(), h->Sval32.as<float>(), nnzF, st));
        CK(launch_to_f32(h->Svalr.as<double>(), h->Svalr32.as<float>(), nnzF, st));
    }
    h->status = dalloc<int32_t>(1, st);
    // Group tables of the one-row-per-warp solves, only when some row is long
    // enough to matter: up to 4x LONG_ROW_SINGLE entries a warp still walks a
    // row in a few rounds of its chunked dot, and the fixed groups avoid
    // building the table (a host pass over the rows) at setup.
    CK(cudaStreamSynchronize(st));
    h->max_row = maxlen;
    if (maxlen > 4 * LONG_ROW_SINGLE) build_group_tables(h, st);
}

// The complete set of solve arrays of several systems at once (the batched
// form): the same steps as finish_handle, run once over the concatenation of
// the systems' factors (their labels are contiguous, so a stable sort by
// (system, level, label) keeps every system in its own position range and the
// CSC / CSR of the relabelled block-diagonal factor are the systems' own
// arrays side by side), then split into the handles with one segmented copy
// per array.  Three small device-to-host reads (entry offsets and depths,
// level histograms, longest rows) replace the per-system synchronisations.
void finish_batch(std::vector<std::unique_ptr<parac_factor_s>> &hs, FactorOut &fo, const std::vector<SysDesc> &sys,
                  const std::vector<int64_t> &nnzL, const DBuf &cp, const DBuf &ri, const DBuf &va, const DBuf &ord,
                  const Opts &O)
{
    cudaStream_t st = O.st;
    const int32_t count = (int32_t)sys.size();
    const int64_t N = sys.back().obase + sys.back().n;
    const int64_t nnzF = fo.nnzF;
    const size_t n1 = (size_t)std::max<int64_t>(N, 1), z1 = (size_t)std::max<int64_t>(nnzF, 1);
    const int prec = O.o.g_precision;
    // system of every label (= position: both keep the systems' ranges)
    std::vector<int32_t> ob_h((size_t)count + 1);
    std::vector<int64_t> ob64((size_t)count + 1);
    for (int32_t s = 0; s < count; ++s) { ob_h[(size_t)s] = (int32_t)sys[(size_t)s].obase; ob64[(size_t)s] = sys[(size_t)s].obase; }
    ob_h[(size_t)count] = (int32_t)N; ob64[(size_t)count] = N;
    DBuf obase = dalloc<int32_t>((size_t)count + 1, st), ob64d = dalloc<int64_t>((size_t)count + 1, st);
    CK(cudaMemcpyAsync(obase.p, ob_h.data(), 4 * ob_h.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ob64d.p, ob64.data(), 8 * ob64.size(), cudaMemcpyHostToDevice, st));
    DBuf sysv = dalloc<int32_t>(n1, st);
    if (N > 0) CK(launch_sys_of_label(count, obase.as<int32_t>(), (int32_t)N, sysv.as<int32_t>(), st));
    // entry offset of every system (Fcp at its first column) and its depth
    std::vector<const int64_t *> fptr((size_t)count + 1, fo.Fcp.as<int64_t>());
    DBuf fptr_d = DBuf(sizeof(void *) * fptr.size(), st), f0d = dalloc<int64_t>((size_t)count + 1, st);
    DBuf dmax = dalloc<int32_t>((size_t)count, st);
    CK(cudaMemcpyAsync(fptr_d.p, fptr.data(), sizeof(void *) * fptr.size(), cudaMemcpyHostToDevice, st));
    CK(launch_gather_ends((const int64_t *const *)fptr_d.p, ob64d.as<int64_t>(), count + 1, f0d.as<int64_t>(), st));
    CK(cudaMemsetAsync(dmax.p, 0, 4 * (size_t)count, st));
    CK(launch_seg_max(N, fo.Lev.as<int32_t>(), sysv.as<int32_t>(), dmax.as<int32_t>(), st));
    std::vector<int64_t> f0((size_t)count + 1);
    std::vector<int32_t> dm((size_t)count);
    CK(cudaMemcpyAsync(f0.data(), f0d.p, 8 * f0.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(dm.data(), dmax.p, 4 * dm.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int64_t> hoff((size_t)count + 1, 0);
    int32_t maxdepth = 1;
    for (int32_t s = 0; s < count; ++s) {
        const int32_t depth = sys[(size_t)s].n > 0 ? dm[(size_t)s] + 1 : 0;
        hoff[(size_t)s + 1] = hoff[(size_t)s] + depth;
        maxdepth = std::max(maxdepth, depth);
    }
    // level histograms of every system -> level starts
    DBuf hoffd = dalloc<int64_t>(hoff.size(), st), hist = dalloc<int32_t>((size_t)std::max<int64_t>(hoff.back(), 1), st);
    CK(cudaMemcpyAsync(hoffd.p, hoff.data(), 8 * hoff.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(hist.p, 0, 4 * (size_t)std::max<int64_t>(hoff.back(), 1), st));
    CK(launch_seg_hist(N, fo.Lev.as<int32_t>(), sysv.as<int32_t>(), hoffd.as<int64_t>(), hist.as<int32_t>(), st));
    std::vector<int32_t> hh((size_t)std::max<int64_t>(hoff.back(), 1));
    CK(cudaMemcpyAsync(hh.data(), hist.p, 4 * hh.size(), cudaMemcpyDeviceToHost, st));
    // positions: stable sort by level, then by system
    DBuf order = dalloc<int32_t>(n1, st), keys = dalloc<int32_t>(n1, st), rtmp(radix_tmp_bytes(N), st);
    CK(cudaMemcpyAsync(keys.p, fo.Lev.p, 4 * (size_t)N, cudaMemcpyDeviceToDevice, st));
    CK(launch_iota_i32(order.as<int32_t>(), N, 0, st));
    auto bits_of = [](int64_t v) { int b = 0; while (b < 31 && (v >> b) != 0) ++b; return b; };
    CK(stable_sort_pairs((int32_t)N, keys.as<int32_t>(), order.as<int32_t>(), bits_of(maxdepth - 1), rtmp.p, st));
    CK(launch_gather_i32((int32_t)N, order.as<int32_t>(), sysv.as<int32_t>(), keys.as<int32_t>(), st));
    CK(stable_sort_pairs((int32_t)N, keys.as<int32_t>(), order.as<int32_t>(), bits_of(count - 1), rtmp.p, st));
    // relabelled CSC (backward) and CSR (forward) of the block-diagonal factor
    DBuf posof = dalloc<int32_t>(n1, st), len = dalloc<int32_t>(n1, st);
    CK(launch_inverse_perm((int32_t)N, order.as<int32_t>(), posof.as<int32_t>(), st));
    CK(launch_relabel_lengths((int32_t)N, order.as<int32_t>(), fo.Fcp.as<int64_t>(), len.as<int32_t>(), st));
    DBuf tmp(scan_tmp_bytes(N + 1), st);
    DBuf Scp = dalloc<int64_t>((size_t)N + 1, st), Srow = dalloc<int32_t>(z1, st), Sval = dalloc<double>(z1, st);
    CK(scan_i32_to_i64(len.as<int32_t>(), Scp.as<int64_t>(), N, tmp.p, st));
    CK(launch_relabel_gather((int32_t)N, order.as<int32_t>(), posof.as<int32_t>(), fo.Fcp.as<int64_t>(),
                             fo.Frow.as<int32_t>(), fo.Fval.as<double>(), Scp.as<int64_t>(), Srow.as<int32_t>(),
                             Sval.as<double>(), st));
    DBuf Srp = dalloc<int64_t>((size_t)N + 1, st), Scol = dalloc<int32_t>(z1, st), Svalr = dalloc<double>(z1, st);
    DBuf cnt = dalloc<int32_t>(n1, st), rmax = dalloc<int32_t>((size_t)count, st);
    CK(cudaMemsetAsync(cnt.p, 0, 4 * n1, st));
    CK(launch_row_count(nnzF, Srow.as<int32_t>(), cnt.as<int32_t>(), st));
    CK(scan_i32_to_i64(cnt.as<int32_t>(), Srp.as<int64_t>(), N, tmp.p, st));
    CK(cudaMemsetAsync(rmax.p, 0, 4 * (size_t)count, st));
    CK(launch_seg_max(N, cnt.as<int32_t>(), sysv.as<int32_t>(), rmax.as<int32_t>(), st));
    CK(launch_seg_max(N, len.as<int32_t>(), sysv.as<int32_t>(), rmax.as<int32_t>(), st));
    std::vector<int32_t> rm((size_t)count);
    CK(cudaMemcpyAsync(rm.data(), rmax.p, 4 * rm.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(cnt.p, 0, 4 * n1, st));
    CK(launch_transpose_scatter((int32_t)N, Scp.as<int64_t>(), Srow.as<int32_t>(), Sval.as<double>(), Srp.as<int64_t>(),
                                cnt.as<int32_t>(), Scol.as<int32_t>(), Svalr.as<double>(), st));
    CK(launch_sort_rows((int32_t)N, Srp.as<int64_t>(), Scol.as<int32_t>(), Svalr.as<double>(), st));
    CK(launch_sort_long_rows((int32_t)N, Srp.as<int64_t>(), Scol.as<int32_t>(), Svalr.as<double>(), st));
    sort_huge_rows(N, Srp.as<int64_t>(), Scol.as<int32_t>(), Svalr.as<double>(), st);
    DBuf Dpos = dalloc<double>(n1, st), Sdinv = dalloc<double>(n1, st), Sperm = dalloc<int32_t>(n1, st);
    CK(launch_gather_f64((int32_t)N, order.as<int32_t>(), fo.D.as<double>(), Dpos.as<double>(), st));
    CK(launch_dinv((int32_t)N, Dpos.as<double>(), Sdinv.as<double>(), st));
    CK(launch_gather_i32((int32_t)N, order.as<int32_t>(), ord.as<int32_t>(), Sperm.as<int32_t>(), st));
    DBuf Sval32, Svalr32;
    if (prec == 32) {
        Sval32 = dalloc<float>(z1, st); Svalr32 = dalloc<float>(z1, st);
        CK(launch_to_f32(Sval.as<double>(), Sval32.as<float>(), nnzF, st));
        CK(launch_to_f32(Svalr.as<double>(), Svalr32.as<float>(), nnzF, st));
    }
    CK(cudaStreamSynchronize(st));             // level histograms and longest rows on the host
    // the handles and their slices
    enum { A_FCP, A_FROW, A_FVAL, A_D, A_LEV, A_PERM, A_LP, A_LI, A_LV, A_SCP, A_SROW, A_SVAL, A_SRP, A_SCOL,
           A_SVALR, A_SDINV, A_SPERM, A_SVAL32, A_SVALR32, A_KINDS };
    std::vector<SplitSeg> seg((size_t)A_KINDS * count);
    int64_t zoff = 0, maxn = 0, maxf = 0, maxl = 0;
    for (int32_t s = 0; s < count; ++s) {
        const int64_t n = sys[(size_t)s].n, ob = sys[(size_t)s].obase, fo0 = f0[(size_t)s], nf = f0[(size_t)s + 1] - fo0;
        const int64_t nl = nnzL[(size_t)s];
        maxn = std::max(maxn, n + 1); maxf = std::max(maxf, nf); maxl = std::max(maxl, nl);
        std::unique_ptr<parac_factor_s> h(new parac_factor_s());
        cudaGetDevice(&h->device);
        h->n = n; h->prec = prec; h->spin_limit = O.o.spin_limit; h->sptrsv = O.o.sptrsv;
        h->check_every = O.o.check_every; h->stream = st;
        h->trsv_blocks = O.o.trsv_blocks; h->poll_ns = O.o.poll_ns; h->pcg_graph = O.o.pcg_graph;
        h->pcg_many = O.o.pcg_many; h->pcg_workers = O.o.pcg_workers; h->host_tables = O.o.host_tables == PARAC_ON;
        h->nnzF = nf; h->nnzL = nl;
        const size_t m1 = (size_t)std::max<int64_t>(n, 1), f1 = (size_t)std::max<int64_t>(nf, 1), l1 = (size_t)std::max<int64_t>(nl, 1);
        h->Fcp = dalloc<int64_t>((size_t)n + 1, st); h->Frow = dalloc<int32_t>(f1, st); h->Fval = dalloc<double>(f1, st);
        h->D = dalloc<double>(m1, st); h->Lev = dalloc<int32_t>(m1, st); h->perm = dalloc<int32_t>(m1, st);
        h->Lp = dalloc<int64_t>((size_t)n + 1, st); h->Li = dalloc<int32_t>(l1, st); h->Lv = dalloc<double>(l1, st);
        h->Scp = dalloc<int64_t>((size_t)n + 1, st); h->Srow = dalloc<int32_t>(f1, st); h->Sval = dalloc<double>(f1, st);
        h->Srp = dalloc<int64_t>((size_t)n + 1, st); h->Scol = dalloc<int32_t>(f1, st); h->Svalr = dalloc<double>(f1, st);
        h->Sdinv = dalloc<double>(m1, st); h->Sperm = dalloc<int32_t>(m1, st);
        if (prec == 32) { h->Sval32 = dalloc<float>(f1, st); h->Svalr32 = dalloc<float>(f1, st); }
        h->status = dalloc<int32_t>(1, st);
        auto at = [&](int k) -> SplitSeg & { return seg[(size_t)k * count + s]; };
        at(A_FCP) = {h->Fcp.p, n + 1, ob, -fo0};       at(A_FROW) = {h->Frow.p, nf, fo0, -ob};
        at(A_FVAL) = {h->Fval.p, nf, fo0, 0};         at(A_D) = {h->D.p, n, ob, 0};
        at(A_LEV) = {h->Lev.p, n, ob, 0};             at(A_PERM) = {h->perm.p, n, ob, -ob};
        at(A_LP) = {h->Lp.p, n + 1, ob, -zoff};        at(A_LI) = {h->Li.p, nl, zoff, -ob};
        at(A_LV) = {h->Lv.p, nl, zoff, 0};            at(A_SCP) = {h->Scp.p, n + 1, ob, -fo0};
        at(A_SROW) = {h->Srow.p, nf, fo0, -ob};       at(A_SVAL) = {h->Sval.p, nf, fo0, 0};
        at(A_SRP) = {h->Srp.p, n + 1, ob, -fo0};       at(A_SCOL) = {h->Scol.p, nf, fo0, -ob};
        at(A_SVALR) = {h->Svalr.p, nf, fo0, 0};       at(A_SDINV) = {h->Sdinv.p, n, ob, 0};
        at(A_SPERM) = {h->Sperm.p, n, ob, -ob};
        at(A_SVAL32) = {h->Sval32.p, prec == 32 ? nf : 0, fo0, 0};
        at(A_SVALR32) = {h->Svalr32.p, prec == 32 ? nf : 0, fo0, 0};
        zoff += nl;
        // level starts of the system's positions, depth and longest row / column
        const int32_t depth = (int32_t)(hoff[(size_t)s + 1] - hoff[(size_t)s]);
        h->depth = depth;
        h->lstart.assign((size_t)depth + 1, 0);
        for (int32_t l = 0; l < depth; ++l) h->lstart[(size_t)l + 1] = h->lstart[(size_t)l] + hh[(size_t)(hoff[(size_t)s] + l)];
        h->max_row = rm[(size_t)s];
        hs[(size_t)s] = std::move(h);
    }
    DBuf segd(sizeof(SplitSeg) * seg.size(), st);
    CK(cudaMemcpyAsync(segd.p, seg.data(), sizeof(SplitSeg) * seg.size(), cudaMemcpyHostToDevice, st));
    const SplitSeg *sd = segd.as<SplitSeg>();
    auto split = [&](int k, int64_t mx, int elem, bool fl, const void *src) {
        CK(launch_split(sd + (size_t)k * count, count, mx, elem, fl, src, st));
    };
    split(A_FCP, maxn, 8, false, fo.Fcp.p); split(A_FROW, maxf, 4, false, fo.Frow.p); split(A_FVAL, maxf, 8, true, fo.Fval.p);
    split(A_D, maxn, 8, true, fo.D.p); split(A_LEV, maxn, 4, false, fo.Lev.p); split(A_PERM, maxn, 4, false, ord.p);
    split(A_LP, maxn, 8, false, cp.p); split(A_LI, maxl, 4, false, ri.p); split(A_LV, maxl, 8, true, va.p);
    split(A_SCP, maxn, 8, false, Scp.p); split(A_SROW, maxf, 4, false, Srow.p); split(A_SVAL, maxf, 8, true, Sval.p);
    split(A_SRP, maxn, 8, false, Srp.p); split(A_SCOL, maxf, 4, false, Scol.p); split(A_SVALR, maxf, 8, true, Svalr.p);
    split(A_SDINV, maxn, 8, true, Sdinv.p); split(A_SPERM, maxn, 4, false, Sperm.p);
    if (prec == 32) { split(A_SVAL32, maxf, 4, true, Sval32.p); split(A_SVALR32, maxf, 4, true, Svalr32.p); }
    CK(cudaStreamSynchronize(st));             // every slice written before the global arrays are freed
    for (int32_t s = 0; s < count; ++s) {
        parac_factor_s *h = hs[(size_t)s].get();
        if (h->max_row > 4 * LONG_ROW_SINGLE) build_group_tables(h, st);
        h->stats = stats_json(h, fo, s);
    }
}

std::string stats_json(const parac_factor_s *h, const FactorOut &fo, int sys_index)
{
    char buf[3072];
    snprintf(buf, sizeof buf,
             "{\"n\": %lld, \"nnz_F\": %lld, \"nnz_G\": %lld, \"labels\": %lld, \"nnz_lower_input\": %lld, "
             "\"fill_entries\": %llu, \"pool_entries_used\": %llu, \"factor_entries_used\": %llu, "
             "\"scratch_bytes_used\": %llu, \"vertices_warp_path\": %llu, \"vertices_block_path\": %llu, "
             "\"vertices_global_path\": %llu, \"vertices_register_path\": %llu, \"handoffs\": %llu, "
             "\"queue_spins\": %llu, \"regrows\": %d, \"max_lower_column\": %d, \"blocks\": %d, "
             "\"warps_per_block\": %d, \"precision\": %d, \"samples\": %d, \"fill_store\": %d, \"system\": %d, \"t_ingest_ms\": %.4f, "
             "\"t_elim_ms\": %.4f, \"t_compact_ms\": %.4f, \"depth\": %d, \"max_row_F\": %d, \"cycles\": {\"wait\": %llu, "
             "\"gather\": %llu, \"sort_merge\": %llu, \"store_sort_scan\": %llu, \"sample_append\": %llu, "
             "\"release\": %llu, \"reg_weight_sort\": %llu, \"reg_scan\": %llu, \"coop_join\": %llu, "
             "\"coop_gather\": %llu, \"coop_row_sort\": %llu, \"coop_merge_store\": %llu, "
             "\"coop_weight_sort\": %llu, \"coop_scan\": %llu, \"coop_sample_append\": %llu, "
             "\"coop_release\": %llu}, \"grid_help_vertices\": %llu, \"grid_help_chunks_helpers\": %llu, "
             "\"grid_help_chunks_owner\": %llu, \"solve_groups\": [%d, %d, %d, %d]}",
             (long long)h->n, (long long)h->nnzF, (long long)(h->nnzF + h->n), (long long)fo.nl,
             (long long)fo.nnz_low, fo.stats[3], fo.pool_used, fo.f_used, fo.scratch_used, fo.stats[0], fo.stats[1],
             fo.stats[2], fo.stats[5], fo.stats[6], fo.stats[4], fo.regrows, fo.max_lower_column, fo.blocks, fo.warps, h->prec, fo.samples, fo.fill_store, sys_index, fo.t_ingest, fo.t_elim,
             fo.t_compact, h->depth, h->max_row, fo.stats[8], fo.stats[9], fo.stats[10], fo.stats[11], fo.stats[12],
             fo.stats[13], fo.stats[14], fo.stats[15], fo.stats[16], fo.stats[17], fo.stats[18], fo.stats[19],
             fo.stats[20], fo.stats[21], fo.stats[22], fo.stats[23], fo.stats[24], fo.stats[25], fo.stats[26], h->sng_f, h->sng_b,
             h->snslot_f, h->snslot_b);
    std::string out = buf;
    if (fo.stats[24] > 0 && (fo.stats[32] | fo.stats[33] | fo.stats[34]) != 0) {
        // grid-help step profile (timing >= 2): per step, the owner's post /
        // own chunks / wait cycles and the helpers' chunk cycles and count
        out.pop_back();
        out += ", \"grid_help_steps\": [";
        for (int op = 1; op <= 12; ++op) {
            char e[256];
            snprintf(e, sizeof e, "%s[%llu, %llu, %llu, %llu, %llu, %llu, %llu, %llu]", op > 1 ? ", " : "",
                     fo.stats[32 + 4 * (op - 1)], fo.stats[33 + 4 * (op - 1)], fo.stats[34 + 4 * (op - 1)],
                     fo.stats[35 + 4 * (op - 1)], fo.stats[80 + op], fo.stats[96 + op], fo.stats[112 + op],
                     fo.stats[128 + op]);
            out += e;
        }
        out += "]}";
    }
    return out;
}

template <typename F>
parac_status guarded(F &&f)
{
    try {
        g_err.clear();
        return f();
    } catch (const StatusFail &e) {
        if (g_err.empty()) g_err = parac_status_string(e.s);
        cudaGetLastError();
        return e.s;
    } catch (const CudaFail &e) {
        set_err("%s failed: %s", e.where, cudaGetErrorString(e.e));
        cudaGetLastError();
        return PARAC_ECUDA;
    } catch (const std::bad_alloc &) {
        set_err("host allocation failed");
        return PARAC_ENOMEM;
    }
}

bool check_csc_host(int64_t n, const int64_t *colptr)
{
    if (!colptr) return n == 0;
    if (is_device_ptr(colptr)) return true;   // checked by kernels
    if (colptr[0] != 0) return false;
    for (int64_t j = 0; j < n; ++j)
        if (colptr[j + 1] < colptr[j]) return false;
    return true;
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

void parac_opts_default(parac_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->kind = PARAC_KIND_AUTO;
    o->g_precision = 64;
    o->pool_mult = 0.0;
    o->max_pool_regrow = 2;
    o->spin_limit = 1ll << 24;
    o->warps_per_block = 8;
    o->queue_chunk = 1;
    o->check_every = 8;
    o->samples = 1;
}

const char *parac_status_string(parac_status s)
{
    switch (s) {
    case PARAC_OK: return "PARAC_OK";
    case PARAC_EINVAL: return "PARAC_EINVAL: invalid argument";
    case PARAC_ENOT_SDD: return "PARAC_ENOT_SDD: matrix is not a Laplacian/SDDM (sign or dominance)";
    case PARAC_ENOMEM: return "PARAC_ENOMEM: allocation failed";
    case PARAC_EPOOL: return "PARAC_EPOOL: fill workspace overflow";
    case PARAC_ETIMEOUT: return "PARAC_ETIMEOUT: device wait exceeded the spin limit";
    case PARAC_ECUDA: return "PARAC_ECUDA: CUDA runtime error";
    case PARAC_ENOCONV: return "PARAC_ENOCONV: PCG did not reach the tolerance";
    }
    return "unknown parac_status";
}

const char *parac_last_error(void) { return g_err.c_str(); }

uint64_t parac_kernel_launches(void) { return (uint64_t)parac::launch_count(); }

parac_status parac_factor(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                          const int32_t *ordering, uint64_t seed, const parac_opts *opts, parac_factor_t *out)
{
    if (out) *out = nullptr;
    return guarded([&]() -> parac_status {
        if (!out || n < 0 || n >= 0x7ffffffeLL) { set_err("bad n or out"); return PARAC_EINVAL; }
        if (n > 0 && (!colptr || !rowind || !val)) { set_err("null matrix array"); return PARAC_EINVAL; }
        if (!check_csc_host(n, colptr)) { set_err("colptr must start at 0 and be non-decreasing"); return PARAC_EINVAL; }
        Opts O = read_opts(opts);
        if (O.o.kind < 0 || O.o.kind > 2) { set_err("bad kind"); return PARAC_EINVAL; }
        set_mempool_keep();
        cudaStream_t st = O.st;
        std::unique_ptr<parac_factor_s> h(new parac_factor_s());
        cudaGetDevice(&h->device);
        h->n = n; h->prec = O.o.g_precision; h->spin_limit = O.o.spin_limit; h->sptrsv = O.o.sptrsv;
        h->check_every = O.o.check_every; h->stream = st;
        h->trsv_blocks = O.o.trsv_blocks; h->poll_ns = O.o.poll_ns; h->pcg_graph = O.o.pcg_graph;
        h->pcg_many = O.o.pcg_many; h->pcg_workers = O.o.pcg_workers; h->host_tables = O.o.host_tables == PARAC_ON;
        DView<int64_t> cp; cp.set(colptr, (size_t)n + 1, st);
        int64_t nnz = 0;
        if (n > 0) {
            if (is_device_ptr(colptr)) {
                CK(cudaMemcpyAsync(&nnz, colptr + n, 8, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            } else {
                nnz = colptr[n];
            }
        }
        h->nnzL = nnz;
        DView<int32_t> ri; ri.set(rowind, (size_t)nnz, st);
        DView<double> va; va.set(val, (size_t)nnz, st);
        if (O.o.order == PARAC_ORDER_NNZ && ordering) {
            set_err("an ordering array and order = PARAC_ORDER_NNZ exclude each other");
            return PARAC_EINVAL;
        }
        DView<int32_t> od; od.set(ordering, (size_t)n, st);
        DBuf nnz_ord;
        if (O.o.order == PARAC_ORDER_NNZ && n > 0) {     // Sec. V NNZ-sorted ordering, on the device
            nnz_ord = dalloc<int32_t>((size_t)n, st);
            DBuf tmp(nnz_order_tmp_bytes(n), st);
            CK(nnz_sorted_order(n, cp.p, nullptr, nullptr, 1, seed, nnz_ord.as<int32_t>(), tmp.p, st));
            od.p = nnz_ord.as<int32_t>();
        }
        std::vector<SysDesc> sys(1);
        sys[0].n = n; sys[0].obase = 0; sys[0].lbase = 0;
        sys[0].ground = O.o.kind == PARAC_KIND_LAPLACIAN ? -1 : (int32_t)n;
        FactorOut fo;
        if (n > 0) {
            run_factor(n, cp.p, ri.p, va.p, od.p, nullptr, sys, O.o.kind, seed, O, fo);
        } else {
            fo.Fcp = dalloc<int64_t>(1, st);
            CK(cudaMemsetAsync(fo.Fcp.p, 0, 8, st));
            fo.Frow = dalloc<int32_t>(1, st); fo.Fval = dalloc<double>(1, st); fo.D = dalloc<double>(1, st);
        }
        h->nnzF = fo.nnzF;
        h->Fcp = std::move(fo.Fcp); h->Frow = std::move(fo.Frow); h->Fval = std::move(fo.Fval); h->D = std::move(fo.D);
        h->Lev = std::move(fo.Lev);
        if (n == 0) h->Lev = dalloc<int32_t>(1, st);
        h->perm = dalloc<int32_t>(std::max<int64_t>(n, 1), st);
        if (od.p) copy_out(h->perm.p, od.p, 4 * (size_t)n, st);
        else CK(launch_iota_i32(h->perm.as<int32_t>(), n, 0, st));
        h->Lp = dalloc<int64_t>(n + 1, st); h->Li = dalloc<int32_t>(std::max<int64_t>(nnz, 1), st);
        h->Lv = dalloc<double>(std::max<int64_t>(nnz, 1), st);
        copy_out(h->Lp.p, cp.p, 8 * ((size_t)n + 1), st);
        copy_out(h->Li.p, ri.p, 4 * (size_t)nnz, st);
        copy_out(h->Lv.p, va.p, 8 * (size_t)nnz, st);
        finish_handle(h.get(), n, fo.nnzF, O);
        CK(cudaStreamSynchronize(st));
        h->stats = stats_json(h.get(), fo, 0);
        *out = h.release();
        return PARAC_OK;
    });
}

parac_status parac_factor_many(int32_t count, const parac_system *systems, uint64_t seed, const parac_opts *opts,
                               parac_factor_t *out)
{
    if (out && count > 0) for (int32_t s = 0; s < count; ++s) out[s] = nullptr;
    return guarded([&]() -> parac_status {
        if (count < 0 || (count > 0 && (!systems || !out))) { set_err("bad count/systems/out"); return PARAC_EINVAL; }
        if (count == 0) return PARAC_OK;
        Opts O = read_opts(opts);
        if (O.o.kind < 0 || O.o.kind > 2) { set_err("bad kind"); return PARAC_EINVAL; }
        set_mempool_keep();
        cudaStream_t st = O.st;
        std::vector<SysDesc> sys(count);
        std::vector<int64_t> nnz(count);
        int64_t N = 0, NNZ = 0, NL = 0;
        // entry counts: colptr[n] of every system, the device-resident ones read
        // by one gather kernel and one copy
        std::vector<const int64_t *> dptr;
        std::vector<int64_t> didx;
        std::vector<int32_t> dsys;
        for (int s = 0; s < count; ++s) {
            const parac_system &y = systems[s];
            if (y.n < 0 || (y.n > 0 && (!y.colptr || !y.rowind || !y.val))) { set_err("system %d: bad arrays", s); return PARAC_EINVAL; }
            if (!check_csc_host(y.n, y.colptr)) { set_err("system %d: bad colptr", s); return PARAC_EINVAL; }
            nnz[s] = 0;
            if (y.n > 0) {
                if (is_device_ptr(y.colptr)) { dptr.push_back(y.colptr); didx.push_back(y.n); dsys.push_back(s); }
                else nnz[s] = y.colptr[y.n];
            }
        }
        if (!dptr.empty()) {
            const int32_t m = (int32_t)dptr.size();
            DBuf pd = DBuf(sizeof(void *) * (size_t)m, st), id = dalloc<int64_t>((size_t)m, st), od = dalloc<int64_t>((size_t)m, st);
            CK(cudaMemcpyAsync(pd.p, dptr.data(), sizeof(void *) * (size_t)m, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(id.p, didx.data(), 8 * (size_t)m, cudaMemcpyHostToDevice, st));
            CK(launch_gather_ends((const int64_t *const *)pd.p, id.as<int64_t>(), m, od.as<int64_t>(), st));
            std::vector<int64_t> ends((size_t)m);
            CK(cudaMemcpyAsync(ends.data(), od.p, 8 * (size_t)m, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int32_t i = 0; i < m; ++i) nnz[(size_t)dsys[(size_t)i]] = ends[(size_t)i];
        }
        for (int s = 0; s < count; ++s) {
            const parac_system &y = systems[s];
            sys[s].n = y.n; sys[s].obase = N; sys[s].lbase = NL;
            sys[s].ground = O.o.kind == PARAC_KIND_LAPLACIAN ? -1 : (int32_t)(NL + y.n);
            N += y.n; NNZ += nnz[s]; NL += y.n + (sys[s].ground >= 0 ? 1 : 0);
        }
        if (NL >= 0x7fffffffLL) { set_err("batch too large for 32-bit labels"); return PARAC_EINVAL; }
        if (O.o.order == PARAC_ORDER_NNZ)
            for (int s = 0; s < count; ++s)
                if (systems[s].ordering) {
                    set_err("system %d: an ordering array and order = PARAC_ORDER_NNZ exclude each other", s);
                    return PARAC_EINVAL;
                }
        // concatenated device input with global indices: one segmented copy per
        // array (host inputs are staged to the device first; a system without
        // an ordering takes the shared 0, 1, 2, ... array)
        DBuf cp = dalloc<int64_t>(N + 1, st), ri = dalloc<int32_t>(std::max<int64_t>(NNZ, 1), st),
             va = dalloc<double>(std::max<int64_t>(NNZ, 1), st), ord = dalloc<int32_t>(std::max<int64_t>(N, 1), st),
             lab = dalloc<int32_t>(std::max<int64_t>(N, 1), st);
        int64_t maxn = 1, maxz = 1;
        for (int s = 0; s < count; ++s) { maxn = std::max(maxn, sys[s].n); maxz = std::max(maxz, nnz[s]); }
        DBuf iota = dalloc<int32_t>((size_t)maxn, st);
        CK(launch_iota_i32(iota.as<int32_t>(), maxn, 0, st));
        enum { K_CP, K_RI, K_VA, K_ORD, K_LAB, K_KINDS };
        std::vector<CatSeg> cs((size_t)K_KINDS * count);
        std::vector<DView<int64_t>> vc(count);
        std::vector<DView<int32_t>> vr(count), vo(count);
        std::vector<DView<double>> vv(count);
        int64_t zb = 0;
        for (int s = 0; s < count; ++s) {
            const parac_system &y = systems[s];
            const int64_t n = y.n, ob = sys[s].obase;
            vc[s].set(y.colptr, (size_t)n + 1, st); vr[s].set(y.rowind, (size_t)nnz[s], st);
            vv[s].set(y.val, (size_t)nnz[s], st); vo[s].set(y.ordering, (size_t)n, st);
            auto at = [&](int k) -> CatSeg & { return cs[(size_t)k * count + s]; };
            at(K_CP) = {vc[s].p, n, ob, zb};
            at(K_RI) = {vr[s].p, nnz[s], zb, ob};
            at(K_VA) = {vv[s].p, nnz[s], zb, 0};
            at(K_ORD) = {vo[s].p ? (const void *)vo[s].p : (const void *)iota.p, n, ob, ob};
            at(K_LAB) = {iota.p, n, ob, sys[s].lbase};
            zb += nnz[s];
        }
        DBuf csd(sizeof(CatSeg) * cs.size(), st);
        CK(cudaMemcpyAsync(csd.p, cs.data(), sizeof(CatSeg) * cs.size(), cudaMemcpyHostToDevice, st));
        const CatSeg *cd = csd.as<CatSeg>();
        CK(launch_cat(cd + (size_t)K_CP * count, count, maxn, 8, false, cp.p, st));
        CK(launch_cat(cd + (size_t)K_RI * count, count, maxz, 4, false, ri.p, st));
        CK(launch_cat(cd + (size_t)K_VA * count, count, maxz, 8, true, va.p, st));
        CK(launch_cat(cd + (size_t)K_ORD * count, count, maxn, 4, false, ord.p, st));
        CK(launch_cat(cd + (size_t)K_LAB * count, count, maxn, 4, false, lab.p, st));
        const int64_t total = zb;
        CK(cudaMemcpyAsync(cp.as<int64_t>() + N, &total, 8, cudaMemcpyHostToDevice, st));
        if (O.o.order == PARAC_ORDER_NNZ && N > 0) {     // every system's NNZ-sorted ordering at once
            std::vector<int32_t> ob_h((size_t)count);
            for (int s = 0; s < count; ++s) ob_h[(size_t)s] = (int32_t)sys[s].obase;
            DBuf obase = dalloc<int32_t>((size_t)count, st), sys_of_v = dalloc<int32_t>((size_t)N, st);
            CK(cudaMemcpyAsync(obase.p, ob_h.data(), 4 * (size_t)count, cudaMemcpyHostToDevice, st));
            CK(launch_sys_of_label(count, obase.as<int32_t>(), (int32_t)N, sys_of_v.as<int32_t>(), st));
            DBuf tmp(nnz_order_tmp_bytes(N), st);
            CK(nnz_sorted_order(N, cp.as<int64_t>(), sys_of_v.as<int32_t>(), obase.as<int32_t>(), count, seed,
                                ord.as<int32_t>(), tmp.p, st));
            CK(cudaStreamSynchronize(st));
        }
        FactorOut fo;
        run_factor(N, cp.as<int64_t>(), ri.as<int32_t>(), va.as<double>(), ord.as<int32_t>(), lab.as<int32_t>(), sys,
                   O.o.kind, seed, O, fo);
        std::vector<std::unique_ptr<parac_factor_s>> hs(count);
        finish_batch(hs, fo, sys, nnz, cp, ri, va, ord, O);
        CK(cudaStreamSynchronize(st));
        for (int s = 0; s < count; ++s) out[s] = hs[s].release();
        return PARAC_OK;
    });
}

parac_status parac_factor_export(parac_factor_t G, int64_t *nnz, int64_t *colptr, int32_t *rowind, double *Fval,
                                 double *D)
{
    return guarded([&]() -> parac_status {
        if (!G || !nnz) { set_err("null handle or nnz"); return PARAC_EINVAL; }
        *nnz = G->nnzF;
        if (!colptr) return PARAC_OK;
        if (!rowind || !Fval || !D) { set_err("null output array"); return PARAC_EINVAL; }
        cudaStream_t st = G->stream;
        copy_out(colptr, G->Fcp.p, 8 * ((size_t)G->n + 1), st);
        copy_out(rowind, G->Frow.p, 4 * (size_t)G->nnzF, st);
        copy_out(Fval, G->Fval.p, 8 * (size_t)G->nnzF, st);
        copy_out(D, G->D.p, 8 * (size_t)G->n, st);
        CK(cudaStreamSynchronize(st));
        return PARAC_OK;
    });
}

parac_status parac_factor_stats(parac_factor_t G, char *json, size_t cap)
{
    if (!G || !json) { g_err = "null handle or buffer"; return PARAC_EINVAL; }
    if (G->stats.size() + 1 > cap) { g_err = "buffer too small"; return PARAC_EINVAL; }
    std::memcpy(json, G->stats.c_str(), G->stats.size() + 1);
    return PARAC_OK;
}

void parac_factor_free(parac_factor_t G)
{
    if (!G) return;
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = G->device;
    cudaStream_t st = G->stream;
    if (cur != dev) cudaSetDevice(dev);
    delete G;
    cudaStreamSynchronize(st);
    if (cur != dev) cudaSetDevice(cur);
}

}  // extern "C"

// ------------------------------------------------------------------ solve
namespace {

// Set by parac_pcg_many for its worker threads: the stream the worker's
// solves are ordered on (instead of the handle's) and the number of solves
// that run at once, which share the resident-block capacity -- the solve
// kernels need their whole grid resident, so concurrent solves together must
// fit on the GPU.
thread_local cudaStream_t t_stream_override = nullptr;
thread_local int t_grid_share = 0;
thread_local bool t_no_graph = false;     // one-shot solves: capturing would cost more than it saves

// Cap of the solves' polling back-off (parac_opts.poll_ns): 64 ns measured
// best on the 128^3 grid with a warp per row (266 ms PCG vs 271 at 256 ns and
// 319 at 1024); the SDDM batch is indifferent.

// Table of the hybrid solves (schedule.h, hybrid_table), built on a handle's
// first single-system solve: a level with more rows than the solve grid has
// warps is cut into runs of at most 32 rows (a lane per row), a narrower one
// lists its rows (a warp per row); O(depth + n / 32 + rows of narrow levels)
// host work on the level starts.
void ensure_tpr_table(parac_factor_s *h)
{
    if (h->tpr_tried || h->n <= 0) return;
    h->tpr_tried = true;
    if (h->max_row > TPR_MAX_ROW || h->sng_f > 0 || (int64_t)h->lstart.size() != (int64_t)h->depth + 1) return;
    const int64_t blocks = h->trsv_blocks > 0 ? h->trsv_blocks : (int64_t)num_sms();
    const std::vector<int32_t> t = hybrid_table({BatchSysLevels{0, 0, h->lstart, nullptr}}, blocks * (TPR_THREADS / 32));
    h->tpr_chunks = DBuf(4 * std::max<size_t>(t.size(), 2), h->stream);
    CK(cudaMemcpyAsync(h->tpr_chunks.p, t.data(), 4 * t.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->ntpr = (int32_t)(t.size() / 2);
}

SolveArgs solve_args(parac_factor_s *G, const int64_t *Lp, const int32_t *Li, const double *Lv, int64_t nnzL)
{
    SolveArgs A{};
    A.n = (int32_t)G->n;
    A.Lp = Lp; A.Li = Li; A.Lv = Lv;
    A.Fcp = G->Scp.as<int64_t>(); A.Frow = G->Srow.as<int32_t>(); A.Fval64 = G->Sval.as<double>();
    A.Fval32 = G->Sval32.as<float>();
    A.Frp = G->Srp.as<int64_t>(); A.Fcol = G->Scol.as<int32_t>(); A.Fvalr64 = G->Svalr.as<double>();
    A.Fvalr32 = G->Svalr32.as<float>();
    A.Dinv = G->Sdinv.as<double>(); A.operm = G->Sperm.as<int32_t>();
    A.prec = G->prec;
    const double n = G->n > 0 ? (double)G->n : 1.0;
    A.lanes_spmv = lanes_for((double)nnzL / n);
    // one row per warp unless the handle asks for sub-warp rows
    A.lanes_trsv = G->sptrsv == PARAC_SPTRSV_SUB8 ? 8 : G->sptrsv == PARAC_SPTRSV_SUB4 ? 4 : 32;
    A.trsv_warps = SOLVE_WARPS;
    int bps = 0;
    trsv_configure(A.lanes_trsv, A.trsv_warps, &bps, A.prec);
    if (bps < 1) bps = 1;
    int max_blocks = num_sms() * bps;            // all co-resident: required by the static schedule
    if (t_grid_share > 1) max_blocks = std::max(1, max_blocks / t_grid_share);
    A.trsv_blocks = max_blocks;
    // Grid sized to the dependency frontier: about two average levels of rows
    // in flight, so that waiting rows do not flood the memory system with polls.
    if (G->depth > 0) {
        const int64_t rows_per_block = (int64_t)A.trsv_warps * (32 / A.lanes_trsv);
        const int64_t want = (2 * G->n / G->depth + rows_per_block - 1) / rows_per_block;
        A.trsv_blocks = (int)std::max<int64_t>(std::min<int64_t>(num_sms(), max_blocks),
                                               std::min<int64_t>(max_blocks, want));
    }
    if (G->trsv_blocks > 0) A.trsv_blocks = std::max(1, std::min(max_blocks, G->trsv_blocks));
    set_poll_backoff((unsigned)G->poll_ns);
    const int64_t rows_per_group = (int64_t)A.trsv_warps * (32 / A.lanes_trsv);
    const int64_t groups = (G->n + rows_per_group - 1) / rows_per_group;
    if (groups < A.trsv_blocks) A.trsv_blocks = (int)std::max<int64_t>(groups, 1);
    // the hybrid solves (THREAD, and AUTO) when no row or column is long
    if (G->sptrsv == PARAC_SPTRSV_THREAD || G->sptrsv == PARAC_SPTRSV_AUTO) ensure_tpr_table(G);
    const bool tpr = G->ntpr > 0 && G->sng_f == 0 &&
                     (G->sptrsv == PARAC_SPTRSV_THREAD || G->sptrsv == PARAC_SPTRSV_AUTO);
    if (tpr) {
        const int tb = std::max(1, tpr_blocks_per_sm(A.prec));
        const int64_t tmax = std::max<int64_t>(1, (int64_t)num_sms() * tb / std::max(1, t_grid_share));  // all co-resident
        const int64_t wpb = TPR_THREADS / 32;
        // one block of 8 warps per SM: measured best on the 128^3 grid (FP64
        // apply 3.45 ms against 3.86 with 1.5 blocks and 4.13 with 2 per SM)
        int64_t want = num_sms();
        if (G->trsv_blocks > 0) want = G->trsv_blocks;
        want = std::min<int64_t>(want, ((int64_t)G->ntpr + wpb - 1) / wpb);
        A.tpr_blocks = (int32_t)std::max<int64_t>(1, std::min<int64_t>(tmax, want));
        A.tpr_chunks = (const int2 *)G->tpr_chunks.p;
        A.ntpr = G->ntpr;
    }
    A.spin_limit = G->spin_limit;
    A.status = G->status.as<int32_t>();
    if (G->sng_f > 0 && A.lanes_trsv == 32 && A.trsv_warps == SOLVE_WARPS) {
        A.gt_f = (const int4 *)G->sgt_f.p; A.ng_f = G->sng_f;
        A.gt_b = (const int4 *)G->sgt_b.p; A.ng_b = G->sng_b;
        A.part_f = G->spart_f.p; A.nslot_f = G->snslot_f;
        A.part_b = G->spart_b.p; A.nslot_b = G->snslot_b;
    }
    return A;
}

void ensure_cache(parac_factor_s *G, const SolveArgs &A, cudaStream_t st)
{
    SolveCache &c = G->cache;
    if (c.n == (int32_t)G->n && c.B.vec_blocks > 0 && c.B.pstride >= A.trsv_blocks) return;
    const size_t n = (size_t)std::max<int64_t>(G->n, 1);
    c.x = dalloc<double>(n, st); c.r = dalloc<double>(n, st); c.z = dalloc<double>(n, st);
    c.p = dalloc<double>(n, st); c.q = dalloc<double>(n, st); c.b = dalloc<double>(n, st);
    if (G->prec == 32) { c.y32 = dalloc<float>(n, st); c.zl32 = dalloc<float>(n, st); }
    else { c.y64 = dalloc<double>(n, st); c.zl64 = dalloc<double>(n, st); }
    int vb = (int)std::min<int64_t>((G->n + 255) / 256, (int64_t)num_sms() * 8);
    if (vb < 1) vb = 1;
    const int pstride = std::max(vb, A.trsv_blocks);
    c.partials = dalloc<double>((size_t)3 * pstride, st);
    c.state = DBuf(pcg_state_bytes(), st);
    c.B.x = c.x.as<double>(); c.B.r = c.r.as<double>(); c.B.z = c.z.as<double>(); c.B.p = c.p.as<double>();
    c.B.q = c.q.as<double>(); c.B.b = c.b.as<double>();
    c.B.yl64 = c.y64.as<double>(); c.B.zl64 = c.zl64.as<double>(); c.B.yl32 = c.y32.as<float>(); c.B.zl32 = c.zl32.as<float>();
    c.B.partials = c.partials.as<double>(); c.B.state = c.state.as<PcgState>();
    c.B.vec_blocks = vb; c.B.pstride = pstride;
    c.n = (int32_t)G->n;
}

int32_t read_dev_status(parac_factor_s *G, cudaStream_t st)
{
    int32_t s = 0;
    CK(cudaMemcpyAsync(&s, G->status.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return s;
}

void ensure_block_cache(parac_factor_s *G, const SolveArgs &A, int nrhs, cudaStream_t st)
{
    BlockCache &c = G->bcache;
    int vb = (int)std::min<int64_t>((G->n * 32 + 255) / 256, (int64_t)num_sms() * 8);
    if (vb < 1) vb = 1;
    const int pstride = std::max(vb, A.trsv_blocks);
    if (c.n == (int32_t)G->n && c.nrhs == nrhs && c.prec == G->prec && c.pstride >= pstride) return;
    const size_t m = (size_t)std::max<int64_t>(G->n, 1) * nrhs;
    c.x = dalloc<double>(m, st); c.r = dalloc<double>(m, st); c.z = dalloc<double>(m, st);
    c.p = dalloc<double>(m, st); c.q = dalloc<double>(m, st); c.b = dalloc<double>(m, st);
    if (G->prec == 32) { c.y = dalloc<float>(m, st); c.zl = dalloc<float>(m, st); }
    else { c.y = dalloc<double>(m, st); c.zl = dalloc<double>(m, st); }
    c.partials = dalloc<double>((size_t)3 * 32 * pstride, st);
    c.state = DBuf(block_state_bytes(), st);
    BlockBuffers &B = c.B;
    B = BlockBuffers{};
    B.x = c.x.as<double>(); B.r = c.r.as<double>(); B.z = c.z.as<double>(); B.p = c.p.as<double>();
    B.q = c.q.as<double>(); B.b = c.b.as<double>();
    if (G->prec == 32) { B.yl32 = c.y.as<float>(); B.zl32 = c.zl.as<float>(); }
    else { B.yl64 = c.y.as<double>(); B.zl64 = c.zl.as<double>(); }
    B.partials = c.partials.as<double>();
    B.state = (BlockState *)c.state.p;
    B.nrhs = nrhs; B.vec_blocks = vb; B.pstride = pstride;
    c.n = (int32_t)G->n; c.nrhs = nrhs; c.prec = G->prec; c.pstride = pstride;
}

// Row groups of the block triangular solves, built once per handle (and
// warps per block) from the relabelled factor's row and column pointers.
void ensure_block_groups(parac_factor_s *G, int warps, cudaStream_t st)
{
    BlockCache &c = G->bcache;
    if (c.g_warps != warps && !G->host_tables) {         // built on the device
        const int64_t n = G->n;
        DBuf tmp(row_groups_tmp_bytes(n), st);
        int64_t ngf = 0, nsf = 0, ngb = 0, nsb = 0;
        CK(row_groups_count(G->Srp.as<int64_t>(), n, false, warps, LONG_ROW_BLOCK, SPLIT_ROW_BLOCK, CHUNK_BLOCK, tmp.p,
                            &ngf, &nsf, st));
        c.gt_f = dalloc<int32_t>((size_t)(4 * ngf), st);
        CK(row_groups_write(G->Srp.as<int64_t>(), n, false, warps, SPLIT_ROW_BLOCK, CHUNK_BLOCK, tmp.p,
                            c.gt_f.as<int32_t>(), st));
        CK(row_groups_count(G->Scp.as<int64_t>(), n, true, warps, LONG_ROW_BLOCK, SPLIT_ROW_BLOCK, CHUNK_BLOCK, tmp.p,
                            &ngb, &nsb, st));
        c.gt_b = dalloc<int32_t>((size_t)(4 * ngb), st);
        CK(row_groups_write(G->Scp.as<int64_t>(), n, true, warps, SPLIT_ROW_BLOCK, CHUNK_BLOCK, tmp.p,
                            c.gt_b.as<int32_t>(), st));
        c.part_f = dalloc<double>((size_t)std::max<int64_t>(nsf, 1) * 32, st);
        c.part_b = dalloc<double>((size_t)std::max<int64_t>(nsb, 1) * 32, st);
        CK(cudaStreamSynchronize(st));
        c.ng_f = (int32_t)ngf; c.ng_b = (int32_t)ngb;
        c.nslot_f = (int32_t)nsf; c.nslot_b = (int32_t)nsb;
        c.g_warps = warps;
    } else if (c.g_warps != warps) {                     // the host builder
        const size_t n = (size_t)G->n;
        std::vector<int64_t> rp(n + 1), cp(n + 1);
        CK(cudaMemcpyAsync(rp.data(), G->Srp.p, 8 * (n + 1), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(cp.data(), G->Scp.p, 8 * (n + 1), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const GroupTable gf = row_groups(rp, false, warps, LONG_ROW_BLOCK, SPLIT_ROW_BLOCK, CHUNK_BLOCK),
                         gb = row_groups(cp, true, warps, LONG_ROW_BLOCK, SPLIT_ROW_BLOCK, CHUNK_BLOCK);
        c.gt_f = dalloc<int32_t>(gf.g.size(), st);
        c.gt_b = dalloc<int32_t>(gb.g.size(), st);
        CK(cudaMemcpyAsync(c.gt_f.p, gf.g.data(), 4 * gf.g.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c.gt_b.p, gb.g.data(), 4 * gb.g.size(), cudaMemcpyHostToDevice, st));
        c.part_f = dalloc<double>((size_t)std::max(gf.nslots, 1) * 32, st);
        c.part_b = dalloc<double>((size_t)std::max(gb.nslots, 1) * 32, st);
        CK(cudaStreamSynchronize(st));       // the host vectors go out of scope
        c.ng_f = gf.ngroups; c.ng_b = gb.ngroups;
        c.nslot_f = gf.nslots; c.nslot_b = gb.nslots;
        c.g_warps = warps;
    }
    c.B.gt_f = (const int4 *)c.gt_f.p; c.B.gt_b = (const int4 *)c.gt_b.p;
    c.B.ng_f = c.ng_f; c.B.ng_b = c.ng_b;
    c.B.part_f = c.part_f.p; c.B.part_b = c.part_b.p;
    c.B.nslot_f = c.nslot_f; c.B.nslot_b = c.nslot_b;
}

// The library's own solve stream for this handle, made to wait for the work
// already queued on the calling stream st (the handle's, or a worker's of
// parac_pcg_many) and on the handle's stream.
cudaStream_t enter_solve_stream(parac_factor_s *G, cudaStream_t st)
{
    SolveStream &ss = G->sstream;
    if (!ss.s) {
        CK(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ss.in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ss.out, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ss.h, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(ss.in, st));
    CK(cudaStreamWaitEvent(ss.s, ss.in, 0));
    if (st != G->stream) {                   // the cached work space was made on the handle's stream
        CK(cudaEventRecord(ss.h, G->stream));
        CK(cudaStreamWaitEvent(ss.s, ss.h, 0));
    }
    return ss.s;
}

// ... and the calling stream made to wait for the solve stream's work.
void leave_solve_stream(parac_factor_s *G, cudaStream_t st)
{
    SolveStream &ss = G->sstream;
    CK(cudaEventRecord(ss.out, ss.s));
    CK(cudaStreamWaitEvent(st, ss.out, 0));
}

bool graphs_enabled(const parac_factor_s *G)
{
    return !t_no_graph && G->pcg_graph != PARAC_OFF;
}

// Run `iters` iterations given by `launch(stream)`: replay the cached graph
// if its key matches, else capture a new one (or launch directly when graphs
// are switched off).
template <class Launch>
cudaError_t run_iterations(parac_factor_s *G, const uint64_t (&key)[GraphCache::KEY], Launch &&launch,
                           cudaStream_t ps)
{
    if (!graphs_enabled(G)) return launch(ps);
    GraphCache &gc = G->graph;
    if (!gc.exec || memcmp(gc.key, key, sizeof key) != 0) {
        gc.reset();
        cudaGraph_t g = nullptr;
        unsigned long long nk = 0;
        cudaError_t e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        capture_launch_counts(&nk);
        const cudaError_t le = launch(ps);
        capture_launch_counts(nullptr);
        e = cudaStreamEndCapture(ps, &g);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return le != cudaSuccess ? le : e;
        }
        e = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { gc.exec = nullptr; return e; }
        memcpy(gc.key, key, sizeof key);
        gc.launches = nk;
    }
    cudaError_t e = cudaGraphLaunch(gc.exec, ps);
    if (e == cudaSuccess) count_graph_launches(gc.launches);
    return e;
}

void graph_key(uint64_t (&k)[GraphCache::KEY], const SolveArgs &A, int form, int nrhs, int iters, const void *x,
               const void *y, const void *partials, const void *state, int vec_blocks, int pstride)
{
    memset(k, 0, sizeof k);
    int i = 0;
    k[i++] = (uint64_t)form; k[i++] = (uint64_t)nrhs; k[i++] = (uint64_t)iters;
    k[i++] = (uint64_t)(uintptr_t)A.Lp; k[i++] = (uint64_t)(uintptr_t)A.Li; k[i++] = (uint64_t)(uintptr_t)A.Lv;
    k[i++] = (uint64_t)(uintptr_t)A.Fcp; k[i++] = (uint64_t)(uintptr_t)A.Frp;
    k[i++] = (uint64_t)A.n; k[i++] = (uint64_t)A.prec; k[i++] = (uint64_t)A.lanes_spmv; k[i++] = (uint64_t)A.lanes_trsv;
    k[i++] = (uint64_t)A.trsv_blocks; k[i++] = (uint64_t)A.trsv_warps; k[i++] = (uint64_t)A.spin_limit;
    k[i++] = (uint64_t)(uintptr_t)A.status;
    k[i++] = (uint64_t)(uintptr_t)x; k[i++] = (uint64_t)(uintptr_t)y; k[i++] = (uint64_t)(uintptr_t)partials;
    k[i++] = (uint64_t)(uintptr_t)state; k[i++] = (uint64_t)vec_blocks; k[i++] = (uint64_t)pstride;
}

// One right-hand side: B, X are n-vectors on the device.
parac_status pcg_single(parac_factor_s *G, const SolveArgs &A, const double *b, double *x, double tol, int32_t maxit,
                        cudaStream_t ps, int32_t *iters, double *relres, bool *converged)
{
    PcgBuffers &Bf = G->cache.B;
    CK(cudaMemcpyAsync(Bf.b, b, 8 * (size_t)A.n, cudaMemcpyDeviceToDevice, ps));
    CK(pcg_init(A, Bf, tol, maxit, ps));
    uint64_t key[GraphCache::KEY];
    graph_key(key, A, 1, 1, G->check_every, Bf.x, Bf.yl64 ? (const void *)Bf.yl64 : (const void *)Bf.yl32,
              Bf.partials, Bf.state, Bf.vec_blocks, Bf.pstride);
    const int every = G->check_every;
    auto step = [&](cudaStream_t s) -> cudaError_t {
        for (int c = 0; c < every; ++c) {
            cudaError_t e = pcg_iteration(A, Bf, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    PcgHostState hs{};
    for (;;) {
        CK(run_iterations(G, key, step, ps));
        CK(pcg_read_state(Bf, &hs, ps));
        if (read_dev_status(G, ps) != ST_OK) return PARAC_ETIMEOUT;
        if (!hs.done) continue;
        CK(pcg_true_residual(A, Bf, ps));
        CK(pcg_read_state(Bf, &hs, ps));
        const bool ok = hs.true_rr <= tol * tol * hs.bb;
        if (ok || hs.iters >= maxit || hs.bb == 0.0) break;
        CK(pcg_clear_done(Bf, ps));
        CK(pcg_resume(A, Bf, ps));
    }
    if (read_dev_status(G, ps) != ST_OK) return PARAC_ETIMEOUT;
    CK(cudaMemcpyAsync(x, Bf.x, 8 * (size_t)A.n, cudaMemcpyDeviceToDevice, ps));
    *iters = hs.iters;
    *relres = hs.bb > 0.0 ? std::sqrt(hs.true_rr / hs.bb) : 0.0;
    *converged = hs.true_rr <= tol * tol * hs.bb || hs.bb == 0.0;
    return PARAC_OK;
}

// Several right-hand sides: Bcm / Xcm are device n x nrhs column-major with
// leading dimensions ldb / ldx.
parac_status pcg_block(parac_factor_s *G, SolveArgs A, int nrhs, const double *Bcm, int64_t ldb, double *Xcm,
                       int64_t ldx, double tol, int32_t maxit, cudaStream_t st, cudaStream_t ps, int32_t *iters,
                       double *relres, bool *all_conv)
{
    // the SpTRSM kernels' own co-residency bound
    const int bps = std::max(1, btrsm_blocks_per_sm(A.trsv_warps, A.prec));
    A.trsv_blocks = std::min(A.trsv_blocks, std::max(1, num_sms() * bps / std::max(1, t_grid_share)));
    ensure_block_cache(G, A, nrhs, G->stream);
    ensure_block_groups(G, A.trsv_warps, G->stream);
    const BlockBuffers &B = G->bcache.B;
    CK(bpack((int32_t)A.n, nrhs, Bcm, ldb, B.b, ps));
    CK(bpcg_init(A, B, tol, maxit, ps));
    uint64_t key[GraphCache::KEY];
    graph_key(key, A, 2, nrhs, G->check_every, B.x, B.yl64 ? (const void *)B.yl64 : (const void *)B.yl32,
              B.partials, B.state, B.vec_blocks, B.pstride);
    const int every = G->check_every;
    auto step = [&](cudaStream_t s) -> cudaError_t {
        for (int c = 0; c < every; ++c) {
            cudaError_t e = bpcg_iteration(A, B, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    BlockHostState hs{};
    for (;;) {
        CK(run_iterations(G, key, step, ps));
        CK(bpcg_read_state(B, &hs, ps));
        if (read_dev_status(G, ps) != ST_OK) return PARAC_ETIMEOUT;
        if (!hs.all_done) continue;
        CK(bpcg_true_residual(A, B, ps));
        CK(bpcg_read_state(B, &hs, ps));
        bool reopen = false;
        for (int j = 0; j < nrhs; ++j)
            if (hs.converged[j] && !(hs.true_rr[j] <= tol * tol * hs.bb[j]) && hs.iters[j] < maxit) reopen = true;
        if (!reopen) break;
        CK(bpcg_reopen(A, B, ps));
    }
    if (read_dev_status(G, ps) != ST_OK) return PARAC_ETIMEOUT;
    CK(bunpack((int32_t)A.n, nrhs, B.x, Xcm, ldx, ps));
    *all_conv = true;
    for (int j = 0; j < nrhs; ++j) {
        iters[j] = hs.iters[j];
        relres[j] = hs.bb[j] > 0.0 ? std::sqrt(hs.true_rr[j] / hs.bb[j]) : 0.0;
        if (!(hs.true_rr[j] <= tol * tol * hs.bb[j]) && hs.bb[j] > 0.0) *all_conv = false;
    }
    return PARAC_OK;
}

}  // namespace

extern "C" parac_status parac_pcg(parac_factor_t G, int64_t n, const int64_t *colptr, const int32_t *rowind,
                                  const double *val, const double *B, int32_t nrhs, int64_t ldb, double tol,
                                  int32_t maxit, double *X, int64_t ldx, int32_t *iters, double *true_relres)
{
    return guarded([&]() -> parac_status {
        if (!G || n != G->n || nrhs < 1 || nrhs > 32 || (n > 0 && (!B || !X)) || ldb < n || ldx < n || maxit < 0) {
            set_err("bad arguments to parac_pcg");
            return PARAC_EINVAL;
        }
        cudaStream_t st = t_stream_override ? t_stream_override : G->stream;
        DView<int64_t> cp; DView<int32_t> ri; DView<double> va;
        const int64_t *Lp = G->Lp.as<int64_t>();
        const int32_t *Li = G->Li.as<int32_t>();
        const double *Lv = G->Lv.as<double>();
        int64_t nnzL = G->nnzL;
        if (colptr) {
            if (!rowind || !val) { set_err("null matrix array"); return PARAC_EINVAL; }
            if (!check_csc_host(n, colptr)) { set_err("bad colptr"); return PARAC_EINVAL; }
            cp.set(colptr, (size_t)n + 1, st);
            if (is_device_ptr(colptr)) {
                CK(cudaMemcpyAsync(&nnzL, colptr + n, 8, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            } else nnzL = colptr[n];
            ri.set(rowind, (size_t)nnzL, st);
            va.set(val, (size_t)nnzL, st);
            Lp = cp.p; Li = ri.p; Lv = va.p;
        }
        if (n == 0) {
            for (int j = 0; j < nrhs; ++j) { if (iters) iters[j] = 0; if (true_relres) true_relres[j] = 0.0; }
            return PARAC_OK;
        }
        SolveArgs A = solve_args(G, Lp, Li, Lv, nnzL);
        const bool bdev = is_device_ptr(B), xdev = is_device_ptr(X);
        // right-hand sides and solutions on the device, column-major
        DBuf Bstage, Xstage;
        const double *Bd = B;
        double *Xd = X;
        int64_t ldbd = ldb, ldxd = ldx;
        if (!bdev) {
            Bstage = dalloc<double>((size_t)n * nrhs, st);
            CK(cudaMemcpy2DAsync(Bstage.p, 8 * (size_t)n, B, 8 * (size_t)ldb, 8 * (size_t)n, (size_t)nrhs,
                                 cudaMemcpyHostToDevice, st));
            Bd = Bstage.as<double>(); ldbd = n;
        }
        if (!xdev) { Xstage = dalloc<double>((size_t)n * nrhs, st); Xd = Xstage.as<double>(); ldxd = n; }
        CK(cudaMemsetAsync(G->status.p, 0, 4, st));
        std::vector<int32_t> it(nrhs, 0);
        std::vector<double> rel(nrhs, 0.0);
        bool all_conv = true;
        parac_status rs = PARAC_OK;
        if (nrhs == 1) {
            ensure_cache(G, A, G->stream);        // cached work space lives on the handle's stream
            cudaStream_t ps = enter_solve_stream(G, st);
            bool conv = true;
            rs = pcg_single(G, A, Bd, Xd, tol, maxit, ps, &it[0], &rel[0], &conv);
            all_conv = conv;
            leave_solve_stream(G, st);
        } else {
            cudaStream_t ps = nullptr;
            {
                // buffers are allocated on the handle's stream before the join
                const int bps = std::max(1, btrsm_blocks_per_sm(A.trsv_warps, A.prec));
                SolveArgs Ab = A;
                Ab.trsv_blocks = std::min(A.trsv_blocks, std::max(1, num_sms() * bps / std::max(1, t_grid_share)));
                ensure_block_cache(G, Ab, nrhs, G->stream);
                ensure_block_groups(G, A.trsv_warps, G->stream);
            }
            ps = enter_solve_stream(G, st);
            rs = pcg_block(G, A, nrhs, Bd, ldbd, Xd, ldxd, tol, maxit, st, ps, it.data(), rel.data(), &all_conv);
            leave_solve_stream(G, st);
        }
        if (rs == PARAC_ETIMEOUT) {
            CK(cudaStreamSynchronize(st));
            set_err("triangular solve wait exceeded the spin limit");
            return PARAC_ETIMEOUT;
        }
        if (!xdev)
            CK(cudaMemcpy2DAsync(X, 8 * (size_t)ldx, Xd, 8 * (size_t)n, 8 * (size_t)n, (size_t)nrhs,
                                 cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int j = 0; j < nrhs; ++j) {
            if (iters) iters[j] = it[j];
            if (true_relres) true_relres[j] = rel[j];
        }
        if (!all_conv) { set_err("PCG reached maxit"); return PARAC_ENOCONV; }
        return PARAC_OK;
    });
}

namespace {

// ------------------------------------------------------------------ batched PCG
// The systems of one parac_pcg_many call solved as one block-diagonal system:
// their matrices, factors and vectors concatenated (system s holds rows
// off[s] .. off[s+1]), one schedule of the triangular solves interleaving the
// systems' dependency levels, and per-system CG scalars and stopping (batch.cu).
// A system's preconditioner apply is the same arithmetic, entry for entry, as
// its own parac_pcg's; only the dot products' reduction trees differ.
constexpr int64_t BATCH_CHUNK_ROWS = 4096;

struct BatchRun {
    DBuf Lp, Li, Lv, Fcp, Frow, Fval, Frp, Fcol, Fvalr, Dinv, operm;
    DBuf gt_f, gt_b, part_f, part_b;
    DBuf hy;                          // hybrid-solve table (int2 entries), when used
    int32_t nhy = 0, hy_blocks = 0;
    DBuf x, r, z, p, q, b, yl, zl, partials, sys, stop, state, status, clo, csys, sys_c0, seg;
};

// Every handle on one device with one precision, and the concatenation within
// the solves' 32-bit positions.
bool batchable(int32_t count, const parac_factor_t *G)
{
    if (count < 2) return false;
    if (G[0] && G[0]->pcg_many == PARAC_OFF) return false;
    int64_t n = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (!G[i] || G[i]->device != G[0]->device || G[i]->prec != G[0]->prec) return false;
        if ((G[i]->n > 0 && (int64_t)G[i]->lstart.size() != (int64_t)G[i]->depth + 1)) return false;
        n += G[i]->n;
    }
    return n > 0 && n < INT32_MAX;
}

parac_status pcg_batch(int32_t count, const parac_factor_t *G, const double *const *bv, double *const *xv,
                       double tol, int32_t maxit, int32_t *iters, double *true_relres)
{
    cudaSetDevice(G[0]->device);
    cudaStream_t st = G[0]->stream;
    set_mempool_keep();
    // start after the work queued on every handle's stream
    for (int32_t i = 1; i < count; ++i) {
        if (G[i]->stream == st) continue;
        cudaEvent_t e0 = nullptr;
        CK(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
        CK(cudaEventRecord(e0, G[i]->stream));
        CK(cudaStreamWaitEvent(st, e0, 0));
        CK(cudaEventDestroy(e0));
    }
    const int prec = G[0]->prec;
    const size_t xs = prec == 32 ? 4 : 8;
    std::vector<int64_t> off((size_t)count + 1, 0), offL((size_t)count + 1, 0), offF((size_t)count + 1, 0);
    int32_t depth = 0;
    long long spin = 0;
    for (int32_t i = 0; i < count; ++i) {
        off[(size_t)i + 1] = off[(size_t)i] + G[i]->n;
        offL[(size_t)i + 1] = offL[(size_t)i] + (G[i]->n > 0 ? G[i]->nnzL : 0);
        offF[(size_t)i + 1] = offF[(size_t)i] + (G[i]->n > 0 ? G[i]->nnzF : 0);
        depth = std::max(depth, G[i]->depth);
        spin = std::max(spin, G[i]->spin_limit);
    }
    const int64_t n = off.back(), nnzL = offL.back(), nnzF = offF.back();
    BatchRun R;
    const size_t n1 = (size_t)n + 1, L1 = (size_t)std::max<int64_t>(nnzL, 1), F1 = (size_t)std::max<int64_t>(nnzF, 1);
    R.Lp = dalloc<int64_t>(n1, st); R.Li = dalloc<int32_t>(L1, st); R.Lv = dalloc<double>(L1, st);
    R.Fcp = dalloc<int64_t>(n1, st); R.Frow = dalloc<int32_t>(F1, st); R.Fval = DBuf(xs * F1, st);
    R.Frp = dalloc<int64_t>(n1, st); R.Fcol = dalloc<int32_t>(F1, st); R.Fvalr = DBuf(xs * F1, st);
    R.Dinv = dalloc<double>((size_t)n, st); R.operm = dalloc<int32_t>((size_t)n, st);
    // concatenation: 11 arrays, one segment per system each
    enum { C_LP, C_LI, C_LV, C_FCP, C_FROW, C_FVAL, C_FRP, C_FCOL, C_FVALR, C_DINV, C_PERM, C_KINDS };
    std::vector<CatSeg> seg((size_t)C_KINDS * count);
    int64_t maxn = 0, maxL = 0, maxF = 0;
    for (int32_t i = 0; i < count; ++i) {
        const parac_factor_s *h = G[i];
        const int64_t ni = h->n, li = ni > 0 ? h->nnzL : 0, fi = ni > 0 ? h->nnzF : 0;
        const int64_t o = off[(size_t)i], oL = offL[(size_t)i], oF = offF[(size_t)i];
        maxn = std::max(maxn, ni); maxL = std::max(maxL, li); maxF = std::max(maxF, fi);
        auto at = [&](int k) -> CatSeg & { return seg[(size_t)k * count + i]; };
        const bool f32 = prec == 32;
        at(C_LP) = {h->Lp.p, ni, o, oL};
        at(C_LI) = {h->Li.p, li, oL, o};
        at(C_LV) = {h->Lv.p, li, oL, 0};
        at(C_FCP) = {h->Scp.p, ni, o, oF};
        at(C_FROW) = {h->Srow.p, fi, oF, o};
        at(C_FVAL) = {f32 ? h->Sval32.p : h->Sval.p, fi, oF, 0};
        at(C_FRP) = {h->Srp.p, ni, o, oF};
        at(C_FCOL) = {h->Scol.p, fi, oF, o};
        at(C_FVALR) = {f32 ? h->Svalr32.p : h->Svalr.p, fi, oF, 0};
        at(C_DINV) = {h->Sdinv.p, ni, o, 0};
        at(C_PERM) = {h->Sperm.p, ni, o, o};
    }
    R.seg = DBuf(sizeof(CatSeg) * seg.size(), st);
    CK(cudaMemcpyAsync(R.seg.p, seg.data(), sizeof(CatSeg) * seg.size(), cudaMemcpyHostToDevice, st));
    const CatSeg *ds = R.seg.as<CatSeg>();
    auto cat = [&](int k, int64_t mx, int elem, bool fl, DBuf &dst) {
        CK(launch_cat(ds + (size_t)k * count, count, mx, elem, fl, dst.p, st));
    };
    cat(C_LP, maxn, 8, false, R.Lp); cat(C_LI, maxL, 4, false, R.Li); cat(C_LV, maxL, 8, true, R.Lv);
    cat(C_FCP, maxn, 8, false, R.Fcp); cat(C_FROW, maxF, 4, false, R.Frow); cat(C_FVAL, maxF, (int)xs, true, R.Fval);
    cat(C_FRP, maxn, 8, false, R.Frp); cat(C_FCOL, maxF, 4, false, R.Fcol); cat(C_FVALR, maxF, (int)xs, true, R.Fvalr);
    cat(C_DINV, maxn, 8, true, R.Dinv); cat(C_PERM, maxn, 4, false, R.operm);
    // closing pointers (host values, copied before this function returns)
    const int64_t ends[3] = {nnzL, nnzF, nnzF};
    CK(cudaMemcpyAsync(R.Lp.as<int64_t>() + n, &ends[0], 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(R.Fcp.as<int64_t>() + n, &ends[1], 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(R.Frp.as<int64_t>() + n, &ends[2], 8, cudaMemcpyHostToDevice, st));
    // schedule of the solves: levels interleaved over the systems
    std::vector<std::vector<int64_t>> rps, cps;
    std::vector<BatchSysLevels> fw, bw;
    rps.reserve((size_t)count); cps.reserve((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        const parac_factor_s *h = G[i];
        if (h->n == 0) continue;
        const std::vector<int64_t> *rp = nullptr, *cp = nullptr;
        if (h->max_row > 4 * LONG_ROW_SINGLE) {     // rows that need the block-wide kinds
            rps.emplace_back((size_t)h->n + 1); cps.emplace_back((size_t)h->n + 1);
            CK(cudaMemcpyAsync(rps.back().data(), h->Srp.p, 8 * ((size_t)h->n + 1), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(cps.back().data(), h->Scp.p, 8 * ((size_t)h->n + 1), cudaMemcpyDeviceToHost, st));
            rp = &rps.back(); cp = &cps.back();
        }
        fw.push_back({i, off[(size_t)i], h->lstart, rp});
        bw.push_back({i, off[(size_t)i], h->lstart, cp});
    }
    CK(cudaStreamSynchronize(st));
    // the hybrid solves, the systems' levels interleaved in one table, when no
    // handle has a row of more than TPR_MAX_ROW entries (measured on the
    // 200-system batch: 150 ms PCG against 272 ms with a warp per row; the
    // handles' sptrsv choice, timed on single-system applies, does not apply)
    bool hybrid = true;
    for (int32_t i = 0; i < count && hybrid; ++i) hybrid = G[i]->max_row <= TPR_MAX_ROW;
    if (hybrid) {
        const int64_t hb = G[0]->trsv_blocks > 0 ? G[0]->trsv_blocks : (int64_t)num_sms();
        const std::vector<int32_t> t = hybrid_table(fw, hb * (TPR_THREADS / 32));
        R.hy = DBuf(4 * std::max<size_t>(t.size(), 2), st);
        CK(cudaMemcpyAsync(R.hy.p, t.data(), 4 * t.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        R.nhy = (int32_t)(t.size() / 2);
        R.hy_blocks = (int32_t)std::max<int64_t>(1, std::min<int64_t>(hb, (int64_t)num_sms() * std::max(1, tpr_blocks_per_sm(prec))));
    }
    // otherwise one row per warp (the stop-flag solves; sub-warp rows measured slower here)
    const int lanes = 32;
    const int rows_per_group = SOLVE_WARPS;
    const GroupTable gf = hybrid ? GroupTable{} : batch_groups(fw, n, false, rows_per_group, LONG_ROW_SINGLE, SPLIT_ROW_SINGLE, CHUNK_SINGLE);
    const GroupTable gb = hybrid ? GroupTable{} : batch_groups(bw, n, true, rows_per_group, LONG_ROW_SINGLE, SPLIT_ROW_SINGLE, CHUNK_SINGLE);
    R.gt_f = dalloc<int32_t>(std::max<size_t>(gf.g.size(), 4), st);
    R.gt_b = dalloc<int32_t>(std::max<size_t>(gb.g.size(), 4), st);
    CK(cudaMemcpyAsync(R.gt_f.p, gf.g.data(), 4 * gf.g.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(R.gt_b.p, gb.g.data(), 4 * gb.g.size(), cudaMemcpyHostToDevice, st));
    R.part_f = DBuf(xs * (size_t)std::max(gf.nslots, 1), st);
    R.part_b = DBuf(xs * (size_t)std::max(gb.nslots, 1), st);
    // row chunks of the dot products (never across systems)
    const RowChunks chunks = row_chunks(off, BATCH_CHUNK_ROWS);
    const std::vector<int64_t> &clo = chunks.lo;
    const std::vector<int32_t> &csys = chunks.sys, &c0 = chunks.first;
    const int32_t nch = (int32_t)csys.size();
    R.clo = dalloc<int64_t>(clo.size(), st); R.csys = dalloc<int32_t>(std::max<size_t>(csys.size(), 1), st);
    R.sys_c0 = dalloc<int32_t>(c0.size(), st);
    CK(cudaMemcpyAsync(R.clo.p, clo.data(), 8 * clo.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(R.csys.p, csys.data(), 4 * csys.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(R.sys_c0.p, c0.data(), 4 * c0.size(), cudaMemcpyHostToDevice, st));
    // vectors and state
    R.x = dalloc<double>((size_t)n, st); R.r = dalloc<double>((size_t)n, st); R.z = dalloc<double>((size_t)n, st);
    R.p = dalloc<double>((size_t)n, st); R.q = dalloc<double>((size_t)n, st); R.b = dalloc<double>((size_t)n, st);
    R.yl = DBuf(xs * (size_t)n, st); R.zl = DBuf(xs * (size_t)n, st);
    R.partials = dalloc<double>(3 * (size_t)std::max(nch, 1), st);
    R.sys = DBuf(sizeof(SysState) * (size_t)count, st);
    R.stop = dalloc<int32_t>((size_t)count, st);
    R.state = DBuf(batch_state_bytes(), st);
    R.status = dalloc<int32_t>(1, st);
    CK(cudaMemsetAsync(R.status.p, 0, 4, st));
    for (int32_t i = 0; i < count; ++i)
        if (G[i]->n > 0)
            CK(cudaMemcpyAsync(R.b.as<double>() + off[(size_t)i], bv[i], 8 * (size_t)G[i]->n, cudaMemcpyDefault, st));
    // solve arguments of the concatenated system
    SolveArgs A{};
    A.n = (int32_t)n;
    A.Lp = R.Lp.as<int64_t>(); A.Li = R.Li.as<int32_t>(); A.Lv = R.Lv.as<double>();
    A.Fcp = R.Fcp.as<int64_t>(); A.Frow = R.Frow.as<int32_t>();
    A.Frp = R.Frp.as<int64_t>(); A.Fcol = R.Fcol.as<int32_t>();
    if (prec == 32) { A.Fval32 = R.Fval.as<float>(); A.Fvalr32 = R.Fvalr.as<float>(); }
    else { A.Fval64 = R.Fval.as<double>(); A.Fvalr64 = R.Fvalr.as<double>(); }
    A.Dinv = R.Dinv.as<double>(); A.operm = R.operm.as<int32_t>();
    A.prec = prec;
    A.lanes_spmv = lanes_for((double)nnzL / (double)n);
    A.lanes_trsv = lanes;
    A.trsv_warps = SOLVE_WARPS;
    int bps = 0;
    trsv_configure(lanes, SOLVE_WARPS, &bps, prec, true);
    const int64_t max_blocks = (int64_t)num_sms() * std::max(bps, 1);   // all co-resident
    const int64_t want = (2 * n / std::max(depth, 1) + rows_per_group - 1) / rows_per_group;
    int64_t tb = std::max<int64_t>(std::min<int64_t>(num_sms(), max_blocks), std::min<int64_t>(max_blocks, want));
    if (G[0]->trsv_blocks > 0) tb = std::max<int64_t>(1, std::min<int64_t>(max_blocks, G[0]->trsv_blocks));
    tb = std::min<int64_t>(tb, std::max<int64_t>(std::max(gf.ngroups, gb.ngroups), 1));
    A.trsv_blocks = (int32_t)tb;
    CK(set_poll_backoff((unsigned)G[0]->poll_ns));
    A.spin_limit = spin;
    A.status = R.status.as<int32_t>();
    if (hybrid) {
        A.tpr_chunks = (const int2 *)R.hy.p; A.ntpr = R.nhy; A.tpr_blocks = R.hy_blocks;
    } else {
        A.gt_f = (const int4 *)R.gt_f.p; A.ng_f = gf.ngroups; A.part_f = R.part_f.p; A.nslot_f = gf.nslots;
        A.gt_b = (const int4 *)R.gt_b.p; A.ng_b = gb.ngroups; A.part_b = R.part_b.p; A.nslot_b = gb.nslots;
    }
    A.skip = R.stop.as<int32_t>();
    BatchBuffers B{};
    B.count = count; B.nchunks = nch;
    B.clo = R.clo.as<int64_t>(); B.csys = R.csys.as<int32_t>(); B.sys_c0 = R.sys_c0.as<int32_t>();
    B.x = R.x.as<double>(); B.r = R.r.as<double>(); B.z = R.z.as<double>(); B.p = R.p.as<double>();
    B.q = R.q.as<double>(); B.b = R.b.as<double>(); B.stop = R.stop.as<int32_t>();
    if (prec == 32) { B.solve.yl32 = R.yl.as<float>(); B.solve.zl32 = R.zl.as<float>(); }
    else { B.solve.yl64 = R.yl.as<double>(); B.solve.zl64 = R.zl.as<double>(); }
    B.partials = R.partials.as<double>(); B.sys = R.sys.as<SysState>(); B.st = R.state.as<BatchState>();
    B.spmv_blocks = (int32_t)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
    // the iteration: rounds of check_every steps, then the stopping tests
    const int every = G[0]->check_every;
    CK(spcg_init(A, B, tol, maxit, st));
    std::vector<SysState> hs((size_t)count);
    auto batch_status = [&]() {
        int32_t s = 0;
        CK(cudaMemcpyAsync(&s, R.status.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return s;
    };
    for (;;) {
        BatchState bs{};
        CK(cudaMemcpyAsync(&bs, R.state.p, sizeof bs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (batch_status() != ST_OK) { set_err("triangular solve wait exceeded the spin limit"); return PARAC_ETIMEOUT; }
        if (!bs.gate.done) {
            for (int c = 0; c < every; ++c) CK(spcg_iteration(A, B, st));
            continue;
        }
        CK(spcg_true_residual(A, B, st));
        CK(cudaMemcpyAsync(hs.data(), R.sys.p, sizeof(SysState) * (size_t)count, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool reopen = false;
        for (const SysState &y : hs)
            if (y.converged && !(y.true_rr <= y.tol2bb) && y.iters < maxit) reopen = true;
        if (!reopen) break;
        CK(spcg_reopen(A, B, st));
    }
    if (batch_status() != ST_OK) { set_err("triangular solve wait exceeded the spin limit"); return PARAC_ETIMEOUT; }
    for (int32_t i = 0; i < count; ++i)
        if (G[i]->n > 0)
            CK(cudaMemcpyAsync(xv[i], R.x.as<double>() + off[(size_t)i], 8 * (size_t)G[i]->n, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    int32_t first = -1;
    for (int32_t i = 0; i < count; ++i) {
        const SysState &y = hs[(size_t)i];
        if (iters) iters[i] = y.iters;
        if (true_relres) true_relres[i] = y.bb > 0.0 ? std::sqrt(y.true_rr / y.bb) : 0.0;
        if (first < 0 && y.bb > 0.0 && !(y.true_rr <= tol * tol * y.bb)) first = i;
    }
    if (first >= 0) { set_err("system %d: PCG reached maxit", first); return PARAC_ENOCONV; }
    return PARAC_OK;
}

}  // namespace

// PCG on several systems at once: as one block-diagonal system (pcg_batch)
// when the handles share a device and a precision; otherwise worker threads
// each take the next system and run parac_pcg on it, every handle on its own
// library stream, so the GPU runs the systems' kernels side by side.
extern "C" parac_status parac_pcg_many(int32_t count, const parac_factor_t *G, const double *const *b,
                                       double *const *x, double tol, int32_t maxit, int32_t *iters,
                                       double *true_relres)
{
    return guarded([&]() -> parac_status {
        if (count < 0 || (count > 0 && (!G || !b || !x))) { set_err("bad arguments to parac_pcg_many"); return PARAC_EINVAL; }
        for (int32_t i = 0; i < count; ++i) {
            if (G[i] && G[i]->n > 0 && (!b[i] || !x[i])) {
                set_err("parac_pcg_many: null right-hand side or solution of system %d", i);
                return PARAC_EINVAL;
            }
            for (int32_t j = 0; j < i && j < 64; ++j)
                if (G[i] == G[j]) { set_err("parac_pcg_many: handle %d repeats handle %d", i, j); return PARAC_EINVAL; }
        }
        // both paths switch to the handles' device (the batch on this thread,
        // one of the workers on this thread too); the caller's device comes back
        struct Restore { int dev = -1; ~Restore() { if (dev >= 0) cudaSetDevice(dev); } } restore;
        bool any = false;
        for (int32_t i = 0; i < count; ++i) any = any || G[i];
        if (any) CK(cudaGetDevice(&restore.dev));
        if (batchable(count, G)) {
            try {
                return pcg_batch(count, G, b, x, tol, maxit, iters, true_relres);
            } catch (const StatusFail &e) {
                // no room for the concatenated copy: solve system by system instead
                if (e.s != PARAC_ENOMEM) throw;
                cudaGetLastError();
                g_err.clear();
            }
        }
        std::vector<parac_status> st((size_t)count, PARAC_OK);
        std::vector<std::string> msg((size_t)count);
        std::vector<int32_t> it((size_t)count, 0);
        std::vector<double> rr((size_t)count, 0.0);
        std::atomic<int32_t> next{0};
        // 4 by default: measured best on 200 SDDM systems (1: 1.65 s, 4: 0.89 s, 16: 1.72 s)
        const int workers = count > 0 && G[0] ? G[0]->pcg_workers : 4;
        const int nth = (int)std::min<int32_t>(count, workers);
        auto worker = [&]() {
            // each worker orders its systems on its own stream and gets 1/nth
            // of the resident-block capacity for its solves
            cudaStream_t ws = nullptr;
            int wdev = -1;
            t_grid_share = nth;
            t_no_graph = true;
            for (;;) {
                const int32_t i = next.fetch_add(1);
                if (i >= count) break;
                if (!G[i]) { st[(size_t)i] = PARAC_EINVAL; msg[(size_t)i] = "null handle"; continue; }
                cudaSetDevice(G[i]->device);
                if (wdev != G[i]->device) {
                    if (ws) { cudaStreamSynchronize(ws); cudaStreamDestroy(ws); }
                    ws = nullptr;
                    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); ws = nullptr; }
                    wdev = G[i]->device;
                    // start after the work already queued on the handles' stream
                    cudaEvent_t e0 = nullptr;
                    if (ws && cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) == cudaSuccess) {
                        cudaEventRecord(e0, G[i]->stream);
                        cudaStreamWaitEvent(ws, e0, 0);
                        cudaEventDestroy(e0);
                    }
                }
                t_stream_override = ws;
                st[(size_t)i] = parac_pcg(G[i], G[i]->n, nullptr, nullptr, nullptr, b[i], 1, G[i]->n, tol, maxit, x[i],
                                          G[i]->n, &it[(size_t)i], &rr[(size_t)i]);
                if (st[(size_t)i] != PARAC_OK) msg[(size_t)i] = parac_last_error();
            }
            t_stream_override = nullptr;
            t_grid_share = 0;
            t_no_graph = false;
            if (ws) { cudaStreamSynchronize(ws); cudaStreamDestroy(ws); }
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nth; ++t) th.emplace_back(worker);
        if (nth > 0) worker();
        for (auto &t : th) t.join();
        parac_status out = PARAC_OK;
        int32_t first = -1;
        for (int32_t i = 0; i < count; ++i) {
            if (iters) iters[i] = it[(size_t)i];
            if (true_relres) true_relres[i] = rr[(size_t)i];
            // errors before non-convergence, the first system's first
            const parac_status s2 = st[(size_t)i];
            if (s2 != PARAC_OK && (out == PARAC_OK || (out == PARAC_ENOCONV && s2 != PARAC_ENOCONV))) { out = s2; first = i; }
        }
        if (first >= 0) set_err("system %d: %s", first, msg[(size_t)first].c_str());
        return out;
    });
}

extern "C" parac_status parac_precond_apply(parac_factor_t G, const double *r, double *z)
{
    return guarded([&]() -> parac_status {
        if (!G || (G->n > 0 && (!r || !z))) { set_err("bad arguments"); return PARAC_EINVAL; }
        if (G->n == 0) return PARAC_OK;
        cudaStream_t st = G->stream;
        SolveArgs A = solve_args(G, G->Lp.as<int64_t>(), G->Li.as<int32_t>(), G->Lv.as<double>(), G->nnzL);
        ensure_cache(G, A, st);
        PcgBuffers &Bf = G->cache.B;
        CK(cudaMemsetAsync(G->status.p, 0, 4, st));
        const size_t bytes = 8 * (size_t)G->n;
        CK(cudaMemcpyAsync(Bf.r, r, bytes, cudaMemcpyDefault, st));
        CK(precond_apply(A, Bf, Bf.r, Bf.z, st));
        CK(cudaMemcpyAsync(z, Bf.z, bytes, cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        if (read_dev_status(G, st) != ST_OK) { set_err("triangular solve wait exceeded the spin limit"); return PARAC_ETIMEOUT; }
        return PARAC_OK;
    });
}

// ------------------------------------------------------------------ autotuner
// Times candidate schedules on the caller's systems and keeps the fastest.
// The elimination candidates vary the worker warps per CTA, the ready-queue
// claim size and the threshold between the per-warp and the CTA-cooperative
// paths; the factor is the same for every candidate (the determinism of the
// schedule), so only time decides.  The solve candidates are the sync-free
// triangular-solve layouts, timed on preconditioner applies with the best
// factor.
extern "C" parac_status parac_autotune(int32_t count, const parac_system *systems, uint64_t seed,
                                       const parac_opts *base, parac_opts *best, char *report, size_t cap)
{
    return guarded([&]() -> parac_status {
        if (count < 1 || !systems || !best) { set_err("bad arguments to parac_autotune"); return PARAC_EINVAL; }
        parac_opts b0;
        parac_opts_default(&b0);
        if (base) b0 = *base;
        struct Cand { int warps, qc, big; double ms; };
        std::vector<Cand> fc = {{8, 1, 0, 0}, {8, 2, 0, 0}, {8, 4, 0, 0}, {8, 1, 64, 0}, {8, 1, 256, 0}, {4, 1, 0, 0}};
        std::vector<parac_factor_t> hs((size_t)count, nullptr);
        auto free_all = [&]() { for (auto &h : hs) { parac_factor_free(h); h = nullptr; } };
        auto run = [&](const parac_opts &o) -> double {
            const auto t0 = std::chrono::steady_clock::now();
            const parac_status r = parac_factor_many(count, systems, seed, &o, hs.data());
            const auto t1 = std::chrono::steady_clock::now();
            if (r != PARAC_OK) { free_all(); throw StatusFail{r}; }
            return std::chrono::duration<double, std::milli>(t1 - t0).count();
        };
        {   // warm-up: allocations, module load
            run(b0);
            free_all();
        }
        int bi = 0;
        for (size_t c = 0; c < fc.size(); ++c) {
            parac_opts o = b0;
            o.warps_per_block = fc[c].warps; o.queue_chunk = fc[c].qc; o.big_threshold = fc[c].big;
            double t = run(o);
            free_all();
            t = std::min(t, run(o));
            free_all();
            fc[c].ms = t;
            if (t < fc[(size_t)bi].ms) bi = (int)c;
        }
        parac_opts o = b0;
        o.warps_per_block = fc[(size_t)bi].warps; o.queue_chunk = fc[(size_t)bi].qc; o.big_threshold = fc[(size_t)bi].big;
        run(o);
        // solve strategies on the best factor
        int64_t nmax = 0;
        for (auto h : hs) nmax = std::max<int64_t>(nmax, h->n);
        cudaStream_t st = (cudaStream_t)b0.stream;
        DBuf r = dalloc<double>((size_t)std::max<int64_t>(nmax, 1), st), z = dalloc<double>((size_t)std::max<int64_t>(nmax, 1), st);
        CK(cudaMemsetAsync(r.p, 0x3f, 8 * (size_t)std::max<int64_t>(nmax, 1), st));   // every entry 0x3f3f...3f
        CK(cudaStreamSynchronize(st));
        struct SCand { int strat; double ms; };
        std::vector<SCand> sc = {{PARAC_SPTRSV_THREAD, 0}, {PARAC_SPTRSV_WARP, 0}, {PARAC_SPTRSV_SUB8, 0},
                                 {PARAC_SPTRSV_SUB4, 0}};
        int si = 0;
        for (size_t c = 0; c < sc.size(); ++c) {
            for (auto h : hs) h->sptrsv = sc[c].strat;
            double t = 1e300;
            for (int rep = 0; rep < 3; ++rep) {
                const auto t0 = std::chrono::steady_clock::now();
                for (auto h : hs) {
                    const parac_status q = parac_precond_apply(h, r.as<double>(), z.as<double>());
                    if (q != PARAC_OK) { free_all(); throw StatusFail{q}; }
                }
                const auto t1 = std::chrono::steady_clock::now();
                t = std::min(t, std::chrono::duration<double, std::milli>(t1 - t0).count());
            }
            sc[c].ms = t;
            if (t < sc[(size_t)si].ms) si = (int)c;
        }
        free_all();
        o.sptrsv = sc[(size_t)si].strat;
        *best = o;
        if (report && cap > 0) {
            std::string js = "{\"factor\": [";
            char buf[256];
            for (size_t c = 0; c < fc.size(); ++c) {
                snprintf(buf, sizeof buf, "%s{\"warps_per_block\": %d, \"queue_chunk\": %d, \"big_threshold\": %d, \"ms\": %.3f}",
                         c ? ", " : "", fc[c].warps, fc[c].qc, fc[c].big, fc[c].ms);
                js += buf;
            }
            js += "], \"solve\": [";
            for (size_t c = 0; c < sc.size(); ++c) {
                snprintf(buf, sizeof buf, "%s{\"sptrsv\": %d, \"ms\": %.3f}", c ? ", " : "", sc[c].strat, sc[c].ms);
                js += buf;
            }
            snprintf(buf, sizeof buf, "], \"best\": {\"warps_per_block\": %d, \"queue_chunk\": %d, \"big_threshold\": %d, \"sptrsv\": %d}}",
                     o.warps_per_block, o.queue_chunk, o.big_threshold, o.sptrsv);
            js += buf;
            if (js.size() + 1 > cap) { set_err("report buffer too small (%zu bytes needed)", js.size() + 1); return PARAC_EINVAL; }
            memcpy(report, js.c_str(), js.size() + 1);
        }
        return PARAC_OK;
    });
}

// Allocation-free preconditioner apply (see include/parac.h).  Uses only the
// handle's arrays and the library's fixed work array: no device allocation
// and no allocating library call happens here.
extern "C" parac_status parac_precond_apply_noalloc(parac_factor_t G, const double *r, double *z)
{
    return guarded([&]() -> parac_status {
        if (!G || (G->n > 0 && (!r || !z))) { set_err("bad arguments"); return PARAC_EINVAL; }
        if (G->n > NOALLOC_MAX_N) {
            set_err("parac_precond_apply_noalloc handles at most %d unknowns (factor has %lld)", NOALLOC_MAX_N,
                    (long long)G->n);
            return PARAC_EINVAL;
        }
        if (G->n == 0) return PARAC_OK;
        if (!on_device(r, G->device) || !on_device(z, G->device)) {
            set_err("r and z must be device memory of the factor's device %d", G->device);
            return PARAC_EINVAL;
        }
        // the caller's current device comes back on every return, errors included
        struct Restore { int dev = -1; ~Restore() { if (dev >= 0) cudaSetDevice(dev); } } restore;
        CK(cudaGetDevice(&restore.dev));
        if (restore.dev != G->device) CK(cudaSetDevice(G->device));
        cudaStream_t st = G->stream;
        SolveArgs A = solve_args(G, G->Lp.as<int64_t>(), G->Li.as<int32_t>(), G->Lv.as<double>(), G->nnzL);
        CK(cudaMemsetAsync(G->status.p, 0, 4, st));
        CK(precond_apply_noalloc(A, r, z, st));
        if (read_dev_status(G, st) != ST_OK) { set_err("triangular solve wait exceeded the spin limit"); return PARAC_ETIMEOUT; }
        return PARAC_OK;
    });
}
