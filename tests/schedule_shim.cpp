// C entry points over the solves' schedule builders (csrc/schedule.cpp), for
// the CPU tests: tables are written as 4 ints per group.
#include <cstring>
#include <vector>

#include "schedule.h"

using namespace parac;

static int64_t emit(const GroupTable &t, int32_t *out, int64_t cap, int32_t *nslots)
{
    if (nslots) *nslots = t.nslots;
    if (out && (int64_t)t.g.size() <= cap) std::memcpy(out, t.g.data(), 4 * t.g.size());
    return t.ngroups;
}

extern "C" int64_t sched_row_groups(const int64_t *ptr, int64_t n, int descending, int warps, int long_row,
                                    int split_row, int chunk, int32_t *out, int64_t cap, int32_t *nslots)
{
    std::vector<int64_t> p(ptr, ptr + n + 1);
    return emit(row_groups(p, descending != 0, warps, long_row, split_row, chunk), out, cap, nslots);
}

// System s: first position off[s], level starts lstart[lo[s] .. lo[s+1]),
// pointers ptr[po[s] .. po[s] + n_s + 1) when po[s] >= 0.
extern "C" int64_t sched_batch_groups(int32_t count, const int64_t *off, const int64_t *lstart, const int64_t *lo,
                                      const int64_t *ptr, const int64_t *po, int64_t n_tot, int descending,
                                      int warps, int long_row, int split_row, int chunk, int32_t *out, int64_t cap,
                                      int32_t *nslots)
{
    std::vector<std::vector<int64_t>> ptrs((size_t)count);
    std::vector<BatchSysLevels> sys;
    for (int32_t s = 0; s < count; ++s) {
        BatchSysLevels y;
        y.sys = s;
        y.off = off[s];
        y.lstart.assign(lstart + lo[s], lstart + lo[s + 1]);
        y.ptr = nullptr;
        if (po[s] >= 0) {
            const int64_t ns = off[s + 1] - off[s];
            ptrs[(size_t)s].assign(ptr + po[s], ptr + po[s] + ns + 1);
            y.ptr = &ptrs[(size_t)s];
        }
        sys.push_back(y);
    }
    return emit(batch_groups(sys, n_tot, descending != 0, warps, long_row, split_row, chunk), out, cap, nslots);
}

// Writes lo (nchunks + 1), sys (nchunks), first (count + 1); returns nchunks.
extern "C" int64_t sched_row_chunks(const int64_t *off, int32_t count, int64_t rows, int64_t *lo, int32_t *sys,
                                    int32_t *first, int64_t cap)
{
    const RowChunks c = row_chunks(std::vector<int64_t>(off, off + count + 1), rows);
    const int64_t nch = (int64_t)c.sys.size();
    if (nch + 1 <= cap) {
        std::memcpy(lo, c.lo.data(), 8 * c.lo.size());
        std::memcpy(sys, c.sys.data(), 4 * c.sys.size());
        std::memcpy(first, c.first.data(), 4 * c.first.size());
    }
    return nch;
}

// Hybrid-solve table of `count` systems (off / lstart / lo as for
// sched_batch_groups); writes 2 ints per entry, returns the entry count.
extern "C" int64_t sched_hybrid_table(int32_t count, const int64_t *off, const int64_t *lstart, const int64_t *lo,
                                      int64_t wide, int32_t *out, int64_t cap)
{
    std::vector<BatchSysLevels> sys;
    for (int32_t s = 0; s < count; ++s) {
        BatchSysLevels y;
        y.sys = s;
        y.off = off[s];
        y.lstart.assign(lstart + lo[s], lstart + lo[s + 1]);
        y.ptr = nullptr;
        sys.push_back(y);
    }
    const std::vector<int32_t> t = hybrid_table(sys, wide);
    if (out && (int64_t)t.size() <= cap) std::memcpy(out, t.data(), 4 * t.size());
    return (int64_t)t.size() / 2;
}
