// schedule.h -- the solves' group schedules (host code, no CUDA): which
// rows each group of the static round robin takes, in which order.
#pragma once

#include <cstdint>
#include <vector>

namespace parac {

// Schedule of the solves: groups in position order, 4 ints each (first
// position in walk order, kind, arg, slot).  GK_ROWS: arg rows, one per warp;
// GK_SHARED: one row for the whole block; GK_CHUNK: entries [arg*chunk,
// (arg+1)*chunk) of one row (in walk order) summed by the block into partial
// slot `slot`; GK_COMBINE: the row's arg partials from `slot` on, summed in
// order, finish the row.  Chunks come before their combine.
enum : int32_t { GK_ROWS = 0, GK_SHARED = 1, GK_CHUNK = 2, GK_COMBINE = 3 };
constexpr int32_t GK_KIND_MASK = 0xff, GK_SYS_SHIFT = 8;   // kind | system << GK_SYS_SHIFT
struct GroupTable {
    std::vector<int32_t> g;       // 4 * ngroups
    int32_t ngroups = 0, nslots = 0;
};
GroupTable row_groups(const std::vector<int64_t> &ptr, bool descending, int warps, int long_row, int split_row,
                      int chunk);
// one system of a concatenated solve: its first global position, its level
// starts (positions, depth + 1 entries) and, for systems with rows longer than
// the block-wide threshold, its row (forward) or column (backward) pointers
struct BatchSysLevels {
    int32_t sys;
    int64_t off;
    std::vector<int64_t> lstart;
    const std::vector<int64_t> *ptr;
};
GroupTable batch_groups(const std::vector<BatchSysLevels> &sys, int64_t n_tot, bool descending, int warps,
                        int long_row, int split_row, int chunk);

// Table of the hybrid solves over one system or several (their levels
// interleaved): entries in level order, systems in order within a level; a
// level with more than `wide` rows (all systems together) is cut into runs of
// at most 32 consecutive rows of one system, entry {first position, rows |
// sys << HY_SYS_SHIFT}; a narrower level lists its rows one per entry,
// {position, 0 | sys << HY_SYS_SHIFT}.  Two ints per entry.  The backward
// solve walks the same table from its end.
constexpr int32_t HY_COUNT_MASK = 63, HY_SYS_SHIFT = 6;
std::vector<int32_t> hybrid_table(const std::vector<BatchSysLevels> &sys, int64_t wide);

// Row chunks of the batched PCG's dot products: system s holds rows off[s] ..
// off[s+1]; chunk c covers rows lo[c] .. lo[c+1] (at most `rows`, never two
// systems), sys[c] is its system, and system s owns chunks first[s] ..
// first[s+1].  lo ends with the total row count.
struct RowChunks {
    std::vector<int64_t> lo;
    std::vector<int32_t> sys, first;
};
RowChunks row_chunks(const std::vector<int64_t> &off, int64_t rows);

}  // namespace parac
