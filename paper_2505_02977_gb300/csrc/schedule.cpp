// schedule.cpp -- the solves' group schedules (host code).  Each table entry
// is an int4 {first position in walk order, kind, arg, slot}; see schedule.h.
#include "schedule.h"

#include <algorithm>

namespace parac {

// Group table over positions in ascending (forward) or descending (backward)
// order; ptr = row pointers [n+1] of the rows in that order's numbering.
GroupTable row_groups(const std::vector<int64_t> &ptr, bool descending, int warps, int long_row, int split_row,
                      int chunk)
{
    const int64_t n = (int64_t)ptr.size() - 1;
    GroupTable t;
    t.g.reserve((size_t)(4 * (n / (warps > 0 ? warps : 1) + 2)));
    auto push = [&](int64_t start, int32_t kind, int32_t arg, int32_t slot) {
        t.g.push_back((int32_t)start); t.g.push_back(kind); t.g.push_back(arg); t.g.push_back(slot);
        ++t.ngroups;
    };
    int cur = 0;
    int64_t start = 0;
    for (int64_t kk = 0; kk < n; ++kk) {
        const int64_t j = descending ? n - 1 - kk : kk;
        const int64_t len = ptr[j + 1] - ptr[j];
        if (len > long_row) {
            if (cur > 0) { push(start, GK_ROWS, cur, 0); cur = 0; }
            if (len > split_row) {
                const int32_t nch = (int32_t)((len + chunk - 1) / chunk);
                for (int32_t c = 0; c < nch; ++c) push(kk, GK_CHUNK, c, t.nslots + c);
                push(kk, GK_COMBINE, nch, t.nslots);
                t.nslots += nch;
            } else {
                push(kk, GK_SHARED, 0, 0);
            }
        } else {
            if (cur == 0) start = kk;
            if (++cur == warps) { push(start, GK_ROWS, cur, 0); cur = 0; }
        }
    }
    if (cur > 0) push(start, GK_ROWS, cur, 0);
    return t;
}

// Schedule of the concatenated solves.  System s holds global positions
// [off[s], off[s+1]); its level l the positions off[s] + lstart[l] .. .  The
// forward walk takes the levels in ascending order and, within a level, the
// systems in order; the backward walk the levels in descending order (a row's
// dependencies sit at strictly lower levels going forward and strictly higher
// ones going back).  Each (level, system) range is cut into GK_ROWS groups of
// up to `warps` consecutive positions; a row longer than long_row entries
// (ptr given) gets the block-wide kinds of row_groups.  Every entry's kind
// carries its system (kind | sys << GK_SYS_SHIFT), so that the solves can
// skip the groups of systems that stopped.
GroupTable batch_groups(const std::vector<BatchSysLevels> &sys, int64_t n_tot, bool descending, int warps,
                        int long_row, int split_row, int chunk)
{
    GroupTable t;
    int32_t depth = 0;
    int64_t approx = 0;
    for (const auto &y : sys) {
        depth = std::max<int32_t>(depth, (int32_t)y.lstart.size() - 1);
        approx += (y.lstart.empty() ? 0 : y.lstart.back()) / std::max(1, warps) + (int64_t)y.lstart.size();
    }
    t.g.reserve((size_t)(4 * approx));
    int32_t sysbits = 0;
    auto push = [&](int64_t start, int32_t kind, int32_t arg, int32_t slot) {
        t.g.push_back((int32_t)start); t.g.push_back(kind | sysbits); t.g.push_back(arg); t.g.push_back(slot);
        ++t.ngroups;
    };
    for (int32_t li = 0; li < depth; ++li) {
        const int32_t l = descending ? depth - 1 - li : li;
        for (const auto &y : sys) {
            if (l + 1 >= (int32_t)y.lstart.size()) continue;
            sysbits = y.sys << GK_SYS_SHIFT;
            const int64_t a = y.off + y.lstart[(size_t)l], b = y.off + y.lstart[(size_t)l + 1];
            // walk positions kk of this range: forward j = kk, backward j = n_tot - 1 - kk
            const int64_t k0 = descending ? n_tot - b : a, k1 = descending ? n_tot - a : b;
            if (!y.ptr) {                      // no long rows: groups of `warps` positions
                for (int64_t kk = k0; kk < k1; kk += warps)
                    push(kk, GK_ROWS, (int32_t)std::min<int64_t>(warps, k1 - kk), 0);
                continue;
            }
            int cur = 0;
            int64_t start = k0;
            for (int64_t kk = k0; kk < k1; ++kk) {
                const int64_t j = (descending ? n_tot - 1 - kk : kk) - y.off;
                const int64_t len = (*y.ptr)[(size_t)j + 1] - (*y.ptr)[(size_t)j];
                if (len > long_row) {
                    if (cur > 0) { push(start, GK_ROWS, cur, 0); cur = 0; }
                    if (len > split_row) {
                        const int32_t nch = (int32_t)((len + chunk - 1) / chunk);
                        for (int32_t c = 0; c < nch; ++c) push(kk, GK_CHUNK, c, t.nslots + c);
                        push(kk, GK_COMBINE, nch, t.nslots);
                        t.nslots += nch;
                    } else {
                        push(kk, GK_SHARED, 0, 0);
                    }
                } else {
                    if (cur == 0) start = kk;
                    if (++cur == warps) { push(start, GK_ROWS, cur, 0); cur = 0; }
                }
            }
            if (cur > 0) push(start, GK_ROWS, cur, 0);
        }
    }
    return t;
}

RowChunks row_chunks(const std::vector<int64_t> &off, int64_t rows)
{
    RowChunks c;
    const int32_t count = (int32_t)off.size() - 1;
    c.first.assign((size_t)std::max(count, 0) + 1, 0);
    for (int32_t s = 0; s < count; ++s) {
        c.first[(size_t)s] = (int32_t)c.sys.size();
        for (int64_t a = off[(size_t)s]; a < off[(size_t)s + 1]; a += rows) {
            c.lo.push_back(a);
            c.sys.push_back(s);
        }
    }
    c.first[(size_t)std::max(count, 0)] = (int32_t)c.sys.size();
    c.lo.push_back(count > 0 ? off[(size_t)count] : 0);
    return c;
}

std::vector<int32_t> hybrid_table(const std::vector<BatchSysLevels> &sys, int64_t wide)
{
    size_t depth = 0;
    int64_t n = 0;
    for (const auto &y : sys) {
        if (y.lstart.size() > depth + 1) depth = y.lstart.size() - 1;
        if (!y.lstart.empty()) n += y.lstart.back() - y.lstart.front();
    }
    std::vector<int32_t> t;
    t.reserve((size_t)(2 * (n / 16 + (int64_t)depth * (int64_t)sys.size() + 2)));
    for (size_t l = 0; l < depth; ++l) {
        int64_t width = 0;
        for (const auto &y : sys)
            if (l + 1 < y.lstart.size()) width += y.lstart[l + 1] - y.lstart[l];
        const bool runs = width > wide;
        for (const auto &y : sys) {
            if (l + 1 >= y.lstart.size()) continue;
            const int64_t q0 = y.off + y.lstart[l], q1 = y.off + y.lstart[l + 1];
            const int32_t tag = y.sys << HY_SYS_SHIFT;
            if (runs) {
                for (int64_t q = q0; q < q1; q += 32) {
                    t.push_back((int32_t)q);
                    t.push_back((int32_t)std::min<int64_t>(32, q1 - q) | tag);
                }
            } else {
                for (int64_t q = q0; q < q1; ++q) { t.push_back((int32_t)q); t.push_back(tag); }
            }
        }
    }
    return t;
}

}  // namespace parac
