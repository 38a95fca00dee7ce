"""Host logic of the solves' static schedules (csrc/schedule.cpp), on the CPU.

The sync-free triangular solves hand row groups to a fully co-resident grid in
a fixed round robin; they always progress because every row's dependencies
sit in earlier groups.  These tests build the group tables for random inputs
and check what the solves rely on: every row in exactly one group, groups in
walk order, long rows given to a whole block or split into chunks followed by
their combine, and -- for the batched solves -- groups that never straddle a
(system, level) segment, carry their system in the kind's upper bits, and put
every dependency of a row in an earlier group."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2505_02977_gb300", "csrc")
GK_ROWS, GK_SHARED, GK_CHUNK, GK_COMBINE = 0, 1, 2, 3
KIND_MASK, SYS_SHIFT = 0xFF, 8


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("sched") / "libsched.so")
    subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(CSRC, "schedule.cpp"), os.path.join(ROOT, "tests", "schedule_shim.cpp"),
                    "-o", out], check=True)
    L = C.CDLL(out)
    P64, P32 = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
    L.sched_row_groups.restype = C.c_int64
    L.sched_row_groups.argtypes = [P64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P32, C.c_int64, P32]
    L.sched_batch_groups.restype = C.c_int64
    L.sched_batch_groups.argtypes = [C.c_int32, P64, P64, P64, P64, P64, C.c_int64, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int, P32, C.c_int64, P32]
    L.sched_hybrid_table.restype = C.c_int64
    L.sched_hybrid_table.argtypes = [C.c_int32, P64, P64, P64, C.c_int64, P32, C.c_int64]
    L.sched_row_chunks.restype = C.c_int64
    L.sched_row_chunks.argtypes = [P64, C.c_int32, C.c_int64, P64, P32, P32, C.c_int64]
    return L


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def row_groups(L, ptr, descending, warps, long_row, split_row, chunk):
    ptr = np.ascontiguousarray(ptr, np.int64)
    n = len(ptr) - 1
    cap = 4 * (2 * n + 16 + int((np.diff(ptr) // chunk).sum()) + n)
    out = np.zeros(cap, np.int32)
    ns = np.zeros(1, np.int32)
    g = L.sched_row_groups(_p(ptr, C.c_int64), n, int(descending), warps, long_row, split_row, chunk,
                           _p(out, C.c_int32), cap, _p(ns, C.c_int32))
    return out[:4 * g].reshape(g, 4), int(ns[0])


def batch_groups(L, systems, descending, warps, long_row, split_row, chunk):
    """systems: list of (n_s, lstart_s, ptr_s or None)."""
    off = np.zeros(len(systems) + 1, np.int64)
    lst, lo, ptrs, po = [], [0], [], []
    used = 0
    for s, (ns, ls, ptr) in enumerate(systems):
        off[s + 1] = off[s] + ns
        lst.append(np.asarray(ls, np.int64)); lo.append(lo[-1] + len(ls))
        if ptr is None:
            po.append(-1)
        else:
            po.append(used); ptrs.append(np.asarray(ptr, np.int64)); used += len(ptr)
    lst = np.concatenate(lst) if lst else np.zeros(1, np.int64)
    lo = np.asarray(lo, np.int64); po = np.asarray(po, np.int64)
    ptrs = np.concatenate(ptrs) if ptrs else np.zeros(1, np.int64)
    n = int(off[-1])
    extra = sum(int((np.diff(p) // chunk).sum()) for (_, _, p) in systems if p is not None)
    cap = 4 * (2 * n + 8 * len(systems) * (max((len(x[1]) for x in systems), default=1)) + extra + 16)
    out = np.zeros(cap, np.int32)
    ns = np.zeros(1, np.int32)
    g = L.sched_batch_groups(len(systems), _p(off, C.c_int64), _p(lst, C.c_int64), _p(lo, C.c_int64),
                             _p(ptrs, C.c_int64), _p(po, C.c_int64), n, int(descending), warps, long_row,
                             split_row, chunk, _p(out, C.c_int32), cap, _p(ns, C.c_int32))
    return out[:4 * g].reshape(g, 4), int(ns[0]), off


def walk(tab, nslots, n, lens, warps, long_row, split_row, chunk, monotone=True):
    """Check one table against the rules the solves rely on; return, per walk
    position kk, the index of the group that finishes it.  monotone: groups
    also come in increasing walk position (one system's table)."""
    done_at = -np.ones(n, np.int64)
    slot_next = 0
    pending = None            # (kk, chunks seen, first slot) of a split row
    last_kk = -1
    for gi, (x, kind_w, arg, slot) in enumerate(tab):
        kind = kind_w & KIND_MASK
        if kind == GK_ROWS:
            assert pending is None and 1 <= arg <= warps and (x > last_kk or not monotone)
            for kk in range(x, x + arg):
                assert done_at[kk] < 0 and lens[kk] <= long_row
                done_at[kk] = gi
            last_kk = x + arg - 1
        elif kind == GK_SHARED:
            assert pending is None and (x > last_kk or not monotone) and done_at[x] < 0
            assert long_row < lens[x] <= split_row
            done_at[x] = gi
            last_kk = x
        elif kind == GK_CHUNK:
            if pending is None:
                assert (x > last_kk or not monotone) and arg == 0 and slot == slot_next
                pending = [x, 0, slot]
            assert pending[0] == x and arg == pending[1] and slot == pending[2] + arg
            pending[1] += 1
        else:
            assert kind == GK_COMBINE and pending is not None and pending[0] == x
            nch = -(-lens[x] // chunk)
            assert lens[x] > split_row and arg == pending[1] == nch and slot == pending[2]
            slot_next = slot + nch
            done_at[x] = gi
            pending = None
            last_kk = x
    assert pending is None and slot_next == nslots
    assert np.all(done_at >= 0)
    return done_at


@pytest.mark.parametrize("descending", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_row_groups(lib, descending, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 400))
    lens = rng.integers(0, 6, n)
    heavy = rng.random(n) < 0.08
    lens[heavy] = rng.integers(6, 80, heavy.sum())
    ptr = np.concatenate([[0], np.cumsum(lens)])
    warps, long_row, split_row, chunk = 4, 5, 20, 8
    tab, nslots = row_groups(lib, ptr, descending, warps, long_row, split_row, chunk)
    wlens = lens[::-1] if descending else lens           # row length at walk position kk
    walk(tab, nslots, n, wlens, warps, long_row, split_row, chunk)
    assert np.all((tab[:, 1] >> SYS_SHIFT) == 0)


def _batch_case(rng, count, with_ptr):
    systems, levels, deps = [], [], []
    for s in range(count):
        ns = int(rng.integers(0, 120))
        if ns == 0:
            systems.append((0, np.zeros(1, np.int64), None)); levels.append(np.zeros(0, np.int64)); deps.append([])
            continue
        depth = int(rng.integers(1, 12))
        lv = np.sort(rng.integers(0, depth, ns))
        lv = np.searchsorted(np.unique(lv), lv)           # levels 0..depth'-1, all used, positions in level order
        depth = int(lv.max()) + 1
        lstart = np.searchsorted(lv, np.arange(depth + 1))
        # a row at level l > 0 depends on at least one row at level l - 1 (and maybe lower)
        dep = []
        for j in range(ns):
            if lv[j] == 0:
                dep.append([]); continue
            prev = np.nonzero(lv == lv[j] - 1)[0]
            lower = np.nonzero(lv < lv[j])[0]
            d = {int(rng.choice(prev))} | {int(v) for v in rng.choice(lower, min(2, len(lower)))}
            dep.append(sorted(d))
        ptr = None
        if with_ptr and rng.random() < 0.5:
            lens = rng.integers(0, 6, ns)
            heavy = rng.random(ns) < 0.1
            lens[heavy] = rng.integers(6, 60, heavy.sum())
            ptr = np.concatenate([[0], np.cumsum(lens)])
        systems.append((ns, lstart, ptr)); levels.append(lv); deps.append(dep)
    return systems, levels, deps


@pytest.mark.parametrize("seed", range(6))
def test_batch_groups(lib, seed):
    rng = np.random.default_rng(100 + seed)
    count = int(rng.integers(1, 9))
    systems, levels, deps = _batch_case(rng, count, with_ptr=seed % 2 == 1)
    warps, long_row, split_row, chunk = 4, 5, 20, 8
    n = sum(s[0] for s in systems)
    if n == 0:
        return
    for descending in (False, True):
        tab, nslots, off = batch_groups(lib, systems, descending, warps, long_row, split_row, chunk)
        # row length and (system, level) of every walk position
        lens = np.zeros(n, np.int64); sysof = np.zeros(n, np.int64); lvof = np.zeros(n, np.int64)
        for s, (ns, ls, ptr) in enumerate(systems):
            if ns == 0:
                continue
            pos = np.arange(off[s], off[s] + ns)
            kk = n - 1 - pos if descending else pos
            if ptr is not None:
                lens[kk] = np.diff(ptr)
            sysof[kk] = s; lvof[kk] = levels[s]
        done_at = walk(tab, nslots, n, lens, warps, long_row, split_row, chunk, monotone=False)
        # every group inside one (system, level) segment, tagged with its system
        for x, kind_w, arg, slot in tab:
            span = range(x, x + arg) if (kind_w & KIND_MASK) == GK_ROWS else [x]
            assert len({(sysof[k], lvof[k]) for k in span}) == 1
            assert kind_w >> SYS_SHIFT == sysof[x]
        # groups by level (ascending forward, descending backward), systems in order within a level
        key = [(lvof[x] if not descending else -lvof[x], sysof[x]) for x, _, _, _ in tab]
        assert key == sorted(key)
        # dependencies finish in earlier groups: forward, a row's dependencies; backward, its dependents
        for s, (ns, ls, ptr) in enumerate(systems):
            for j in range(ns):
                for d in deps[s][j]:
                    a, b = off[s] + j, off[s] + d            # global positions: a depends on b
                    if descending:
                        assert done_at[n - 1 - b] > done_at[n - 1 - a]
                    else:
                        assert done_at[b] < done_at[a]


@pytest.mark.parametrize("seed", range(4))
def test_row_chunks(lib, seed):
    """The batched PCG's dot-product chunks partition the rows, never cross a
    system, hold at most `rows` rows, and each system owns a contiguous run
    of them (systems without rows own none)."""
    rng = np.random.default_rng(200 + seed)
    count = int(rng.integers(1, 12))
    ns = rng.integers(0, 50, count)
    ns[rng.random(count) < 0.2] = 0
    off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    rows = int(rng.integers(1, 9))
    cap = int(off[-1]) + count + 2
    lo = np.zeros(cap, np.int64); sy = np.zeros(cap, np.int32); first = np.zeros(count + 1, np.int32)
    nch = lib.sched_row_chunks(_p(off, C.c_int64), count, rows, _p(lo, C.c_int64), _p(sy, C.c_int32),
                               _p(first, C.c_int32), cap)
    assert nch == sum(-(-int(k) // rows) for k in ns)
    lo, sy = lo[:nch + 1], sy[:nch]
    assert lo[0] == 0 and lo[-1] == off[-1] and np.all(np.diff(lo) >= 1) and np.all(np.diff(lo) <= rows)
    for c in range(nch):
        s = sy[c]
        assert off[s] <= lo[c] and lo[c + 1] <= off[s + 1]
    for s in range(count):
        assert np.all(sy[first[s]:first[s + 1]] == s)
        assert (first[s + 1] - first[s]) == -(-int(ns[s]) // rows)
    assert first[count] == nch


HY_COUNT_MASK, HY_SYS_SHIFT = 63, 6


@pytest.mark.parametrize("seed", range(6))
def test_hybrid_table(lib, seed):
    """The hybrid solves' table: every position in exactly one entry; entries
    in level order with systems in order within a level; a run holds at most
    32 consecutive positions of one (system, level) segment and is used only
    where the level (all systems) is wider than `wide`, single rows elsewhere;
    each entry carries its system; and every dependency of a row sits in an
    earlier entry, so walking the table from its end (the backward solve)
    meets every dependent before its dependencies."""
    rng = np.random.default_rng(300 + seed)
    count = int(rng.integers(1, 7))
    systems, levels, deps = _batch_case(rng, count, with_ptr=False)
    off = np.zeros(count + 1, np.int64)
    lst, lo = [], [0]
    for s_, (ns, ls, _) in enumerate(systems):
        off[s_ + 1] = off[s_] + ns
        lst.append(np.asarray(ls, np.int64)); lo.append(lo[-1] + len(ls))
    n = int(off[-1])
    if n == 0:
        return
    lst = np.concatenate(lst); lo = np.asarray(lo, np.int64)
    wide = int(rng.integers(0, 12))
    cap = 2 * (n + 8)
    out = np.zeros(cap, np.int32)
    ne = lib.sched_hybrid_table(count, _p(off, C.c_int64), _p(lst, C.c_int64), _p(lo, C.c_int64), wide,
                                _p(out, C.c_int32), cap)
    tab = out[:2 * ne].reshape(ne, 2)
    sysof = np.zeros(n, np.int64); lvof = np.zeros(n, np.int64)
    for s_, (ns, ls, _) in enumerate(systems):
        sysof[off[s_]:off[s_ + 1]] = s_; lvof[off[s_]:off[s_ + 1]] = levels[s_]
    width = np.bincount(lvof, minlength=lvof.max() + 1)
    entry_of = -np.ones(n, np.int64)
    keys = []
    for e, (x, y) in enumerate(tab):
        cnt, sy = y & HY_COUNT_MASK, y >> HY_SYS_SHIFT
        span = range(x, x + cnt) if cnt > 0 else [x]
        assert 1 <= len(span) <= 32
        assert len({(sysof[k], lvof[k]) for k in span}) == 1 and sysof[x] == sy
        assert (cnt > 0) == (width[lvof[x]] > wide)
        for k in span:
            assert entry_of[k] < 0
            entry_of[k] = e
        keys.append((lvof[x], sy))
    assert np.all(entry_of >= 0) and keys == sorted(keys)
    for s_, (ns, ls, _) in enumerate(systems):
        for j in range(ns):
            for d in deps[s_][j]:
                assert entry_of[off[s_] + d] < entry_of[off[s_] + j]


def scan_row_groups(ptr, descending, warps, long_row, split_row, chunk):
    """The device builder's construction of the same table (csrc/compact.cu,
    row_groups_count / row_groups_write), step for step in numpy: long-row
    flags, their exclusive ranks and compacted positions, groups emitted at
    each position (a long row's own groups; one where a run of short rows
    starts a group of `warps`), exclusive offsets of groups and slots, and
    every group written at its offset."""
    ptr = np.asarray(ptr, np.int64)
    n = len(ptr) - 1
    kk = np.arange(n)
    j = n - 1 - kk if descending else kk
    ln = ptr[j + 1] - ptr[j]
    islong = ln > long_row
    nch = (ln + chunk - 1) // chunk
    split = islong & (ln > split_row)
    slots = np.where(split, nch, 0)
    lrank = np.concatenate([[0], np.cumsum(islong)])          # exclusive, lrank[n] = long rows
    longpos = kk[islong]
    prev = np.where(lrank[:n] > 0, longpos[np.maximum(lrank[:n] - 1, 0)] if len(longpos) else -1, -1)
    start = (~islong) & (((kk - prev - 1) % warps) == 0)
    cnt = np.where(islong, np.where(split, nch + 1, 1), start.astype(np.int64))
    goff = np.concatenate([[0], np.cumsum(cnt)])
    soff = np.concatenate([[0], np.cumsum(slots)])
    g = np.zeros((int(goff[n]), 4), np.int32)
    nlong = int(lrank[n])
    for k in range(n):
        g0 = int(goff[k])
        if not islong[k]:
            if not start[k]:
                continue
            nxt = int(longpos[lrank[k]]) if lrank[k] < nlong else n
            g[g0] = (k, GK_ROWS, min(warps, nxt - k), 0)
        elif split[k]:
            for c in range(int(nch[k])):
                g[g0 + c] = (k, GK_CHUNK, c, int(soff[k]) + c)
            g[g0 + int(nch[k])] = (k, GK_COMBINE, int(nch[k]), int(soff[k]))
        else:
            g[g0] = (k, GK_SHARED, 0, 0)
    return g, int(soff[n])


@pytest.mark.parametrize("seed", range(6))
def test_scan_construction_matches_row_groups(lib, seed):
    """The scan-based construction used on the device gives row_groups'
    table exactly: random row lengths with runs of long rows, long rows at
    both ends, and rows above the split length."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    ln = rng.integers(0, 40, n)
    hot = rng.random(n) < [0.0, 0.01, 0.05, 0.2, 0.5, 0.9][seed]
    ln[hot] = rng.integers(41, 400, hot.sum())
    if n > 2 and seed % 2:
        ln[0] = 500; ln[-1] = 300
    ptr = np.concatenate([[0], np.cumsum(ln)])
    for desc in (False, True):
        for warps in (1, 3, 8):
            ref, ns_ref = row_groups(lib, ptr, desc, warps, 40, 120, 50)
            got, ns = scan_row_groups(ptr, desc, warps, 40, 120, 50)
            assert ns == ns_ref
            assert np.array_equal(got, ref), (desc, warps)
