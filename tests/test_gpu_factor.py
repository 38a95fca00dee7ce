"""GPU factor parity: the CUDA elimination (through the C ABI) must produce the
oracle's factor bit for bit -- structure, F values and pivots -- whatever the
schedule (grid size, warps, queue chunking, working-set path)."""
import numpy as np
import pytest

import oracle
from paper_2505_02977_gb300 import workloads as W
from tests.helpers import same_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_02977_gb300 import parac
    return parac


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_factor(P, A, perm, seed, on_device=True, **opts):
    o = P.parac_opts_default(**opts) if opts else None
    if on_device:
        G = P.parac_factor(A.n, _dev(A.colptr), _dev(A.rowind), _dev(A.val),
                           None if perm is None else _dev(perm), seed, o)
    else:
        G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, o)
    F = G.export()
    st = G.stats()
    G.free()
    return F, st


def _check(P, A, perm, seed, kind=0, **opts):
    ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, kind=kind)
    got, st = _gpu_factor(P, A, perm, seed, kind=kind, **opts)
    assert same_factor(got, ref), _first_diff(got, ref)
    return got, st


def _first_diff(a, b):
    if a["n"] != b["n"]:
        return f"n {a['n']} vs {b['n']}"
    if not np.array_equal(a["colptr"], b["colptr"]):
        j = int(np.argmax(a["colptr"] != b["colptr"]))
        return f"colptr differs from column {j - 1}"
    if not np.array_equal(a["row"], b["row"]):
        return f"rows differ at {int(np.argmax(a['row'] != b['row']))}"
    if not np.array_equal(a["D"].view(np.uint64), b["D"].view(np.uint64)):
        k = int(np.argmax(a["D"] != b["D"]))
        return f"D differs at {k}: {a['D'][k]!r} vs {b['D'][k]!r}"
    t = int(np.argmax(a["val"].view(np.uint64) != b["val"].view(np.uint64)))
    return f"values differ at {t}: {a['val'][t]!r} vs {b['val'][t]!r}"


def test_grid2d_64_bit_identical(P):
    A, perm, seed, _ = W.config("grid2d-64")
    _check(P, A, perm, seed)
    got, _ = _gpu_factor(P, A, perm, seed, on_device=False)          # host-pointer inputs
    assert same_factor(got, oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed))


@pytest.mark.parametrize("sched", [
    dict(),
    dict(blocks=1, warps_per_block=1),
    dict(blocks=3, warps_per_block=2, queue_chunk=4),
    dict(queue_chunk=8),
    dict(big_threshold=32),
    dict(big_threshold=32, warps_per_block=2),
])
def test_random_graphs_any_schedule(P, sched):
    rng = np.random.default_rng(5)
    for trial in range(6):
        n = int(rng.integers(50, 3000))
        a, b = W.sparse_random_edges(n, int(rng.integers(1, 6)) * n, trial, connected=trial % 3 != 0)
        w = rng.lognormal(0, 1.5, len(a))
        exc = rng.uniform(0, 0.3, n) * (rng.random(n) < 0.3) if trial % 2 else None
        A = W.laplacian_from_edges(n, a, b, w, exc)
        perm = W.random_ordering(n, trial)
        _check(P, A, perm, 100 + trial, **sched)


def test_identity_ordering_and_unit_weights(P):
    A, _, _, _ = W.config("grid2d-64")
    _check(P, A, None, 9)


def test_grid3d_32_bit_identical(P):
    A, perm, seed, _ = W.config("grid3d-32")
    _check(P, A, perm, seed)


def test_grid3d_64_bit_identical(P):
    A, perm, seed, _ = W.config("grid3d-64")
    _, st = _check(P, A, perm, seed)
    assert st["nnz_G"] == st["nnz_F"] + A.n


def test_high_degree_paths(P):
    """A hub of degree several thousand forces the CTA-cooperative path with
    the CTA buffer and with global scratch; small caps force it on moderate
    degrees as well."""
    rng = np.random.default_rng(3)
    n = 6000
    hub = np.zeros(n - 1, np.int64)
    a = np.concatenate([hub, rng.integers(1, n, 3 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 3 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    a, b = key // n, key % n
    A = W.laplacian_from_edges(n, a, b, rng.uniform(0.5, 2, len(a)))
    for perm in (W.random_ordering(n, 1), np.concatenate([np.arange(1, n), [0]]).astype(np.int32),
                 np.arange(n, dtype=np.int32)):
        _check(P, A, perm, 4)
        _check(P, A, perm, 4, big_threshold=32, blocks=2)


def test_sddm_ground_node(P):
    for s in range(3):
        rng = np.random.default_rng(s)
        n = 2000
        a, b = W.sparse_random_edges(n, 4 * n, s)
        w = rng.uniform(0.1, 10, len(a))
        deg = np.bincount(a, weights=w, minlength=n) + np.bincount(b, weights=w, minlength=n)
        A = W.laplacian_from_edges(n, a, b, w, rng.uniform(0, 0.1, n) * deg)
        perm = W.random_ordering(n, s)
        for kind in (0, 2):
            got, _ = _check(P, A, perm, 7 + s, kind=kind)
            assert np.all(got["D"] > 0)


def test_edge_cases(P):
    # single vertex, two vertices, edgeless graph, empty matrix
    for n, a, b in ((1, [], []), (2, [0], [1]), (5, [], [])):
        A = W.laplacian_from_edges(n, np.array(a, np.int64), np.array(b, np.int64), np.ones(len(a)))
        _check(P, A, None, 1)
    G = P.parac_factor(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), None, 0)
    assert G.export()["n"] == 0
    G.free()


def test_errors_are_reported(P):
    A, perm, seed, _ = W.config("grid2d-64")
    bad = A.val.copy()
    off = np.where(A.rowind != np.repeat(np.arange(A.n), np.diff(A.colptr)))[0][0]
    bad[off] = 0.5
    with pytest.raises(P.ParacError) as e:
        P.parac_factor(A.n, A.colptr, A.rowind, bad, perm, seed)
    assert e.value.status == "PARAC_ENOT_SDD"
    with pytest.raises(P.ParacError) as e:
        P.parac_factor(A.n, A.colptr, A.rowind, A.val, np.zeros(A.n, np.int32), seed)
    assert e.value.status == "PARAC_EINVAL"
    exc = W.laplacian_from_edges(4, np.array([0, 1]), np.array([1, 2]), np.ones(2), np.array([0, 0, 1.0, 0]))
    with pytest.raises(P.ParacError) as e:
        P.parac_factor(exc.n, exc.colptr, exc.rowind, exc.val, None, 0, P.parac_opts_default(kind=1))
    assert e.value.status == "PARAC_EINVAL"
    badrow = A.rowind.copy(); badrow[3] = A.n + 5
    with pytest.raises(P.ParacError) as e:
        P.parac_factor(A.n, A.colptr, badrow, A.val, perm, seed)
    assert e.value.status == "PARAC_EINVAL"


def test_pool_overflow_and_regrow(P):
    """A tiny fill workspace overflows: without regrowth the call fails with
    EPOOL; with regrowth it reruns and gives the same factor."""
    A, perm, seed, _ = W.config("grid3d-32")
    with pytest.raises(P.ParacError) as e:
        _gpu_factor(P, A, perm, seed, pool_mult=0.01, max_pool_regrow=0)
    assert e.value.status == "PARAC_EPOOL"
    got, st = _check(P, A, perm, seed, pool_mult=0.01, max_pool_regrow=12)
    assert st["regrows"] >= 1


def test_watchdog_timeout_then_recover(P):
    """A spin limit of one poll makes a device wait give up: the call returns
    ETIMEOUT (no hang) and the library keeps working afterwards."""
    A, perm, seed, _ = W.config("grid3d-32")
    with pytest.raises(P.ParacError) as e:
        _gpu_factor(P, A, perm, seed, spin_limit=1, blocks=8)
    assert e.value.status == "PARAC_ETIMEOUT"
    _check(P, A, perm, seed)


def test_batched_factor_matches_per_system_oracle(P):
    systems = W.sddm_batch(count=12, nmin=200, nmax=5000, seed=17)
    Gs = P.parac_factor_many([(A.n, A.colptr, A.rowind, A.val, perm) for A, perm, _ in systems], seed=99)
    for s, ((A, perm, _), G) in enumerate(zip(systems, Gs)):
        ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=99, sys=s)
        got = G.export()
        assert same_factor(got, ref), (s, _first_diff(got, ref))
        G.free()


def test_warp_only_paths_match(P):
    """With the CTA-cooperative path switched off every working set is handled
    by single warps (shared buffer, CTA buffer under a lock, global scratch):
    the factor must not change."""
    rng = np.random.default_rng(8)
    n = 3000
    hub = np.zeros(n - 1, np.int64)
    a = np.concatenate([hub, rng.integers(1, n, 4 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 4 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    A = W.laplacian_from_edges(n, key // n, key % n, rng.uniform(0.5, 2, len(key)))
    perm = W.random_ordering(n, 3)
    _check(P, A, perm, 5, coop=P.OFF)
    _check(P, A, perm, 5, big_threshold=32, coop=P.OFF)


@pytest.mark.parametrize("sample_sort", ["on", "off"])
def test_rmat_bit_identical(P, sample_sort):
    """R-MAT scale 15 (hubs of a few thousand neighbours, fill that piles up
    on the last vertices): the cooperative path with working sets in global
    memory, by sample sort and by the bitonic network, gives the oracle's
    factor."""
    A, perm, seed, _ = W.config("rmat-15")
    _, st = _check(P, A, perm, seed, sample_sort=P.ON if sample_sort == "on" else P.OFF)
    assert st["vertices_global_path"] > 0


@pytest.mark.parametrize("name,samples", [("rmat-15", 1), ("grid3d-64", 1), ("rmat-15", 2)])
def test_grid_help_bit_identical(P, name, samples):
    """Grid help: with a 256-entry CTA buffer every working set above 256
    gathered entries is offered to the grid's idle warps, which take chunks
    of its gather, both sample sorts, the scan, the sampling and the counter
    releases.  The factor equals the oracle's and the one without help (also
    with two samples per slot, MS(2)); on R-MAT the board was used (a grid's
    gathers may stay under the buffer)."""
    A, perm, seed, _ = W.config(name)
    kw = dict(block_cap=256, samples=samples)
    ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=samples)
    on, st = _gpu_factor(P, A, perm, seed, grid_help=P.ON, grid_help_min=0, **kw)
    off, st_off = _gpu_factor(P, A, perm, seed, grid_help=P.OFF, **kw)
    assert same_factor(on, ref), _first_diff(on, ref)
    assert same_factor(off, ref), _first_diff(off, ref)
    assert st_off["grid_help_vertices"] == 0
    if name.startswith("rmat"):
        assert st["grid_help_vertices"] > 0
        assert st["grid_help_chunks_helpers"] + st["grid_help_chunks_owner"] > 0


@pytest.mark.parametrize("field", ["uniform", "aniso", "contrast"])
def test_poisson_stand_ins_bit_identical(P, field):
    """Dirichlet Poisson stand-ins (SDDM: boundary rows ground through the
    ground node) on a 24^3 grid."""
    A, perm, seed, _ = W.config(f"poisson-{field}-24")
    _, st = _check(P, A, perm, seed)
    assert st["n"] == A.n


def test_ac2_bit_identical(P):
    """MS(2) (two samples per clique-tree slot) on every elimination path:
    register and warp paths (grid, random graphs), the CTA path with shared and
    global working sets (hub graph, R-MAT scale 15), and a grounded SDDM."""
    cases = [W.config("grid2d-64")[:3]]
    rng = np.random.default_rng(12)
    for s in range(2):
        n = int(rng.integers(500, 3000))
        a, b = W.sparse_random_edges(n, 4 * n, s)
        cases.append((W.laplacian_from_edges(n, a, b, rng.lognormal(0, 1, len(a))), W.random_ordering(n, s), s))
    n = 4000
    a = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, 3 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 3 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    cases.append((W.laplacian_from_edges(n, key // n, key % n, rng.uniform(0.5, 2, len(key))),
                  W.random_ordering(n, 9), 9))
    cases.append(W.config("rmat-15")[:3])
    cases.append(W.config("poisson-contrast-16")[:3])
    for A, perm, seed in cases:
        ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=2)
        one = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
        got, st = _gpu_factor(P, A, perm, seed, samples=2)
        assert same_factor(got, ref), _first_diff(got, ref)
        assert st["samples"] == 2 and ref["fill"] > one["fill"]


def test_hashmap_fill_store_bit_identical(P):
    """The hashmap fill store W (Sec. IV-C) instead of the per-column slabs: the
    same factor on every elimination path (register, warp, CTA with shared and
    global working sets), with MS(2), SDDM, a batch, and a small table that
    forces regrowth."""
    cases = [W.config("grid2d-64")[:3], W.config("rmat-15")[:3], W.config("poisson-contrast-16")[:3]]
    rng = np.random.default_rng(31)
    n = 4000
    a = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, 3 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 3 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    cases.append((W.laplacian_from_edges(n, key // n, key % n, rng.uniform(0.5, 2, len(key))),
                  W.random_ordering(n, 9), 9))
    for A, perm, seed in cases:
        ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
        got, st = _gpu_factor(P, A, perm, seed, fill_store=1)
        assert same_factor(got, ref), _first_diff(got, ref)
        assert st["fill_store"] == 1 and st["regrows"] == 0   # hubs (R-MAT, the star) fit without regrowth
    A, perm, seed = cases[0]
    ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=2)
    got, _ = _gpu_factor(P, A, perm, seed, fill_store=1, samples=2)
    assert same_factor(got, ref)
    A, perm, seed = cases[1]                      # R-MAT: a table far too small for its live fill
    got, st = _gpu_factor(P, A, perm, seed, fill_store=1, pool_mult=0.02, max_pool_regrow=10)
    assert same_factor(got, oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)) and st["regrows"] > 0
    batch = W.sddm_batch(5, nmin=300, nmax=3000, seed=4)
    systems = [(Ab.n, Ab.colptr, Ab.rowind, Ab.val, pb) for (Ab, pb, bb) in batch]
    Gs = P.parac_factor_many(systems, seed=99, opts=P.parac_opts_default(fill_store=1))
    for s, ((Ab, pb, bb), G) in enumerate(zip(batch, Gs)):
        ref = oracle.factor(Ab.colptr, Ab.rowind, Ab.val, pb, seed=99, sys=s)
        assert same_factor(G.export(), ref)
        G.free()


@pytest.mark.parametrize("name", ["grid3d-32", "rmat-15"])
def test_nnz_sorted_ordering_on_device(P, name):
    """order = PARAC_ORDER_NNZ builds Sec. V's NNZ-sorted ordering on the
    device: the factor is bit-identical to the oracle's under the numpy
    definition of that ordering (any other permutation would change it)."""
    A, _, seed, _ = W.config(name)
    G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, None, seed, P.parac_opts_default(order=P.ORDER_NNZ))
    ref = oracle.factor(A.colptr, A.rowind, A.val, W.nnz_sorted_ordering(A, seed), seed=seed)
    got = G.export()
    assert same_factor(got, ref), _first_diff(got, ref)
    G.free()
    with pytest.raises(P.ParacError) as e:     # an ordering array as well: refused
        P.parac_factor(A.n, A.colptr, A.rowind, A.val, np.arange(A.n, dtype=np.int32), seed,
                       P.parac_opts_default(order=P.ORDER_NNZ))
    assert e.value.status == "PARAC_EINVAL"


def test_nnz_sorted_ordering_batch(P):
    """The batched form orders every system by its own NNZ-sorted ordering."""
    batch = W.sddm_batch(8, nmin=300, nmax=6000, seed=23)
    systems = [(A.n, A.colptr, A.rowind, A.val, None) for (A, perm, b) in batch]
    Gs = P.parac_factor_many(systems, seed=11, opts=P.parac_opts_default(order=P.ORDER_NNZ))
    for s, ((A, perm, b), G) in enumerate(zip(batch, Gs)):
        ref = oracle.factor(A.colptr, A.rowind, A.val, W.nnz_sorted_ordering(A, 11), seed=11, sys=s)
        got = G.export()
        assert same_factor(got, ref), (s, _first_diff(got, ref))
        G.free()
