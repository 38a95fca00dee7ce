"""Pins for the CPU oracle: facts fixed by the ParAC paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine (numpy's Philox), exact arithmetic, closed forms (degree <= 2 pivots
are exact eliminations), invariants (zero row sums, spanning trees,
dependency counters), the paper's worked example (Fig. 1, Sec. III), a
statistical identity (E[G G^T] = L, Sec. II-B) and a dense direct solve.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2505_02977_gb300 import workloads as W
from tests.helpers import reconstruct, same_factor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_matches_numpy_bitgenerator():
    """Philox4x64-10 equals numpy's Philox (which advances the counter by one
    before producing its first block)."""
    rng = np.random.default_rng(1234)
    for _ in range(50):
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64)
        ctr = rng.integers(0, 2 ** 63, 4, dtype=np.uint64)
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        ctr1 = ctr.copy(); ctr1[0] += np.uint64(1)
        assert np.array_equal(oracle.philox4x64_10(ctr1, key), ref)


def test_slot_uniform_definition_and_range():
    rng = np.random.default_rng(7)
    for _ in range(200):
        seed, k, p, s = (int(x) for x in rng.integers(0, 2 ** 40, 4))
        raw = np.random.Philox(key=np.array([seed, 0], np.uint64),
                               counter=np.array([k - 1 if k else 0, p, s, 0], np.uint64)).random_raw(1)[0] \
            if k else None
        v = oracle.slot_uniform(seed, k, p, s)
        assert 0.0 < v <= 1.0
        if raw is not None:
            assert v == ((int(raw) >> 11) + 1) * 2.0 ** -53


# ----------------------------------------------------------------- suffix sums
def test_suffix_scan_exact_on_integers():
    """Integer weights make every partial sum exact: any misplaced index shows."""
    rng = np.random.default_rng(3)
    for d in list(range(1, 70)) + [95, 96, 97, 128, 129, 300, 1025]:
        w = rng.integers(1, 1000, d).astype(float)
        S = oracle.suffix_scan(w)
        assert np.array_equal(S, np.cumsum(w[::-1])[::-1])


def test_suffix_scan_error_bound():
    rng = np.random.default_rng(4)
    for d in (1, 5, 31, 32, 33, 200, 5000):
        w = np.sort(rng.lognormal(0, 2, d))
        S = oracle.suffix_scan(w)
        ref = np.array([math.fsum(w[i:]) for i in range(d)])
        # every sum has at most ~(5 + d/32) rounded additions of positive terms
        bound = (6 + d / 32 + 1) * 2.0 ** -53 * ref
        assert np.all(np.abs(S - ref) <= bound)


# ----------------------------------------------------------------- sampling search
def test_pick_search_equals_literal_rule():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        d = int(rng.integers(1, 40))
        S = np.cumsum(rng.random(d)[::-1])[::-1]
        if rng.random() < 0.5:          # break monotonicity on purpose
            S = S * (1 + 1e-15 * rng.standard_normal(d))
            S[rng.integers(0, d)] *= 1.0 + rng.random() * 0.3
        lo = int(rng.integers(0, d))
        R = S[lo] * (rng.random() if rng.random() < 0.9 else 1.0)
        assert oracle.pick_search(S, lo, R) == oracle.pick_bruteforce(S, lo, R)


# ----------------------------------------------------------------- one pivot
def _union_find_tree(nodes, edges):
    parent = {v: v for v in nodes}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra == rb:
            return False
        parent[ra] = rb
    return len({find(v) for v in nodes}) == 1


def test_eliminate_merge_factor_column_and_spanning_tree():
    rng = np.random.default_rng(6)
    for trial in range(300):
        d0 = int(rng.integers(1, 30))
        base = np.sort(rng.choice(np.arange(10, 10000), d0, replace=False)).astype(np.int32)
        mult = rng.integers(1, 4, d0)
        rows = np.repeat(base, mult)
        w = rng.lognormal(0, 1, len(rows))
        perm = rng.permutation(len(rows))
        out = oracle.eliminate_one(rows[perm], w[perm], seed=trial, k=5)
        assert out["d"] == d0
        assert np.array_equal(out["rows"], base)
        assert np.array_equal(out["mult"], mult)
        for u, wu in zip(base, out["w"]):
            assert wu == pytest.approx(w[rows == u].sum(), rel=1e-14)
        assert out["D"] == pytest.approx(w.sum(), rel=1e-13)
        assert np.all(out["fval"] == -out["w"] / out["D"])
        # Alg. 2: d-1 sampled edges forming a spanning tree of N_k, each slot
        # linked to a later slot of the weight order (Sec. II-B)
        assert len(out["lo"]) == d0 - 1
        assert np.all(out["lo"] < out["hi"])
        assert np.all(out["pick"] >= np.arange(1, d0))
        assert _union_find_tree(list(base), list(zip(out["lo"], out["hi"]))) if d0 > 1 else True


def _expected_update(out):
    """E[sampled clique] from the oracle's slot weights and Alg. 2's probabilities."""
    rows = out["rows"]; w = out["w"]; D = out["D"]
    order = np.lexsort((rows, w))          # weight order
    ws = w[order]; rs = rows[order]
    idx = {r: i for i, r in enumerate(rows)}
    d = len(rows)
    E = np.zeros((d, d))
    S = np.cumsum(ws[::-1])[::-1]
    for p in range(1, d):
        c = out["c"][p - 1]                  # the oracle's weight for slot p
        u = rs[p - 1]
        for j in range(p, d):
            prob = ws[j] / S[p]
            a, b = idx[u], idx[rs[j]]
            E[a, a] += prob * c; E[b, b] += prob * c; E[a, b] -= prob * c; E[b, a] -= prob * c
    return E


def test_unbiased_update_by_enumeration():
    """Sum over all sampling outcomes of P(outcome) * C = C_exact (Sec. II-B)."""
    rng = np.random.default_rng(8)
    for trial in range(200):
        d = int(rng.integers(1, 7))
        rows = np.arange(100, 100 + d, dtype=np.int32)
        w = rng.lognormal(0, 1, d)
        out = oracle.eliminate_one(rows, w, seed=trial, k=1)
        E = _expected_update(out)
        wm = out["w"]; D = out["D"]
        Cex = np.diag(wm) - np.outer(wm, wm) / D       # L^(k) - l_k l_k^T / l_kk on N_k
        assert np.allclose(E, Cex, rtol=0, atol=1e-14 * max(1.0, np.abs(Cex).max()))


def test_sampler_frequencies_chi_square():
    """Slot p picks later entry j with probability w_j / S[p] (Alg. 2/3)."""
    from scipy.stats import chi2
    w = np.array([0.3, 0.5, 1.0, 1.7, 2.9, 4.1])
    rows = np.arange(50, 56, dtype=np.int32)
    d = len(w)
    N = 20000
    counts = np.zeros((d, d))
    for k in range(N):
        out = oracle.eliminate_one(rows, w, seed=99, k=k)
        for p in range(1, d):
            counts[p, out["pick"][p - 1]] += 1
    S = np.cumsum(w[::-1])[::-1]
    for p in range(1, d - 1):
        exp = N * w[p:] / S[p]
        stat = ((counts[p, p:] - exp) ** 2 / exp).sum()
        assert chi2.sf(stat, d - p - 1) > 1e-4, (p, counts[p], exp)
    assert counts[d - 1, d - 1] == N


# ----------------------------------------------------------------- whole factors
def _mat(n, a, b, w, excess=None):
    return W.laplacian_from_edges(n, a, b, w, excess)


@pytest.mark.parametrize("n", [2, 3, 10, 57])
def test_path_and_cycle_exact_under_any_order(n):
    """Pivots of degree <= 2 sample their only pair with weight w_i w_j/(w_i+w_j):
    an exact series reduction, so F D F^T = L under every ordering."""
    rng = np.random.default_rng(n)
    for edges in (W.path_edges(n), W.cycle_edges(n) if n > 2 else W.path_edges(n)):
        a, b = edges
        A = _mat(n, a, b, rng.uniform(0.5, 5, len(a)))
        Ad = A.dense()
        for s in range(3):
            perm = W.random_ordering(n, 10 * n + s)
            F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s)
            assert np.allclose(reconstruct(F, perm), Ad, rtol=0, atol=1e-13 * np.abs(Ad).max())
            assert np.sum(F["D"] == 0) == 1


def test_tree_exact_with_leaf_first_order():
    for s in range(5):
        n = 40 + 13 * s
        a, b = W.random_tree_edges(n, s)
        A = _mat(n, a, b, np.random.default_rng(s).uniform(0.1, 9, len(a)))
        perm = W.leaf_first_ordering(n, a, b, s)
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s)
        Ad = A.dense()
        assert np.allclose(reconstruct(F, perm), Ad, rtol=0, atol=1e-13 * np.abs(Ad).max())


def test_tree_random_order_is_not_exact():
    """Sanity check of the above: with degree-3 pivots the sample is a proper approximation."""
    n = 60
    a, b = W.random_tree_edges(n, 3)
    A = _mat(n, a, b, np.ones(len(a)))
    perm = W.random_ordering(n, 5)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=1)
    assert F["max_gather"] >= 3
    assert not np.allclose(reconstruct(F, perm), A.dense(), atol=1e-8)


def test_sddm_with_ground_node_exact_on_a_path():
    """SDDM -> Laplacian through a ground node (Sec. V); a path whose end has the
    only excess stays a path after augmentation, so the factor is exact."""
    n = 30
    a, b = W.path_edges(n)
    rng = np.random.default_rng(2)
    exc = np.zeros(n); exc[n - 1] = 0.75
    A = _mat(n, a, b, rng.uniform(1, 2, n - 1), exc)
    for s in range(3):
        perm = W.random_ordering(n, s)
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s, kind=oracle.KIND_SDDM)
        Ad = A.dense()
        assert np.allclose(reconstruct(F, perm), Ad, rtol=0, atol=1e-13 * np.abs(Ad).max())
        assert np.all(F["D"] > 0)


def test_zero_row_sums_of_reconstruction():
    """Each sampled update is a Laplacian (Sec. II-B), so F D F^T 1 = 0."""
    for s in range(6):
        n = 300
        a, b = W.sparse_random_edges(n, 900, s)
        A = _mat(n, a, b, np.random.default_rng(s).lognormal(0, 1.5, len(a)))
        perm = W.random_ordering(n, s + 100)
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s)
        G = reconstruct(F, perm)
        assert np.abs(G.sum(axis=1)).max() <= 1e-13 * np.abs(np.diag(G)).max()
        assert np.allclose(G, G.T, atol=1e-13 * np.abs(np.diag(G)).max())


def test_sample_mean_matches_L():
    """E[G G^T] = L (Sec. II-B): the mean of F D F^T over 1e5 seeds on small
    graphs lies within 4 standard errors of L, entry by entry."""
    rng = np.random.default_rng(11)
    graphs = []
    n = 6
    ia, ib = np.triu_indices(n, 1)
    graphs.append((n, ia, ib, rng.uniform(0.2, 3, len(ia))))             # K6
    n2 = 8
    a, b = W.sparse_random_edges(n2, 14, 4)
    graphs.append((n2, a, b, rng.lognormal(0, 1, len(a))))
    nseeds = 100_000
    for n, a, b, w in graphs:
        A = _mat(n, a, b, w)
        perm = W.random_ordering(n, 77)
        L = oracle.lib()
        acc = np.zeros((n, n)); acc2 = np.zeros((n, n))
        for s in range(nseeds):
            F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s, L=L)
            G = reconstruct(F, perm)
            acc += G; acc2 += G * G
        mean = acc / nseeds
        var = acc2 / nseeds - mean ** 2
        se = np.sqrt(np.maximum(var, 0) / nseeds)
        Ad = A.dense()
        dev = np.abs(mean - Ad)
        # entries that are deterministic (zero variance) only carry summation rounding
        assert np.all(dev <= 4 * se + 1e-10 * np.abs(Ad).max()), (dev / (se + 1e-300)).max()
        assert var.max() > 0          # genuinely random


# ----------------------------------------------------------------- dependency counters
def _golden_fig1():
    vals = {}
    with open(os.path.join(GOLDEN, "fig1_dependency_counters.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(":", 1)
            vals[k.strip()] = v.split()
    return vals


def test_fig1_worked_example():
    g = _golden_fig1()
    edges = [tuple(int(x) for x in e.split("-")) for e in g["edges"]]
    n = 6
    a = np.array([e[0] for e in edges]); b = np.array([e[1] for e in edges])
    A = _mat(n, a, b, np.ones(len(edges)))
    low = oracle.ingest(A.colptr, A.rowind, A.val, None, oracle.KIND_LAPLACIAN)
    dp0 = np.bincount(low["row"], minlength=n)          # counters start (R8)
    assert list(dp0) == [int(x) for x in g["initial_counts"]]
    samples = [tuple(int(x) for x in e.split("-")) for e in g["sampled_edges"]]
    nbrs = [int(x) for x in g["pivot_neighbours"]]
    dp_ins, _ = oracle.dp_update(dp0, samples, [], [])
    assert dp_ins[5] == int(g["counts_after_inserts_d5"][0])
    dp1, enq = oracle.dp_update(dp0, samples, nbrs, [1] * len(nbrs))
    assert list(dp1[1:]) == [int(x) for x in g["counts_after_d1_to_d5"]]
    assert sorted(enq) == [int(x) for x in g["enqueued"]]


def test_insert_before_delete_hazard():
    """Sec. III: deleting before inserting can enqueue a vertex whose incoming
    sampled edge is not yet recorded."""
    dp = np.array([0, 1, 1])
    dp_ok, enq_ok = oracle.dp_update(dp, [(1, 2)], [1, 2], [1, 1])
    assert list(enq_ok) == [1] and dp_ok[2] == 1
    _, enq_bad = oracle.dp_update(dp, [(1, 2)], [1, 2], [1, 1], deletes_first=True)
    assert sorted(enq_bad) == [1, 2]


@pytest.mark.parametrize("s", range(6))
def test_tracked_schedule_invariants_and_bit_identity(s):
    """Counters equal recomputed d_t(i) after every pivot, ready pivots are
    pairwise non-adjacent, and every counter-respecting schedule gives the
    label-order factor bit for bit (Sec. III 'Distribution Preservation')."""
    rng = np.random.default_rng(s)
    n = int(rng.integers(20, 120))
    a, b = W.sparse_random_edges(n, 3 * n, s, connected=(s % 3 != 0))
    w = rng.lognormal(0, 1, len(a))
    exc = rng.uniform(0, 0.5, n) if s % 2 else None
    A = _mat(n, a, b, w, exc)
    perm = W.random_ordering(n, s + 1)
    ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=1000 + s)
    for sched in range(3):
        T = oracle.factor_tracked(A.colptr, A.rowind, A.val, perm, seed=1000 + s, sched_seed=sched, check=True)
        assert T["violations"] == 0
        assert same_factor(T, ref)


# ----------------------------------------------------------------- ingest
def test_ingest_conventions_and_errors():
    n = 5
    a, b = W.path_edges(n)
    A = _mat(n, a, b, np.ones(n - 1))
    lo = oracle.ingest(A.colptr, A.rowind, A.val, None)
    assert lo["n"] == n and not lo["ground"] and len(lo["row"]) == n - 1
    assert np.all(lo["w"] == 1.0)
    # SDDM: ground node labelled last with edges of the row excess
    S = _mat(n, a, b, np.ones(n - 1), np.array([0.5, 0, 0, 0, 0.25]))
    lo = oracle.ingest(S.colptr, S.rowind, S.val, None)
    assert lo["ground"] and lo["n"] == n + 1
    gw = sorted(lo["w"][lo["row"] == n])
    assert gw == [0.25, 0.5]
    with pytest.raises(oracle.OracleError) as e:
        oracle.ingest(S.colptr, S.rowind, S.val, None, oracle.KIND_LAPLACIAN)
    assert e.value.code == 1
    bad = S.val.copy(); bad[np.where((S.rowind != np.repeat(np.arange(n), np.diff(S.colptr))))[0][0]] = 0.3
    with pytest.raises(oracle.OracleError) as e:
        oracle.ingest(S.colptr, S.rowind, bad, None)
    assert e.value.code == 2
    neg = A.val.copy(); neg[0] = 0.5           # diagonal below the off-diagonal sum
    with pytest.raises(oracle.OracleError) as e:
        oracle.ingest(A.colptr, A.rowind, neg, None)
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError):
        oracle.ingest(A.colptr, A.rowind, A.val, np.array([0, 1, 1, 2, 3]))


# ----------------------------------------------------------------- preconditioner / PCG
def test_precond_inverts_exact_factor():
    """For an exact factor (a path) and r orthogonal to 1, L M^{-1} r = r."""
    n = 80
    a, b = W.path_edges(n)
    A = _mat(n, a, b, np.random.default_rng(1).uniform(1, 3, n - 1))
    perm = W.random_ordering(n, 2)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=3)
    r = np.random.default_rng(4).standard_normal(n); r -= r.mean()
    z = oracle.precond_apply(F, perm, r)
    assert np.allclose(A.dense() @ z, r, atol=1e-11 * np.abs(r).max())


def test_pcg_matches_dense_solve():
    for s in range(4):
        n = 200 + 100 * s
        a, b = W.sparse_random_edges(n, 4 * n, s)
        rng = np.random.default_rng(s)
        exc = rng.uniform(0, 1, n) if s % 2 else None
        A = _mat(n, a, b, rng.lognormal(0, 1, len(a)), exc)
        perm = W.random_ordering(n, s)
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s)
        bvec = W.gaussian_rhs(n, 1, s, center=exc is None)
        x, it, rr = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, bvec, 1e-13, 2000)
        Ad = A.dense()
        xs = np.linalg.lstsq(Ad, bvec, rcond=None)[0]
        if exc is None:
            x = x - x.mean(); xs = xs - xs.mean()
        assert rr <= 1e-13
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_pcg_path_converges_at_once():
    n = 500
    a, b = W.path_edges(n)
    A = _mat(n, a, b, np.random.default_rng(0).uniform(1, 2, n - 1))
    perm = W.random_ordering(n, 1)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=2)
    bvec = W.gaussian_rhs(n, 1, 3)
    _, it, rr = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, bvec, 1e-8, 50)
    assert it <= 2 and rr <= 1e-8


# ----------------------------------------------------------------- mixed precision (FP32 factor)
# The mixed form keeps the elimination and PCG's recurrences in FP64 and
# applies the factor in FP32: F rounded to FP32, FP32 triangular solves, D^+
# applied in FP64 with the product rounded to FP32 (readings M1-M5 in the
# oracle's source).

U32 = 2.0 ** -24


def _path_identity(n, w):
    """Path 0-1-...-(n-1) with edge weights w, eliminated in label order: every
    pivot has one neighbour, so the factor is exact with F(j+1,j) = -1 and
    D_j = w_j (D_{n-1} = 0), and every solve row and column has one entry."""
    a, b = W.path_edges(n)
    A = _mat(n, a, b, w)
    return A, oracle.factor(A.colptr, A.rowind, A.val, None, seed=1)


def test_fp32_apply_exact_when_the_arithmetic_is_exact():
    """Unit-weight path, integer residual: every FP32 operation is exact, so
    the mixed apply equals the FP64 apply bit for bit, and both equal the
    closed form (prefix sums, then suffix sums of all but the last)."""
    n = 200
    A, F = _path_identity(n, np.ones(n - 1))
    assert np.all(F["val"] == -1.0) and np.all(F["D"][:-1] == 1.0) and F["D"][-1] == 0.0
    r = np.random.default_rng(3).integers(-10, 11, n).astype(float)
    z64 = oracle.precond_apply(F, None, r)
    z32 = oracle.precond_apply(F, None, r, prec=32)
    s = np.cumsum(r); s[-1] = 0.0
    closed = np.cumsum(s[::-1])[::-1]
    assert np.array_equal(z32, z64) and np.array_equal(z64, closed)


def test_fp32_apply_error_on_a_path_grows_with_its_length():
    """Exact path factor with weights in [1, 2): F = -1 exactly, so the only
    roundings are r -> FP32, one addition per forward step, the FP32 scale
    and one addition per backward step.  With R1 = sum |r| bounding every
    forward partial sum and Z1 = sum |s| every backward one,
      |y^_j - y_j| <= (j+1) 2u R1,   |s^_j - s_j| <= (|y^_j - y_j| + 2u R1)/w_j,
      |z^_j - z_j| <= sum_{i>=j} |s^_i - s_i| + (n-j) 2u Z1,
    a bound linear in the path length per solve.  The FP32 apply stays within
    it, and within the oracle's own running-error bound."""
    for n in (10, 300, 3000):
        rng = np.random.default_rng(n)
        w = rng.uniform(1, 2, n - 1)
        A, F = _path_identity(n, w)
        r = rng.standard_normal(n)
        z64 = oracle.precond_apply(F, None, r)
        z32, bd = oracle.precond_apply(F, None, r, prec=32, bound=True)
        R1 = np.abs(r).sum()
        ey = (np.arange(n) + 1) * 2 * U32 * R1
        s = np.cumsum(r)[:-1] / w
        Z1 = np.abs(s).sum() * (1 + 1e-6)
        es = np.append((ey[:-1] + 2 * U32 * R1) / w, 0.0)
        ez = np.cumsum(es[::-1])[::-1] + (n - np.arange(n)) * 2 * U32 * Z1
        err = np.abs(z32 - z64)
        assert np.all(err <= ez * (1 + 1e-6))
        assert np.all(err <= bd * (1 + 2.0 ** -20))
        assert err.max() > 0.0 or n == 10


def _fp32_cases():
    out = [W.config("grid2d-64")[:2]]
    rng = np.random.default_rng(8)
    for s in range(3):
        n = int(rng.integers(200, 2000))
        a, b = W.sparse_random_edges(n, 4 * n, 30 + s)
        exc = rng.uniform(0, 0.5, n) if s == 1 else None
        out.append((_mat(n, a, b, rng.lognormal(0, 1, len(a)), exc), W.random_ordering(n, s)))
    n = 500
    a, b = W.path_edges(n)
    out.append((_mat(n, a, b, rng.uniform(1, 2, n - 1)), W.random_ordering(n, 9)))
    return out


@pytest.mark.parametrize("case", range(5))
def test_fp32_apply_within_running_error_bound(case):
    """On grids, random (also SDDM) graphs and a randomly ordered path, the
    mixed apply differs from the FP64 apply by at most the componentwise
    running-error bound, which is not vacuous (below 1% of |z|), and the
    difference is FP32-sized (FP32 arithmetic was really used)."""
    A, perm = _fp32_cases()[case]
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=case)
    r = np.random.default_rng(case).standard_normal(A.n)
    z64 = oracle.precond_apply(F, perm, r)
    z32, bd = oracle.precond_apply(F, perm, r, prec=32, bound=True)
    err = np.abs(z32 - z64)
    assert np.all(err <= bd * (1 + 2.0 ** -20))
    assert bd.max() <= 1e-2 * np.abs(z64).max()
    assert 1e-10 * np.abs(z64).max() < err.max()


def test_fp32_bound_catches_a_dropped_term():
    """A factor with one entry removed (a plausible kernel mistake, planted
    here on the CPU) moves the apply far outside the bound."""
    A, perm = _fp32_cases()[1]
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=1)
    r = np.random.default_rng(5).standard_normal(A.n)
    z64 = oracle.precond_apply(F, perm, r)
    Fm = dict(F); Fm["val"] = F["val"].copy()
    Fm["val"][len(F["val"]) // 2] = 0.0
    zb, _ = oracle.precond_apply(Fm, perm, r, prec=32, bound=True)
    _, bd = oracle.precond_apply(F, perm, r, prec=32, bound=True)
    assert np.any(np.abs(zb - z64) > bd)


def test_fp32_pcg():
    """PCG with the FP32 factor keeps FP64 recurrences and reaches the same
    true relative residual.  With an exact factor (a path) the FP64 apply is
    L's pseudo-inverse on the range, so PCG stops after one iteration; the FP32
    apply is that inverse perturbed by an FP32-sized error, which one more
    iteration removes to 1e-8."""
    for A, perm in _fp32_cases()[:4]:
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=4)
        sddm = A.dense().sum(axis=1).max() > 1e-9
        b = W.gaussian_rhs(A.n, 1, 6, center=not sddm)
        _, it64, rr64 = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 1000)
        _, it32, rr32 = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 1000, prec=32)
        assert rr64 <= 1e-8 and rr32 <= 1e-8
    n = 200
    A, F = _path_identity(n, np.ones(n - 1))
    b = np.random.default_rng(1).integers(-10, 11, n).astype(float); b -= b.mean()
    x64, i64, r64 = oracle.pcg(A.colptr, A.rowind, A.val, F, None, b, 1e-8, 50)
    x32, i32, r32 = oracle.pcg(A.colptr, A.rowind, A.val, F, None, b, 1e-8, 50, prec=32)
    assert i64 == 1 and r64 <= 1e-8 and i32 <= 2 and r32 <= 1e-8


# ----------------------------------------------------------------- per-slot multi-sampling MS(k)
# MS(k): every slot of the clique tree, at every pivot, draws k neighbours,
# sample q with Philox counter (k, p, sys, q), each edge weighted c_p / k.
# k = 1 is Alg. 2.  Not Sec. VI's AC(2), which doubles the samples of the
# input matrix's own entries only.

def test_ac2_counter_word_and_weights():
    """Sample q of slot p uses counter word 3 = q (checked against numpy's
    Philox); sample 0 of MS(2) picks exactly Alg. 2's neighbour with half its
    weight; sample 1 follows the literal "largest j >= p with S[j] >= R" rule
    with its own uniform."""
    rng = np.random.default_rng(17)
    for trial in range(100):
        d = int(rng.integers(2, 12))
        rows = np.arange(10, 10 + d, dtype=np.int32)
        w = rng.lognormal(0, 1, d)
        k = int(rng.integers(1, 1000))
        one = oracle.eliminate_one(rows, w, seed=trial, k=k)
        two = oracle.eliminate_one(rows, w, seed=trial, k=k, samples=2)
        m = d - 1
        assert len(two["c"]) == 2 * m
        assert np.array_equal(two["pick"][:m], one["pick"])
        assert np.array_equal(two["c"][:m], one["c"] / 2)
        order = np.lexsort((two["rows"], two["w"]))
        ws = two["w"][order]
        S = oracle.suffix_scan(ws)
        for p in range(1, d):
            raw = np.random.Philox(key=np.array([trial, 0], np.uint64),
                                   counter=np.array([k - 1, p, 0, 1], np.uint64)).random_raw(1)[0]
            v = ((int(raw) >> 11) + 1) * 2.0 ** -53
            assert oracle.slot_uniform(trial, k, p, 0, q=1) == v
            assert two["pick"][m + p - 1] == oracle.pick_bruteforce(S, p, S[p] * v)
            assert two["c"][m + p - 1] == two["c"][p - 1]


def test_ms2_unbiased_by_enumeration():
    """MS(2): summed over all outcomes of both samples of every slot, the
    expected update equals the exact Schur complement update, as for Alg. 2."""
    rng = np.random.default_rng(19)
    for trial in range(200):
        d = int(rng.integers(1, 7))
        rows = np.arange(100, 100 + d, dtype=np.int32)
        w = rng.lognormal(0, 1, d)
        out = oracle.eliminate_one(rows, w, seed=trial, k=3, samples=2)
        order = np.lexsort((out["rows"], out["w"]))
        ws = out["w"][order]; rs = out["rows"][order]
        idx = {r: i for i, r in enumerate(out["rows"])}
        S = np.cumsum(ws[::-1])[::-1]
        E = np.zeros((d, d))
        for q in range(2):
            for p in range(1, d):
                c = out["c"][q * (d - 1) + p - 1]
                for j in range(p, d):
                    prob = ws[j] / S[p]
                    a, b = idx[rs[p - 1]], idx[rs[j]]
                    E[a, a] += prob * c; E[b, b] += prob * c; E[a, b] -= prob * c; E[b, a] -= prob * c
        wm = out["w"]; D = out["D"]
        Cex = np.diag(wm) - np.outer(wm, wm) / D
        assert np.allclose(E, Cex, rtol=0, atol=1e-14 * max(1.0, np.abs(Cex).max()))


def test_ms2_factor_counts_mean_and_variance():
    """MS(2) appends twice the fill edges of Alg. 2; paths stay exact; the mean
    of F D F^T over seeds matches L within 4 standard errors, with a smaller
    variance than Alg. 2's (the reason for more samples)."""
    A = _mat(8, np.arange(7), np.arange(1, 8), np.linspace(0.5, 2.0, 7))
    perm = W.random_ordering(8, 3)
    F2 = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=1, samples=2)
    assert np.allclose(reconstruct(F2, perm), A.dense(), rtol=0, atol=1e-13)
    rng = np.random.default_rng(23)
    n = 6
    ia, ib = np.triu_indices(n, 1)
    A = _mat(n, ia, ib, rng.uniform(0.2, 3, len(ia)))
    perm = W.random_ordering(n, 77)
    F1 = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=5)
    F2 = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=5, samples=2)
    assert F2["fill"] == 2 * F1["fill"]
    L = oracle.lib()
    nseeds = 20_000
    stats = {}
    for ks in (1, 2):
        acc = np.zeros((n, n)); acc2 = np.zeros((n, n))
        for s in range(nseeds):
            G = reconstruct(oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s, samples=ks, L=L), perm)
            acc += G; acc2 += G * G
        mean = acc / nseeds
        var = np.maximum(acc2 / nseeds - mean ** 2, 0)
        se = np.sqrt(var / nseeds)
        Ad = A.dense()
        assert np.all(np.abs(mean - Ad) <= 4 * se + 1e-10 * np.abs(Ad).max())
        stats[ks] = var.sum()
    assert stats[2] < stats[1]


# ----------------------------------------------------------------- AC(k): Sec. VI's multigraph variant
def _ac_expected_update(rows_e, w_e, out):
    """E[sampled clique] of one AC(k) pivot over every outcome: slots are the
    entries in (weight, row) order, slot p picks later entry j with
    probability w_j / S[p] and adds c_p (b_u - b_x)(b_u - b_x)^T, which is
    zero for a self-loop (u = x)."""
    order = np.lexsort((rows_e, w_e))
    ws = w_e[order]; rs = rows_e[order]
    g = len(ws)
    idx = {r: i for i, r in enumerate(out["rows"])}
    d = len(out["rows"])
    S = np.cumsum(ws[::-1])[::-1]
    E = np.zeros((d, d))
    for p in range(1, g):
        c = out["c"][p - 1]
        a = idx[rs[p - 1]]
        for j in range(p, g):
            b = idx[rs[j]]
            if a == b:
                continue
            prob = ws[j] / S[p]
            E[a, a] += prob * c; E[b, b] += prob * c; E[a, b] -= prob * c; E[b, a] -= prob * c
    return E


def test_acsplit_unbiased_by_enumeration():
    """AC(k), one pivot on a multiset with repeated rows (split copies of equal
    weight, fill entries of other weights): summed over every outcome of
    every slot the update is the exact Schur complement of the merged star,
    diag(w_u) - w w^T / D (Sec. II-B, with the self-loop terms zero); the
    pivot is the total weight, F(u,k) = -w_u / D, self-loops are exactly the
    slots whose pick shares their row, and every slot carries c_p = S[p] w_p / D."""
    rng = np.random.default_rng(31)
    for trial in range(300):
        nr = int(rng.integers(1, 5))
        base = np.arange(200, 200 + nr, dtype=np.int32)
        mult = rng.integers(1, 4, nr)
        rows_e = np.repeat(base, mult)
        w_e = np.concatenate([np.full(m, rng.lognormal(0, 1)) if rng.random() < 0.5 else rng.lognormal(0, 1, m)
                              for m in mult])
        perm = rng.permutation(len(rows_e))
        rows_e, w_e = rows_e[perm], w_e[perm]
        out = oracle.eliminate_one_ac(rows_e, w_e, seed=trial, k=4)
        g = len(rows_e)
        assert out["d"] == nr and len(out["c"]) == g - 1
        wm = np.array([w_e[rows_e == r].sum() for r in out["rows"]])
        assert np.allclose(out["w"], wm, rtol=1e-15, atol=0)
        assert np.array_equal(out["mult"], [int((rows_e == r).sum()) for r in out["rows"]])
        D = out["D"]
        assert abs(D - w_e.sum()) <= 1e-14 * w_e.sum()
        assert np.allclose(out["fval"], -out["w"] / D, rtol=1e-15, atol=0)
        order = np.lexsort((rows_e, w_e))
        ws, rs = w_e[order], rows_e[order]
        S = np.cumsum(ws[::-1])[::-1]
        for p in range(1, g):
            assert abs(out["c"][p - 1] - S[p] * ws[p - 1] / D) <= 1e-14 * abs(out["c"][p - 1]) + 1e-300
            j = out["pick"][p - 1]
            assert p <= j < g
            loop = rs[j] == rs[p - 1]
            assert (out["lo"][p - 1] == -1) == loop and (out["hi"][p - 1] == -1) == loop
            if not loop:
                assert (out["lo"][p - 1], out["hi"][p - 1]) == (min(rs[j], rs[p - 1]), max(rs[j], rs[p - 1]))
        E = _ac_expected_update(rows_e, w_e, out)
        Cex = np.diag(out["w"]) - np.outer(out["w"], out["w"]) / D
        assert np.allclose(E, Cex, rtol=0, atol=1e-13 * max(1.0, np.abs(Cex).max()))


@pytest.mark.parametrize("n", [2, 5, 40])
def test_acsplit_one_copy_on_paths_is_alg2(n):
    """With one copy per entry and no repeated row in any gathered list (a
    path: eliminating a vertex links its two neighbours, which were not
    adjacent), AC(1) takes exactly Alg. 2's steps: the same factor, bit for
    bit, under any ordering."""
    rng = np.random.default_rng(n)
    a, b = W.path_edges(n)
    A = _mat(n, a, b, rng.uniform(0.5, 2.0, len(a)))
    for s in range(5):
        perm = W.random_ordering(n, s)
        F1 = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s)
        Fa = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s, ac=1)
        assert np.array_equal(F1["colptr"], Fa["colptr"]) and np.array_equal(F1["row"], Fa["row"])
        assert np.array_equal(F1["val"].view(np.uint64), Fa["val"].view(np.uint64))
        assert np.array_equal(np.asarray(F1["D"]).view(np.uint64), np.asarray(Fa["D"]).view(np.uint64))


def test_acsplit_factor_mean_matches_L():
    """AC(2) on a dense 6-vertex graph: every sampled factor has the zero row
    sums of a Laplacian, and over 20,000 seeds the mean of F D F^T is L
    within 4 standard errors (the factorization is unbiased, Sec. II-B)."""
    rng = np.random.default_rng(41)
    n = 6
    ia, ib = np.triu_indices(n, 1)
    A = _mat(n, ia, ib, rng.uniform(0.2, 3, len(ia)))
    perm = W.random_ordering(n, 5)
    L = oracle.lib()
    nseeds = 20_000
    acc = np.zeros((n, n)); acc2 = np.zeros((n, n))
    for s in range(nseeds):
        G = reconstruct(oracle.factor(A.colptr, A.rowind, A.val, perm, seed=s, ac=2, L=L), perm)
        assert np.abs(G.sum(axis=1)).max() <= 1e-12 * np.abs(G).max()
        acc += G; acc2 += G * G
    mean = acc / nseeds
    se = np.sqrt(np.maximum(acc2 / nseeds - mean ** 2, 0) / nseeds)
    Ad = A.dense()
    assert np.all(np.abs(mean - Ad) <= 4 * se + 1e-10 * np.abs(Ad).max())


def test_acsplit_denser_than_alg2_far_below_ms2():
    """On the 64x64 grid AC(2) keeps more of the factor than Alg. 2 (more
    slots per pivot) while its fill stays within a small multiple of Alg.
    2's; MS(2), whose fill entries are resampled at every later pivot,
    grows far more.  Grounded SDDM input splits its ground edges too."""
    A, perm, seed, _ = W.config("grid2d-64")
    F1 = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    Fa = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, ac=2)
    Fm = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=2)
    assert len(Fa["row"]) > len(F1["row"]) and Fa["fill"] > F1["fill"]
    assert Fa["fill"] < 4 * F1["fill"] < Fm["fill"]
    B, pb, sb, _ = W.config("poisson-contrast-16")
    Fb = oracle.factor(B.colptr, B.rowind, B.val, pb, seed=sb, ac=2)
    assert Fb["n"] == B.n and np.all(np.asarray(Fb["D"]) > 0)


@pytest.mark.parametrize("s", range(3))
def test_acsplit_counter_schedule_invariants_and_bit_identity(s):
    """AC(2) under the dependency counters of Sec. III: the counters start at
    the split copies (two per input entry), self-loop samples add no edge and
    no increment, and after every pivot they equal a recount of the entries
    still waiting; ready vertices are pairwise non-adjacent; and whatever
    ready vertex is taken next, the factor is the label-order one, bit for
    bit (entries of equal key are identical, so the sorts are canonical)."""
    rng = np.random.default_rng(500 + s)
    n = int(rng.integers(40, 160))
    a, b = W.sparse_random_edges(n, 3 * n, s)
    A = _mat(n, a, b, rng.lognormal(0, 1, len(a)))
    perm = W.random_ordering(n, s)
    ref = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=70 + s, ac=2)
    for sched in (1, 2, 3):
        T = oracle.factor_tracked(A.colptr, A.rowind, A.val, perm, seed=70 + s, sched_seed=sched, check=True, ac=2)
        assert T["violations"] == 0
        assert same_factor(T, ref)
