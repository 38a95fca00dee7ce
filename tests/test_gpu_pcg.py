"""GPU solve parity: preconditioner apply and PCG against the oracle (FP64),
and the FP32-stored factor inside FP64 PCG."""
import numpy as np
import pytest

import oracle
from paper_2505_02977_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_02977_gb300 import parac
    return parac


def _factor(P, A, perm, seed, **opts):
    return P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, P.parac_opts_default(**opts) if opts else None)


def _cases():
    out = [W.config("grid2d-64")]
    rng = np.random.default_rng(2)
    for s in range(3):
        n = int(rng.integers(300, 4000))
        a, b = W.sparse_random_edges(n, 3 * n, s)
        A = W.laplacian_from_edges(n, a, b, rng.lognormal(0, 1, len(a)))
        out.append((A, W.random_ordering(n, s), s, W.gaussian_rhs(n, 1, s)))
    return out


@pytest.mark.parametrize("case", range(4))
def test_precond_apply_matches_oracle(P, case):
    A, perm, seed, b = _cases()[case]
    G = _factor(P, A, perm, seed)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    r = np.random.default_rng(case).standard_normal(A.n)
    z = P.parac_precond_apply(G, r)
    zr = oracle.precond_apply(F, perm, r)
    assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    G.free()


@pytest.mark.parametrize("case", range(4))
def test_pcg_matches_oracle(P, case):
    """Same stopping rule as the oracle: converged to 1e-8 within one iteration
    of the oracle's count; solutions converged to 1e-12 agree to 1e-10
    relative; after the same iteration count the iterates agree to 1e-8 (the
    dot products and sparse sums are reduced in different orders, and CG
    amplifies that rounding from one iteration to the next)."""
    A, perm, seed, b = _cases()[case]
    G = _factor(P, A, perm, seed)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    xo, ito, rro = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 1000)
    x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-8, maxit=1000)
    assert status == "PARAC_OK" and rr[0] <= 1e-8
    assert abs(int(it[0]) - ito) <= 1
    xo12, _, _ = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-12, 2000)
    x12, _, rr12, _ = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-12, maxit=2000)
    xa, xb = x12 - x12.mean(), xo12 - xo12.mean()
    assert np.linalg.norm(xa - xb) <= 1e-10 * np.linalg.norm(xb)
    x2, it2, _, _ = P.parac_pcg(G, A.n, None, None, None, b, tol=0.0, maxit=ito)
    assert it2[0] == ito
    xa, xb = x2 - x2.mean(), xo - xo.mean()
    assert np.linalg.norm(xa - xb) <= 1e-8 * np.linalg.norm(xb)
    G.free()


def test_pcg_with_caller_matrix_and_device_arrays(P):
    import torch
    A, perm, seed, b = W.config("grid2d-64")
    G = _factor(P, A, perm, seed)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, it, rr, status = P.parac_pcg(G, A.n, dev(A.colptr), dev(A.rowind), dev(A.val), dev(b), tol=1e-8)
    assert status == "PARAC_OK" and rr[0] <= 1e-8
    xh, ith, rrh, _ = P.parac_pcg(G, A.n, A.colptr, A.rowind, A.val, b, tol=1e-8)
    assert it[0] == ith[0]
    assert np.allclose(x.cpu().numpy(), xh, rtol=0, atol=1e-12 * np.abs(xh).max())
    G.free()


def test_pcg_sddm_matches_dense_solve(P):
    rng = np.random.default_rng(4)
    n = 600
    a, b = W.sparse_random_edges(n, 4 * n, 4)
    w = rng.uniform(0.1, 10, len(a))
    deg = np.bincount(a, weights=w, minlength=n) + np.bincount(b, weights=w, minlength=n)
    A = W.laplacian_from_edges(n, a, b, w, rng.uniform(0, 0.1, n) * deg)
    perm = W.random_ordering(n, 1)
    bvec = rng.standard_normal(n)
    G = _factor(P, A, perm, 3)
    x, it, rr, status = P.parac_pcg(G, n, None, None, None, bvec, tol=1e-12, maxit=500)
    xs = np.linalg.solve(A.dense(), bvec)
    assert status == "PARAC_OK"
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    G.free()


def test_fp32_factor_converges(P):
    """FP32-stored G applied in FP32 inside FP64 PCG reaches the same 1e-8 true
    residual, within a few iterations of the FP64 solve."""
    A, perm, seed, b = W.config("grid3d-32")
    G64 = _factor(P, A, perm, seed)
    G32 = _factor(P, A, perm, seed, g_precision=32)
    _, it64, rr64, s64 = P.parac_pcg(G64, A.n, None, None, None, b, tol=1e-8, maxit=500)
    _, it32, rr32, s32 = P.parac_pcg(G32, A.n, None, None, None, b, tol=1e-8, maxit=500)
    assert s64 == s32 == "PARAC_OK" and rr32[0] <= 1e-8 and rr64[0] <= 1e-8
    assert it32[0] <= it64[0] + 3
    G64.free(); G32.free()


def test_pcg_multiple_rhs(P):
    """Block PCG on 5 right-hand sides: every column converges to 1e-8 within
    one iteration of the oracle's single-vector PCG on that column, and after
    the oracle's iteration count its iterate agrees with the oracle's to 1e-8
    (reduction orders differ; see test_pcg_matches_oracle)."""
    A, perm, seed, _ = W.config("grid2d-64")
    B = W.gaussian_rhs(A.n, 5, 9)
    G = _factor(P, A, perm, seed)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    X, it, rr, status = P.parac_pcg(G, A.n, None, None, None, B, tol=1e-8, maxit=500)
    assert status == "PARAC_OK" and X.shape == (A.n, 5) and np.all(rr <= 1e-8)
    kmin = None
    for j in range(5):
        xo, ito, rro = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, B[:, j], 1e-8, 500)
        assert abs(int(it[j]) - ito) <= 1
        kmin = ito if kmin is None else min(kmin, ito)
    X2, it2, _, _ = P.parac_pcg(G, A.n, None, None, None, B, tol=0.0, maxit=kmin)
    assert np.all(it2 == kmin)
    for j in range(5):
        xo, _, _ = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, B[:, j], 0.0, kmin)
        xa, xb = X2[:, j] - X2[:, j].mean(), xo - xo.mean()
        assert np.linalg.norm(xa - xb) <= 1e-8 * np.linalg.norm(xb)
    G.free()


@pytest.mark.parametrize("prec", [64, 32])
def test_block_pcg_columns_independent(P, prec):
    """32 right-hand sides (the maximum) with leading dimensions above n:
    a column scaled by 2^20 gives exactly 2^20 times the other's iterate
    (power-of-two scaling is exact in every step, so any mixing between the
    lanes of different columns shows), a zero column stops at once with x = 0,
    columns stop on their own counts, and the padding rows of X are left
    untouched."""
    A, perm, seed, _ = W.config("grid2d-64")
    n, k = A.n, 32
    B = np.zeros((n + 7, k), order="F")
    B[:n] = W.gaussian_rhs(n, k, 17)
    B[:n, 1] = B[:n, 0] * 2.0 ** 20
    B[:n, 2] = 0.0
    B[:n, 3] = B[:n, 4] * 1e-3 + B[:n, 5] * 1e-6
    B[n:] = 123.0                                                       # padding: must not be read
    X = np.full((n + 3, k), -7.0, order="F")
    G = _factor(P, A, perm, seed, g_precision=prec)
    Xo, it, rr, status = P.parac_pcg(G, n, None, None, None, B, tol=1e-8, maxit=500, X=X)
    assert status == "PARAC_OK" and np.all(rr <= 1e-8)
    assert np.all(X[n:] == -7.0)
    assert np.array_equal(X[:n, 1], X[:n, 0] * 2.0 ** 20) and it[1] == it[0]
    assert np.all(X[:n, 2] == 0.0) and it[2] == 0 and rr[2] == 0.0
    for j in (0, 5, 31):
        xj, itj, rrj, _ = P.parac_pcg(G, n, None, None, None, np.ascontiguousarray(B[:n, j]), tol=1e-8, maxit=500)
        assert abs(int(itj[0]) - int(it[j])) <= 1
        assert np.linalg.norm((xj - xj.mean()) - (X[:n, j] - X[:n, j].mean())) <= 1e-6 * np.linalg.norm(xj)
    G.free()


def test_block_pcg_device_arrays(P):
    import torch
    A, perm, seed, _ = W.config("grid2d-64")
    B = W.gaussian_rhs(A.n, 8, 21)
    G = _factor(P, A, perm, seed)
    Xh, ith, rrh, _ = P.parac_pcg(G, A.n, None, None, None, B, tol=1e-8)
    Xd, itd, rrd, status = P.parac_pcg(G, A.n, None, None, None, torch.from_numpy(B).cuda(), tol=1e-8)
    assert status == "PARAC_OK" and tuple(Xd.shape) == (A.n, 8)
    assert np.array_equal(ith, itd) and np.array_equal(Xd.cpu().numpy(), Xh)
    G.free()


@pytest.mark.parametrize("nrhs", [1, 6])
def test_graph_replay_matches_direct_launches(P, nrhs):
    """The captured-graph replay of the PCG iterations runs the same kernels
    in the same order as direct launches: identical bits."""
    A, perm, seed, _ = W.config("grid2d-64")
    B = W.gaussian_rhs(A.n, nrhs, 23)
    G = _factor(P, A, perm, seed)
    Xg, itg, rrg, _ = P.parac_pcg(G, A.n, None, None, None, B, tol=1e-10, maxit=500)
    Xg2, itg2, _, _ = P.parac_pcg(G, A.n, None, None, None, B, tol=1e-10, maxit=500)    # replay of a cached graph
    Gd = _factor(P, A, perm, seed, pcg_graph=P.OFF)          # same factor, iterations launched directly
    Xd, itd, rrd, _ = P.parac_pcg(Gd, A.n, None, None, None, B, tol=1e-10, maxit=500)
    Gd.free()
    assert np.array_equal(itg, itd) and np.array_equal(Xg, Xd) and np.array_equal(rrg, rrd)
    assert np.array_equal(itg2, itd) and np.array_equal(Xg2, Xd)
    G.free()


def test_pcg_noconv_status(P):
    A, perm, seed, b = W.config("grid2d-64")
    G = _factor(P, A, perm, seed)
    x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-14, maxit=3)
    assert status == "PARAC_ENOCONV" and it[0] == 3 and rr[0] > 1e-14
    G.free()


def test_grid3d_128_full_size(P):
    """The 128^3 workload at full size: the factor is bit-identical to the
    oracle's, and PCG reaches 1e-8 within two iterations of the oracle."""
    import torch
    from tests.helpers import same_factor
    A, perm, seed, b = W.config("grid3d-128")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    G = P.parac_factor(A.n, dev(A.colptr), dev(A.rowind), dev(A.val), dev(perm), seed)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    assert same_factor(G.export(), F)
    x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, dev(b), tol=1e-8, maxit=1000)
    xo, ito, rro = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 1000)
    assert status == "PARAC_OK" and rr[0] <= 1e-8 and rro <= 1e-8
    assert abs(int(it[0]) - ito) <= 2
    G.free()


@pytest.mark.parametrize("strategy", [1, 2, 3, 4])
def test_sptrsv_strategies(P, strategy):
    """Every triangular-solve layout applies the same preconditioner (up to
    the order of the row sums) and PCG reaches 1e-8 within one iteration of
    the oracle."""
    for case in (0, 1):
        A, perm, seed, b = _cases()[case]
        G = _factor(P, A, perm, seed, sptrsv=strategy)
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
        r = np.random.default_rng(case).standard_normal(A.n)
        z = P.parac_precond_apply(G, r)
        zr = oracle.precond_apply(F, perm, r)
        assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
        xo, ito, _ = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 1000)
        x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-8, maxit=1000)
        assert status == "PARAC_OK" and rr[0] <= 1e-8 and abs(int(it[0]) - ito) <= 1
        G.free()


def test_autotune(P):
    """The tuner returns a complete schedule; factors made with it are the
    default schedule's, bit for bit; every candidate was timed."""
    from tests.helpers import same_factor
    batch = W.sddm_batch(6, nmin=500, nmax=5000, seed=5)
    systems = [(A.n, A.colptr, A.rowind, A.val, perm) for (A, perm, b) in batch]
    best, rep = P.parac_autotune(systems, seed=7)
    assert len(rep["factor"]) >= 4 and len(rep["solve"]) == 4
    assert all(c["ms"] > 0 for c in rep["factor"] + rep["solve"])
    assert best.sptrsv in (1, 2, 3, 4) and best.warps_per_block in (4, 8) and best.queue_chunk >= 1
    tuned = P.parac_factor_many(systems, seed=7, opts=best)
    plain = P.parac_factor_many(systems, seed=7)
    for Gt, Gp in zip(tuned, plain):
        assert same_factor(Gt.export(), Gp.export())
        Gt.free(); Gp.free()


def test_split_rows(P):
    """A hub adjacent to every vertex and eliminated last gives a factor row of
    ~40,000 entries: the solves split it into chunks summed by separate
    blocks and combined in order (8,192 entries per chunk with one right-hand
    side, 512 with several).  The preconditioner still matches the oracle's,
    and block PCG matches single-vector PCG."""
    rng = np.random.default_rng(21)
    n = 40000
    a = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, 2 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 2 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    A = W.laplacian_from_edges(n, key // n, key % n, rng.uniform(0.5, 2.0, len(key)))
    perm = np.concatenate([rng.permutation(np.arange(1, n)), [0]]).astype(np.int32)
    G = _factor(P, A, perm, 3)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=3)
    assert np.bincount(F["row"], minlength=n).max() > 32768
    for case in range(2):
        r = np.random.default_rng(case).standard_normal(n)
        z = P.parac_precond_apply(G, r)
        zr = oracle.precond_apply(F, perm, r)
        assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    B = W.gaussian_rhs(n, 4, 5)
    X, it, rr, status = P.parac_pcg(G, n, None, None, None, B, tol=1e-8, maxit=500)
    assert status == "PARAC_OK" and np.all(rr <= 1e-8)
    for j in range(4):
        xj, itj, _, _ = P.parac_pcg(G, n, None, None, None, np.ascontiguousarray(B[:, j]), tol=1e-8, maxit=500)
        assert abs(int(itj[0]) - int(it[j])) <= 1
        assert np.linalg.norm((xj - xj.mean()) - (X[:, j] - X[:, j].mean())) <= 1e-6 * np.linalg.norm(xj)
    G.free()


def _hub_system(n, seed):
    """A hub adjacent to every vertex, eliminated last: one factor row of about
    n entries (split into chunks by the solves)."""
    rng = np.random.default_rng(seed)
    a = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, 2 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 2 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    A = W.laplacian_from_edges(n, key // n, key % n, rng.uniform(0.5, 2.0, len(key)),
                               excess=rng.uniform(0.0, 0.1, n))
    perm = np.concatenate([rng.permutation(np.arange(1, n)), [0]]).astype(np.int32)
    return A, perm, W.gaussian_rhs(n, 1, seed + 1, center=False)


def _relres(A, x, b):
    import scipy.sparse as sp
    M = sp.csc_matrix((A.val, A.rowind, A.colptr), shape=(A.n, A.n))
    return np.linalg.norm(b - M @ x) / np.linalg.norm(b)


def test_pcg_many_thread_path_matches_single_calls(P):
    """With the per-system worker threads (pcg_many = PARAC_OFF) every
    system's result is bit-identical to its own parac_pcg call (host and device
    right-hand sides)."""
    import torch
    batch = W.sddm_batch(12, nmin=500, nmax=20000, seed=13)
    systems = [(A.n, A.colptr, A.rowind, A.val, perm) for (A, perm, b) in batch]
    Gs = P.parac_factor_many(systems, seed=3, opts=P.parac_opts_default(pcg_many=P.OFF))
    bs = [b for (A, perm, b) in batch]
    xs, its, rrs, status = P.parac_pcg_many(Gs, bs, tol=1e-8, maxit=500)
    assert status == "PARAC_OK" and np.all(rrs <= 1e-8)
    xd, itd, rrd, _ = P.parac_pcg_many(Gs, [torch.from_numpy(b).cuda() for b in bs], tol=1e-8, maxit=500)
    for i, ((A, perm, b), G) in enumerate(zip(batch, Gs)):
        x1, it1, rr1, _ = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-8, maxit=500)
        assert it1[0] == its[i] == itd[i] and rr1[0] == rrs[i]
        assert np.array_equal(x1, xs[i]) and np.array_equal(x1, xd[i].cpu().numpy())
    for G in Gs:
        G.free()


@pytest.mark.parametrize("prec", [64, 32])
def test_pcg_many_batched(P, prec):
    """The batched PCG (all systems as one block-diagonal system, levels
    interleaved in one schedule, per-system scalars): each system converges to
    the tolerance (true residual recomputed here), within one iteration of its
    own parac_pcg call (the systems' preconditioner applies are the same
    arithmetic; only the dot products' reduction order differs), and the
    result does not depend on where the right-hand sides live.  The batch
    includes a system with a split factor row (hub) and mixes sizes."""
    import torch
    batch = W.sddm_batch(11, nmin=300, nmax=30000, seed=17)
    batch.append(_hub_system(40000, 5))
    systems = [(A.n, A.colptr, A.rowind, A.val, perm) for (A, perm, b) in batch]
    Gs = P.parac_factor_many(systems, seed=9, opts=P.parac_opts_default(g_precision=prec))
    bs = [b for (A, perm, b) in batch]
    xs, its, rrs, status = P.parac_pcg_many(Gs, bs, tol=1e-8, maxit=800)
    assert status == "PARAC_OK" and np.all(rrs <= 1e-8)
    xd, itd, rrd, _ = P.parac_pcg_many(Gs, [torch.from_numpy(b).cuda() for b in bs], tol=1e-8, maxit=800)
    for i, ((A, perm, b), G) in enumerate(zip(batch, Gs)):
        assert np.array_equal(xs[i], xd[i].cpu().numpy()) and its[i] == itd[i] and rrs[i] == rrd[i]
        assert _relres(A, xs[i], b) <= 1.0001e-8
        assert abs(_relres(A, xs[i], b) - rrs[i]) <= 1e-3 * rrs[i] + 1e-14
        x1, it1, rr1, _ = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-8, maxit=800)
        assert abs(int(it1[0]) - int(its[i])) <= 1
        assert np.linalg.norm(x1 - xs[i]) <= 1e-5 * np.linalg.norm(x1)
    for G in Gs:
        G.free()


def test_pcg_many_batched_maxit(P):
    """A batched run stopped by maxit reports PARAC_ENOCONV with every system's
    iterations (= maxit unless it converged first) and true residual written."""
    batch = W.sddm_batch(6, nmin=2000, nmax=20000, seed=19)
    systems = [(A.n, A.colptr, A.rowind, A.val, perm) for (A, perm, b) in batch]
    Gs = P.parac_factor_many(systems, seed=4)
    bs = [b for (A, perm, b) in batch]
    xs, its, rrs, status = P.parac_pcg_many(Gs, bs, tol=1e-12, maxit=3)
    assert status == "PARAC_ENOCONV"
    for i, (A, perm, b) in enumerate(batch):
        assert its[i] == 3
        assert abs(_relres(A, xs[i], b) - rrs[i]) <= 1e-6 * rrs[i]
    for G in Gs:
        G.free()


@pytest.mark.parametrize("n", [40000, 120000])
def test_device_group_tables_match_host(P, n):
    """The warp-per-row solves' group tables (factors with rows of more than
    2,048 entries) built on the device equal the host builder's: the same
    group and partial-slot counts, and preconditioner applies and block PCG
    solves (which walk those tables, and the block solves' own ones) that
    agree bit for bit (every CSR row, the hub's included, is sorted by
    column, so two handles of one factor sum in the same order).  The hub
    row is longer than the split length, so chunk and combine groups are
    exercised."""
    A, perm, b = _hub_system(n, 7)
    r = np.ascontiguousarray(b, np.float64).reshape(-1)
    Bm = W.gaussian_rhs(n, 4, 9, center=False)
    out = []
    for host in (P.ON, P.DEFAULT):
        G = P.parac_factor(n, A.colptr, A.rowind, A.val, perm, 3,
                           P.parac_opts_default(host_tables=host, sptrsv=P.SPTRSV_WARP))
        st = G.stats()
        z = P.parac_precond_apply(G, r)
        X, it, rr, status = P.parac_pcg(G, n, A.colptr, A.rowind, A.val, Bm, tol=1e-8, maxit=200)
        out.append((st["solve_groups"], st["max_row_F"], z, X, it))
        G.free()
    (g0, m0, z0, X0, it0), (g1, m1, z1, X1, it1) = out
    assert m0 > 2048 and g0[0] > 0 and g0[1] > 0
    assert g0 == g1
    assert g0[2] > 0                           # the hub row (forward solve) is split: partial slots
    assert np.array_equal(z0.view(np.uint64), z1.view(np.uint64))
    assert np.array_equal(np.asarray(it0), np.asarray(it1))
    assert np.array_equal(np.asarray(X0).view(np.uint64), np.asarray(X1).view(np.uint64))
