"""GPU parity of the mixed-precision form and of the batched PCG against the
oracle.

Mixed form: the factor is stored and applied in FP32 while PCG's
recurrences stay FP64.  The oracle's FP32 apply follows the same reading
(F and the right-hand side rounded to FP32, FP32 triangular solves, D^+ in
FP64 with the product rounded to FP32) and comes with a componentwise
running-error bound that holds for any order of the FP32 sums.  The GPU and
the oracle add the terms of a row in different orders, so:
  * where every solve row and column has at most one entry (an exactly
    factored path in label order) the two are bit-identical;
  * elsewhere each evaluation lies within its own bound of the exact apply,
    so they differ by at most the sum of the two bounds.  The bounds differ
    only through the computed intermediates, which agree to well under 1%,
    so 2.1 times the oracle's bound covers both.
Batched PCG: every system of parac_pcg_many is checked against the oracle's
PCG for that system (same factor, same precision), not against parac_pcg.
"""
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


def _factor(P, A, perm, seed, **opts):
    return P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, P.parac_opts_default(**opts))


def _hub_system(n, seed):
    """A hub adjacent to every vertex, eliminated last, plus random edges and
    a small diagonal excess (SDDM): one factor row of about n entries, which
    the solves split into chunks summed by separate blocks."""
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


def test_fp32_apply_bit_identical_on_exact_path(P):
    """Path in label order, weights in [1, 2): F(j+1,j) = -1, D_j = w_j, every
    forward row and backward column holds one entry, so the GPU's FP32 apply
    performs exactly the oracle's roundings."""
    n = 20000
    rng = np.random.default_rng(41)
    a, b = W.path_edges(n)
    A = W.laplacian_from_edges(n, a, b, rng.uniform(1, 2, n - 1))
    G = _factor(P, A, None, 1, g_precision=32)
    F = oracle.factor(A.colptr, A.rowind, A.val, None, seed=1)
    assert same_factor(G.export(), F)
    for call in range(2):
        r = rng.standard_normal(n)
        z = P.parac_precond_apply(G, r)
        zo = oracle.precond_apply(F, None, r, prec=32)
        assert np.array_equal(z, zo), call
    G.free()


def _mixed_cases():
    out = {}
    A, perm, seed, _ = W.config("grid3d-32")
    out["grid3d-32"] = (A, perm, seed)
    A, perm, _ = _hub_system(40000, 5)
    out["hub-40000"] = (A, perm, 7)
    A, perm, seed, _ = W.config("rmat-15")
    out["rmat-15"] = (A, perm, seed)
    return out


@pytest.mark.parametrize("name", ["grid3d-32", "hub-40000", "rmat-15"])
def test_fp32_apply_within_bound_of_oracle(P, name):
    """The GPU's FP32 apply against the oracle's, element by element, within
    2.1 times the oracle's running-error bound; the FP64 apply on the same
    factor within 1e-12 of the oracle's FP64 apply."""
    A, perm, seed = _mixed_cases()[name]
    G32 = _factor(P, A, perm, seed, g_precision=32)
    G64 = _factor(P, A, perm, seed, g_precision=64)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    assert same_factor(G32.export(), F)
    rng = np.random.default_rng(3)
    for _ in range(2):
        r = rng.standard_normal(A.n)
        z = P.parac_precond_apply(G32, r)
        zo, bd = oracle.precond_apply(F, perm, r, prec=32, bound=True)
        err = np.abs(z - zo)
        worst = int(np.argmax(err - 2.1 * bd))
        assert np.all(err <= 2.1 * bd), (worst, err[worst], bd[worst])
        z64 = P.parac_precond_apply(G64, r)
        zo64 = oracle.precond_apply(F, perm, r)
        assert np.linalg.norm(z64 - zo64) <= 1e-12 * np.linalg.norm(zo64)
    G32.free(); G64.free()


@pytest.mark.parametrize("name", ["grid3d-32", "hub-40000", "rmat-15"])
def test_fp32_pcg_matches_oracle(P, name):
    """PCG with the FP32 factor reaches a true relative residual of 1e-8 (also
    recomputed here), within one iteration of the oracle's mixed-form PCG; the
    FP64 oracle's count is reported beside it."""
    import scipy.sparse as sp
    A, perm, seed = _mixed_cases()[name]
    sddm = name.startswith("hub")
    b = W.gaussian_rhs(A.n, 1, 77, center=not sddm)
    G = _factor(P, A, perm, seed, g_precision=32)
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed)
    x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, b, tol=1e-8, maxit=2000)
    xo, ito, rro = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 2000, prec=32)
    _, it64, rr64 = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 2000)
    M = sp.csc_matrix((A.val, A.rowind, A.colptr), shape=(A.n, A.n))
    true_rr = np.linalg.norm(b - M @ x) / np.linalg.norm(b)
    print(f"{name}: FP32-G PCG iterations GPU {int(it[0])}, oracle {ito}; FP64 oracle {it64}; "
          f"true relres GPU {true_rr:.2e}, oracle {rro:.2e}")
    assert status == "PARAC_OK" and rr[0] <= 1e-8 and true_rr <= 1.0001e-8 and rro <= 1e-8 and rr64 <= 1e-8
    assert abs(int(it[0]) - ito) <= 1
    G.free()


def _batch():
    batch = W.sddm_batch(9, nmin=300, nmax=30000, seed=17)
    batch.append(_hub_system(40000, 5))
    return batch


@pytest.mark.parametrize("prec", [64, 32])
def test_pcg_many_each_system_matches_oracle(P, prec):
    """parac_pcg_many on a mixed batch (three families, a split-row hub
    system): each system's factor is the oracle's for its batch index; each
    converges to 1e-8 within one iteration of the oracle's PCG in the same
    precision; and after the same number of iterations (tol = 0) each iterate
    agrees with the oracle's to 1e-8 (FP64) or 1e-5 (FP32 factor: the FP32
    sums are reduced in another order, an FP32-sized difference per apply
    that CG carries forward) relative."""
    batch = _batch()
    systems = [(A.n, A.colptr, A.rowind, A.val, perm) for (A, perm, b) in batch]
    seed = 9
    Gs = P.parac_factor_many(systems, seed=seed, opts=P.parac_opts_default(g_precision=prec))
    bs = [b for (A, perm, b) in batch]
    xs, its, rrs, status = P.parac_pcg_many(Gs, bs, tol=1e-8, maxit=800)
    assert status == "PARAC_OK" and np.all(rrs <= 1e-8)
    Fs, ito = [], []
    for s, ((A, perm, b), G) in enumerate(zip(batch, Gs)):
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, sys=s)
        assert same_factor(G.export(), F), s
        xo, it_o, rr_o = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, b, 1e-8, 800, prec=prec)
        assert rr_o <= 1e-8
        assert abs(int(its[s]) - it_o) <= 1, (s, int(its[s]), it_o)
        Fs.append(F); ito.append(it_o)
    k = min(ito)
    xk, itk, _, _ = P.parac_pcg_many(Gs, bs, tol=0.0, maxit=k)
    tol = 1e-8 if prec == 64 else 1e-5
    for s, (A, perm, b) in enumerate(batch):
        assert itk[s] == k
        xo, _, _ = oracle.pcg(A.colptr, A.rowind, A.val, Fs[s], perm, b, 0.0, k, prec=prec)
        assert np.linalg.norm(xk[s] - xo) <= tol * np.linalg.norm(xo), s
    for G in Gs:
        G.free()
