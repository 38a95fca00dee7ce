"""Input generators: the Poisson stand-ins against an independent construction."""
import numpy as np
import scipy.sparse as sp

from paper_2505_02977_gb300 import workloads as W


def _tridiag(m):
    # 1D Dirichlet Laplacian: 2 on the diagonal (ghost neighbours at both ends), -1 off it
    return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])


def test_poisson_uniform_and_aniso_are_kronecker_sums():
    """7-point Dirichlet Poisson = eps_z T(x)I(x)I + I(x)T(x)I + I(x)I(x)T with x
    the fastest index (uniform: eps = 1; aniso: eps = 0.01 along z)."""
    m = 6
    I, T = sp.identity(m), _tridiag(m)
    for field, eps in (("uniform", 1.0), ("aniso", 0.01)):
        A = W.poisson3d(m, field).scipy().toarray()
        K = (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + eps * sp.kron(sp.kron(T, I), I)).toarray()
        assert np.allclose(A, K, rtol=0, atol=1e-14)


def test_poisson_contrast_field():
    """Contrast field: the coefficient is constant on 8^3 cell blocks with
    values 1 and 1e4 (both present); every grid edge carries minus the
    harmonic mean of its cells' coefficients, no other off-diagonal exists, and
    each row sums to its cell's coefficient times its number of boundary faces."""
    m, blk = 16, 8
    A = W.poisson3d(m, "contrast", seed=3, block=blk)
    k = A.meta["kappa"].reshape(m, m, m)
    for bz in range(0, m, blk):
        for by in range(0, m, blk):
            for bx in range(0, m, blk):
                cell = k[bz:bz + blk, by:by + blk, bx:bx + blk]
                assert np.all(cell == cell.flat[0]) and cell.flat[0] in (1.0, 1e4)
    assert set(np.unique(k)) == {1.0, 1e4}
    D = A.scipy().toarray()
    kf = k.ravel()
    expect = np.zeros_like(D)
    idx = np.arange(m ** 3).reshape(m, m, m)
    for sl_a, sl_b in (((slice(None), slice(None), slice(0, m - 1)), (slice(None), slice(None), slice(1, m))),
                       ((slice(None), slice(0, m - 1), slice(None)), (slice(None), slice(1, m), slice(None))),
                       ((slice(0, m - 1), slice(None), slice(None)), (slice(1, m), slice(None), slice(None)))):
        a, b = idx[sl_a].ravel(), idx[sl_b].ravel()
        w = 2 * kf[a] * kf[b] / (kf[a] + kf[b])
        expect[a, b] = -w; expect[b, a] = -w
    off = D - np.diag(np.diag(D))
    assert np.allclose(off, expect, rtol=1e-15, atol=0)
    z, y, x = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    faces = ((x == 0) * 1 + (x == m - 1) + (y == 0) + (y == m - 1) + (z == 0) + (z == m - 1)).ravel()
    assert np.allclose(D.sum(1), kf * faces, rtol=1e-12, atol=1e-9)


def test_splitmix64_outputs():
    """The vectorised splitmix64 matches a plain integer restatement of the
    published generator, whose first output from state 0 is 0xE220A8397B1DCDAF."""
    M = (1 << 64) - 1

    def ref(seed, count):
        out, st = [], seed
        for _ in range(count):
            st = (st + 0x9E3779B97F4A7C15) & M
            z = st
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            out.append(z ^ (z >> 31))
        return out
    assert int(W.splitmix64_outputs(0, 1)[0]) == 0xE220A8397B1DCDAF
    for seed in (0, 1, 12345, 2 ** 63 + 7):
        assert [int(v) for v in W.splitmix64_outputs(seed, 50)] == ref(seed, 50)


def test_nnz_sorted_ordering_definition():
    """Sec. V NNZ-sorted ordering: a permutation, stored-entry counts
    non-decreasing along it, equal counts ordered by the seeded key, then index."""
    A, _, _, _ = W.config("grid2d-64")
    for seed in (0, 5):
        o = W.nnz_sorted_ordering(A, seed)
        assert np.array_equal(np.sort(o), np.arange(A.n))
        deg = np.diff(A.colptr)[o]
        assert np.all(np.diff(deg) >= 0)
        key = (W.splitmix64_outputs(seed, A.n) >> np.uint64(33)).astype(np.int64)[o]
        same = np.diff(deg) == 0
        assert np.all((np.diff(key) > 0) | ((np.diff(key) == 0) & (np.diff(o) > 0)) | ~same)
