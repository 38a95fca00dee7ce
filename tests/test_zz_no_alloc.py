"""The allocation-free preconditioner apply (parac_precond_apply_noalloc).

It serves callers that cannot allocate device memory where they apply the
preconditioner.  Called through the C ABI, it must give the same z = M^{-1} r
as parac_precond_apply on consecutive calls (the shared work array keeps the
previous call's values, which must not leak into the next result), and it must
refuse factors larger than its fixed work array and host pointers.  This file
is collected last, so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_2505_02977_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_allocating_apply_twice():
    import torch
    from paper_2505_02977_gb300 import parac as P
    A, perm, seed, _ = W.config("grid3d-32")
    for prec in (64, 32):
        G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, P.parac_opts_default(g_precision=prec))
        rng = np.random.default_rng(prec)
        for call in range(2):
            r_host = rng.standard_normal(A.n)
            z_ref = P.parac_precond_apply(G, r_host)
            r = torch.from_numpy(r_host).cuda()
            z = torch.full_like(r, float("nan"))
            P.parac_precond_apply_noalloc(G, r, z)
            torch.cuda.synchronize()
            zd = z.cpu().numpy()
            assert np.all(np.isfinite(zd)), (prec, call)
            assert np.linalg.norm(zd - z_ref) <= 1e-12 * np.linalg.norm(z_ref), (prec, call)
        G.free()


def test_noalloc_apply_limits():
    import torch
    from paper_2505_02977_gb300 import parac as P
    A, perm, seed, _ = W.config("grid2d-64")
    G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed)
    dev0 = torch.cuda.current_device()
    r = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.ParacError) as e:       # host memory is refused
        P._check(P._lib.parac_precond_apply_noalloc(G.handle, np.zeros(A.n).ctypes.data, r.data_ptr()), "noalloc")
    assert e.value.status == "PARAC_EINVAL"
    G.free()
    assert torch.cuda.current_device() == dev0     # an error return leaves the caller's device current
    big = W.config("grid3d-64")[0]                # 262,144 unknowns: exactly at the limit
    for prec in (64, 32):                          # the backward unknowns end at the array's last element
        Gb = P.parac_factor(big.n, big.colptr, big.rowind, big.val, None, 1, P.parac_opts_default(g_precision=prec))
        rh = np.random.default_rng(prec + 1).standard_normal(big.n)
        rb = torch.from_numpy(rh).cuda()
        zb = torch.full_like(rb, float("nan"))
        P.parac_precond_apply_noalloc(Gb, rb, zb)
        torch.cuda.synchronize()
        z_ref = P.parac_precond_apply(Gb, rh)
        zd = zb.cpu().numpy()
        assert np.linalg.norm(zd - z_ref) <= 1e-12 * np.linalg.norm(z_ref), prec
        Gb.free()
    n = (1 << 18) + 1                              # one unknown too many
    a, b = W.path_edges(n)
    Pm = W.laplacian_from_edges(n, a, b, np.ones(n - 1))
    Gp = P.parac_factor(n, Pm.colptr, Pm.rowind, Pm.val, None, 1)
    rp = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.ParacError) as e:
        P.parac_precond_apply_noalloc(Gp, rp, torch.empty_like(rp))
    assert e.value.status == "PARAC_EINVAL"
    Gp.free()


def _hub(n, seed):
    """A hub adjacent to every vertex and eliminated last: its factor row has
    about n entries, which the solves split into chunks whose partial sums
    meet in slots of the handle (reset by every apply)."""
    rng = np.random.default_rng(seed)
    a = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, 2 * n)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, 2 * n)])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    A = W.laplacian_from_edges(n, key // n, key % n, rng.uniform(0.5, 2.0, len(key)))
    perm = np.concatenate([rng.permutation(np.arange(1, n)), [0]]).astype(np.int32)
    return A, perm


def test_noalloc_apply_split_rows_twice():
    """A factor with a row of ~40,000 entries (split-row chunks) under the
    2^18 limit: two calls in a row equal the allocating apply."""
    import torch
    from paper_2505_02977_gb300 import parac as P
    A, perm = _hub(40000, 3)
    for prec in (64, 32):
        G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, 3, P.parac_opts_default(g_precision=prec))
        assert np.bincount(G.export()["row"], minlength=A.n).max() > 4 * 8192
        rng = np.random.default_rng(prec)
        for call in range(2):
            r_host = rng.standard_normal(A.n)
            z_ref = P.parac_precond_apply(G, r_host)
            r = torch.from_numpy(r_host).cuda()
            z = torch.full_like(r, float("nan"))
            P.parac_precond_apply_noalloc(G, r, z)
            torch.cuda.synchronize()
            zd = z.cpu().numpy()
            assert np.linalg.norm(zd - z_ref) <= 1e-12 * np.linalg.norm(z_ref), (prec, call)
        G.free()


def test_noalloc_apply_rejects_another_devices_memory():
    """Vectors on a device other than the factor's are refused (needs two GPUs)."""
    import torch
    from paper_2505_02977_gb300 import parac as P
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible device")
    A, perm, seed, _ = W.config("grid2d-64")
    G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed)
    r = torch.zeros(A.n, dtype=torch.float64, device="cuda:1")
    with pytest.raises(P.ParacError) as e:
        P.parac_precond_apply_noalloc(G, r, torch.empty_like(r))
    assert e.value.status == "PARAC_EINVAL"
    G.free()
