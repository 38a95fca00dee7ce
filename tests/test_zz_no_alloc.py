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
    r = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.ParacError) as e:       # host memory is refused
        P._check(P._lib.parac_precond_apply_noalloc(G.handle, np.zeros(A.n).ctypes.data, r.data_ptr()), "noalloc")
    assert e.value.status == "PARAC_EINVAL"
    G.free()
    big = W.config("grid3d-64")[0]                # 262,144 unknowns: exactly at the limit
    Gb = P.parac_factor(big.n, big.colptr, big.rowind, big.val, None, 1)
    rb = torch.ones(big.n, dtype=torch.float64, device="cuda")
    rb -= rb.mean()
    zb = torch.empty_like(rb)
    P.parac_precond_apply_noalloc(Gb, rb, zb)
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
