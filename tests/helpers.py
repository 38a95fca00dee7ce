"""Test-side helpers: dense reconstructions used to check factors."""
import numpy as np


def dense_factor(F):
    """Dense unit-lower F (label space) and D from a CSC factor dict."""
    n = F["n"]
    Fd = np.eye(n)
    for k in range(n):
        for t in range(F["colptr"][k], F["colptr"][k + 1]):
            Fd[F["row"][t], k] = F["val"][t]
    return Fd, np.asarray(F["D"][:n], float)


def reconstruct(F, ordering):
    """F D F^T mapped back to original vertex numbering."""
    Fd, D = dense_factor(F)
    G = Fd @ np.diag(D) @ Fd.T
    n = F["n"]
    perm = np.arange(n) if ordering is None else np.asarray(ordering)
    A = np.zeros((n, n))
    A[np.ix_(perm, perm)] = G
    return A


def same_factor(F1, F2):
    """Bitwise equality of two CSC factors (structure, values, pivots)."""
    return (F1["n"] == F2["n"] and np.array_equal(F1["colptr"], F2["colptr"])
            and np.array_equal(F1["row"], F2["row"])
            and np.array_equal(F1["val"].view(np.uint64), F2["val"].view(np.uint64))
            and np.array_equal(np.asarray(F1["D"]).view(np.uint64), np.asarray(F2["D"]).view(np.uint64)))
