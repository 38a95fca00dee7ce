"""Seeded synthetic inputs shaped like the ParAC paper's workloads.

This module only builds inputs: graphs, their Laplacian/SDDM matrices in full
symmetric CSC form (Sec. V sign convention: positive diagonal, non-positive
off-diagonals), elimination orderings and right-hand sides.  It holds none of
the factorisation or solver arithmetic, and both the CUDA path and the CPU
oracle consume exactly the arrays it returns.

Stand-ins for the paper's matrices (Table I), which are not available here:
  * 2D / 3D grid Laplacians (5- and 7-point stencils) for the structured PDE
    rows (uniform / contrast 3D Poisson);
  * R-MAT power-law graphs for com-LiveJournal (17.35 nnz/col, Sec. V);
  * random geometric, Erdos-Renyi and grid SDDM systems with random diagonal
    excess for the 200 SDDM2023 "chimera" systems (Sec. V-C).
"""
import os

import numpy as np

__all__ = [
    "Matrix", "laplacian_from_edges", "grid2d_edges", "grid3d_edges", "rmat_edges",
    "rgg_edges", "er_edges", "largest_component", "random_ordering", "nnz_sorted_ordering",
    "gaussian_rhs", "path_edges", "cycle_edges", "random_tree_edges", "leaf_first_ordering",
    "sparse_random_edges", "config", "sddm_batch", "CONFIGS",
]


class Matrix:
    """Full symmetric CSC matrix (colptr int64[n+1], rowind int32[nnz], val f64[nnz])."""

    def __init__(self, n, colptr, rowind, val, meta=None):
        self.n = int(n)
        self.colptr = np.ascontiguousarray(colptr, np.int64)
        self.rowind = np.ascontiguousarray(rowind, np.int32)
        self.val = np.ascontiguousarray(val, np.float64)
        self.meta = dict(meta or {})

    @property
    def nnz(self):
        return int(self.colptr[-1])

    def dense(self):
        A = np.zeros((self.n, self.n))
        for j in range(self.n):
            for t in range(self.colptr[j], self.colptr[j + 1]):
                A[self.rowind[t], j] += self.val[t]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csc_matrix((self.val, self.rowind, self.colptr), shape=(self.n, self.n))


def laplacian_from_edges(n, i, j, w, excess=None):
    """Laplacian (plus optional diagonal excess -> SDDM) of an undirected graph.

    Each undirected edge (i, j, w > 0) appears once in the input; duplicate
    edges are allowed and simply add up.  Self-loops must be removed first.
    The diagonal is the weighted degree plus ``excess``.  Rows are sorted
    within each column; every column stores its diagonal entry.
    """
    i = np.asarray(i, np.int64); j = np.asarray(j, np.int64); w = np.asarray(w, np.float64)
    assert np.all(i != j), "self-loops are not edges of a Laplacian"
    deg = np.bincount(i, weights=w, minlength=n) + np.bincount(j, weights=w, minlength=n)
    diag = deg if excess is None else deg + np.asarray(excess, np.float64)
    rows = np.concatenate([i, j, np.arange(n)])
    cols = np.concatenate([j, i, np.arange(n)])
    vals = np.concatenate([-w, -w, diag])
    key = cols * n + rows
    order = np.argsort(key, kind="stable")
    rows = rows[order]; cols = cols[order]; vals = vals[order]
    colptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(cols, minlength=n), out=colptr[1:])
    return Matrix(n, colptr, rows.astype(np.int32), vals)


# --------------------------------------------------------------------------- graphs
def grid2d_edges(nx, ny):
    idx = np.arange(nx * ny).reshape(ny, nx)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return a, b


def grid3d_edges(nx, ny, nz):
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    a = np.concatenate([idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()])
    b = np.concatenate([idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()])
    return a, b


def _sorted_unique(x):
    """np.unique(x) for an int64 array, by sort and neighbour comparison."""
    x = np.sort(x)
    if len(x) == 0:
        return x
    keep = np.empty(len(x), bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def rmat_edges(scale, edge_factor, a=0.57, b=0.19, c=0.19, seed=0, chunk=1 << 24):
    """R-MAT (Chakrabarti et al.) edge list: symmetrised, self-loops dropped, deduplicated."""
    rng = np.random.default_rng(seed)
    m = edge_factor << scale
    n = 1 << scale
    keys = []
    for s0 in range(0, m, chunk):
        cnt = min(chunk, m - s0)
        src = np.zeros(cnt, np.int64); dst = np.zeros(cnt, np.int64)
        for lvl in range(scale):
            u = rng.random(cnt)
            ibit = u >= (a + b)
            jbit = ((u >= a) & (u < a + b)) | (u >= a + b + c)
            src |= ibit.astype(np.int64) << lvl
            dst |= jbit.astype(np.int64) << lvl
        keep = src != dst
        lo = np.minimum(src[keep], dst[keep]); hi = np.maximum(src[keep], dst[keep])
        keys.append(_sorted_unique(lo * n + hi))
    key = _sorted_unique(np.concatenate(keys))
    return n, (key // n), (key % n)


def rgg_edges(n, radius, seed=0):
    """Random geometric graph in the unit square."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
    return pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)


def er_edges(n, p, seed=0):
    """Erdos-Renyi G(n, p) by geometric skipping over the pairs i < j."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    out = []
    pos = -1
    while True:
        gaps = rng.geometric(p, size=max(1024, int(total * p * 1.1) + 16))
        idx = pos + np.cumsum(gaps)
        keep = idx[idx < total]
        out.append(keep)
        if len(keep) < len(idx):
            break
        pos = int(idx[-1])
    t = np.concatenate(out).astype(np.int64)
    # pair index t enumerates (i, j), i < j, row by row
    i = np.floor((2 * n - 1 - np.sqrt((2.0 * n - 1) ** 2 - 8.0 * t)) / 2).astype(np.int64)
    start = i * (2 * n - i - 1) // 2
    fix_lo = t < start
    i[fix_lo] -= 1
    start = i * (2 * n - i - 1) // 2
    fix_hi = t >= start + (n - 1 - i)
    i[fix_hi] += 1
    start = i * (2 * n - i - 1) // 2
    j = t - start + i + 1
    return i, j


def path_edges(n):
    return np.arange(n - 1), np.arange(1, n)


def cycle_edges(n):
    return np.arange(n), (np.arange(n) + 1) % n


def random_tree_edges(n, seed=0):
    """Random recursive tree: vertex v > 0 attaches to a uniform earlier vertex."""
    rng = np.random.default_rng(seed)
    par = np.array([rng.integers(0, v) for v in range(1, n)], np.int64)
    return par, np.arange(1, n)


def leaf_first_ordering(n, a, b, seed=0):
    """An ordering of a tree in which every vertex is a leaf of the remaining tree when
    eliminated (repeatedly strip a random current leaf)."""
    rng = np.random.default_rng(seed)
    adj = [set() for _ in range(n)]
    for x, y in zip(a, b):
        adj[int(x)].add(int(y)); adj[int(y)].add(int(x))
    deg = np.array([len(s) for s in adj])
    leaves = [v for v in range(n) if deg[v] <= 1]
    order = []
    alive = np.ones(n, bool)
    while leaves:
        t = int(rng.integers(0, len(leaves)))
        v = leaves[t]; leaves[t] = leaves[-1]; leaves.pop()
        if not alive[v]:
            continue
        alive[v] = False
        order.append(v)
        for u in adj[v]:
            if alive[u]:
                adj[u].discard(v)
                deg[u] -= 1
                if deg[u] == 1 or (deg[u] == 0 and len(order) == n - 1):
                    leaves.append(u)
    for v in range(n):
        if alive[v]:
            order.append(v)
    return np.array(order, np.int32)


def sparse_random_edges(n, m, seed=0, connected=True):
    """Random simple graph with about m edges (plus a random spanning tree if connected)."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, m); b = rng.integers(0, n, m)
    if connected and n > 1:
        ta, tb = random_tree_edges(n, seed + 7)
        a = np.concatenate([a, ta]); b = np.concatenate([b, tb])
    keep = a != b
    lo = np.minimum(a[keep], b[keep]); hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    return key // n, key % n


def largest_component(n, a, b):
    """Restrict an edge list to its largest connected component, relabelled 0..n'-1."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    if n == 0:
        return 0, a, b
    g = sp.coo_matrix((np.ones(len(a), np.int8), (a, b)), shape=(n, n))
    ncomp, lab = connected_components(g, directed=False)
    big = np.argmax(np.bincount(lab))
    keepv = lab == big
    newid = -np.ones(n, np.int64)
    newid[keepv] = np.arange(int(keepv.sum()))
    ke = keepv[a]
    return int(keepv.sum()), newid[a[ke]], newid[b[ke]]


# --------------------------------------------------------------------------- orderings / rhs
def random_ordering(n, seed):
    """Uniformly random elimination order: ordering[k] = vertex eliminated k-th."""
    return np.random.default_rng(seed).permutation(n).astype(np.int32)


def splitmix64_outputs(seed, count):
    """Outputs 1..count of the splitmix64 generator started from state `seed`
    (Steele, Lea, Flood, OOPSLA 2014), as uint64."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.arange(1, count + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def nnz_sorted_ordering(mat, seed):
    """Sec. V 'NNZ-Sorted' ordering: columns by ascending stored-entry count,
    ties by the top 31 bits of the (v+1)-th splitmix64 output from state
    `seed`, then by index v."""
    n = mat.n
    deg = np.diff(mat.colptr)
    tie = (splitmix64_outputs(seed, n) >> np.uint64(33)).astype(np.int64)
    return np.lexsort((np.arange(n), tie, deg)).astype(np.int32)


def gaussian_rhs(n, nrhs=1, seed=0, center=True):
    """Zero-mean Gaussian right-hand sides, column-major n x nrhs (mean-centred per column)."""
    B = np.random.default_rng(seed).standard_normal((nrhs, n))
    if center:
        B -= B.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(B.T if nrhs > 1 else B[0])


# --------------------------------------------------------------------------- configurations
def _grid2d(side, weights, seed):
    a, b = grid2d_edges(side, side)
    if weights == "unit":
        w = np.ones(len(a))
    else:
        lo, hi = weights
        w = np.random.default_rng(seed).uniform(lo, hi, len(a))
    return laplacian_from_edges(side * side, a, b, w)


def _grid3d(side, weights, seed):
    a, b = grid3d_edges(side, side, side)
    lo, hi = weights
    w = np.random.default_rng(seed).uniform(lo, hi, len(a))
    return laplacian_from_edges(side ** 3, a, b, w)


def poisson3d(side, field="uniform", seed=0, eps=0.01, block=8, contrast=1e4):
    """7-point finite-difference Poisson matrix on a side^3 grid with Dirichlet
    boundary (a ghost neighbour beyond each face: SDDM, the boundary rows carry
    the missing neighbours' weights as excess).  Coefficient fields:
      uniform   every edge weight 1
      aniso     weights 1, 1, eps along x, y, z (eps = 0.01: 100:1 anisotropy)
      contrast  per-cell coefficient 1 or `contrast` (1e4) on block^3 cell blocks,
                each block's value drawn with probability 1/2 (seed); an edge gets the
                harmonic mean 2 k_a k_b / (k_a + k_b) of its cells' coefficients
    The paper's anisotropy and contrast fields are not specified; these are
    stated stand-ins."""
    n = side ** 3
    idx = np.arange(n).reshape(side, side, side)          # [z, y, x]
    if field == "contrast":
        nb = (side + block - 1) // block
        kb = np.where(np.random.default_rng(seed).random((nb, nb, nb)) < 0.5, 1.0, contrast)
        z, y, x = np.meshgrid(np.arange(side), np.arange(side), np.arange(side), indexing="ij")
        kappa = kb[z // block, y // block, x // block].ravel()
    else:
        kappa = np.ones(n)
    dir_w = {"x": 1.0, "y": 1.0, "z": eps if field == "aniso" else 1.0}
    a_l, b_l, w_l = [], [], []
    exc = np.zeros(n)
    for axis, name in ((2, "x"), (1, "y"), (0, "z")):
        lo = [slice(None)] * 3; hi = [slice(None)] * 3
        lo[axis] = slice(0, side - 1); hi[axis] = slice(1, side)
        a = idx[tuple(lo)].ravel(); b = idx[tuple(hi)].ravel()
        ka, kb2 = kappa[a], kappa[b]
        w = dir_w[name] * 2.0 * ka * kb2 / (ka + kb2)
        a_l.append(a); b_l.append(b); w_l.append(w)
        # ghost neighbours beyond the two faces along this axis
        first = [slice(None)] * 3; last = [slice(None)] * 3
        first[axis] = 0; last[axis] = side - 1
        for face in (idx[tuple(first)].ravel(), idx[tuple(last)].ravel()):
            exc[face] += dir_w[name] * kappa[face]
    A = laplacian_from_edges(n, np.concatenate(a_l), np.concatenate(b_l), np.concatenate(w_l), excess=exc)
    A.meta.update(field=field, side=side, kappa=kappa)
    return A


def _rmat(scale, seeds):
    n, a, b = rmat_edges(scale, 16, seed=seeds[0])
    n, a, b = largest_component(n, a, b)
    w = np.random.default_rng(seeds[1]).lognormal(0.0, 1.0, len(a))
    return laplacian_from_edges(n, a, b, w)


def config(name, side=None):
    """Workload by name: returns (Matrix, ordering, factor seed, rhs); cached as
    an .npz file in the directory named by PARAC_WORKLOAD_CACHE when that is set
    (the generators are deterministic, so the cache only saves time)."""
    cache = os.environ.get("PARAC_WORKLOAD_CACHE")
    if cache:
        path = os.path.join(cache, f"{name}.npz")
        if os.path.exists(path):
            z = np.load(path)
            A = Matrix(int(z["n"]), z["colptr"], z["rowind"], z["val"])
            return A, z["perm"], int(z["seed"]), z["b"]
        out = _config(name)
        os.makedirs(cache, exist_ok=True)
        A, perm, seed, b = out
        np.savez(path, n=A.n, colptr=A.colptr, rowind=A.rowind, val=A.val, perm=perm, seed=seed, b=b)
        return out
    return _config(name)


def _config(name):
    """Workload by name: returns (Matrix, ordering, factor seed, rhs).

    grid2d-64     64x64 5-point grid, unit weights (n = 4096)
    grid3d-128    128^3 7-point grid, weights U[1,10) (n = 2,097,152)
    rmat-22       R-MAT scale 22, edge factor 16, (.57,.19,.19,.05), lognormal(0,1) weights, LCC
    rmat-24       as rmat-22 at scale 24, 32 right-hand sides
    grid3d-N      N^3 grid as grid3d-128 (smaller cases for tests)
    poisson-F-N   N^3 Dirichlet Poisson (F = uniform, aniso, contrast; see poisson3d)
    """
    if name == "grid2d-64":
        A = _grid2d(64, "unit", 0)
        return A, random_ordering(A.n, 1), 2, gaussian_rhs(A.n, 1, 3)
    if name.startswith("grid3d-"):
        s = int(name.split("-")[1])
        A = _grid3d(s, (1.0, 10.0), 11)
        return A, random_ordering(A.n, 12), 13, gaussian_rhs(A.n, 1, 14)
    if name == "rmat-22":
        A = _rmat(22, (21, 22))
        return A, random_ordering(A.n, 23), 24, gaussian_rhs(A.n, 1, 25)
    if name == "rmat-24":
        A = _rmat(24, (41, 42))
        return A, random_ordering(A.n, 43), 45, gaussian_rhs(A.n, 32, 44)
    if name.startswith("poisson-"):                # poisson-{uniform,aniso,contrast}-N
        _, field, side = name.split("-")
        A = poisson3d(int(side), field, seed=51)
        return A, random_ordering(A.n, 52), 53, gaussian_rhs(A.n, 1, 54, center=False)
    if name.startswith("rmat-"):
        s = int(name.split("-")[1])
        A = _rmat(s, (21 + s, 22 + s))
        return A, random_ordering(A.n, 23 + s), 24 + s, gaussian_rhs(A.n, 1, 25 + s)
    raise KeyError(name)


CONFIGS = ("grid2d-64", "grid3d-128", "rmat-22", "sddm-batch-200", "rmat-24")


def sddm_batch(count=200, nmin=1000, nmax=200000, seed=31):
    """Heterogeneous SDDM systems: n log-uniform in [nmin, nmax], families in equal
    thirds (2D grid, random geometric graph with mean degree ~8, Erdos-Renyi with
    mean degree 10); weights U[0.1,10); diagonal excess U[0,0.1] x weighted degree;
    degree-0 vertices dropped.  Returns a list of (Matrix, ordering, rhs)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        fam = s % 3
        sub = int(rng.integers(0, 2 ** 31))
        if fam == 0:
            side = max(2, int(round(np.sqrt(n))))
            a, b = grid2d_edges(side, side); nv = side * side
        elif fam == 1:
            a, b = rgg_edges(n, np.sqrt(8.0 / (np.pi * n)), seed=sub); nv = n
        else:
            a, b = er_edges(n, 10.0 / (n - 1), seed=sub); nv = n
        used = np.zeros(nv, bool); used[a] = True; used[b] = True
        newid = -np.ones(nv, np.int64); newid[used] = np.arange(int(used.sum()))
        a = newid[a]; b = newid[b]; nv = int(used.sum())
        r2 = np.random.default_rng(sub + 1)
        w = r2.uniform(0.1, 10.0, len(a))
        deg = np.bincount(a, weights=w, minlength=nv) + np.bincount(b, weights=w, minlength=nv)
        exc = r2.uniform(0.0, 0.1, nv) * deg
        A = laplacian_from_edges(nv, a, b, w, excess=exc)
        A.meta.update(family=("grid2d", "rgg", "er")[fam], index=s)
        out.append((A, random_ordering(nv, sub + 2), gaussian_rhs(nv, 1, sub + 3, center=False)))
    return out
