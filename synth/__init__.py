"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module builds matrices and right-hand sides only.  It holds none of the
solver's arithmetic (no message, aggregate or residual formula): it draws
random numbers from ``numpy.random.default_rng(seed)`` (PCG64, identical on
x86-64 and aarch64) and assembles symmetric CSR matrices.

Every matrix is returned as a :class:`CSR` holding the FULL symmetric matrix,
diagonal included, with strictly increasing column indices inside each row.

Workload shapes follow the paper's experiments and the benchmark configurations:

* ``grid2d``      -- 2-D 5-point Poisson stencil (Sec. "2-D Poisson's Equation").
* ``random_sym``  -- sparse random symmetric diagonally dominant matrix; stands
  in for the paper's social-network graphs (Sec. "Rating Users ...", 1M nodes,
  about 10M edges), whose data is not available.
* ``grid3d``      -- 3-D 7-point heterogeneous diffusion stencil.
* ``rgg_batch``   -- many random geometric graphs of power-law sizes.
* ``random_tree`` -- trees, on which GaBP is exact (Sec. "Convergence and Exactness").
* ``toy3x3`` / ``nonpsd3x3`` / ``cdma_r3`` / ``cdma_r4`` / ``run_gabp_3x3`` --
  the small matrices printed in the paper's numerical examples.
* ``random_rect`` -- a sparse rectangular matrix (``RectCSR``), the data matrix of the
  least-squares / MMSE-detection workloads (Sec. "Extension to General Linear Systems",
  Chapter "Extending GaBP to support non-square matrices"); stands in for a sparse
  spreading or measurement matrix.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "from_coo", "from_dense", "to_dense",
    "grid2d", "poisson2d", "random_sym", "grid3d", "rgg_batch", "random_tree",
    "toy3x3", "nonpsd3x3", "cdma_r3", "cdma_r4", "run_gabp_3x3",
    "rhs", "rhs_batch", "spd_seed", "block_diag", "RectCSR", "random_rect",
]


@dataclass
class CSR:
    """Full symmetric sparse matrix in CSR form (diagonal stored explicitly)."""
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def num_edges(self) -> int:
        """Directed edges = off-diagonal stored entries."""
        return self.nnz - self.n


@dataclass
class RectCSR:
    """Rectangular sparse matrix (m rows, k columns) in CSR form, strictly increasing columns."""
    m: int
    k: int
    rowptr: np.ndarray  # int32 [m+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.k))
        A[np.repeat(np.arange(self.m), np.diff(self.rowptr)), self.col] = self.val
        return A


def random_rect(m: int, k: int, per_row: int, seed: int) -> RectCSR:
    """m x k matrix whose every row holds ``per_row`` distinct uniformly drawn columns with
    values N(0, 1) / sqrt(per_row) (unit expected row norm, as a normalised spreading code)."""
    if per_row > k:
        raise ValueError("per_row exceeds the column count")
    rng = np.random.default_rng(seed)
    cols = np.empty((m, per_row), dtype=np.int64)
    # distinct columns per row: draw with replacement, redraw the rows that repeat one
    cols[:] = rng.integers(0, k, size=(m, per_row))
    for _ in range(1000):
        s = np.sort(cols, axis=1)
        bad = np.nonzero(np.any(s[:, 1:] == s[:, :-1], axis=1))[0] if per_row > 1 else np.zeros(0, np.int64)
        if bad.size == 0:
            break
        cols[bad] = rng.integers(0, k, size=(bad.size, per_row))
    else:
        raise RuntimeError("could not draw distinct columns")
    cols.sort(axis=1)
    vals = rng.standard_normal((m, per_row)) / np.sqrt(per_row)
    vals[vals == 0.0] = 1e-3  # a stored zero is not an entry
    rowptr = np.arange(0, m * per_row + 1, per_row, dtype=np.int64)
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return RectCSR(m, k, rowptr.astype(np.int32), cols.ravel().astype(np.int32), vals.ravel(),
                   {"kind": "random_rect", "per_row": per_row, "seed": seed})


def from_coo(n: int, rows, cols, vals, meta=None) -> CSR:
    """Assemble CSR from COO triplets that contain no duplicate (row, col)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate (row, col) entries")
    r = rows[order]
    counts = np.bincount(r, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSR(n, rowptr.astype(np.int32), cols[order].astype(np.int32), vals[order], dict(meta or {}))


def from_dense(A) -> CSR:
    A = np.asarray(A, dtype=np.float64)
    r, c = np.nonzero(A)
    return from_coo(A.shape[0], r, c, A[r, c])


def to_dense(m: CSR) -> np.ndarray:
    A = np.zeros((m.n, m.n))
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    A[rows, m.col] = m.val
    return A


def _assemble_symmetric(n, iu, ju, w, diag_factor, isolated_diag=1.0, meta=None):
    """Symmetric matrix from undirected edges (iu, ju, w) with
    A_ii = diag_factor * sum_j |A_ij| (isolated_diag where a node has no edge)."""
    iu = np.asarray(iu, dtype=np.int64)
    ju = np.asarray(ju, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    absrow = np.bincount(iu, weights=np.abs(w), minlength=n) + np.bincount(ju, weights=np.abs(w), minlength=n)
    d = diag_factor * absrow
    d[absrow == 0] = isolated_diag
    rows = np.concatenate([iu, ju, np.arange(n)])
    cols = np.concatenate([ju, iu, np.arange(n)])
    vals = np.concatenate([w, w, d])
    return from_coo(n, rows, cols, vals, meta)


def block_diag(mats) -> CSR:
    """Block-diagonal assembly; meta['offsets'] holds the system row offsets."""
    offs = [0]
    rowptrs, cols, vals = [], [], []
    nnz0 = 0
    for m in mats:
        rowptrs.append(m.rowptr[:-1].astype(np.int64) + nnz0)
        cols.append(m.col.astype(np.int64) + offs[-1])
        vals.append(m.val)
        nnz0 += m.nnz
        offs.append(offs[-1] + m.n)
    rowptr = np.concatenate(rowptrs + [np.array([nnz0])])
    if nnz0 >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSR(offs[-1], rowptr.astype(np.int32), np.concatenate(cols).astype(np.int32),
               np.concatenate(vals), {"offsets": np.asarray(offs, dtype=np.int64)})


# --------------------------------------------------------------------------- paper's small systems
def toy3x3():
    """The 3-node tree system of the paper's first numerical example (Sec. "Toy Linear System")."""
    A = np.array([[1.0, -2.0, 3.0], [-2.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    b = np.array([-6.0, 0.0, 2.0])
    return A, b


def nonpsd3x3():
    """Symmetric non-PSD 3x3 matrix of Sec. "Symmetric Non-PSD Data Matrix"; b is all ones."""
    return np.array([[1.0, 2.0, 3.0], [2.0, 2.0, 1.0], [3.0, 1.0, 1.0]]), np.ones(3)


def cdma_r3():
    """Gold-code cross-correlation matrix R3 (Sec. "Linear Detection"), b all ones."""
    return np.array([[7.0, -1, 3], [-1, 7, -5], [3, -5, 7]]) / 7.0, np.ones(3)


def cdma_r4():
    """Gold-code cross-correlation matrix R4 (Sec. "Linear Detection"), b all ones."""
    return np.array([[7.0, -1, 3, 3], [-1, 7, 3, -1], [3, 3, 7, -1], [3, -1, -1, 7]]) / 7.0, np.ones(4)


def run_gabp_3x3():
    """The 3x3 example the paper's appendix runs (A with 0.3/0.1 couplings, b all ones)."""
    return np.array([[1.0, 0.3, 0.1], [0.3, 1.0, 0.1], [0.1, 0.1, 1.0]]), np.ones(3)


def poisson2d(p: int) -> CSR:
    """Paper's 2-D Poisson system on a p x p interior grid: 4 on the diagonal, -1 to neighbours."""
    return grid2d(p, offdiag=-1.0, diag=4.0)


# --------------------------------------------------------------------------- generators
def grid2d(p: int, offdiag: float = -1.0, diag: float = 4.5) -> CSR:
    """p x p 5-point grid in natural (row-major) order with constant coefficients."""
    idx = np.arange(p * p).reshape(p, p)
    iu = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    ju = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    rows = np.concatenate([iu, ju, np.arange(p * p)])
    cols = np.concatenate([ju, iu, np.arange(p * p)])
    vals = np.concatenate([np.full(2 * iu.size, offdiag), np.full(p * p, diag)])
    return from_coo(p * p, rows, cols, vals, {"kind": "grid2d", "p": p})


def random_sym(n: int, picks: int, diag_factor: float, seed: int) -> CSR:
    """Random sparse symmetric matrix.

    Every row i picks ``picks`` distinct partners j != i uniformly at random; each
    pick carries a value U(-1, 1).  The pattern is symmetrised (A_ij = A_ji); when
    both i->j and j->i were drawn, the value drawn first (row-major pick order)
    is kept.  The diagonal is ``diag_factor`` times the row's absolute sum.
    """
    if n < picks + 1:
        raise ValueError("n must exceed picks")
    rng = np.random.default_rng(seed)
    j = rng.integers(0, n - 1, size=(n, picks), dtype=np.int64)
    w = rng.uniform(-1.0, 1.0, size=(n, picks))
    rows = np.arange(n, dtype=np.int64)[:, None]
    j = j + (j >= rows)  # skip self
    # re-draw duplicate picks inside a row until all picks of the row are distinct
    for _ in range(100):
        s = np.sort(j, axis=1)
        bad = np.nonzero(np.any(s[:, 1:] == s[:, :-1], axis=1))[0]
        if bad.size == 0:
            break
        for r in bad:
            seen = set()
            for c in range(picks):
                while int(j[r, c]) in seen:
                    v = int(rng.integers(0, n - 1))
                    j[r, c] = v + (v >= r)
                seen.add(int(j[r, c]))
    iu = np.minimum(rows, j).ravel()
    ju = np.maximum(rows, j).ravel()
    key = iu * n + ju
    _, first = np.unique(key, return_index=True)
    first.sort()
    return _assemble_symmetric(n, iu[first], ju[first], w.ravel()[first], diag_factor,
                               meta={"kind": "random_sym", "picks": picks, "diag_factor": diag_factor, "seed": seed})


def grid3d(m: int, diag_factor: float, seed: int) -> CSR:
    """m^3 7-point grid, natural order, face coefficients k_f ~ LogNormal(0, 1).

    A_ij = -k_f on each interior face, A_ii = diag_factor * sum of the row's k_f
    (no boundary faces are added).  Faces are drawn x-faces, y-faces, z-faces,
    each in C order of the lower cell.
    """
    rng = np.random.default_rng(seed)
    idx = np.arange(m ** 3, dtype=np.int64).reshape(m, m, m)  # [z, y, x]
    pairs = [
        (idx[:, :, :-1], idx[:, :, 1:]),
        (idx[:, :-1, :], idx[:, 1:, :]),
        (idx[:-1, :, :], idx[1:, :, :]),
    ]
    iu = np.concatenate([a.ravel() for a, _ in pairs])
    ju = np.concatenate([c.ravel() for _, c in pairs])
    k = rng.lognormal(0.0, 1.0, size=iu.size)
    return _assemble_symmetric(m ** 3, iu, ju, -k, diag_factor,
                               meta={"kind": "grid3d", "m": m, "diag_factor": diag_factor, "seed": seed})


def rgg_batch(num: int, nmin: int, nmax: int, alpha: float, seed: int, degree: float = 6.0,
              diag_factor: float = 1.1):
    """Batch of random geometric graphs (unit square), sizes n ~ p(n) ∝ n^-alpha on [nmin, nmax].

    Radius r = sqrt(degree / (pi n)); weights -U(0.5, 1); A_ii = diag_factor * row
    abs-sum, 1 for an isolated node.  Returns the list of per-system CSR matrices.
    """
    from scipy.spatial import cKDTree  # available on both machines

    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=num)
    if alpha == 1.0:
        sizes = nmin * (nmax / nmin) ** u
    else:
        a, b = nmin ** (1 - alpha), nmax ** (1 - alpha)
        sizes = (a + u * (b - a)) ** (1.0 / (1 - alpha))
    sizes = np.clip(np.floor(sizes).astype(np.int64), nmin, nmax)
    mats = []
    for s, n in enumerate(sizes):
        pts = rng.uniform(0.0, 1.0, size=(int(n), 2))
        r = np.sqrt(degree / (np.pi * n))
        pr = cKDTree(pts).query_pairs(r, output_type="ndarray")
        pr = pr[np.lexsort((pr[:, 1], pr[:, 0]))]
        w = -rng.uniform(0.5, 1.0, size=pr.shape[0])
        mats.append(_assemble_symmetric(int(n), pr[:, 0], pr[:, 1], w, diag_factor,
                                        meta={"kind": "rgg", "system": s}))
    return mats


def random_tree(n: int, seed: int, diag_scale: float = 1.0, dd: bool = False) -> CSR:
    """Random labelled tree (each node i>0 attaches to a uniform earlier node).

    Off-diagonal values U(-1, 1) (magnitude at least 0.1).  The diagonal is
    U(0.5, 1.5) * diag_scale, or the row abs-sum + that when ``dd``; the matrix
    need not be positive definite unless ``dd``.
    """
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int64)
    child = np.arange(1, n, dtype=np.int64)
    w = rng.uniform(0.1, 1.0, size=n - 1) * rng.choice([-1.0, 1.0], size=n - 1)
    d = rng.uniform(0.5, 1.5, size=n) * diag_scale
    if dd:
        d = d + np.bincount(parent, np.abs(w), minlength=n) + np.bincount(child, np.abs(w), minlength=n)
    rows = np.concatenate([parent, child, np.arange(n)])
    cols = np.concatenate([child, parent, np.arange(n)])
    vals = np.concatenate([w, w, d])
    m = from_coo(n, rows, cols, vals, {"kind": "tree", "seed": seed})
    m.meta["parent"] = np.concatenate([[-1], parent])
    return m


def rhs(n: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(n)


def rhs_batch(n: int, nrhs: int, seed: int) -> np.ndarray:
    """[nrhs, n] matrix of N(0, 1) right-hand sides (row r is right-hand side r)."""
    return np.random.default_rng(seed).standard_normal((nrhs, n))


def spd_seed(make, seed0: int, tries: int = 50):
    """First seed >= seed0 whose matrix make(seed) has a dense Cholesky factor."""
    for s in range(seed0, seed0 + tries):
        m = make(s)
        try:
            np.linalg.cholesky(to_dense(m))
            return s, m
        except np.linalg.LinAlgError:
            continue
    raise RuntimeError("no SPD seed found")


def dense_dd(n: int, diag_factor: float, seed: int) -> np.ndarray:
    """Dense symmetric n x n matrix: off-diagonal U(-1, 1), diagonal diag_factor x the row's
    off-diagonal absolute sum (diagonally dominant for diag_factor > 1; 1 for n = 1)."""
    rng = np.random.default_rng(seed)
    A = np.triu(rng.uniform(-1.0, 1.0, size=(n, n)), 1)
    A = A + A.T
    rs = np.abs(A).sum(axis=1)
    A[np.diag_indices(n)] = np.where(rs > 0.0, diag_factor * rs, 1.0)
    return A


def rbf_kernel_system(n: int, d: int, sigma: float, diag_factor: float, seed: int,
                      block: int = 2048) -> np.ndarray:
    """Dense kernel-regression system: n points uniform in [0, 1]^d, Gaussian kernel
    K_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)) off the diagonal, and the main diagonal weighted to
    diag_factor x the row's off-diagonal sum, so that the matrix is diagonally dominant.  Built in
    row blocks (n = 16384 is 2 GB of FP64)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(n, d))
    A = np.empty((n, n), dtype=np.float64)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        d2 = np.zeros((r1 - r0, n))
        for k in range(d):  # (x_ik - x_jk)^2 is the same for (i, j) and (j, i): A is exactly symmetric
            diff = X[r0:r1, k][:, None] - X[None, :, k]
            d2 += diff * diff
        blk = np.exp(d2 * (-0.5 / (sigma * sigma)))
        idx = np.arange(r0, r1)
        blk[idx - r0, idx] = 0.0
        A[r0:r1] = blk
    A[np.diag_indices(n)] = diag_factor * A.sum(axis=1)
    return A
