"""Dense symmetric matrices (gabp_create_dense): the broadcast rounds on every entry of a dense
row, against the FP64 CPU oracle on the same matrix, the dense solution, and the CSR handle of
the same entries.

The kernel-regression chapter's construction (its main diagonal weighted until the kernel
matrix is diagonally dominant) is the workload shape: synth.rbf_kernel_system.  Tolerances as
for the sparse FP64 path: 1e-13 at a fixed round, 1e-12 at convergence, equal round counts;
FP32 messages + FP64 refinement: 1e-10 relative residual and cond(A)-scaled error.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_0811_2518_gb300 as m

    return m


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("n", [1, 2, 37, 300])
def test_dense_equals_csr_handle_and_oracle(gb, n):
    """n = 1, 2 (degenerate), 37 and 300 (ragged warps and blocks): the dense entry gives bitwise
    the result of a CSR handle of the same entries, the oracle's round count and iterate, and the
    dense solution."""
    A = synth.dense_dd(n, 1.1, 3 + n)
    b = synth.rhs(n, n)
    sd = gb.Solver.from_dense(A)
    assert sd.nnz == n * n
    xd, st, it, rel = sd.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=2000)
    sd.close()
    m = synth.from_dense(A)
    sc = gb.Solver.from_csr(m)
    xc, stc, itc, _ = sc.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=2000)
    sc.close()
    assert st == stc == gb.GABP_OK and it == itc
    assert torch.equal(xd, xc)
    ref = oracle.gabp_broadcast(m, b, max_iter=2000, tol=1e-12)
    assert ref["status"] == oracle.OK and ref["iters"] == it
    x = xd.cpu().numpy()
    assert _maxrel(x, ref["x"]) <= 1e-12
    assert _maxrel(x, np.linalg.solve(A, b)) <= 1e-11


def test_dense_fixed_rounds_and_device_input(gb):
    """A device matrix with lda > n (rows of a wider array): x after 1, 4 and 9 rounds equals the
    oracle's iterate to 1e-13, element by element."""
    n, N = 257, 300
    big = np.zeros((N, N))
    big[:n, :n] = synth.dense_dd(n, 1.2, 21)
    A = big[:n, :n]
    b = synth.rhs(n, 22)
    At = torch.from_numpy(big).cuda()[:n, :n]
    assert At.stride(0) == N
    m = synth.from_dense(A)
    for t in (1, 4, 9):
        s = gb.Solver.from_dense(At)
        x, st, it, _ = s.solve(torch.from_numpy(b).cuda(), tol=0.0, max_iter=t)
        s.close()
        assert st == gb.GABP_NOT_CONVERGED and it == t
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0)
        assert np.allclose(x.cpu().numpy(), r["x"], rtol=1e-13, atol=1e-15 * np.max(np.abs(r["x"])))


@pytest.mark.parametrize("precision,n", [(0, 600), (1, 2000)])
def test_rbf_kernel_system(gb, precision, n):
    """The kernel-regression shape: points in [0, 1]^3, Gaussian kernel (sigma 0.1), main
    diagonal 1.1 x the row sum; FP64 to 1e-12 (600 points: also the oracle's round count and
    iterate) and FP32 messages + FP64 refinement to 1e-10 (2000 points), against the dense
    solution.  (The oracle's input check scans rows: O(n^3) on a dense matrix.)"""
    A = synth.rbf_kernel_system(n, 3, 0.1, 1.1, 7)
    b = synth.rhs(n, 8)
    tol = 1e-12 if precision == 0 else 1e-10
    s = gb.Solver.from_dense(A, precision=precision)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=2000)
    s.close()
    assert st == gb.GABP_OK and rel <= tol
    x = x.cpu().numpy()
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 2 * tol * np.linalg.cond(A) * np.linalg.norm(xs)
    r = b - A @ x
    assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(b)
    if precision == 0:
        ref = oracle.gabp_broadcast(synth.from_dense(A), b, max_iter=2000, tol=tol)
        assert ref["iters"] == it and _maxrel(x, ref["x"]) <= 1e-12


def test_dense_zeros_kept_pattern_and_rejections(gb):
    """Exact zeros are left out (a banded dense array keeps its band and diagonal); an asymmetric
    matrix, a zero diagonal entry or a NaN are rejected; bad arguments too."""
    n = 64
    A = synth.dense_dd(n, 1.1, 5)
    i, j = np.indices((n, n))
    A[np.abs(i - j) > 3] = 0.0
    A[np.diag_indices(n)] = 1.1 * (np.abs(A).sum(axis=1) - np.abs(np.diag(A)))
    s = gb.Solver.from_dense(A)
    assert s.nnz == int(np.count_nonzero(A))
    b = synth.rhs(n, 6)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12)
    s.close()
    assert st == gb.GABP_OK and _maxrel(x.cpu().numpy(), np.linalg.solve(A, b)) <= 1e-11
    for bad in ("asym", "zero_diag", "nan"):
        B = A.copy()
        if bad == "asym":
            B[0, 1] += 0.5
        elif bad == "zero_diag":
            B[5, 5] = 0.0
        else:
            B[2, 3] = B[3, 2] = np.nan
        with pytest.raises(gb.GaBPError) as ei:
            gb.Solver.from_dense(B)
        assert ei.value.status == gb.GABP_ERR_INVALID, bad
    with pytest.raises(ValueError):
        gb.Solver.from_dense(np.zeros((3, 4)))
