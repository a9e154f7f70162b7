"""Degenerate inputs on every solver path, against the dense solution: one row, two rows (one
edge), a chain of three, a graph with no edges at all, and a disconnected pair; batched solves of one
and of three right-hand sides; independent systems of one row each and a single system; the dense
and least-squares entries at their smallest sizes.  GaBP is exact on these trees, so every path must
reach the tolerance and the dense answer (relative error <= 1e-9; FP64 paths to 1e-12)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_0811_2518_gb300 as m

    return m


MATS = {
    "one_row": np.array([[2.5]]),
    "two_rows": np.array([[2.0, -1.0], [-1.0, 3.0]]),
    "chain3": np.array([[4.0, 1.0, 0.0], [1.0, 3.0, -1.0], [0.0, -1.0, 2.0]]),
    "no_edges": np.diag([1.5, 2.0, 0.5, 4.0]),
    "two_pairs": np.array([[3.0, 1.0, 0.0, 0.0], [1.0, 2.0, 0.0, 0.0], [0.0, 0.0, 5.0, -2.0], [0.0, 0.0, -2.0, 4.0]]),
}

PATHS = {
    "fp64_node": {},
    "fp64_edge": {"variant": 1},
    "fp64_serial": {"schedule": 1},
    "fp64_freeze": {"freeze_precisions": 1},
    "fp32_refine": {"precision": 1},
    "fp32_refine_serial": {"precision": 1, "schedule": 1},
}


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("path", list(PATHS))
def test_single_solve_paths(gb, mat, path):
    A = MATS[mat]
    b = np.arange(1.0, A.shape[0] + 1.0)
    opts = PATHS[path]
    tol = 1e-12 if opts.get("precision", 0) == 0 else 1e-10
    s = gb.Solver.from_csr(synth.from_dense(A), **opts)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=100)
    s.close()
    assert st == gb.GABP_OK and rel <= tol, (st, rel)
    assert _relerr(x.cpu().numpy(), np.linalg.solve(A, b)) <= (1e-12 if tol == 1e-12 else 1e-9)


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("R", [1, 3])
@pytest.mark.parametrize("schedule", [0, 1])
def test_batched_tiny(gb, mat, R, schedule):
    A = MATS[mat]
    n = A.shape[0]
    B = np.stack([np.arange(1.0, n + 1.0) * (r + 1) + r for r in range(R)])  # R columns, column-major rows
    s = gb.Solver.from_csr(synth.from_dense(A), precision=1, schedule=schedule)
    X, st, its, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-10)
    s.close()
    assert st == gb.GABP_OK and np.all(rel <= 1e-10)
    Xr = np.linalg.solve(A, B.T).T
    assert _relerr(X.cpu().numpy(), Xr) <= 1e-9


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_systems_of_one_row_and_one_system(gb, mode):
    """Four systems of one row each (offsets 0..4 of the diagonal matrix), and the chain as a
    single system, on every independent-systems kernel."""
    A = MATS["no_edges"]
    b = np.array([1.0, -2.0, 3.0, 0.5])
    s = gb.Solver.from_csr(synth.from_dense(A), multi_mode=mode)
    x, st, sts, its, rel = s.solve_systems(torch.from_numpy(b).cuda(), np.arange(5), tol=1e-10)
    s.close()
    assert st == gb.GABP_OK and np.all(sts == 0)
    assert _relerr(x.cpu().numpy(), b / np.diag(A)) <= 1e-9
    A = MATS["chain3"]
    b = np.array([1.0, 2.0, 3.0])
    s = gb.Solver.from_csr(synth.from_dense(A), multi_mode=mode)
    x, st, sts, its, rel = s.solve_systems(torch.from_numpy(b).cuda(), np.array([0, 3]), tol=1e-10)
    s.close()
    assert st == gb.GABP_OK and _relerr(x.cpu().numpy(), np.linalg.solve(A, b)) <= 1e-9


def test_dense_and_least_squares_smallest(gb):
    for A in (np.array([[3.0]]), MATS["two_rows"]):
        s = gb.Solver.from_dense(A)
        b = np.ones(A.shape[0])
        x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12)
        s.close()
        assert st == gb.GABP_OK and _relerr(x.cpu().numpy(), np.linalg.solve(A, b)) <= 1e-12
    # J is 1 x 1 and 2 x 1: x = (J^T J + gamma)^{-1} J^T y
    for Jd in (np.array([[2.0]]), np.array([[1.0], [-3.0]])):
        m_, k_ = Jd.shape
        rp = np.arange(m_ + 1, dtype=np.int32)
        J = synth.RectCSR(m_, k_, rp, np.zeros(m_, dtype=np.int32), Jd[:, 0].copy())
        y = np.arange(1.0, m_ + 1.0)
        s = gb.LSQSolver.from_rect(J, 0.5)
        x, z, st, it, rel = s.solve_lsq(torch.from_numpy(y).cuda(), tol=1e-12, max_iter=500)
        s.close()
        xr = np.linalg.solve(Jd.T @ Jd + 0.5 * np.eye(k_), Jd.T @ y)
        assert st == gb.GABP_OK and _relerr(x.cpu().numpy(), xr) <= 1e-12
