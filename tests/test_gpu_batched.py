"""GPU batched multi-RHS solve (FP32 messages, shared precision state, FP64 refinement)
against the FP64 oracle, through the C ABI.  Refined tolerance 1e-10 relative per column."""
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


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("R", [1, 5, 64, 130])
def test_batched_matches_oracle(gb, R):
    m = synth.grid3d(12, 1.05, 3)  # 1728 unknowns, heterogeneous 7-point diffusion
    B = synth.rhs_batch(m.n, R, 11)
    B[min(3, R - 1)] = 0.0  # one zero right-hand side
    s = gb.Solver.from_csr(m)
    X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-12)
    s.close()
    assert st == gb.GABP_OK and np.all(rel <= 1e-12)
    X = X.cpu().numpy()
    A = oracle.to_dense(m)
    for r in range(R):
        if not np.any(B[r]):
            assert not np.any(X[r])
            continue
        ref = oracle.gabp_broadcast(m, B[r], max_iter=5000, tol=1e-13)
        assert _relerr(X[r], ref["x"]) <= 1e-10
    assert _relerr(X[R - 1], oracle.dense_solve(A, B[R - 1])) <= 1e-10


def test_batched_equals_single_rhs_solves(gb):
    m = synth.random_sym(20011, 8, 1.1, 2)
    B = synth.rhs_batch(m.n, 40, 12)
    s = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE)
    X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-11)
    assert st == gb.GABP_OK
    for r in (0, 17, 39):
        x, st1, it1, rel1 = s.solve(torch.from_numpy(B[r]).cuda(), tol=1e-11)
        assert st1 == gb.GABP_OK
        assert _relerr(X[r].cpu().numpy(), x.cpu().numpy()) <= 1e-9
    s.close()


def test_batched_rejects_bad_ld(gb):
    m = synth.grid2d(8)
    s = gb.Solver.from_csr(m)
    B = torch.zeros(3, m.n, dtype=torch.float64, device="cuda")
    st, it = gb.gabp_solve_batched(s.handle, 3, B.data_ptr(), B.data_ptr(), m.n - 1, 1e-10, 100)
    s.close()
    assert st == gb.GABP_ERR_INVALID


@pytest.mark.parametrize("schedule", [1, 0])
def test_full_size_grid3d_64rhs(gb, schedule):
    """The 64-right-hand-side workload at full size (128^3 7-point grid, LogNormal(0,1) faces,
    diagonal 1.05 x row abs-sum, right-hand sides seed 3) in the launch configuration the
    benchmark times (serial schedule, and the parallel one): every column's residual,
    recomputed on the host in FP64, meets the 1e-10 tolerance.  (The max-norm error bound the
    residual implies, |r|_inf / min_i (A_ii - sum_j |A_ij|), is loose here -- the margin is
    0.05 x the row sum and some rows' sums are small -- so only the residual is asserted.)"""
    sp = pytest.importorskip("scipy.sparse")
    m = synth.grid3d(128, 1.05, 3)
    R = 64
    B = synth.rhs_batch(m.n, R, 3)
    s = gb.Solver.from_csr(m, schedule=schedule)
    X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-10, max_iter=5000)
    s.close()
    assert st == gb.GABP_OK and np.all(rel <= 1e-10)
    X = X.cpu().numpy()
    A = sp.csr_matrix((m.val, m.col, m.rowptr), shape=(m.n, m.n))
    Rm = B.T - A @ X.T
    rn = np.linalg.norm(Rm, axis=0) / np.linalg.norm(B, axis=1)
    assert np.all(rn <= 1e-10), rn.max()


def test_full_size_grid3d_columns_vs_oracle(gb):
    """Two columns of the full 128^3 x 64 batched solve (the benchmark's serial schedule) against
    the oracle's FP64 GaBP solution of the same column (parallel schedule, to 1e-13), entry by
    entry: at tolerance 1e-12 the max-norm difference is below 1e-10 of max |x|; at the benchmark's
    1e-10 it is below 1e-8."""
    m = synth.grid3d(128, 1.05, 3)
    B = synth.rhs_batch(m.n, 64, 3)
    cols = (0, 37)
    oracle.gabp_broadcast(m, B[0], max_iter=0, tol=0.0)  # input checks
    par = oracle.host_threads() is not None
    refs = {}
    for c in cols:
        r, _ = oracle.broadcast_timed(m, B[c], 2000, threads=par, tol=1e-13)
        assert r["status"] == oracle.OK
        refs[c] = r["x"]
    s = gb.Solver.from_csr(m, schedule=1)
    for tol, bar in ((1e-12, 1e-10), (1e-10, 1e-8)):
        X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=tol, max_iter=5000)
        assert st == gb.GABP_OK and np.all(rel <= tol)
        for c in cols:
            x = X[c].cpu().numpy()
            assert np.max(np.abs(x - refs[c])) <= bar * np.max(np.abs(refs[c]))
    s.close()
