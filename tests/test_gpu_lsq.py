"""Regularised least squares through the augmented symmetric system (Sec. "Extension to General
Linear Systems"; Chapter "Extending GaBP to support non-square matrices") on the GPU, through the
C ABI (gabp_create_lsq / gabp_solve_lsq): iterates against the oracle's GaBP on its own augmented
matrix, converged solutions against the dense normal equations, every solver path, device input,
the auxiliary block, invalid inputs, and the benchmark-sized problem by its normal equations."""
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


SHAPES = [(300, 120, 4, 0.5), (1000, 1000, 6, 1.0), (250, 700, 5, 2.0), (3000, 1500, 8, 1.0)]


def _lsq(gb, J, y, gamma, tol, max_iter, **opts):
    s = gb.LSQSolver.from_rect(J, gamma, **opts)
    x, z, st, it, rel = s.solve_lsq(torch.from_numpy(y).cuda(), tol=tol, max_iter=max_iter, want_z=True, check=False)
    s.close()
    return x.cpu().numpy(), z.cpu().numpy(), st, it, rel


@pytest.mark.parametrize("m,k,per_row,gamma", SHAPES)
@pytest.mark.parametrize("rounds", [1, 4, 11])
def test_iterates_match_oracle(gb, m, k, per_row, gamma, rounds):
    J = synth.random_rect(m, k, per_row, 11)
    y = synth.rhs(m, 12)
    r = oracle.gabp_lsq(J, y, gamma, max_iter=rounds, tol=0.0)
    x, z, st, it, _ = _lsq(gb, J, y, gamma, 0.0, rounds, precision=gb.GABP_PREC_FP64)
    assert st == gb.GABP_NOT_CONVERGED and it == rounds
    assert np.max(np.abs(x - r["x"])) <= 1e-12 * np.max(np.abs(r["x"]))
    assert np.max(np.abs(z - r["z"])) <= 1e-12 * np.max(np.abs(r["z"]))


@pytest.mark.parametrize("m,k,per_row,gamma", SHAPES)
def test_converged_fp64_equals_normal_equations(gb, m, k, per_row, gamma):
    J = synth.random_rect(m, k, per_row, 11)
    y = synth.rhs(m, 12)
    r = oracle.gabp_lsq(J, y, gamma, max_iter=5000, tol=1e-12)
    x, z, st, it, rel = _lsq(gb, J, y, gamma, 1e-12, 5000, precision=gb.GABP_PREC_FP64)
    assert st == gb.GABP_OK and r["status"] == oracle.OK and it == r["iters"] and rel <= 1e-12
    Jd = J.dense()
    xr = oracle.ridge_solve(Jd, y, gamma)
    assert np.max(np.abs(x - xr)) <= 1e-10 * np.max(np.abs(xr))
    assert np.max(np.abs(x - r["x"])) <= 1e-12 * np.max(np.abs(r["x"]))
    assert np.allclose(z, (Jd @ x - y) / gamma, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("opts", [dict(precision=1), dict(precision=1, device_loop=0), dict(precision=0, schedule=1),
                                  dict(precision=1, schedule=1), dict(precision=0, variant=1),
                                  dict(precision=0, accel=2, schedule=1)])
def test_every_path_reaches_the_ridge_solution(gb, opts):
    m, k, per_row, gamma = SHAPES[3]
    J = synth.random_rect(m, k, per_row, 11)
    y = synth.rhs(m, 12)
    x, z, st, it, rel = _lsq(gb, J, y, gamma, 1e-10, 5000, **opts)
    assert st == gb.GABP_OK and rel <= 1e-10
    xr = oracle.ridge_solve(J.dense(), y, gamma)
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)


def test_serial_schedule_matches_oracle(gb):
    m, k, per_row, gamma = SHAPES[0]
    J = synth.random_rect(m, k, per_row, 11)
    y = synth.rhs(m, 12)
    Ja = oracle.lsq_augmented(J, gamma)
    for t in (1, 3, 8):
        ref = oracle.gabp_serial(Ja, np.concatenate([np.zeros(k), y]), max_iter=t, tol=0.0)
        x, z, st, it, _ = _lsq(gb, J, y, gamma, 0.0, t, precision=0, schedule=1)
        assert it == t
        assert np.max(np.abs(x - ref["x"][:k])) <= 1e-12 * np.max(np.abs(ref["x"][:k]))


def test_device_input_equals_host_input(gb):
    J = synth.random_rect(800, 300, 5, 3)
    y = torch.from_numpy(synth.rhs(800, 4)).cuda()
    a = gb.LSQSolver.from_rect(J, 1.0)
    b = gb.LSQSolver(J.m, J.k, torch.from_numpy(J.rowptr).cuda(), torch.from_numpy(J.col).cuda(),
                     torch.from_numpy(J.val).cuda(), 1.0)
    xa = a.solve_lsq(y, tol=1e-12, max_iter=3000)
    xb = b.solve_lsq(y, tol=1e-12, max_iter=3000)
    assert xa[2] == xb[2] == gb.GABP_OK and xa[3] == xb[3]
    assert torch.equal(xa[0], xb[0])
    # the base-class solve acts on the augmented system itself
    bt = torch.cat([torch.zeros(J.k, dtype=torch.float64, device="cuda"), y])
    xt, st, it, rel = a.solve(bt, tol=1e-12, max_iter=3000)
    assert torch.equal(xt[:J.k], xa[0])
    a.close()
    b.close()


def test_invalid_inputs(gb):
    J = synth.random_rect(50, 20, 3, 1)
    for gamma in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(gb.GaBPError) as ei:
            gb.LSQSolver.from_rect(J, gamma)
        assert ei.value.status == gb.GABP_ERR_INVALID
    bad_col = J.col.copy()
    bad_col[0], bad_col[1] = bad_col[1], bad_col[0]  # not increasing
    zero = J.val.copy()
    zero[7] = 0.0
    oob = J.col.copy()
    oob[4] = J.k
    for rp, cl, vl in ((J.rowptr, bad_col, J.val), (J.rowptr, J.col, zero), (J.rowptr, oob, J.val)):
        with pytest.raises(gb.GaBPError) as ei:
            gb.LSQSolver(J.m, J.k, rp, cl, vl, 1.0)
        assert ei.value.status == gb.GABP_ERR_INVALID
    s = gb.Solver.from_csr(synth.grid2d(4, -1.0, 4.5))
    x = torch.empty(16, dtype=torch.float64, device="cuda")
    st, _, _ = gb.gabp_solve_lsq(s.handle, x.data_ptr(), x.data_ptr(), None, 1e-10, 10)
    assert st == gb.GABP_ERR_INVALID
    s.close()


def test_empty_rows_and_columns(gb):
    """A row of J without entries leaves its z = -y_r / gamma; a column without entries gives x_c = 0."""
    from scipy.sparse import csr_matrix

    Jd = synth.random_rect(60, 30, 4, 2).dense()
    Jd[5, :] = 0.0
    Jd[:, 7] = 0.0
    c = csr_matrix(Jd)
    J = synth.RectCSR(60, 30, c.indptr.astype(np.int32), c.indices.astype(np.int32), c.data.copy())
    y = synth.rhs(60, 3)
    x, z, st, it, rel = _lsq(gb, J, y, 0.8, 1e-12, 3000, precision=0)
    assert st == gb.GABP_OK and x[7] == 0.0
    assert z[5] == pytest.approx(-y[5] / 0.8, rel=1e-14)
    assert np.allclose(x, oracle.ridge_solve(Jd, y, 0.8), rtol=1e-9, atol=1e-12)


def test_full_size_normal_equations(gb):
    """The benchmark's least-squares workload (J: 2^20 x 2^19, 8 entries per row, gamma = 1) solved
    by the default FP32 + refinement path to 1e-10: the normal-equation residual
    ||J^T (y - J x) - gamma x|| / ||J^T y|| recomputed on the host, and the FP64 path's answer
    agreeing with it to the accuracy both residuals imply."""
    from scipy.sparse import csr_matrix

    J = synth.random_rect(1 << 20, 1 << 19, 8, 21)
    y = synth.rhs(J.m, 22)
    S = csr_matrix((J.val, J.col, J.rowptr), shape=(J.m, J.k))
    jty = S.T @ y
    out = {}
    for name, prec in (("fp32", 1), ("fp64", 0)):
        x, z, st, it, rel = _lsq(gb, J, y, 1.0, 1e-10, 5000, precision=prec)
        assert st == gb.GABP_OK and rel <= 1e-10
        ne = S.T @ (y - S @ x) - x
        assert np.linalg.norm(ne) <= 1e-8 * np.linalg.norm(jty)
        out[name] = x
    assert np.linalg.norm(out["fp32"] - out["fp64"]) <= 1e-8 * np.linalg.norm(out["fp64"])
