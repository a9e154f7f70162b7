"""Serial schedule on the GPU (one message store, nodes firing colour by colour) against the
FP64 oracle's serial schedule, through the C ABI.

The colouring is integer work: bit-exact against the oracle's greedy colouring.  FP64 sweeps:
messages and x after a fixed number of sweeps within 1e-12 relative of the oracle (the GPU
forms each message from the sender's aggregate minus the reverse message, the oracle from an
explicit cavity sum: the rounding differs, not the arithmetic), equal sweep counts at
convergence.  FP32 sweeps with FP64 refinement: 1e-10 relative error after refinement, 1e-5
unrefined, as for the parallel schedule."""
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


def _path(n):
    """Tridiagonal chain numbered along itself: the colouring's dependency chain is n long (the
    device passes stop early and the host finishes the greedy colouring)."""
    rng = np.random.default_rng(7)
    w = -rng.uniform(0.5, 1.0, n - 1)
    rows = np.concatenate([np.arange(n - 1), np.arange(1, n), np.arange(n)])
    cols = np.concatenate([np.arange(1, n), np.arange(n - 1), np.arange(n)])
    d = np.zeros(n)
    d[:-1] += np.abs(w)
    d[1:] += np.abs(w)
    return synth.from_coo(n, rows, cols, np.concatenate([w, w, 1.1 * d]))


def _star(n):
    """Node 0 joined to every other node: one row far longer than the device's per-row slot sort
    handles (sorted on the host)."""
    rng = np.random.default_rng(8)
    w = -rng.uniform(0.5, 1.0, n - 1)
    leaves = np.arange(1, n)
    rows = np.concatenate([np.zeros(n - 1, dtype=np.int64), leaves, np.arange(n)])
    cols = np.concatenate([leaves, np.zeros(n - 1, dtype=np.int64), np.arange(n)])
    d = np.concatenate([[1.1 * np.abs(w).sum()], 2.0 * np.abs(w)])
    return synth.from_coo(n, rows, cols, np.concatenate([w, w, d]))


MATS = {
    "path": lambda: _path(3000),
    "star": lambda: _star(2000),
    "grid2d": lambda: synth.grid2d(32, -1.0, 4.5),
    "grid3d": lambda: synth.grid3d(12, 1.05, 3),
    "random": lambda: synth.random_sym(3001, 8, 1.1, 2),
    "rgg": lambda: synth.rgg_batch(1, 3000, 3001, 2.0, 4)[0],
    "tree": lambda: synth.random_tree(500, 3, dd=True),
    "random_l2": lambda: synth.random_sym(1000, 8, 1.1, 6),
    "random_l4": lambda: synth.random_sym(500, 16, 1.1, 7),
}
# Graphs of at most 128 warps' rows (32 / L rows a warp, L = 1, 2 or 4 lanes a row by the mean
# degree) run every sweep in one thread-block cluster: grid2d and tree with two warps a CTA, star,
# grid3d, random_l2 (L = 2) and random_l4 (L = 4) with four, path and rgg with eight; "random"
# (3001 rows, L = 2: 188 warps) takes a launch per pass.


@pytest.mark.parametrize("name", list(MATS))
def test_colouring_bit_exact(gb, name):
    m = MATS[name]()
    s = gb.Solver.from_csr(m, schedule=1)
    c, nc = s.serial_colours()
    s.close()
    ref, nref = oracle.colour_greedy(m)
    assert nc == nref
    assert np.array_equal(c.cpu().numpy(), ref)


def test_colouring_large_random(gb):
    """n = 2^18, degree ~16: many tiles, long Jones-Plassmann chains resolved."""
    m = synth.random_sym(1 << 18, 8, 1.1, 5)
    s = gb.Solver.from_csr(m, schedule=1)
    c, nc = s.serial_colours()
    s.close()
    ref, nref = oracle.colour_greedy(m)
    assert nc == nref and np.array_equal(c.cpu().numpy(), ref)


def _fp64(gb, m, b, sweeps, tol=0.0):
    s = gb.Solver.from_csr(m, schedule=1, precision=gb.GABP_PREC_FP64)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=sweeps)
    P, hm = s.messages()
    Pi = s.marginal_precisions()
    s.close()
    return st, it, x.cpu().numpy(), P.cpu().numpy(), hm.cpu().numpy(), Pi.cpu().numpy()


@pytest.mark.parametrize("name", ["grid2d", "grid3d", "random", "rgg", "tree", "path", "star", "random_l2",
                                  "random_l4"])
@pytest.mark.parametrize("sweeps", [1, 2, 7])
def test_fp64_sweeps_match_oracle(gb, name, sweeps):
    m = MATS[name]()
    b = synth.rhs(m.n, 7)
    st, it, x, P, hm, Pi = _fp64(gb, m, b, sweeps)
    r = oracle.gabp_serial(m, b, max_iter=sweeps, tol=0.0, messages=True)
    assert it == r["iters"] == sweeps
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    off = rows != m.col
    assert np.allclose(P[off], r["Pmsg"][off], rtol=1e-12, atol=0)
    hm_ref = r["Pmsg"] * r["mumsg"]
    assert np.max(np.abs(hm[off] - hm_ref[off])) <= 1e-12 * np.max(np.abs(hm_ref[off]))
    # x_i = (b_i + sum_k h_ki) / (A_ii + sum_k P_ki): a 1e-12 rounding difference in the sums is
    # amplified by their cancellation (random trees are not diagonally dominant)
    absP = np.bincount(rows, np.abs(np.where(off, r["Pmsg"], m.val)), minlength=m.n)
    absh = np.abs(b) + np.bincount(rows[off], np.abs(hm_ref[off]), minlength=m.n)
    bound = 1e-12 * (absP * np.abs(r["x"]) + absh) / np.abs(r["P"]) + 1e-300
    assert np.all(np.abs(x - r["x"]) <= bound)
    assert np.all(np.abs(Pi - r["P"]) <= 1e-12 * absP)


@pytest.mark.parametrize("name", ["grid2d", "random", "rgg", "path", "random_l2", "random_l4"])
def test_fp64_converged_equal_sweeps(gb, name):
    m = MATS[name]()
    b = synth.rhs(m.n, 3)
    st, it, x, P, hm, Pi = _fp64(gb, m, b, 5000, tol=1e-12)
    r = oracle.gabp_serial(m, b, max_iter=5000, tol=1e-12)
    assert st == gb.GABP_OK and r["status"] == oracle.OK
    assert it == r["iters"]
    assert _relerr(x, r["x"]) <= 1e-12
    par = oracle.gabp_broadcast(m, b, max_iter=5000, tol=1e-12)
    assert it < par["iters"]  # the serial schedule needs fewer sweeps than rounds


@pytest.mark.parametrize("name,one_launch", [("grid2d", True), ("path", True), ("random_l4", True),
                                             ("random", False)])
def test_fp64_small_graphs_one_launch(gb, name, one_launch):
    """Graphs whose rows fit 128 warps (32 / L rows a warp) run every sweep of a solve in one
    thread-block cluster launch; the 3001-row graph of mean degree 16 (two lanes a row: 188 warps)
    launches its passes.  Both reach the oracle's sweep count and answer."""
    m = MATS[name]()
    b = synth.rhs(m.n, 5)
    s = gb.Solver.from_csr(m, schedule=1, precision=gb.GABP_PREC_FP64, profile=1)
    s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=5000)
    s.profile(reset=True)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=5000)
    launches = s.profile()["launches"]
    s.close()
    r = oracle.gabp_serial(m, b, max_iter=5000, tol=1e-12)
    assert st == gb.GABP_OK and it == r["iters"]
    assert _relerr(x.cpu().numpy(), r["x"]) <= 1e-12
    assert (launches == 1) == one_launch, launches


def test_fp64_tree_exact(gb):
    m = MATS["tree"]()
    b = synth.rhs(m.n, 4)
    A = oracle.to_dense(m)
    st, it, x, P, hm, Pi = _fp64(gb, m, b, 500, tol=1e-13)
    assert st == gb.GABP_OK
    assert _relerr(x, np.linalg.solve(A, b)) <= 1e-12
    assert np.allclose(Pi, oracle.marginal_precisions_exact(A), rtol=1e-11)


def test_fp64_breakdown_and_zero_rhs(gb):
    A = np.array([[2.0, 1.0, 0.0, 0.0], [1.0, 3.0, 1.0, 1.0], [0.0, 1.0, 1.0, 0.0], [0.0, 1.0, 0.0, 0.5]])
    m = synth.from_dense(A)
    b = np.ones(4)
    r = oracle.gabp_serial(m, b, max_iter=20, tol=1e-14)
    s = gb.Solver.from_csr(m, schedule=1)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-14, max_iter=20)
    s.close()
    assert st == r["status"]
    if r["status"] == oracle.BREAKDOWN:
        assert it == r["iters"]
    m = MATS["grid2d"]()
    s = gb.Solver.from_csr(m, schedule=1)
    x, st, it, rel = s.solve(torch.zeros(m.n, dtype=torch.float64, device="cuda"), tol=1e-12)
    assert st == gb.GABP_OK and it == 0 and not torch.any(x)
    s.close()


@pytest.mark.parametrize("name", ["grid2d", "grid3d", "random", "rgg"])
def test_fp32_serial_refined(gb, name):
    m = MATS[name]()
    b = synth.rhs(m.n, 5)
    x0 = oracle.dense_solve(oracle.to_dense(m), b)
    out = {}
    for sched in (0, 1):
        s = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, schedule=sched, overlap_precision=0)
        x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=20000)
        out[sched] = (st, it, x.cpu().numpy(), s.stats())
        s.close()
    st, it, x, stats = out[1]
    assert st == gb.GABP_OK and _relerr(x, x0) <= 1e-10
    assert stats["refine_steps"] >= 1
    if name != "random":  # grids and geometric graphs: far fewer sweeps than rounds
        assert it < 0.8 * out[0][1]


def test_fp32_serial_unrefined_within_1e5(gb):
    m = MATS["grid3d"]()
    b = synth.rhs(m.n, 6)
    ref = oracle.gabp_serial(m, b, max_iter=5000, tol=1e-13)
    s = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, schedule=1, max_refine=1, inner_tol=1e-7,
                           inner_max_iter=2000, prec_stop_log2=22)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=5000)
    assert s.stats()["refine_steps"] == 1
    s.close()
    assert _relerr(x.cpu().numpy(), ref["x"]) <= 1e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_repeated_solves_one_handle(gb, precision):
    """The captured serial sweeps are replayed for new right-hand sides and new output arrays."""
    m = MATS["grid3d"]()
    s = gb.Solver.from_csr(m, schedule=1, precision=precision)
    A = oracle.to_dense(m)
    for seed in (1, 2, 3):
        b = synth.rhs(m.n, seed)
        x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-11, max_iter=5000)
        assert st == gb.GABP_OK
        assert _relerr(x.cpu().numpy(), np.linalg.solve(A, b)) <= 1e-9
    s.close()


@pytest.mark.parametrize("R", [5, 64, 130])
def test_batched_serial_refined(gb, R):
    """R right-hand sides with serial sweeps (warp per row, lanes over right-hand sides):
    every column within 1e-10 of the dense solution, fewer sweeps than parallel rounds."""
    m = MATS["grid3d"]()
    B = synth.rhs_batch(m.n, R, 9)  # [R, n]
    A = oracle.to_dense(m)
    X0 = np.linalg.solve(A, B.T).T
    its = {}
    for sched in (0, 1):
        s = gb.Solver.from_csr(m, schedule=sched)
        X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-11)
        its[sched] = it
        s.close()
        assert st == gb.GABP_OK and np.all(rel <= 1e-11)
        Xh = X.cpu().numpy()
        for r in range(R):
            assert _relerr(Xh[r], X0[r]) <= 1e-9, r
    assert its[1] < its[0]


def test_set_values_serial_fp64(gb):
    """New values on the same pattern reach the serial layout's copies (FP64 serial sweeps)."""
    m = MATS["grid3d"]()
    s = gb.Solver.from_csr(m, schedule=1, precision=gb.GABP_PREC_FP64)
    b = synth.rhs(m.n, 4)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-11, max_iter=5000)
    v2 = m.val.copy()
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    v2[rows == m.col] *= 1.3  # heavier diagonal, same pattern
    s.set_values(v2)
    x2, st2, it2, rel2 = s.solve(torch.from_numpy(b).cuda(), tol=1e-11, max_iter=5000)
    s.close()
    m2 = synth.CSR(m.n, m.rowptr, m.col, v2, {})
    assert st2 == gb.GABP_OK
    assert _relerr(x2.cpu().numpy(), np.linalg.solve(oracle.to_dense(m2), b)) <= 1e-9
    assert it2 < it
