"""GPU parity of the plain FP64 GaBP path against the FP64 CPU oracle (through the C ABI).

Tolerances: the paper's iterates are reproduced round for round; at a fixed
round the GPU and the oracle agree to 1e-13 relative on x and the messages
(they differ only in summation order and in the reciprocal's last bit), and at
convergence to 1e-12 relative (the FP64 target), with equal round counts.
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


def _solver(gb, m, **opts):
    return gb.Solver.from_csr(m, **opts)


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu_solve(gb, m, b, tol, max_iter, **opts):
    s = _solver(gb, m, **opts)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=max_iter)
    out = {"x": x.cpu().numpy(), "status": st, "iters": it, "relres": rel}
    if st >= 0 and opts.get("precision", 0) == 0 and opts.get("gamma_mode", 0) == 0:
        P, hm = s.messages()
        out["Pmsg"], out["hmsg"] = P.cpu().numpy(), hm.cpu().numpy()
        out["P"] = s.marginal_precisions().cpu().numpy()
    out["stats"] = s.stats()
    s.close()
    return out


def _diag_mask(m):
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    return rows == m.col


@pytest.mark.parametrize("variant", [0, 1])
def test_toy_tables_gpu(gb, variant):
    """Sec. "Toy Linear System": messages and tentative means at t = 1, 2, 3."""
    A, b = synth.toy3x3()
    m = synth.from_dense(A)
    off = ~_diag_mask(m)
    for t in (1, 2, 3):
        ref = oracle.gabp_naive(m, b, max_iter=t, tol=0.0, messages=True)
        g = _gpu_solve(gb, m, b, 0.0, t, variant=variant)
        assert g["status"] == ref["status"] and g["iters"] == ref["iters"], (t, g["status"], g["iters"])
        assert np.allclose(g["x"], ref["x"], rtol=1e-14, atol=1e-14)
        assert np.allclose(g["Pmsg"][off], ref["Pmsg"][off], rtol=1e-14, atol=1e-14)
        assert np.allclose(g["hmsg"][off], (ref["Pmsg"] * ref["mumsg"])[off], rtol=1e-14, atol=1e-14)
    assert np.allclose(g["P"], [-12.0, 1.5, 4.0], rtol=1e-14)


def _diameter(m):
    from collections import deque

    def bfs(s):
        dist = np.full(m.n, -1)
        dist[s] = 0
        q = deque([s])
        while q:
            u = q.popleft()
            for p in range(m.rowptr[u], m.rowptr[u + 1]):
                v = m.col[p]
                if v != u and dist[v] < 0:
                    dist[v] = dist[u] + 1
                    q.append(v)
        return dist

    return int(bfs(int(np.argmax(bfs(0)))).max())


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tree_exact_gpu(gb, seed):
    """Trees: after diameter-many rounds the means are A^{-1} b and the precisions
    1/(A^{-1})_ii (Sec. "Convergence and Exactness")."""
    n = 31 if seed % 2 else 400
    m = synth.random_tree(n, seed, dd=(seed % 2 == 0), diag_scale=2.0)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 100 + seed)
    d = _diameter(m)
    g = _gpu_solve(gb, m, b, 0.0, d)
    assert g["status"] in (gb.GABP_OK, gb.GABP_NOT_CONVERGED) and g["iters"] <= d
    xs = oracle.dense_solve(A, b)
    assert _relerr(g["x"], xs) <= 1e-12
    assert np.allclose(g["P"], oracle.marginal_precisions_exact(A), rtol=1e-11)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("lanes", [0, 1, 4, 32])
def test_parity_grid_c1(gb, variant, lanes):
    """32 x 32 grid, diagonal 4.5: same round count as the oracle; 1e-12 at convergence;
    1e-13 on x and messages at a fixed round."""
    m = synth.grid2d(32, -1.0, 4.5)
    b = synth.rhs(m.n, 1)
    ref = oracle.gabp_naive(m, b, max_iter=1000, tol=1e-12)
    g = _gpu_solve(gb, m, b, 1e-12, 1000, variant=variant, lanes=lanes)
    assert g["status"] == ref["status"] == 0
    assert g["iters"] == ref["iters"]
    assert _relerr(g["x"], ref["x"]) <= 1e-12
    off = ~_diag_mask(m)
    for t in (1, 5, 17):
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0, messages=True)
        gg = _gpu_solve(gb, m, b, 0.0, t, variant=variant, lanes=lanes)
        assert _relerr(gg["x"], r["x"]) <= 1e-13
        assert np.allclose(gg["Pmsg"][off], r["Pmsg"][off], rtol=1e-13, atol=1e-15)
        assert np.allclose(gg["hmsg"][off], (r["Pmsg"] * r["mumsg"])[off], rtol=1e-12, atol=1e-14)


def test_parity_grid_tight(gb):
    """Both sides to 1e-13 residual, then compared (and against the dense solution)."""
    m = synth.grid2d(32, -1.0, 4.5)
    b = synth.rhs(m.n, 1)
    ref = oracle.gabp_broadcast(m, b, max_iter=2000, tol=1e-13)
    g = _gpu_solve(gb, m, b, 1e-13, 2000)
    assert _relerr(g["x"], ref["x"]) <= 1e-12
    assert _relerr(g["x"], oracle.dense_solve(oracle.to_dense(m), b)) <= 1e-12


@pytest.mark.parametrize("n,picks,c", [(20011, 8, 1.1), (30001, 3, 1.2)])
def test_parity_random_several_tiles(gb, n, picks, c):
    """Random symmetric graphs spanning many blocks with a ragged last tile."""
    m = synth.random_sym(n, picks, c, 2)
    b = synth.rhs(m.n, 2)
    ref = oracle.gabp_broadcast(m, b, max_iter=500, tol=1e-12)
    for variant in (0, 1):
        g = _gpu_solve(gb, m, b, 1e-12, 500, variant=variant)
        assert g["status"] == ref["status"] == 0
        assert g["iters"] == ref["iters"]
        assert _relerr(g["x"], ref["x"]) <= 1e-12
        assert np.allclose(g["P"], ref["P"], rtol=1e-12)


def test_variants_agree(gb):
    m = synth.random_sym(5000, 5, 1.1, 4)
    b = synth.rhs(m.n, 4)
    a = _gpu_solve(gb, m, b, 0.0, 9, variant=0)
    c = _gpu_solve(gb, m, b, 0.0, 9, variant=1)
    assert _relerr(a["x"], c["x"]) <= 1e-14
    assert np.allclose(a["Pmsg"], c["Pmsg"], rtol=1e-14, atol=0)


def test_check_every_does_not_change_result(gb):
    m = synth.grid2d(24, -1.0, 4.5)
    b = synth.rhs(m.n, 8)
    a = _gpu_solve(gb, m, b, 1e-11, 1000, check_every=1)
    c = _gpu_solve(gb, m, b, 1e-11, 1000, check_every=37)
    assert a["iters"] == c["iters"] and np.array_equal(a["x"], c["x"])


def test_breakdown_gpu(gb):
    A = np.array([[2.0, 1.0, 0.0, 0.0], [1.0, 3.0, 1.0, 1.0], [0.0, 1.0, 1.0, 0.0], [0.0, 1.0, 0.0, 0.5]])
    m = synth.from_dense(A)
    for variant in (0, 1):
        g = _gpu_solve(gb, m, np.ones(4), 1e-14, 10, variant=variant)
        assert g["status"] == gb.GABP_BREAKDOWN and g["iters"] == 2


def test_not_converged_and_max_iter(gb):
    m = synth.grid2d(16, -1.0, 4.5)
    b = synth.rhs(m.n, 3)
    ref = oracle.gabp_naive(m, b, max_iter=7, tol=1e-14)
    g = _gpu_solve(gb, m, b, 1e-14, 7)
    assert g["status"] == ref["status"] == gb.GABP_NOT_CONVERGED and g["iters"] == 7
    assert _relerr(g["x"], ref["x"]) <= 1e-13


def test_divergence_reported(gb):
    """A non-walk-summable, indefinite system (diagonal 0.5 x row abs-sum): no hang, a status."""
    m = synth.random_sym(2000, 3, 0.5, 5)
    g = _gpu_solve(gb, m, synth.rhs(m.n, 5), 1e-10, 3000)
    assert g["status"] in (gb.GABP_DIVERGED, gb.GABP_NOT_CONVERGED, gb.GABP_BREAKDOWN)


def test_zero_rhs_and_tiny(gb):
    m = synth.grid2d(4)
    g = _gpu_solve(gb, m, np.zeros(m.n), 1e-12, 10)
    assert g["status"] == gb.GABP_OK and g["iters"] == 0 and not np.any(g["x"])
    m1 = synth.from_dense(np.array([[2.0]]))
    g = _gpu_solve(gb, m1, np.array([3.0]), 1e-14, 10)
    assert g["status"] == gb.GABP_OK and abs(g["x"][0] - 1.5) < 1e-15


@pytest.mark.parametrize("bad", ["asym_value", "asym_pattern", "zero_diag", "unsorted", "col_range"])
def test_invalid_matrix_rejected(gb, bad):
    A, _ = synth.toy3x3()
    m = synth.from_dense(A)
    rp, col, val = m.rowptr.copy(), m.col.copy(), m.val.copy()
    if bad == "asym_value":
        val[1] = 7.0
    elif bad == "asym_pattern":
        m = synth.from_coo(3, [0, 0, 1, 2, 2], [0, 1, 1, 0, 2], [1.0, 2.0, 1.0, 2.0, 1.0])
        rp, col, val = m.rowptr, m.col, m.val
    elif bad == "zero_diag":
        val[0] = 0.0
    elif bad == "unsorted":
        col[0], col[1] = col[1], col[0]
        val[0], val[1] = val[1], val[0]
    elif bad == "col_range":
        col[2] = 9
    with pytest.raises(gb.GaBPError) as ei:
        gb.Solver(3, rp, col, val)
    assert ei.value.status == gb.GABP_ERR_INVALID


def test_solve_host_matches_device(gb):
    m = synth.random_sym(3000, 4, 1.1, 6)
    b = synth.rhs(m.n, 6)
    s = _solver(gb, m)
    xd, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=500)
    xh = np.zeros(m.n)
    st2, it2, rel2 = s.solve_host(b.copy(), xh, tol=1e-12, max_iter=500)
    s.close()
    assert st == st2 == 0 and it == it2 and np.array_equal(xd.cpu().numpy(), xh)


def test_device_csr_input(gb):
    m = synth.grid2d(20, -1.0, 4.5)
    b = synth.rhs(m.n, 9)
    s = gb.Solver(m.n, torch.from_numpy(m.rowptr).cuda(), torch.from_numpy(m.col).cuda(),
                  torch.from_numpy(m.val).cuda())
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12)
    s.close()
    ref = oracle.gabp_naive(m, b, max_iter=1000, tol=1e-12)
    assert st == 0 and it == ref["iters"] and _relerr(x.cpu().numpy(), ref["x"]) <= 1e-12


def test_full_size_random_sym_c2(gb):
    """The benchmark workload (n = 2^20, 8 picks per row, diagonal 1.1 x row abs-sum) in the
    launch configuration the benchmark times: the residual recomputed on the host meets
    the tolerance, the round count equals the oracle's, and sampled entries agree with it."""
    m = synth.random_sym(1 << 20, 8, 1.1, 2)
    b = synth.rhs(m.n, 2)
    g = _gpu_solve(gb, m, b, 1e-10, 200)
    assert g["status"] == gb.GABP_OK
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    r = b - np.bincount(rows, m.val * g["x"][m.col], minlength=m.n)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    ref = oracle.gabp_broadcast(m, b, max_iter=200, tol=1e-10)
    assert g["iters"] == ref["iters"]
    idx = np.random.default_rng(0).choice(m.n, 4096, replace=False)
    assert np.allclose(g["x"][idx], ref["x"][idx], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("variant", [0, 1])
def test_residual_history(gb, variant):
    """options.history: the relative residual of every iterate x^(t) of an FP64 run, against the
    oracle's iterates after t rounds (x^(0) = b_i / A_ii); the last entry is the returned residual;
    an FP32 + refinement solve records none."""
    m = synth.grid2d(20, -1.0, 4.5)
    b = synth.rhs(m.n, 3)
    A = oracle.to_dense(m)
    s = gb.Solver.from_csr(m, variant=variant, history=256)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=500)
    h = s.residual_history()
    assert st == gb.GABP_OK and h.size == it + 1
    assert abs(h[-1] - rel) <= 1e-12 * max(rel, 1e-300) + 1e-300
    assert h[-1] <= 1e-10 < h[-2]
    nb = np.linalg.norm(b)
    x0 = b / np.diag(A)
    assert abs(h[0] - np.linalg.norm(b - A @ x0) / nb) <= 1e-12 * h[0]
    for t in (1, 2, 7, it):
        xt = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0)["x"]
        ref = np.linalg.norm(b - A @ xt) / nb
        assert abs(h[t] - ref) <= 1e-9 * ref + 1e-15, (t, h[t], ref)
    s.set_options(history=4)
    s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=500)
    assert s.residual_history().size == 4
    s.close()
    s32 = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, history=64)
    s32.solve(torch.from_numpy(b).cuda(), tol=1e-10)
    assert s32.residual_history().size == 0
    s32.close()


def test_warm_start_and_checkpoint(gb):
    """options.warm_start: round 0 takes the last FP64 solve's messages with the new b.  The same b
    is accepted after one round; a nearby b needs fewer rounds than a cold start and reaches the
    oracle's solution; messages exported (gabp_get_messages) and loaded into another handle
    (gabp_set_messages) resume the solve; b = 0 gives x = 0; new values disable the warm start."""
    m = synth.random_sym(3001, 8, 1.1, 2)
    b = synth.rhs(m.n, 3)
    b2 = b + 1e-3 * synth.rhs(m.n, 4)
    tb, tb2 = torch.from_numpy(b).cuda(), torch.from_numpy(b2).cuda()
    cold = gb.Solver.from_csr(m)
    x0, st, it0, _ = cold.solve(tb, tol=1e-12)
    assert st == gb.GABP_OK
    s = gb.Solver.from_csr(m, warm_start=1)
    xa, st, ita, _ = s.solve(tb, tol=1e-12)  # no state yet: a cold start
    assert st == gb.GABP_OK and ita == it0
    x1, st, it1, _ = s.solve(tb, tol=1e-12)
    assert st == gb.GABP_OK and it1 == 1
    assert _relerr(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-12
    x2w, st, it2w, _ = s.solve(tb2, tol=1e-12)
    x2c, st2, it2c, _ = cold.solve(tb2, tol=1e-12)
    assert st == st2 == gb.GABP_OK and it2w < it2c
    ref = oracle.gabp_broadcast(m, b2, max_iter=1000, tol=1e-13)
    assert _relerr(x2w.cpu().numpy(), ref["x"]) <= 1e-10
    P, hm = s.messages()
    r = gb.Solver.from_csr(m, warm_start=1)
    r.set_messages(P, hm)
    x3, st, it3, _ = r.solve(tb2, tol=1e-12)
    assert st == gb.GABP_OK and it3 == 1
    assert _relerr(x3.cpu().numpy(), x2w.cpu().numpy()) <= 1e-12
    xz, st, itz, _ = r.solve(torch.zeros_like(tb), tol=1e-12)
    assert st == gb.GABP_OK and not torch.any(xz)
    r.close()
    s.set_values(m.val)
    x4, st, it4, _ = s.solve(tb, tol=1e-12)
    assert st == gb.GABP_OK and it4 == it0
    s.close()
    cold.close()


def test_fp64_tuning_after_other_handles_freed(gb):
    """The FP64 autotuner's scratch control block is initialised in full (no field read from
    recycled device memory): an FP32 handle solves and is destroyed, then a new FP64 handle tunes
    and solves in the same process, as the benchmark does."""
    m = synth.random_sym(1 << 16, 8, 1.1, 2)
    b = torch.from_numpy(synth.rhs(m.n, 2)).cuda()
    for _ in range(2):
        s32 = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, reuse_precisions=0)
        for _ in range(3):
            s32.solve(b, tol=1e-10)
        s32.close()
        s64 = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP64)
        x, st, it, rel = s64.solve(b, tol=1e-10, max_iter=2000)
        s64.close()
        assert st == gb.GABP_OK and rel <= 1e-10


@pytest.mark.parametrize("p", [362, 363])
def test_cooperative_threshold(gb, p):
    """Graphs of up to 4096 slices of 32 rows run every round of a plain FP64 solve in one cooperative
    launch, larger ones launch a round kernel per round: a 362 x 362 grid (131,044 rows, 4096 slices)
    and a 363 x 363 grid (131,769 rows, 4118 slices) on either side of the threshold give the oracle's
    iterates at fixed rounds (1e-13), its round count at convergence, and the expected launches."""
    m = synth.grid2d(p, -1.0, 4.5)
    b = synth.rhs(m.n, 7)
    for t in (1, 9):
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0)
        g = _gpu_solve(gb, m, b, 0.0, t)
        assert g["iters"] == t and _relerr(g["x"], r["x"]) <= 1e-13
    ref = oracle.gabp_broadcast(m, b, max_iter=3000, tol=1e-10)
    s = _solver(gb, m, profile=1)
    s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=3000)
    s.profile(reset=True)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=3000)
    launches = s.profile()["launches"]
    s.close()
    assert st == gb.GABP_OK and it == ref["iters"]
    assert _relerr(x.cpu().numpy(), ref["x"]) <= 1e-9
    if (m.n + 31) // 32 <= 4096:
        assert launches == 3  # round 0, every round, the answer
    else:
        assert launches > 3


@pytest.mark.parametrize("p", [64, 65])
def test_cluster_rounds_grid64(gb, p):
    """The 64x64 grid (128 slices of width 4) runs in one cluster of 16 CTAs of eight warps with its
    state in shared memory; the 65x65 grid (133 slices) takes the cooperative grid.  Iterates and
    messages at fixed rounds are the oracle's to 1e-13, the converged round count is the oracle's,
    and the solve is three launches."""
    m = synth.grid2d(p, -1.0, 4.5)
    b = synth.rhs(m.n, 9)
    off = ~_diag_mask(m)
    for t in (1, 5):
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0, messages=True)
        g = _gpu_solve(gb, m, b, 0.0, t)
        assert g["iters"] == t and _relerr(g["x"], r["x"]) <= 1e-13, t
        assert np.allclose(g["Pmsg"][off], r["Pmsg"][off], rtol=1e-13, atol=1e-15), t
        assert np.allclose(g["hmsg"][off], (r["Pmsg"] * r["mumsg"])[off], rtol=1e-12, atol=1e-14), t
    ref = oracle.gabp_broadcast(m, b, max_iter=3000, tol=1e-12)
    s = _solver(gb, m, profile=1)
    s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=3000)
    s.profile(reset=True)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=3000)
    launches = s.profile()["launches"]
    s.close()
    assert st == gb.GABP_OK and it == ref["iters"]
    assert _relerr(x.cpu().numpy(), ref["x"]) <= 1e-12
    assert launches == 3


def test_cluster_handles_interleaved(gb):
    """The on-chip cluster rounds' shared memory differs per graph (about 80 KB a CTA on the
    1280-row random graph, 44 KB on the 45x45 grid with four warps a CTA, 4 KB on the 8x8 grid) and
    the kernel's launch limit is shared by every handle: handles set up and solved in alternation
    all run and all reach the oracle's answer in the oracle's round count."""
    mats = {"big": synth.random_sym(1280, 4, 1.1, 3), "mid": synth.grid2d(45, -1.0, 4.5),
            "small": synth.grid2d(8, -1.0, 4.5)}
    solvers = {k: _solver(gb, m) for k, m in mats.items()}
    refs = {}
    for k in ("big", "small", "big", "mid", "small", "mid", "big"):
        m = mats[k]
        b = synth.rhs(m.n, 5)
        if k not in refs:
            refs[k] = oracle.gabp_broadcast(m, b, max_iter=3000, tol=1e-12)
        x, st, it, rel = solvers[k].solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=3000)
        assert st == gb.GABP_OK and it == refs[k]["iters"], k
        assert _relerr(x.cpu().numpy(), refs[k]["x"]) <= 1e-12, k
    for s in solvers.values():
        s.close()


@pytest.mark.parametrize("n,deg", [(1, 0), (33, 4), (200, 4), (1024, 4), (1280, 4), (1280, 20), (1281, 4),
                                   (2048, 4), (2048, 20), (2049, 4), (4096, 4), (4096, 16), (4097, 4),
                                   (8192, 4)])
def test_cluster_rounds_small_graphs(gb, n, deg):
    """Graphs of at most 64 slices (2048 rows) run every plain FP64 round in one thread-block
    cluster (hardware cluster barrier, sums through distributed shared memory; two warps a CTA up
    to 32 slices, four up to 64); those whose state fits in the cluster's shared memory keep it
    there (every degree-4 case up to 2048 rows), the graphs of degree 20 read it from global
    memory.  From 65 to 128 slices (eight warps a CTA) only graphs whose slices are at most 8 slots
    wide take the cluster (test_cluster_rounds_grid64): these random graphs of 4096 rows, and 4097
    and 8192 rows, take the cooperative grid.  Iterates and messages at fixed rounds equal the
    oracle's to 1e-13, the converged round count is the oracle's, and the solve is three launches."""
    m = synth.random_sym(n, deg, 1.1, 3) if n > 1 else synth.from_dense(np.array([[2.0]]))
    b = synth.rhs(m.n, 8)
    for t in (1, 2, 7):
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0, messages=True)
        g = _gpu_solve(gb, m, b, 0.0, t)
        # a residual of exactly 0 meets tol = 0 (the one-node system is solved at round 1)
        assert g["iters"] == t or (g["status"] == gb.GABP_OK and g["relres"] == 0.0), t
        assert _relerr(g["x"], r["x"]) <= 1e-13, t
        if g["iters"] == t and n > 1:  # the messages of round t, written back from the cluster
            off = ~_diag_mask(m)
            assert np.allclose(g["Pmsg"][off], r["Pmsg"][off], rtol=1e-13, atol=1e-15), t
            assert np.allclose(g["hmsg"][off], (r["Pmsg"] * r["mumsg"])[off], rtol=1e-12, atol=1e-14), t
    ref = oracle.gabp_broadcast(m, b, max_iter=3000, tol=1e-12)
    s = _solver(gb, m, profile=1)
    s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=3000)
    s.profile(reset=True)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=3000)
    launches = s.profile()["launches"]
    s.close()
    assert st == gb.GABP_OK and it == ref["iters"]
    assert _relerr(x.cpu().numpy(), ref["x"]) <= 1e-12
    assert launches == 3
