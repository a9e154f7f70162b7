"""The FP64 precision freeze (options.freeze_precisions = 1) against the plain FP64 path and the
FP64 CPU oracle, through the C ABI.

The precision update of Algorithm 1 involves A only, so the precision messages settle by
themselves (the convergence section gives a condition for the variances alone); the freeze
stores the edge coefficients -A_ki / P_k\\i and 1/P~ of the round in which every precision message
was verified stagnant (16 units in the last place) and then updates only the mean messages.  Bars:

* every round up to the stored one (gabp_last_freeze) is bitwise the plain solve's: the residual
  history entries and, at a fixed round at or before it, x and every message are equal;
* after it, x and the mean messages at a fixed round agree with the oracle's iterate of that round
  to 1e-12 relative element by element (the frozen coefficients differ from recomputed ones by
  rounding, and the mean iteration contracts);
* at convergence the round count is the plain solve's within one and x agrees with the oracle's
  converged x to the FP64 target, element by element.
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


def _solve(gb, m, b, tol, max_iter, messages=False, **opts):
    s = gb.Solver.from_csr(m, history=8192, **opts)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=max_iter)
    out = {"x": x.cpu().numpy(), "status": st, "iters": it, "relres": rel,
           "hist": s.residual_history().copy(), **s.stats()}
    if messages:
        P, hm = s.messages()
        out["Pmsg"], out["hmsg"] = P.cpu().numpy(), hm.cpu().numpy()
    s.close()
    return out


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _offdiag(m):
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    return rows != m.col


# (name, matrix, tol): the first three run in one thread-block cluster (two, four and eight warps
# a CTA; the plain rounds with their state in shared memory), the next in the cooperative launch
# (<= 131,072 rows), the last two in the launch-per-round path (CUDA graphs of check_every rounds)
CASES = [
    ("grid2d_32", lambda: synth.grid2d(32, -1.0, 4.5), 1e-12),
    ("grid2d_45", lambda: synth.grid2d(45, -1.0, 4.5), 1e-12),
    ("grid2d_64", lambda: synth.grid2d(64, -1.0, 4.5), 1e-12),
    ("random_20011", lambda: synth.random_sym(20011, 8, 1.1, 2), 1e-12),
    ("random_262144", lambda: synth.random_sym(1 << 18, 8, 1.1, 2), 1e-12),
    ("grid3d_64", lambda: synth.grid3d(64, 1.1, 2), 1e-10),
]


@pytest.mark.parametrize("name,make,tol", CASES, ids=[c[0] for c in CASES])
def test_freeze_matches_plain_and_oracle(gb, name, make, tol):
    m = make()
    b = synth.rhs(m.n, 2)
    p = _solve(gb, m, b, tol, 3000)
    f = _solve(gb, m, b, tol, 3000, freeze_precisions=1)
    assert p["status"] == f["status"] == gb.GABP_OK
    assert p["freeze_round"] == 0 and p["freeze_checks"] == 0
    F = f["freeze_round"]
    assert 0 < F < f["iters"], (F, f["iters"])  # engaged before the end
    assert f["freeze_checks"] >= 1
    # rounds 0..F bitwise the plain solve's (entry t is the residual of x^(t))
    assert np.array_equal(f["hist"][:F + 1], p["hist"][:F + 1])
    assert abs(f["iters"] - p["iters"]) <= 1
    assert f["relres"] <= tol
    ref = oracle.gabp_broadcast(m, b, max_iter=3000, tol=tol)
    assert ref["status"] == oracle.OK and abs(ref["iters"] - f["iters"]) <= 1
    assert _maxrel(f["x"], ref["x"]) <= 100 * tol
    assert _maxrel(f["x"], p["x"]) <= 100 * tol


@pytest.mark.parametrize("name,make", [("grid2d_32", lambda: synth.grid2d(32, -1.0, 4.5)),
                                       ("random_262144", lambda: synth.random_sym(1 << 18, 8, 1.1, 2))],
                         ids=["grid2d_32", "random_262144"])
def test_fixed_rounds_vs_oracle(gb, name, make):
    """x and every message at fixed rounds: bitwise the plain solve's up to the stored round,
    the oracle's iterate to 1e-12 (x, mean messages) and 1e-13 (precision messages) after it."""
    m = make()
    b = synth.rhs(m.n, 5)
    F = _solve(gb, m, b, 0.0, 60, freeze_precisions=1)["freeze_round"]
    assert F > 0
    off = _offdiag(m)
    for t in (F, F + 1, F + 7, F + 30):
        g = _solve(gb, m, b, 0.0, t, messages=True, freeze_precisions=1)
        assert g["iters"] == t and g["status"] == gb.GABP_NOT_CONVERGED
        if t <= F:
            p = _solve(gb, m, b, 0.0, t, messages=True)
            assert np.array_equal(g["x"], p["x"])
            assert np.array_equal(g["Pmsg"], p["Pmsg"]) and np.array_equal(g["hmsg"], p["hmsg"])
            continue
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0, messages=True)
        assert _maxrel(g["x"], r["x"]) <= 1e-12
        assert np.allclose(g["x"], r["x"], rtol=1e-12, atol=1e-14 * np.max(np.abs(r["x"])))
        hm = (r["Pmsg"] * r["mumsg"])[off]
        assert np.allclose(g["hmsg"][off], hm, rtol=1e-12, atol=1e-14 * np.max(np.abs(hm)))
        assert np.allclose(g["Pmsg"][off], r["Pmsg"][off], rtol=1e-13, atol=0.0)


def _scaled_sym(seed):
    """Small symmetric matrices with rows scaled over six decades and a diagonal just above the
    row's absolute off-diagonal sum: some cavities P~_k - P_ik nearly cancel, so a message can
    still move while every aggregate it enters is stagnant."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.6)
    M = np.triu(M, 1)
    M = M + M.T
    s = 10.0 ** rng.uniform(-3, 3, n)
    A = M * np.sqrt(np.outer(s, s))
    A[np.diag_indices(n)] = np.abs(A).sum(1) * rng.uniform(1.0001, 1.2, n) + 1e-12
    return A


SCALED_SEEDS = (65, 55, 111, 160, 171, 0, 2, 3, 6, 9)


def test_failed_verification_then_freeze(gb):
    """On badly scaled systems a verification can fail (a message moved although no aggregate
    did): the screen resumes with a longer run and a later verification may freeze.  Over 300
    rounds at least one of these systems takes that path, bitwise the plain run up to its stored
    round; every one converges (to 1e-10) in the plain solve's rounds within one, and its x is
    within cond(A) x the residual of the dense solution."""
    seen_retry = False
    for seed in SCALED_SEEDS:
        A = _scaled_sym(seed)
        m = synth.from_dense(A)
        b = synth.rhs(m.n, seed)
        p = _solve(gb, m, b, 0.0, 300)
        f = _solve(gb, m, b, 0.0, 300, freeze_precisions=1)
        F, checks = f["freeze_round"], f["freeze_checks"]
        if F > 0:
            assert np.array_equal(f["hist"][:F + 1], p["hist"][:F + 1]), seed
        seen_retry |= F > 0 and checks >= 2
        p = _solve(gb, m, b, 1e-10, 20000)
        f = _solve(gb, m, b, 1e-10, 20000, freeze_precisions=1)
        assert p["status"] == f["status"] == gb.GABP_OK, (seed, p["status"], f["status"])
        assert abs(f["iters"] - p["iters"]) <= 1, (seed, f["iters"], p["iters"])
        r = b - A @ f["x"]
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b), seed
        x = np.linalg.solve(A, b)  # relative error <= cond(A) x relative residual
        assert np.linalg.norm(f["x"] - x) <= 2e-10 * np.linalg.cond(A) * np.linalg.norm(x), seed
    assert seen_retry


def test_paths_without_freeze_unchanged(gb):
    """The option applies to plain FP64 node rounds and plain serial sweeps only: Aitken, Steffensen
    (both schedules), the edge variant and FP32 + refinement give bitwise the same result with it on."""
    m = synth.grid2d(32, -1.0, 4.5)
    b = synth.rhs(m.n, 1)
    for opts in ({"accel": 1}, {"accel": 2}, {"variant": 1}, {"schedule": 1, "accel": 2},
                 {"precision": gb.GABP_PREC_FP32_REFINE}):
        a = _solve(gb, m, b, 1e-12, 2000, **opts)
        c = _solve(gb, m, b, 1e-12, 2000, freeze_precisions=1, **opts)
        assert a["status"] == c["status"] == gb.GABP_OK, opts
        assert a["iters"] == c["iters"] and np.array_equal(a["x"], c["x"]), opts
        assert c["freeze_round"] == 0 and c["freeze_checks"] == 0, opts


def test_launch_shapes_agree(gb):
    """Launch-per-round path: the graph length (check_every) and stream launches instead of graphs
    do not change a bit of the result or the stored round."""
    m = synth.random_sym(1 << 18, 8, 1.1, 2)
    b = synth.rhs(m.n, 3)
    runs = [_solve(gb, m, b, 1e-12, 500, freeze_precisions=1, check_every=k, graphs=g)
            for k, g in ((16, 1), (1, 1), (5, 0))]
    for r in runs[1:]:
        assert r["status"] == runs[0]["status"] == gb.GABP_OK
        assert r["iters"] == runs[0]["iters"] and r["freeze_round"] == runs[0]["freeze_round"]
        assert np.array_equal(r["x"], runs[0]["x"])


def test_warm_start_zero_rhs_and_options(gb):
    """A warm start from frozen-precision messages reaches the oracle's solution; b = 0 gives
    x = 0 with no freeze; freeze_precisions outside {0, 1} is rejected."""
    m = synth.random_sym(3001, 8, 1.1, 2)
    b = synth.rhs(m.n, 3)
    b2 = b + 1e-3 * synth.rhs(m.n, 4)
    s = gb.Solver.from_csr(m, freeze_precisions=1, warm_start=1)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=1000)
    assert st == gb.GABP_OK and s.stats()["freeze_round"] > 0
    x2, st2, it2, rel2 = s.solve(torch.from_numpy(b2).cuda(), tol=1e-12, max_iter=1000)
    ref = oracle.gabp_broadcast(m, b2, max_iter=1000, tol=1e-12)
    assert st2 == gb.GABP_OK and it2 < ref["iters"]
    assert _maxrel(x2.cpu().numpy(), ref["x"]) <= 1e-10
    x0, st0, it0, rel0 = s.solve(torch.zeros(m.n, dtype=torch.float64, device="cuda"), tol=1e-12, max_iter=100)
    assert st0 == gb.GABP_OK and float(x0.abs().max()) == 0.0 and s.stats()["freeze_round"] == 0
    s.close()
    with pytest.raises(gb.GaBPError):
        gb.Solver.from_csr(m, freeze_precisions=2)


SERIAL_CASES = [
    ("grid2d_32", lambda: synth.grid2d(32, -1.0, 4.5), 1e-12),
    ("grid3d_32", lambda: synth.grid3d(32, 1.1, 2), 1e-10),
    ("random_20011", lambda: synth.random_sym(20011, 8, 1.1, 2), 1e-12),
]


@pytest.mark.parametrize("name,make,tol", SERIAL_CASES, ids=[c[0] for c in SERIAL_CASES])
def test_serial_freeze(gb, name, make, tol):
    """The serial schedule (sweeps of colour passes, one message store): a screen on the marginal
    precisions after each sweep, a verifying sweep that stores the coefficients, then mean-only
    sweeps.  x after a fixed number of sweeps is bitwise the plain sweeps' up to the stored sweep
    and the oracle's serial iterate to 1e-12 after it; converged, the sweep count is the plain one
    within one and x the oracle's to 100 tol."""
    m = make()
    b = synth.rhs(m.n, 4)
    p = _solve(gb, m, b, tol, 5000, schedule=1)
    f = _solve(gb, m, b, tol, 5000, schedule=1, freeze_precisions=1)
    assert p["status"] == f["status"] == gb.GABP_OK
    F = f["freeze_round"]
    assert 0 < F < f["iters"] and f["freeze_checks"] >= 1, (F, f["iters"], f["freeze_checks"])
    assert abs(f["iters"] - p["iters"]) <= 1
    ref = oracle.gabp_serial(m, b, max_iter=5000, tol=tol)
    assert ref["status"] == oracle.OK
    assert _maxrel(f["x"], ref["x"]) <= 100 * tol
    for t in (F, F + 1, F + 7):
        g = _solve(gb, m, b, 0.0, t, schedule=1, freeze_precisions=1)
        assert g["iters"] == t
        if t <= F:
            q = _solve(gb, m, b, 0.0, t, schedule=1)
            assert np.array_equal(g["x"], q["x"]), t
        else:
            r = oracle.gabp_serial(m, b, max_iter=t, tol=0.0)
            assert np.allclose(g["x"], r["x"], rtol=1e-12, atol=1e-14 * np.max(np.abs(r["x"]))), t
