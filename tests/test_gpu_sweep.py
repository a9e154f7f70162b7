"""A seeded sweep of small systems of uneven size and density through every single-RHS path and
the batched and independent-systems entry points, against the dense solution (through the C ABI).

Sizes from 1 to a few hundred rows cover ragged tails of every tile and sub-warp shape; the
matrices are symmetric, strictly diagonally dominant (diagonal 1.1-1.5 x the row abs-sum), so
every path converges and the dense LU solution is the fixed point (Sec. "Convergence and
Exactness": walk-summable models)."""
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


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 300))
    p = float(rng.uniform(0.0, min(1.0, 12.0 / max(n, 1))))
    M = np.triu(rng.uniform(-1.0, 1.0, (n, n)) * (rng.random((n, n)) < p), 1)
    M = M + M.T
    d = np.abs(M).sum(axis=1) * rng.uniform(1.1, 1.5) + (np.abs(M).sum(axis=1) == 0)
    A = M + np.diag(d)
    return synth.from_dense(A), A, rng.standard_normal(n)


PATHS = [dict(precision=0), dict(precision=0, variant=1), dict(precision=0, schedule=1),
         dict(precision=0, accel=1), dict(precision=0, accel=2), dict(precision=0, schedule=1, accel=2),
         dict(precision=0, graphs=0), dict(precision=1), dict(precision=1, device_loop=0),
         dict(precision=1, schedule=1), dict(precision=1, overlap_precision=0)]


@pytest.mark.parametrize("seed", range(12))
def test_small_systems_every_path(gb, seed):
    m, A, b = _case(seed)
    x_ref = np.linalg.solve(A, b)
    cond_bound = 1.0 / (1.0 - 1.0 / 1.1)  # strict dominance: ||A^{-1}|| ||A|| bounded by (1 + r) / (1 - r)
    for opts in PATHS:
        s = gb.Solver.from_csr(m, **opts)
        x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=5000)
        s.close()
        assert st == gb.GABP_OK, (seed, opts, st)
        err = np.linalg.norm(x.cpu().numpy() - x_ref) / max(np.linalg.norm(x_ref), 1e-300)
        assert err <= 1e-12 * 3 * cond_bound, (seed, opts, err)


@pytest.mark.parametrize("seed", range(4))
def test_small_systems_batched_and_independent(gb, seed):
    m, A, b = _case(seed + 20)
    R = 3
    B = np.stack([b, 2.0 * b[::-1].copy(), np.zeros_like(b)])
    s = gb.Solver.from_csr(m)
    X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-12)
    s.close()
    assert st == gb.GABP_OK
    X = X.cpu().numpy()
    for r in range(R):
        ref = np.linalg.solve(A, B[r])
        assert np.linalg.norm(X[r] - ref) <= 1e-10 * max(np.linalg.norm(ref), 1e-300)
    mats = [_case(seed + 40 + j)[0] for j in range(3)]
    big = synth.block_diag(mats)
    bb = synth.rhs(big.n, seed)
    sm = gb.Solver.from_csr(big)
    x, st, sts, its, rels = sm.solve_systems(torch.from_numpy(bb).cuda(), big.meta["offsets"], tol=1e-12)
    sm.close()
    assert st == gb.GABP_OK and np.all(sts == gb.GABP_OK)
    ref = np.linalg.solve(oracle.to_dense(big), bb)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("seed", range(6))
def test_small_rectangular_least_squares(gb, seed):
    """Rectangular J of random shape (1 to ~200 rows and columns, over- and under-determined, some
    empty rows and columns) through the augmented system, against the dense ridge normal equations.
    Plain FP64 GaBP with gamma in [0.5, 2] (models that are NOT walk-summable: rho(|R|) up to ~14, and
    it converged on every case tried); FP32 + refinement with gamma = 1.5 sigma_max(|J|)^2, the loading
    for which the general-linear-systems section states the model is walk-summable (its frozen
    coefficients diverge on some of the loosely loaded cases, reported as GABP_DIVERGED)."""
    from scipy.sparse import csr_matrix

    rng = np.random.default_rng(500 + seed)
    m_, k_ = int(rng.integers(1, 200)), int(rng.integers(1, 200))
    Jd = rng.standard_normal((m_, k_)) * (rng.random((m_, k_)) < min(1.0, 6.0 / k_))
    c = csr_matrix(Jd)
    J = synth.RectCSR(m_, k_, c.indptr.astype(np.int32), c.indices.astype(np.int32), c.data.copy())
    y = rng.standard_normal(m_)
    g_loose = float(rng.uniform(0.5, 2.0))
    g_ws = 1.5 * max(float(np.linalg.norm(np.abs(Jd), 2)) ** 2, 1e-3)
    for prec, gamma in ((0, g_loose), (0, g_ws), (1, g_ws)):
        xr = np.linalg.solve(Jd.T @ Jd + gamma * np.eye(k_), Jd.T @ y)
        s = gb.LSQSolver.from_rect(J, gamma, precision=prec)
        x, z, st, it, rel = s.solve_lsq(torch.from_numpy(y).cuda(), tol=1e-12, max_iter=20000)
        s.close()
        assert st == gb.GABP_OK, (seed, prec, gamma, st)
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-9 * max(np.linalg.norm(xr), 1e-300), (seed, prec)
