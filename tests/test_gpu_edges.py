"""Degenerate inputs across every path (through the C ABI): a matrix without edges (diagonal
only: one colour, every message set empty), a single node, isolated nodes inside a graph,
a star (one row holding most of the edges, the other rows one each), and a one-column batch.
Each result is checked against the exact solution (x_i = b_i / A_ii where there are no
edges) or the FP64 oracle."""
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


PATHS = [
    dict(precision=0),
    dict(precision=0, variant=1),
    dict(precision=0, schedule=1),
    dict(precision=1),
    dict(precision=1, device_loop=0),
    dict(precision=1, schedule=1),
    dict(precision=1, overlap_precision=0),
    dict(precision=0, gamma_mode=1, fix_single_loop=1),
    dict(precision=1, gamma_mode=1),
]


def _solve(gb, m, b, **opts):
    s = gb.Solver.from_csr(m, **opts)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=1e-12, max_iter=20000)
    s.close()
    return x.cpu().numpy(), st


@pytest.mark.parametrize("opts", PATHS, ids=[str(p) for p in PATHS])
def test_diagonal_only(gb, opts):
    n = 777
    d = np.random.default_rng(3).uniform(0.5, 3.0, n)
    m = synth.from_coo(n, np.arange(n), np.arange(n), d)
    b = synth.rhs(n, 2)
    x, st = _solve(gb, m, b, **opts)
    assert st == gb.GABP_OK
    assert np.allclose(x, b / d, rtol=1e-12)


@pytest.mark.parametrize("opts", PATHS, ids=[str(p) for p in PATHS])
def test_single_node(gb, opts):
    m = synth.from_coo(1, [0], [0], [2.5])
    x, st = _solve(gb, m, np.array([5.0]), **opts)
    # GaBP is exact after one round; the convergence fix is a geometric outer iteration that
    # stops at the 1e-12 residual
    assert st == gb.GABP_OK and abs(x[0] - 2.0) <= (4e-12 if opts.get("gamma_mode") else 1e-14)


@pytest.mark.parametrize("opts", PATHS, ids=[str(p) for p in PATHS])
def test_isolated_nodes_and_star(gb, opts):
    """Rows 0..9 isolated, a star centred on row 10 with 300 leaves, a path on the rest."""
    n = 400
    rows, cols, vals = [], [], []
    rng = np.random.default_rng(5)
    for k in range(11, 311):
        w = rng.uniform(-1, 1) * 0.5
        rows += [10, k]; cols += [k, 10]; vals += [w, w]
    for k in range(311, n - 1):
        w = rng.uniform(-1, 1)
        rows += [k, k + 1]; cols += [k + 1, k]; vals += [w, w]
    A = np.zeros((n, n))
    A[rows, cols] = vals
    d = np.abs(A).sum(axis=1) * 1.3 + 1.0
    m = synth.from_coo(n, rows + list(range(n)), cols + list(range(n)), vals + list(d))
    b = synth.rhs(n, 6)
    x, st = _solve(gb, m, b, **opts)
    assert st == gb.GABP_OK
    assert _relerr(x, np.linalg.solve(oracle.to_dense(m), b)) <= 1e-10


@pytest.mark.parametrize("sched", [0, 1])
def test_batched_one_column_and_diagonal(gb, sched):
    m = synth.grid2d(20, -1.0, 4.5)
    B = synth.rhs_batch(m.n, 1, 4)
    s = gb.Solver.from_csr(m, schedule=sched)
    X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-12)
    s.close()
    assert st == gb.GABP_OK
    assert _relerr(X.cpu().numpy()[0], np.linalg.solve(oracle.to_dense(m), B[0])) <= 1e-10
    n = 300
    d = np.linspace(1.0, 2.0, n)
    md = synth.from_coo(n, np.arange(n), np.arange(n), d)
    B = synth.rhs_batch(n, 3, 7)
    s = gb.Solver.from_csr(md, schedule=sched)
    X, st, it, rel = s.solve_batched(torch.from_numpy(B).cuda(), tol=1e-12)
    s.close()
    assert st == gb.GABP_OK and np.allclose(X.cpu().numpy(), B / d, rtol=1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_systems_with_edgeless_and_single_node_systems(gb, mode):
    """Independent systems including a 1-node system and an edgeless one among ordinary ones."""
    mats = synth.rgg_batch(3, 1024, 2048, 2.0, 9)
    mats.insert(1, synth.from_coo(1, [0], [0], [4.0]))
    mats.insert(3, synth.from_coo(50, np.arange(50), np.arange(50), np.linspace(1, 2, 50)))
    big = synth.block_diag(mats)
    off = big.meta["offsets"]
    b = synth.rhs(big.n, 3)
    s = gb.Solver.from_csr(big, multi_mode=mode)
    x, st, sts, its, rel = s.solve_systems(torch.from_numpy(b).cuda(), off, tol=1e-12)
    s.close()
    assert st == gb.GABP_OK and np.all(sts == 0)
    assert _relerr(x.cpu().numpy(), np.linalg.solve(oracle.to_dense(big), b)) <= 1e-10


def test_binding_rejects_mismatched_buffers(gb):
    """The binding hands raw pointers to the library, so every buffer the library reads or writes
    is checked first: wrong length, dtype, layout or device raise ValueError before any launch,
    and the solver stays usable."""
    m = synth.grid2d(8, -1.0, 4.5)
    s = gb.Solver.from_csr(m)
    b = torch.from_numpy(synth.rhs(m.n, 1)).cuda()
    with pytest.raises(ValueError):
        s.solve(b[:-1])
    with pytest.raises(ValueError):
        s.solve(b, x=torch.empty(m.n, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        s.solve(b, x=torch.empty(2 * m.n, dtype=torch.float64, device="cuda")[::2])
    with pytest.raises(ValueError):
        s.solve(b, x=torch.empty(m.n - 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        s.solve_host(np.zeros(m.n - 1), np.zeros(m.n))
    with pytest.raises(ValueError):
        s.solve_host(np.zeros(m.n), np.zeros(m.n, dtype=np.float32))
    with pytest.raises(ValueError):
        s.solve_batched(torch.zeros(2, m.n, dtype=torch.float64, device="cuda"),
                        X=torch.empty(3, m.n, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        s.set_values(m.val[:-1])
    with pytest.raises(ValueError):
        s.grad_values(b[:-1], b)
    x, st, it, rel = s.solve(b, tol=1e-12)
    s.close()
    assert st == gb.GABP_OK
    # residual 1e-12, condition number ~17: the error is within 1e-10
    assert _relerr(x.cpu().numpy(), np.linalg.solve(oracle.to_dense(m), synth.rhs(m.n, 1))) <= 1e-10
