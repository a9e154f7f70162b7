"""Many independent systems in one persistent launch (GPU, through the C ABI), against the
FP64 oracle per system.  Refined tolerance: 1e-10 relative error per system."""
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


def _check(gb, mats, split, zero_system=None, mode=0):
    big = synth.block_diag(mats)
    off = big.meta["offsets"]
    b = synth.rhs(big.n, 21)
    if zero_system is not None:
        b[off[zero_system]:off[zero_system + 1]] = 0.0
    s = gb.Solver.from_csr(big, multi_split=split, multi_mode=mode)
    x, st, sts, its, rel = s.solve_systems(torch.from_numpy(b).cuda(), off, tol=1e-12)
    tuned = s.tuned()
    s.close()
    if mode or split:
        assert tuned["multi_mode"] == 0  # a forced kernel is not recorded as a tuning choice
    else:
        assert tuned["multi_mode"] in (1, 2)
    assert st == gb.GABP_OK and np.all(sts == 0) and np.all(rel <= 1e-12)
    x = x.cpu().numpy()
    for k, m in enumerate(mats):
        xs, bs = x[off[k]:off[k + 1]], b[off[k]:off[k + 1]]
        if not np.any(bs):
            assert not np.any(xs)
            continue
        ref = oracle.gabp_broadcast(m, bs, max_iter=5000, tol=1e-13)
        assert _relerr(xs, ref["x"]) <= 1e-10, k


@pytest.mark.parametrize("split", [1, 1 << 30, 9000])
def test_systems_cluster_single_and_mixed(gb, split):
    """split 1: every system solved by a whole cluster; 2^30: every system by one block;
    9000: mixed (systems of rows + entries >= 9000 on clusters)."""
    mats = synth.rgg_batch(12, 1024, 8192, 2.0, 4)
    _check(gb, mats, split, zero_system=3)


def test_systems_autotuned_split(gb):
    mats = synth.rgg_batch(20, 1024, 16384, 2.0, 5)
    _check(gb, mats, 0)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_systems_forced_kernel(gb, mode):
    """mode 1: the grid-persistent kernel (one global round sweeps the rows of every running
    system); mode 2: cluster / single-block teams with an autotuned split; mode 3: the
    grid-persistent kernel on the sliced layout (32-row slices of degree-sorted rows, each
    system padded to whole slices)."""
    mats = synth.rgg_batch(16, 1024, 16384, 2.0, 7)
    _check(gb, mats, 0, zero_system=5, mode=mode)


@pytest.mark.parametrize("mode", [1, 3])
def test_systems_grid_breakdown_isolated(gb, mode):
    """One system whose precision recursion breaks down (a zero cavity precision) stops with
    BREAKDOWN in the grid-persistent kernel (row CSR or sliced) while the others still converge."""
    good = synth.rgg_batch(3, 1024, 2048, 2.0, 8)
    star = synth.from_dense(np.array([[2.0, 1, 0, 0], [1, 3, 1, 1], [0, 1, 1, 0], [0, 1, 0, 0.5]]))
    mats = [good[0], star, good[1], good[2]]
    big = synth.block_diag(mats)
    off = big.meta["offsets"]
    b = synth.rhs(big.n, 3)
    s = gb.Solver.from_csr(big, multi_mode=mode)
    x, st, sts, its, rel = s.solve_systems(torch.from_numpy(b).cuda(), off, tol=1e-12)
    s.close()
    assert st == gb.GABP_BREAKDOWN
    assert sts[1] == gb.GABP_BREAKDOWN and sts[0] == sts[2] == sts[3] == gb.GABP_OK
    x = x.cpu().numpy()
    for k in (0, 2, 3):
        sl = slice(off[k], off[k + 1])
        ref = oracle.gabp_broadcast(mats[k], b[sl], max_iter=5000, tol=1e-13)
        assert _relerr(x[sl], ref["x"]) <= 1e-10


def test_systems_coupled_rejected(gb):
    mats = synth.rgg_batch(2, 1024, 2048, 2.0, 6)
    big = synth.block_diag(mats)
    off = big.meta["offsets"].copy()
    off[1] += 1  # the boundary now cuts through the first system's edges
    s = gb.Solver.from_csr(big)
    b = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GaBPError) as ei:
        s.solve_systems(b, off)
    s.close()
    assert ei.value.status == gb.GABP_ERR_INVALID


def test_512_power_law_systems(gb):
    """The benchmark batch: 512 random geometric graphs, sizes ~ n^-2 on [1024, 65536].
    Every system's residual recomputed on the host meets the tolerance; 8 systems are
    compared with the oracle."""
    mats = synth.rgg_batch(512, 1024, 65536, 2.0, 4)
    big = synth.block_diag(mats)
    off = big.meta["offsets"]
    b = synth.rhs(big.n, 4)
    s = gb.Solver.from_csr(big)
    x, st, sts, its, rel = s.solve_systems(torch.from_numpy(b).cuda(), off, tol=1e-10)
    s.close()
    assert st == gb.GABP_OK and np.all(sts == 0)
    x = x.cpu().numpy()
    rows = np.repeat(np.arange(big.n), np.diff(big.rowptr))
    r = b - np.bincount(rows, big.val * x[big.col], minlength=big.n)
    for k in range(len(mats)):
        sl = slice(off[k], off[k + 1])
        assert np.linalg.norm(r[sl]) <= 1.0001e-10 * np.linalg.norm(b[sl])
    sizes = np.diff(off)
    for k in list(np.argsort(sizes)[:4]) + list(np.argsort(sizes)[-4:]):
        sl = slice(off[k], off[k + 1])
        ref = oracle.gabp_broadcast(mats[k], b[sl], max_iter=5000, tol=1e-12)
        assert _relerr(x[sl], ref["x"]) <= 1e-9


def test_sliced_layout_new_values_and_offsets(gb):
    """The sliced layout follows the handle: new values (gabp_set_values: A scaled by 2 halves x)
    are picked up, and another offsets array (two neighbouring systems merged into one, still a
    block-diagonal split) rebuilds it; each result against the oracle per system."""
    mats = synth.rgg_batch(9, 1024, 8192, 2.0, 11)
    big = synth.block_diag(mats)
    off = big.meta["offsets"]
    b = synth.rhs(big.n, 12)
    bt = torch.from_numpy(b).cuda()
    s = gb.Solver.from_csr(big, multi_mode=3)
    x1, st, sts, its, rel = s.solve_systems(bt, off, tol=1e-12)
    assert st == gb.GABP_OK
    assert s.tuned()["multi_mode"] == 0 and s.tuned()["multi_grid_sliced"]
    s.set_values(2.0 * big.val)
    x2, st2, _, _, _ = s.solve_systems(bt, off, tol=1e-12)
    assert st2 == gb.GABP_OK
    x1, x2 = x1.cpu().numpy(), x2.cpu().numpy()
    for k, m in enumerate(mats):
        sl = slice(off[k], off[k + 1])
        ref = oracle.gabp_broadcast(m, b[sl], max_iter=5000, tol=1e-13)
        assert _relerr(x1[sl], ref["x"]) <= 1e-10, k
        assert _relerr(x2[sl], 0.5 * ref["x"]) <= 1e-10, k
    off2 = np.concatenate([off[:3], off[4:]])  # systems 2 and 3 as one
    x3, st3, sts3, _, _ = s.solve_systems(bt, off2, tol=1e-12)
    s.close()
    assert st3 == gb.GABP_OK and len(sts3) == len(mats) - 1
    x3 = x3.cpu().numpy()
    assert _relerr(x3, x2) <= 1e-10
