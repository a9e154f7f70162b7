"""Changing options on a live handle (gabp_set_options) between solves.

A handle caches captured CUDA graphs of its rounds; a cached graph holds
`check_every` rounds and, for the single-loop convergence fix, the damping step.
After the options change, a solve on the old handle must give what a fresh handle
with the new options gives: the same status and round count and the same iterate.
The sequence raises `check_every` from 1 to 64 so that a graph holding the old,
shorter round count would run out of host polls before the stop rule fires.  The
fresh handle also solves twice: a second solve reuses the converged precision
messages of the first (reuse_precisions), so only second solves compare."""
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


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


PATHS = {
    "fp64_parallel": dict(),
    "fp64_serial": dict(schedule=1),
    "fp64_aitken": dict(accel=1),
    "fp32_parallel": dict(precision=1),
    "fp32_serial": dict(precision=1, schedule=1),
    "fix_single_loop": dict(gamma_mode=1, gamma=0.25, fix_single_loop=1),
}


@pytest.mark.parametrize("path", sorted(PATHS))
def test_check_every_change(gb, path):
    # n = 4096, 3-D grid with a weak diagonal: 73 FP64 rounds to 1e-10; max_iter = 1000
    # with a stale 1-round graph would give up after 1000 // 64 + 3 polls
    m = synth.grid3d(16, 1.15, 3)
    b = torch.from_numpy(synth.rhs(m.n, 4)).cuda()
    opts = PATHS[path]
    s = gb.Solver.from_csr(m, check_every=1, **opts)
    s.solve(b, tol=1e-10, max_iter=1000)
    s.set_options(check_every=64)
    x, st, it, rel = s.solve(b, tol=1e-10, max_iter=1000)
    x = x.cpu().numpy()
    s.close()
    f = gb.Solver.from_csr(m, check_every=64, **opts)
    f.solve(b, tol=1e-10, max_iter=1000)
    xf, stf, itf, relf = f.solve(b, tol=1e-10, max_iter=1000)
    f.close()
    assert st == stf == gb.GABP_OK, (st, stf)
    assert it == itf
    assert _relerr(x, xf.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("schedule", [0, 1])
def test_check_every_change_batched(gb, schedule):
    m = synth.grid3d(16, 1.15, 3)
    B = torch.from_numpy(synth.rhs_batch(m.n, 5, 6)).cuda()
    s = gb.Solver.from_csr(m, check_every=1, schedule=schedule)
    s.solve_batched(B, tol=1e-10, max_iter=1000)
    s.set_options(check_every=64)
    X, st, it, rel = s.solve_batched(B, tol=1e-10, max_iter=1000)
    X = X.cpu().numpy()
    s.close()
    f = gb.Solver.from_csr(m, check_every=64, schedule=schedule)
    f.solve_batched(B, tol=1e-10, max_iter=1000)
    Xf, stf, itf, relf = f.solve_batched(B, tol=1e-10, max_iter=1000)
    f.close()
    assert st == stf == gb.GABP_OK
    assert it == itf
    assert _relerr(X, Xf.cpu().numpy()) <= 1e-12


def test_fix_step_change(gb):
    """The single loop's damping step is an argument of its captured rounds."""
    m = synth.random_sym(1024, 3, 0.8, 7)
    b = torch.from_numpy(synth.rhs(m.n, 5)).cuda()
    s = gb.Solver.from_csr(m, gamma_mode=1, gamma=0.3, fix_single_loop=1, fix_step=0.5)
    x1, st1, it1, _ = s.solve(b, tol=1e-10, max_iter=20000)
    s.set_options(fix_step=0.25)
    x2, st2, it2, _ = s.solve(b, tol=1e-10, max_iter=20000)
    s.close()
    f = gb.Solver.from_csr(m, gamma_mode=1, gamma=0.3, fix_single_loop=1, fix_step=0.25)
    f.solve(b, tol=1e-10, max_iter=20000)
    xf, stf, itf, _ = f.solve(b, tol=1e-10, max_iter=20000)
    f.close()
    assert st1 == st2 == stf == gb.GABP_OK
    assert it2 == itf and it2 != it1
    assert _relerr(x2.cpu().numpy(), xf.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("path", ["fp64_parallel", "fp64_serial", "fp32_parallel", "fp32_serial"])
def test_runs_are_bitwise_reproducible(gb, path):
    """The synchronous rounds read round t-1 and write round t, and every reduction is a
    fixed-order last-block reduction (no floating-point atomics): two handles give bit-identical
    iterates and round counts."""
    m = synth.random_sym(20011, 8, 1.1, 2)
    b = torch.from_numpy(synth.rhs(m.n, 5)).cuda()
    out = []
    for _ in range(2):
        s = gb.Solver.from_csr(m, lanes=4, **PATHS[path])
        x, st, it, rel = s.solve(b, tol=1e-10, max_iter=2000)
        s.close()
        out.append((x.cpu().numpy(), st, it, rel))
    assert out[0][1] == out[1][1] == gb.GABP_OK
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("opts", [dict(precision=1), dict(precision=1, device_loop=0), dict(precision=0),
                                  dict(precision=0, schedule=1), dict(precision=1, gamma_mode=1)])
def test_initial_guess(gb, opts):
    """options.initial_guess: x holds x0 on entry, the path solves A d = b - A x0 and returns x0 + d.
    From the solution of a nearby right-hand side it needs fewer rounds than from zero and meets
    the same stop rule (checked on the host and against the oracle); an x0 that already meets the
    tolerance comes back unchanged after no round; b = 0 gives x = 0; host buffers work too."""
    import oracle

    m = synth.random_sym(20011, 8, 1.1, 2)
    b = synth.rhs(m.n, 5)
    b2 = b + 1e-4 * synth.rhs(m.n, 6)
    tb, tb2 = torch.from_numpy(b).cuda(), torch.from_numpy(b2).cuda()
    cold = gb.Solver.from_csr(m, **opts)
    x1, st, it1, _ = cold.solve(tb, tol=1e-10, max_iter=5000)
    xc, stc, itc, _ = cold.solve(tb2, tol=1e-10, max_iter=5000)
    cold.close()
    assert st == stc == gb.GABP_OK
    s = gb.Solver.from_csr(m, initial_guess=1, **opts)
    xg = x1.clone()
    xg, stg, itg, relg = s.solve(tb2, x=xg, tol=1e-10, max_iter=5000)
    assert stg == gb.GABP_OK and itg < itc and relg <= 1e-10
    xh = xg.cpu().numpy()
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    r = b2 - np.bincount(rows, m.val * xh[m.col], minlength=m.n)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b2) * (1 + 1e-6)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b2) - relg) <= 1e-3 * relg + 1e-16
    ref = oracle.gabp_broadcast(m, b2, max_iter=2000, tol=1e-13)
    assert np.linalg.norm(xh - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    keep = xg.clone()
    x3, st3, it3, rel3 = s.solve(tb2, x=keep.clone(), tol=1e-8, max_iter=5000)
    assert st3 == gb.GABP_OK and it3 == 0 and torch.equal(x3, keep)
    xz, stz, itz, _ = s.solve(torch.zeros_like(tb), x=keep.clone(), tol=1e-10)
    assert stz == gb.GABP_OK and not torch.any(xz)
    xhost = x1.cpu().numpy().copy()
    sth, ith, relh = s.solve_host(b2.copy(), xhost, tol=1e-10, max_iter=5000)
    # (a second FP32 solve on the handle reuses the frozen precision state: not bit-identical)
    assert sth == gb.GABP_OK and relh <= 1e-10
    assert np.linalg.norm(xhost - xh) <= 1e-8 * np.linalg.norm(xh)
    with pytest.raises(ValueError):
        s.solve(tb2)  # initial_guess needs x
    s.close()


@pytest.mark.parametrize("path", ["fp64_parallel", "fp64_serial", "fp32_parallel", "fp32_serial", "fix_single_loop"])
def test_graphs_off_same_results(gb, path):
    """options.graphs = 0 launches every kernel on its own (for per-kernel profilers) instead of
    replaying captured graphs: the same kernels in the same order, so bit-identical results."""
    m = synth.grid3d(16, 1.15, 3)
    b = torch.from_numpy(synth.rhs(m.n, 4)).cuda()
    out = []
    for graphs in (1, 0):
        s = gb.Solver.from_csr(m, lanes=4, graphs=graphs, **PATHS[path])
        x, st, it, rel = s.solve(b, tol=1e-10, max_iter=1000)
        s.close()
        out.append((x.cpu().numpy(), st, it, rel))
    assert out[0][1] == out[1][1] == gb.GABP_OK
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]
    assert np.array_equal(out[0][0], out[1][0])


def test_streams(gb):
    """A handle on a caller's stream and one on its own stream (created with the default stream)
    give bit-identical results; gabp_set_stream moves a handle to another stream and back to its
    own (NULL), and inputs written on the default stream just before a call are seen by it."""
    m = synth.random_sym(20011, 8, 1.1, 2)
    b = torch.from_numpy(synth.rhs(m.n, 5)).cuda()
    kw = dict(lanes=4, precision=gb.GABP_PREC_FP32_REFINE, reuse_precisions=0)  # every solve alike
    own = gb.Solver.from_csr(m, **kw)
    x0, st0, it0, rel0 = own.solve(b, tol=1e-10)
    user = torch.cuda.Stream()
    with torch.cuda.stream(user):
        s = gb.Solver.from_csr(m, stream=user, **kw)
        x1, st1, it1, rel1 = s.solve(b, tol=1e-10)
    user.synchronize()
    assert st0 == st1 == gb.GABP_OK and it0 == it1 and torch.equal(x0, x1)
    assert gb.gabp_set_stream(s.handle, 0) == gb.GABP_OK  # back to a stream of its own
    bb = torch.empty_like(b)
    bb.copy_(b)  # queued on the default stream right before the solve
    x2, st2, it2, rel2 = s.solve(bb, tol=1e-10)
    assert st2 == gb.GABP_OK and it2 == it0 and torch.equal(x2, x0)
    other = torch.cuda.Stream()
    assert gb.gabp_set_stream(s.handle, other.cuda_stream) == gb.GABP_OK
    with torch.cuda.stream(other):
        x3, st3, it3, rel3 = s.solve(b, tol=1e-10)
    other.synchronize()
    assert st3 == gb.GABP_OK and torch.equal(x3, x0)
    s.close()
    own.close()
