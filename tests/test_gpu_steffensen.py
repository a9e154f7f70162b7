"""Steffensen's iterations (Sec. "Convergence Acceleration") on the GPU, parallel and serial
schedules, against the oracle's Steffensen iterations through the C ABI: the iterates after a
fixed number of rounds (odd counts end a cycle's first round, even counts its extrapolation),
equal round counts at convergence, the fixed point, and the sweeps saved on the serial schedule."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCHED = {"parallel": 0, "serial": 1}


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_0811_2518_gb300 as m

    return m


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _solve(gb, m, b, tol, max_iter, schedule, accel=2, **kw):
    s = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP64, accel=accel, schedule=SCHED[schedule], **kw)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=max_iter, check=False)
    s.close()
    return x.cpu().numpy(), st, it, rel


CASES = {
    "grid32": lambda: (synth.grid2d(32, -1.0, 4.5), synth.rhs(1024, 1)),
    "random5000": lambda: (synth.random_sym(5000, 4, 1.1, 6), synth.rhs(5000, 6)),
    "grid3d_12": lambda: (synth.grid3d(12, 1.05, 3), synth.rhs(12 ** 3, 3)),
}


@pytest.mark.parametrize("schedule", ["parallel", "serial"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("rounds", [1, 2, 5, 8, 13])
def test_iterates_match_oracle(gb, schedule, case, rounds):
    m, b = CASES[case]()
    r = oracle.gabp_steffensen(m, b, schedule, max_iter=rounds, tol=0.0)
    x, st, it, _ = _solve(gb, m, b, 0.0, rounds, schedule)
    assert st == gb.GABP_NOT_CONVERGED and it == rounds
    assert np.max(np.abs(x - r["x"])) <= 1e-11 * np.max(np.abs(r["x"]))


@pytest.mark.parametrize("schedule", ["parallel", "serial"])
@pytest.mark.parametrize("case", list(CASES))
def test_converged_rounds_and_fixed_point(gb, schedule, case):
    m, b = CASES[case]()
    r = oracle.gabp_steffensen(m, b, schedule, max_iter=3000, tol=1e-12)
    x, st, it, rel = _solve(gb, m, b, 1e-12, 3000, schedule)
    assert st == gb.GABP_OK and r["status"] == oracle.OK and rel <= 1e-12
    assert abs(it - r["iters"]) <= 2
    assert _relerr(x, np.linalg.solve(oracle.to_dense(m), b)) <= 1e-10


def test_serial_saves_sweeps(gb):
    """On the 32 x 32 grid serial GaBP needs 59 sweeps to 1e-12, with Steffensen's iterations
    about 37 (the oracle's counts)."""
    m, b = CASES["grid32"]()
    _, st0, it0, _ = _solve(gb, m, b, 1e-12, 3000, "serial", accel=0)
    _, st1, it1, _ = _solve(gb, m, b, 1e-12, 3000, "serial")
    assert st0 == st1 == gb.GABP_OK
    assert it1 <= 0.7 * it0


def test_zero_rhs_and_graph_lengths(gb):
    """b = 0 gives x = 0; odd rounds per graph replay (the cycle pairing is kept on the device)
    give the same iterates as the default replay length."""
    m, b = CASES["random5000"]()
    for sched in ("parallel", "serial"):
        x, st, it, _ = _solve(gb, m, np.zeros(m.n), 1e-12, 100, sched)
        assert st == gb.GABP_OK and it == 0 and not np.any(x)
        xa, _, ita, _ = _solve(gb, m, b, 0.0, 11, sched, check_every=3)
        xb, _, itb, _ = _solve(gb, m, b, 0.0, 11, sched)
        assert ita == itb == 11 and np.array_equal(xa, xb)


def test_aitken_with_serial_rejected(gb):
    with pytest.raises(gb.GaBPError) as ei:
        gb.Solver.from_csr(synth.grid2d(4, -1.0, 4.5), accel=1, schedule=1)
    assert ei.value.status == gb.GABP_ERR_INVALID
