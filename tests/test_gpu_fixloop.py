"""Single-loop convergence fix on the GPU (one FP64 GaBP round on A + Gamma per outer step,
damped potential update) against the oracle's single loop, through the C ABI.

Same arithmetic form on both sides (aggregate minus reverse message, information form), so
the iterates agree to 1e-12 relative round for round; converged solutions are compared with
the dense solution."""
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


def _gpu(gb, m, b, tol, max_iter, gamma_mode=1, gamma=0.25, s=0.5):
    sv = gb.Solver.from_csr(m, gamma_mode=gamma_mode, gamma=gamma, fix_single_loop=1, fix_step=s)
    x, st, it, rel = sv.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=max_iter)
    sv.close()
    return x.cpu().numpy(), st, it, rel


@pytest.mark.parametrize("make,gamma", [(lambda: synth.random_sym(2000, 3, 1.2, 3), 0.25),
                                        (lambda: synth.random_sym(1024, 3, 0.8, 7), 0.3)])
@pytest.mark.parametrize("rounds", [1, 2, 9])
def test_rounds_match_oracle(gb, make, gamma, rounds):
    m = make()
    b = synth.rhs(m.n, 2)
    G = oracle.diagonal_loading(oracle.to_dense(m), "uniform", gamma)
    ref = oracle.convergence_fix_single_loop(m, b, G, s=0.5, tol=0.0, max_iter=rounds, history=True)
    x, st, it, rel = _gpu(gb, m, b, 0.0, rounds, gamma=gamma)
    assert it == rounds
    assert _relerr(x, ref["xs"][-1]) <= 1e-12


@pytest.mark.parametrize("s", [0.5, 0.25])
def test_converges_where_plain_fails(gb, s):
    """n = 1024, diagonal 0.8 x row abs-sum (SPD, not walk-summable): plain GaBP fails, the single
    loop with uniform loading reaches A^{-1} b; the round count equals the oracle's."""
    m = synth.random_sym(1024, 3, 0.8, 7)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 5)
    x, st, it, rel = _gpu(gb, m, b, 1e-10, 20000, gamma=0.3, s=s)
    assert st == gb.GABP_OK and rel <= 1e-10
    assert _relerr(x, np.linalg.solve(A, b)) <= 1e-8
    ref = oracle.convergence_fix_single_loop(m, b, oracle.diagonal_loading(A, "uniform", 0.3), s=s, tol=1e-10)
    assert abs(it - ref["iters"]) <= 1


def test_non_walk_summable_4096_and_dd_mode(gb):
    """The n = 4096, diagonal 0.9 x case of the benchmark's convergence-fix workload, uniform and
    diagonally-dominant loading."""
    m = synth.random_sym(4096, 3, 0.9, 5)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 5)
    x0 = np.linalg.solve(A, b)
    for mode, gamma in ((1, 0.25), (2, 0.05)):
        x, st, it, rel = _gpu(gb, m, b, 1e-11, 50000, gamma_mode=mode, gamma=gamma)
        assert st == gb.GABP_OK
        assert _relerr(x, x0) <= 1e-9


@pytest.mark.parametrize("mode,gamma,G", [(1, 0.25, [0.125, 0.375]), (2, 0.2, [0.5, 0.3])])
@pytest.mark.parametrize("s", [0.25, 0.8])
def test_two_node_tree_closed_form(gb, mode, gamma, G, s):
    """On a 2-node tree one GaBP round solves (A + Gamma) x = h exactly, so the single loop is the
    recurrence h^(1) = b, x^(t) = (A + Gamma)^{-1} h^(t), h^(t+1) = (1 - s) h^(t) + s (b + Gamma x^(t)).
    Gamma is worked out by hand for A = [[0.5, -0.9], [-0.9, 1.5]]: uniform gamma 0.25 -> (0.125,
    0.375); diagonally dominant loading max(0, sum_j |A_ij| - A_ii) + 0.2 A_ii -> (0.4 + 0.1, 0 + 0.3).
    The GPU's iterate after t rounds must follow the recurrence."""
    A = np.array([[0.5, -0.9], [-0.9, 1.5]])
    b = np.array([1.0, -0.5])
    J = A + np.diag(G)
    m = synth.from_dense(A)
    h = b.copy()
    for t in range(1, 9):
        xt = np.linalg.solve(J, h)
        x, st, it, rel = _gpu(gb, m, b, 0.0, t, gamma_mode=mode, gamma=gamma, s=s)
        assert it == t
        assert np.allclose(x, xt, rtol=1e-13, atol=1e-15)
        h = (1.0 - s) * h + s * (b + np.asarray(G) * xt)
