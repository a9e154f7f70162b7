"""Pins of the FP64 oracle to facts the paper and the mathematics fix (CPU only).

Each test names the passage it checks.  None of them compares the oracle with
itself through a retyped formula: the references are printed values, dense
linear algebra, closed forms and theorems.
"""
import math
from collections import deque

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def _slot(m, i, k):
    lo, hi = m.rowptr[i], m.rowptr[i + 1]
    hits = np.nonzero(m.col[lo:hi] == k)[0]
    assert hits.size == 1
    return lo + hits[0]


# ----------------------------------------------------------------------------- worked example
@pytest.mark.parametrize("variant", ["naive", "broadcast"])
def test_toy_tables_exact(variant):
    """Sec. "Toy Linear System": every message and tentative mean of the printed
    tables at t = 0..3 (parallel schedule), and the marginal precisions."""
    g = read_golden("toy3x3_tables.txt")
    A, b = synth.toy3x3()
    m = synth.from_dense(A)
    run = oracle.gabp_naive if variant == "naive" else oracle.gabp_broadcast
    names = {"x": 0, "y": 1, "z": 2}
    for t in range(0, 4):
        r = run(m, b, max_iter=t, tol=0.0, messages=True)
        for key, vals in g.items():
            if key.startswith("P_") or key.startswith("mu_"):
                kind, pair = key.split("_")
                snd, rcv = names[pair[0]], names[pair[1]]
                p = _slot(m, rcv, snd)  # message snd -> rcv lives in row rcv
                got = r["Pmsg"][p] if kind == "P" else r["mumsg"][p]
                assert abs(got - vals[t]) <= 1e-15, (key, t, got, vals[t])
            elif key.startswith("mean_"):
                assert abs(r["x"][names[key[-1]]] - vals[t]) <= 1e-15, (key, t)
    r = run(m, b, max_iter=3, tol=0.0)
    for key in ("Pm_x", "Pm_y", "Pm_z"):
        assert abs(r["P"][names[key[-1]]] - g[key][0]) <= 1e-15
    # and both agree with the dense inverse: x* = (1, 2, -1), P_i = 1/(A^-1)_ii
    assert np.allclose(r["x"], oracle.dense_solve(A, b), rtol=0, atol=1e-15)
    assert np.allclose(r["P"], oracle.marginal_precisions_exact(A), rtol=1e-14)


def test_toy_converges_in_diameter_rounds():
    """Sec. "Toy Linear System": on the 3-node tree GaBP converges in two rounds,
    the tree's diameter; the residual stop rule fires at t = 2."""
    A, b = synth.toy3x3()
    r = oracle.gabp_naive(synth.from_dense(A), b, max_iter=10, tol=1e-15)
    assert r["status"] == oracle.OK and r["iters"] == 2


# ----------------------------------------------------------------------------- trees
def _diameter(m):
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
    d0 = bfs(0)
    return int(bfs(int(np.argmax(d0))).max())


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("variant", ["naive", "broadcast"])
def test_tree_exact_after_diameter_rounds(seed, variant):
    """Sec. "Convergence and Exactness" and the Gaussian-elimination proposition:
    on a tree GaBP is exact -- means A^{-1} b and precisions 1/(A^{-1})_ii -- and
    its messages stop changing once information has crossed the tree."""
    m = synth.random_tree(31, seed, dd=(seed % 2 == 0), diag_scale=2.0)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 100 + seed)
    diam = _diameter(m)
    run = oracle.gabp_naive if variant == "naive" else oracle.gabp_broadcast
    r = run(m, b, max_iter=diam, tol=0.0, messages=True)
    xs = oracle.dense_solve(A, b)
    assert np.linalg.norm(r["x"] - xs) <= 1e-12 * np.linalg.norm(xs)
    assert np.allclose(r["P"], oracle.marginal_precisions_exact(A), rtol=1e-11, atol=0)
    r2 = run(m, b, max_iter=diam + 1, tol=0.0, messages=True)
    if variant == "naive":
        # the explicit sum over N(i)\j sees only converged inputs: bit-for-bit stationary
        assert np.array_equal(r2["Pmsg"], r["Pmsg"]) and np.array_equal(r2["mumsg"], r["mumsg"])
    else:
        # the broadcast form subtracts the reverse message from the full aggregate;
        # the cancellation rounds differently once that message has settled
        assert np.allclose(r2["Pmsg"], r["Pmsg"], rtol=1e-12, atol=1e-15)
        assert np.allclose(r2["mumsg"], r["mumsg"], rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------------------------- fixed point
@pytest.mark.parametrize("variant", ["naive", "broadcast"])
def test_fixed_point_diagonally_dominant_grid(variant):
    """Diagonal-dominance theorem (Sec. "Convergence and Exactness"): the means
    converge to A^{-1} b.  32 x 32 5-point grid, diagonal 4.5."""
    m = synth.grid2d(32, -1.0, 4.5)
    b = synth.rhs(m.n, 1)
    run = oracle.gabp_naive if variant == "naive" else oracle.gabp_broadcast
    r = run(m, b, max_iter=2000, tol=1e-13)
    assert r["status"] == oracle.OK
    xs = oracle.dense_solve(oracle.to_dense(m), b)
    assert np.linalg.norm(r["x"] - xs) <= 1e-12 * np.linalg.norm(xs)


def test_fixed_point_walk_summable_random():
    """Spectral-radius theorem: rho(|R|) < 1 gives convergence to A^{-1} b."""
    m = synth.random_sym(400, 4, 1.1, 7)
    A = oracle.to_dense(m)
    assert oracle.rho_abs_normalized(A) < 1
    b = synth.rhs(m.n, 7)
    r = oracle.gabp_broadcast(m, b, max_iter=2000, tol=1e-13)
    assert r["status"] == oracle.OK
    xs = oracle.dense_solve(A, b)
    assert np.linalg.norm(r["x"] - xs) <= 1e-12 * np.linalg.norm(xs)


def test_run_gabp_appendix_example():
    """Appendix example (A with couplings 0.3 / 0.1, b = 1): the solution equals inv(A) b."""
    A, b = synth.run_gabp_3x3()
    r = oracle.gabp_naive(synth.from_dense(A), b, max_iter=100, tol=1e-14)
    assert r["status"] == oracle.OK
    assert np.allclose(r["x"], np.linalg.inv(A) @ b, rtol=1e-13)


def test_broadcast_equals_naive():
    """Sec. "GaBP Broadcast Variant": subtracting the reverse message from the full
    aggregate gives the same messages as the explicit sum over N(i)\\j."""
    m = synth.random_sym(300, 4, 1.1, 3)
    b = synth.rhs(m.n, 3)
    for t in (1, 2, 7, 25):
        a = oracle.gabp_naive(m, b, max_iter=t, tol=0.0, messages=True)
        c = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0, messages=True)
        assert np.allclose(a["Pmsg"], c["Pmsg"], rtol=1e-12, atol=1e-15)
        hm_a, hm_c = a["Pmsg"] * a["mumsg"], c["Pmsg"] * c["mumsg"]
        assert np.allclose(hm_a, hm_c, rtol=1e-11, atol=1e-13)
        assert np.allclose(a["x"], c["x"], rtol=1e-12, atol=1e-14)


def test_info_form_messages_match_paper_mean_form():
    """eq_mean_message: P_ij mu_ij = -A_ij mu_{i\\j}; at the fixed point of a tree the
    information-form mean message therefore equals -A_ij times the cavity mean,
    which on a tree is the exact conditional mean with x_j removed."""
    A, b = synth.toy3x3()
    m = synth.from_dense(A)
    r = oracle.gabp_naive(m, b, max_iter=3, tol=0.0, messages=True)
    # message x -> y: cavity of x without y is (P_xx, mu_xx) combined with z -> x
    p = _slot(m, 1, 0)
    Pcav = 1.0 + r["Pmsg"][_slot(m, 0, 2)]
    hcav = -6.0 + r["Pmsg"][_slot(m, 0, 2)] * r["mumsg"][_slot(m, 0, 2)]
    assert abs(r["Pmsg"][p] * r["mumsg"][p] - (-A[0, 1] * hcav / Pcav)) <= 1e-14


# ----------------------------------------------------------------------------- walk-summability
def test_rho_cdma_printed_values():
    """Sec. "Linear Detection": rho(|I - R3|) = 0.9008, rho(|I - R4|) = 0.8747 (printed to 4 decimals)."""
    g = read_golden("cdma_rho.txt")
    for key, make in (("R3", synth.cdma_r3), ("R4", synth.cdma_r4)):
        A, _ = make()
        assert abs(oracle.rho_abs_normalized(A) - g[key][0]) <= 5e-5


@pytest.mark.parametrize("c", [1.05, 1.1, 1.2, 0.9])
def test_rho_closed_form_row_sum_diagonal(c):
    """For A_ii = c * sum_j |A_ij|, D^{-1}|A_off| has constant row sums 1/c and is
    similar to |R|, so rho(|R|) = 1/c exactly (Perron-Frobenius)."""
    m = synth.random_sym(300, 3, c, 11)
    assert abs(oracle.rho_abs_normalized(oracle.to_dense(m)) - 1.0 / c) <= 1e-12


def test_rho_closed_form_grid():
    """32 x 32 grid, diagonal 4.5: |R| = (path Laplacian adjacency)/4.5, whose
    largest eigenvalue is 4 cos(pi / 33) / 4.5."""
    m = synth.grid2d(32, -1.0, 4.5)
    want = 4.0 * math.cos(math.pi / 33) / 4.5
    assert abs(oracle.rho_abs_normalized(oracle.to_dense(m)) - want) <= 1e-12


# ----------------------------------------------------------------------------- rate bound
def test_rate_bound_diagonally_dominant():
    """Sec. "Upper Bound on Convergence Rate": after ceil(log eps / log gamma)
    rounds, |x* - x_t| < eps ||b||_inf."""
    m = synth.grid2d(12, -1.0, 4.5)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 4)
    eps = 1e-8
    t = oracle.rate_bound_rounds(A, eps)
    # interior node: eps_i = 0.5, |N(i)| = 4, gamma = 1 / (1 + 0.5 / 4)
    assert t == math.ceil(math.log(eps) / math.log(1.0 / (1.0 + 0.5 / 4)))
    r = oracle.gabp_naive(m, b, max_iter=t, tol=0.0)
    xs = oracle.dense_solve(A, b)
    assert np.max(np.abs(xs - r["x"])) < eps * np.max(np.abs(b))


# ----------------------------------------------------------------------------- iteration counts (soft)
def _soft(got, paper):
    return 0.7 * paper <= got <= 1.3 * paper


def test_soft_counts_nonpsd():
    """Table tab_nonPSD: parallel GaBP converges on the symmetric non-PSD 3x3 (paper: 38 rounds)."""
    g = read_golden("iteration_counts.txt")
    A, b = synth.nonpsd3x3()
    r = oracle.gabp_naive(synth.from_dense(A), b, max_iter=1000, tol=1e-6, stop_rule="message")
    assert r["status"] == oracle.OK and _soft(r["iters"], g["nonpsd3x3"][0])
    assert np.allclose(r["x"], np.linalg.solve(A, b), atol=1e-4)


def test_soft_counts_poisson():
    """Table tab_2D_Poisson: 2-D Poisson, p = 10, f = -1, b = -f h^2 (paper: 134 rounds)."""
    g = read_golden("iteration_counts.txt")
    p = 10
    m = synth.poisson2d(p)
    b = np.full(m.n, (1.0 / (p + 1)) ** 2)
    r = oracle.gabp_naive(m, b, max_iter=1000, tol=1e-6, stop_rule="message")
    assert r["status"] == oracle.OK and _soft(r["iters"], g["poisson10"][0])


@pytest.mark.parametrize("name", ["cdma_r3", "cdma_r4"])
def test_soft_counts_cdma(name):
    """Table tab_1: parallel GaBP on the CDMA correlation matrices (paper: 23 / 24)."""
    g = read_golden("iteration_counts.txt")
    A, b = getattr(synth, name)()
    r = oracle.gabp_naive(synth.from_dense(A), b, max_iter=1000, tol=1e-6, stop_rule="message")
    assert r["status"] == oracle.OK and _soft(r["iters"], g[name][0])
    assert np.allclose(r["x"], np.linalg.solve(A, b), atol=1e-4)


# ----------------------------------------------------------------------------- failure modes
def test_breakdown_zero_cavity():
    """A cavity precision that is exactly zero stops the run (the paper's listing
    asserts P_{i\\j} != 0).  Star y with leaves x, z, w: in round 2
    P_{y\\x} = A_yy - A_yz^2 / A_zz - A_yw^2 / A_ww = 3 - 1 - 2 = 0 exactly, while
    every marginal precision of round 1 is nonzero."""
    A = np.array([[2.0, 1.0, 0.0, 0.0], [1.0, 3.0, 1.0, 1.0], [0.0, 1.0, 1.0, 0.0], [0.0, 1.0, 0.0, 0.5]])
    for run in (oracle.gabp_naive, oracle.gabp_broadcast):
        r = run(synth.from_dense(A), np.ones(4), max_iter=10, tol=1e-14)
        assert r["status"] == oracle.BREAKDOWN and r["iters"] == 2


def test_invalid_inputs():
    A, b = synth.toy3x3()
    bad = A.copy()
    bad[0, 1] = 5.0  # asymmetric value
    assert oracle.gabp_naive(synth.from_dense(bad), b)["status"] == oracle.INVALID
    bad = A.copy()
    bad[1, 1] = 0.0  # zero diagonal
    assert oracle.gabp_naive(synth.from_dense(bad), b)["status"] == oracle.INVALID


def test_zero_rhs():
    m = synth.grid2d(4)
    r = oracle.gabp_naive(m, np.zeros(m.n))
    assert r["status"] == oracle.OK and r["iters"] == 0 and not np.any(r["x"])


# ----------------------------------------------------------------------------- convergence fix
def _H_radius(A, G):
    import scipy.linalg as sl
    return float(np.max(sl.eigh(np.diag(G), A + np.diag(G), eigvals_only=True)))


@pytest.mark.parametrize("gamma", [0.25, 0.5])
def test_convergence_fix_non_walk_summable(gamma):
    """Chapter "Fixing convergence of GaBP": J + Gamma is walk-summable for
    gamma > rho(|R|) - 1, the double loop converges to J^{-1} h, and its error
    contracts by rho((J + Gamma)^{-1} Gamma) < 1 per outer step (the lemma's proof).
    A: n = 1024, 3 picks per row, diagonal 0.9 x row abs-sum (rho(|R|) = 1/0.9), SPD."""
    m = synth.random_sym(1024, 3, 0.9, 5)
    A = oracle.to_dense(m)
    np.linalg.cholesky(A)
    assert oracle.rho_abs_normalized(A) > 1.0
    G = oracle.diagonal_loading(A, "uniform", gamma)
    assert oracle.rho_abs_normalized(A + np.diag(G)) < 1.0
    b = synth.rhs(m.n, 5)
    f = oracle.convergence_fix(m, b, G, tol=1e-10, inner_tol=1e-13)
    assert f["status"] == oracle.OK
    xs = oracle.dense_solve(A, b)
    assert np.linalg.norm(f["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
    h = f["history"]
    ratio = float(np.median([h[i + 1] / h[i] for i in range(len(h) // 2, len(h) - 1)]))
    rho_h = _H_radius(A, G)
    assert rho_h < 1.0
    assert abs(ratio - rho_h) <= 0.1 * rho_h


def test_convergence_fix_where_plain_gabp_fails():
    """An SPD matrix on which plain GaBP does not converge (diagonal 0.8 x row abs-sum):
    the double loop still reaches A^{-1} b."""
    m = synth.random_sym(1024, 3, 0.8, 7)
    A = oracle.to_dense(m)
    np.linalg.cholesky(A)
    b = synth.rhs(m.n, 5)
    plain = oracle.gabp_broadcast(m, b, max_iter=300, tol=1e-10)
    assert plain["status"] != oracle.OK
    G = oracle.diagonal_loading(A, "uniform", 0.3)
    f = oracle.convergence_fix(m, b, G, tol=1e-8, inner_tol=1e-11, max_outer=3000)
    assert f["status"] == oracle.OK
    xs = oracle.dense_solve(A, b)
    assert np.linalg.norm(f["x"] - xs) <= 1e-6 * np.linalg.norm(xs)


# ----------------------------------------------------------------------------- gradient reference
def test_dense_gradient_against_finite_differences():
    """dL/db and the symmetrised dL/dA of L = 0.5 ||A^{-1} b - x*||^2 against central
    differences (b_i; the pair A_ij = A_ji moved together; A_ii)."""
    m = synth.random_sym(30, 3, 1.2, 9)
    A = oracle.to_dense(m)
    b = synth.rhs(30, 9)
    xstar = synth.rhs(30, 10)
    x, gb, G = oracle.dense_gradient(A, b, xstar)

    def loss(A_, b_):
        y = np.linalg.solve(A_, b_)
        return 0.5 * np.sum((y - xstar) ** 2)

    h = 1e-6
    for i in (0, 7, 29):
        e = np.zeros(30)
        e[i] = h
        fd = (loss(A, b + e) - loss(A, b - e)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-7 * max(1.0, abs(fd))
    rows, cols = np.nonzero(np.triu(A, 1))
    for i, j in list(zip(rows, cols))[:6]:
        E = np.zeros_like(A)
        E[i, j] = E[j, i] = h
        fd = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
        assert abs(fd - (G[i, j] + G[j, i])) <= 1e-7 * max(1.0, abs(fd))
    for i in (3, 11):
        E = np.zeros_like(A)
        E[i, i] = h
        fd = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
        assert abs(fd - G[i, i]) <= 1e-7 * max(1.0, abs(fd))


# ----------------------------------------------------------------------------- serial schedule
def test_colour_greedy_facts():
    """The colouring of the serial sweeps: proper; on a grid in index order the red-black
    pattern (x + y) mod 2; on a path alternating; on a complete graph one colour per node in
    index order; never more than max degree + 1 colours."""
    m = synth.grid2d(7, -1.0, 4.5)
    colour, nc = oracle.colour_greedy(m)
    xy = np.arange(m.n)
    assert nc == 2 and np.array_equal(colour, (xy // 7 + xy % 7) % 2)
    n = 6
    A = 4.0 * np.eye(n)
    for i in range(n - 1):
        A[i, i + 1] = A[i + 1, i] = -1.0
    colour, nc = oracle.colour_greedy(synth.from_dense(A))
    assert nc == 2 and np.array_equal(colour, np.arange(n) % 2)
    K = np.full((5, 5), 0.1) + 5.0 * np.eye(5)
    colour, nc = oracle.colour_greedy(synth.from_dense(K))
    assert nc == 5 and np.array_equal(colour, np.arange(5))
    for seed in (1, 2, 3):
        m = synth.random_sym(300, 4, 1.1, seed)
        colour, nc = oracle.colour_greedy(m)
        rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
        off = rows != m.col
        assert not np.any(colour[rows[off]] == colour[m.col[off]])  # proper
        assert nc == colour.max() + 1 <= np.diff(m.rowptr).max()  # <= (max degree + 1), diagonal stored


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_serial_tree_exact(seed):
    """On a tree the serial schedule is exact too (Sec. "Convergence and Exactness"): after at
    most diameter sweeps x = A^{-1} b and P_i = 1 / (A^{-1})_ii."""
    m = synth.random_tree(40, seed)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, seed)
    r = oracle.gabp_serial(m, b, max_iter=40, tol=0.0)
    assert np.allclose(r["x"], np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    assert np.allclose(r["P"], oracle.marginal_precisions_exact(A), rtol=1e-10)


@pytest.mark.parametrize("make", [lambda: synth.grid2d(20, -1.0, 4.5), lambda: synth.random_sym(500, 4, 1.1, 3)])
def test_serial_fixed_point_and_fewer_sweeps(make):
    """The serial schedule converges to A^{-1} b on diagonally dominant A, in fewer sweeps than
    the parallel schedule needs rounds (the paper's observation in every table)."""
    m = make()
    b = synth.rhs(m.n, 4)
    x0 = np.linalg.solve(oracle.to_dense(m), b)
    s = oracle.gabp_serial(m, b, max_iter=2000, tol=1e-12)
    p = oracle.gabp_naive(m, b, max_iter=2000, tol=1e-12)
    assert s["status"] == oracle.OK and np.allclose(s["x"], x0, rtol=1e-9, atol=1e-12)
    assert s["iters"] < p["iters"]


def test_serial_soft_counts():
    """Tables tab_nonPSD and tab_2D_Poisson, serial GaBP (paper: 25 and 73 iterations)."""
    g = read_golden("iteration_counts.txt")
    A, b = synth.nonpsd3x3()
    r = oracle.gabp_serial(synth.from_dense(A), b, max_iter=1000, tol=1e-6, stop_rule="message")
    assert r["status"] == oracle.OK and _soft(r["iters"], g["nonpsd3x3_serial"][0])
    p = 10
    m = synth.poisson2d(p)
    r = oracle.gabp_serial(m, np.full(m.n, (1.0 / (p + 1)) ** 2), max_iter=1000, tol=1e-6, stop_rule="message")
    assert r["status"] == oracle.OK and _soft(r["iters"], g["poisson10_serial"][0])


def test_serial_matches_sequential_broadcast_form():
    """A second, independent form of the serial schedule: nodes fire one at a time in colour
    order, each forming its aggregate over ALL of N(i) and subtracting the reverse message
    (the broadcast form of Algorithm 2, in the information form), messages in a dict.  After
    4 sweeps every message agrees with the C oracle's cavity-sum form."""
    m = synth.random_sym(30, 3, 1.2, 8)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 8)
    colour, nc = oracle.colour_greedy(m)
    nbr = [np.flatnonzero((A[i] != 0) & (np.arange(m.n) != i)) for i in range(m.n)]
    P, h = {}, {}  # (k, i): message k -> i
    for i in range(m.n):
        for k in nbr[i]:
            P[(k, i)] = h[(k, i)] = 0.0
    order = [i for c in range(nc) for i in range(m.n) if colour[i] == c]
    for _ in range(4):
        for i in order:
            Pt = A[i, i] + sum(P[(k, i)] for k in nbr[i])
            ht = b[i] + sum(h[(k, i)] for k in nbr[i])
            for j in nbr[i]:
                Pc, hc = Pt - P[(j, i)], ht - h[(j, i)]
                P[(i, j)] = -A[i, j] ** 2 / Pc
                h[(i, j)] = -A[i, j] * hc / Pc
    r = oracle.gabp_serial(m, b, max_iter=4, tol=0.0, messages=True)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    for p in range(m.nnz):
        i, k = rows[p], m.col[p]
        if i == k:
            continue
        assert abs(r["Pmsg"][p] - P[(k, i)]) <= 1e-13 * abs(P[(k, i)])
        hm = r["Pmsg"][p] * r["mumsg"][p]  # information form h = P mu
        assert abs(hm - h[(k, i)]) <= 1e-12 * (abs(h[(k, i)]) + 1e-12)


# ----------------------------------------------------------------------------- single-loop convergence fix
def test_single_loop_reduces_to_plain_gabp():
    """With Gamma = 0 and s = 1 the potentials never move (h^(t) = b): the single loop is plain
    GaBP, round for round equal to the C oracle's Algorithm 2."""
    m = synth.random_sym(300, 4, 1.1, 4)
    b = synth.rhs(m.n, 4)
    sl = oracle.convergence_fix_single_loop(m, b, np.zeros(m.n), s=1.0, tol=0.0, max_iter=6, history=True)
    for t in (1, 3, 6):
        r = oracle.gabp_broadcast(m, b, max_iter=t, tol=0.0)
        assert np.allclose(sl["xs"][t - 1], r["x"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("s", [0.5, 0.25])
def test_single_loop_converges_where_plain_fails(s):
    """The non-walk-summable SPD case on which plain GaBP fails (n = 1024, diagonal 0.8 x row
    abs-sum): the single loop with uniform loading reaches A^{-1} b."""
    m = synth.random_sym(1024, 3, 0.8, 7)
    A = oracle.to_dense(m)
    b = synth.rhs(m.n, 5)
    assert oracle.gabp_broadcast(m, b, max_iter=300, tol=1e-10)["status"] != oracle.OK
    g = oracle.convergence_fix_single_loop(m, b, oracle.diagonal_loading(A, "uniform", 0.3), s=s, tol=1e-10)
    assert g["status"] == oracle.OK
    assert np.linalg.norm(g["x"] - np.linalg.solve(A, b)) <= 1e-8 * np.linalg.norm(np.linalg.solve(A, b))


# ----------------------------------------------------------------------------- Aitken acceleration
def test_aitken_exact_on_geometric_sequences():
    """Aitken's method is exact on x_n = L + C a^n (any |a| != 1, per component)."""
    L = np.array([1.5, -2.0, 0.25, 3.0])
    C = np.array([0.7, -1.3, 2.0, 0.01])
    q = np.array([0.9, -0.6, 0.3, 0.99])
    x = [L + C * q ** k for k in range(3)]
    assert np.allclose(oracle.aitken(*x), L, rtol=1e-12, atol=1e-12)
    assert np.array_equal(oracle.aitken(L, L, L), L)  # zero second difference: the last iterate


def test_aitken_poisson_table():
    """Table tab_2D_Poisson: on the 2-D Poisson system (p = 10, f = -1) Aitken's method reaches
    max-error 1e-6 in ~25 rounds where plain parallel GaBP needs ~134 (both printed in the paper)."""
    g = read_golden("iteration_counts.txt")
    p = 10
    m = synth.poisson2d(p)
    b = np.full(m.n, (1.0 / (p + 1)) ** 2)
    xs = np.linalg.solve(oracle.to_dense(m), b)
    r = oracle.gabp_aitken(m, b, max_iter=300, tol=0.0, history=True)
    first = lambda seq: next(t + 1 for t, v in enumerate(seq) if np.max(np.abs(v - xs)) < 1e-6)
    assert _soft(first(r["ys"]), g["poisson10_aitken"][0])
    assert _soft(first(r["xs"]), g["poisson10"][0])
    # the unaccelerated iterates are the C oracle's Algorithm 2 rounds
    assert np.allclose(r["xs"][9], oracle.gabp_broadcast(m, b, max_iter=10, tol=0.0)["x"], rtol=1e-12)


def test_aitken_converges_to_solution():
    m = synth.grid2d(16, -1.0, 4.5)
    b = synth.rhs(m.n, 3)
    r = oracle.gabp_aitken(m, b, max_iter=500, tol=1e-12)
    assert r["status"] == oracle.OK
    assert np.allclose(r["x"], np.linalg.solve(oracle.to_dense(m), b), rtol=1e-9, atol=1e-11)


# ----------------------------------------------------------------------------- single loop: closed forms
@pytest.mark.parametrize("s", [0.25, 0.5, 0.8])
def test_single_loop_error_ratio_without_edges(s):
    """Chapter "Fixing convergence of GaBP", single loop, on a diagonal A (no edges: one GaBP round
    is the exact solve x = h / (A_ii + Gamma_ii)).  With x* = b / A_ii the damped update
    h <- (1 - s) h + s (b + Gamma x) gives, per node, e^(t+1) = (1 - s A_ii / (A_ii + Gamma_ii)) e^(t)
    (derived by hand from the update; e^(1) = -b Gamma / (A (A + Gamma)) since h^(1) = b).  Swapping
    s and 1 - s, or using x one round late, changes these ratios."""
    n = 5
    a = np.array([1.0, 2.5, 0.75, 4.0, 1.6])
    G = np.array([0.5, 1.0, 0.25, 3.0, 0.1])
    b = np.array([1.0, -2.0, 0.5, 3.0, -1.25])
    m = synth.from_dense(np.diag(a))
    r = oracle.convergence_fix_single_loop(m, b, G, s=s, tol=0.0, max_iter=8, history=True)
    xs = b / a
    e = [x - xs for x in r["xs"]]
    assert np.allclose(e[0], -b * G / (a * (a + G)), rtol=1e-14, atol=0)
    q = 1.0 - s * a / (a + G)
    for t in range(1, 8):
        assert np.allclose(e[t] / e[t - 1], q, rtol=1e-9, atol=0)


@pytest.mark.parametrize("s", [0.25, 0.8])
def test_single_loop_two_node_tree_closed_form(s):
    """Single loop on a 2-node tree: GaBP is exact after one round on it (diameter 1; each cavity is
    the node's own potential, so round t's messages depend only on the potentials h^(t)), hence
    x^(t) = (A + Gamma)^{-1} h^(t), and the chapter's update gives the linear recurrence
    h^(1) = b, h^(t+1) = (1 - s) h^(t) + s (b + Gamma x^(t)).  The oracle's iterates must follow it
    (dense 2x2 solves), round by round."""
    A = np.array([[2.0, -0.9], [-0.9, 1.5]])
    G = np.array([0.6, 0.3])
    b = np.array([1.0, -0.5])
    r = oracle.convergence_fix_single_loop(synth.from_dense(A), b, G, s=s, tol=0.0, max_iter=10, history=True)
    J = A + np.diag(G)
    h = b.copy()
    for t in range(10):
        x = np.linalg.solve(J, h)
        assert np.allclose(r["xs"][t], x, rtol=1e-13, atol=1e-15)
        h = (1.0 - s) * h + s * (b + G * x)


def test_diagonal_loading_dd_hand_values():
    """Diagonal loading that makes A + Gamma diagonally dominant (the chapter's DD-making loading):
    Gamma_ii = max(0, sum_{j != i} |A_ij| - A_ii) + delta A_ii.  Values worked out by hand on a 3x3:
    off-diagonal abs-sums (4, 1.5, 3.5), diagonal (2, 4, 1), delta 0.1 -> (2.2, 0.4, 2.6); every row
    of A + Gamma then exceeds its off-diagonal abs-sum by at least delta A_ii."""
    A = np.array([[2.0, -1.0, 3.0], [-1.0, 4.0, 0.5], [3.0, 0.5, 1.0]])
    G = oracle.diagonal_loading(A, "dd", delta=0.1)
    assert np.allclose(G, [2.2, 0.4, 2.6], rtol=1e-15, atol=1e-15)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) + G - off >= 0.1 * np.diag(A) - 1e-15)
    assert np.allclose(oracle.diagonal_loading(A, "uniform", 0.25), [0.5, 1.0, 0.25], rtol=1e-15)


# ----------------------------------------------------------------------------- Steffensen's iterations
def test_steffensen_step_exact_on_vector_geometric_sequences():
    """x_n = x* + c q^n with one scalar ratio q: the scalar-step extrapolation returns x* (both
    for contracting and for oscillating sequences); nothing moving gives the last iterate."""
    xs_ = np.array([1.5, -2.0, 0.25, 3.0])
    c = np.array([0.7, -1.3, 2.0, 0.01])
    for q in (0.9, -0.6, 0.3):
        y, lam = oracle.steffensen_step(*(xs_ + c * q ** k for k in range(3)))
        assert np.allclose(y, xs_, rtol=1e-12, atol=1e-12)
        assert lam == pytest.approx(q / (q - 1.0), rel=1e-12)
    y, lam = oracle.steffensen_step(xs_, xs_, xs_)
    assert lam == 0.0 and np.array_equal(y, xs_)


def test_jacobi_steffensen_cdma_table():
    """Table tab_2 prints Jacobi + Steffensen on CDMA R3: 59 iterations to 1e-6.  Jacobi's state is
    its iterate, so the only modelling choice is the extrapolation formula: two Jacobi steps, then
    the extrapolated vector replaces the iterate.  The scalar step reproduces the count within the
    soft band; component-wise extrapolation (130-140) or anchoring at x_n (112-118) do not."""
    g = read_golden("iteration_counts.txt")
    A, b = synth.cdma_r3()
    xs_ = np.linalg.solve(A, b)
    d = np.diag(A)
    R = A - np.diag(d)
    x, t = np.zeros(3), 0
    while t < 1000:
        x1 = (b - R @ x) / d
        x2 = (b - R @ x1) / d
        t += 2
        x, _ = oracle.steffensen_step(x, x1, x2)
        if np.max(np.abs(x - xs_)) < 1e-6:
            break
    assert _soft(t, g["cdma_r3_jacobi_steffensen"][0])


@pytest.mark.parametrize("schedule", ["parallel", "serial"])
def test_steffensen_first_round_is_plain_gabp(schedule):
    """Before the first extrapolation the iteration is plain GaBP: round 1 equals the C oracle's
    Algorithm 2 round (parallel) or serial sweep."""
    m = synth.random_sym(500, 4, 1.1, 6)
    b = synth.rhs(m.n, 6)
    r = oracle.gabp_steffensen(m, b, schedule, max_iter=1, tol=0.0, history=True)
    ref = (oracle.gabp_broadcast if schedule == "parallel" else oracle.gabp_serial)(m, b, max_iter=1, tol=0.0)
    assert np.allclose(r["xs"][0], ref["x"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("schedule", ["parallel", "serial"])
def test_steffensen_messages_realise_the_extrapolated_means(schedule):
    """Once the precisions are stationary, moving the mean messages by the cycle's scalar step
    gives a state whose marginal means are exactly the extrapolated vector y = x2 - lam (x2 - x1)
    (x is affine in the mean messages).  Checked on the 32 x 32 grid after the precisions have
    settled (t > 60)."""
    m = synth.grid2d(32, -1.0, 4.5)
    b = synth.rhs(m.n, 1)
    r = oracle.gabp_steffensen(m, b, schedule, max_iter=100, tol=0.0, history=True)
    xs = r["xs"]
    for k in range(35, 50):  # cycle k ends at round 2k + 2 (index 2k + 1)
        x0, x1, x2 = xs[2 * k - 1], xs[2 * k], r["pre"][k]
        y, lam = oracle.steffensen_step(x0, x1, x2)
        assert lam == pytest.approx(r["lams"][k], rel=1e-12, abs=1e-300)
        assert np.allclose(xs[2 * k + 1], y, rtol=1e-11, atol=1e-13 * np.max(np.abs(y)))


@pytest.mark.parametrize("schedule", ["parallel", "serial"])
def test_steffensen_converges_to_solution(schedule):
    """The fixed point is unchanged (the region of convergence is the plain method's, as the
    section remarks): A^{-1} b on diagonally dominant systems."""
    for m, seed in ((synth.grid2d(16, -1.0, 4.5), 3), (synth.random_sym(800, 5, 1.1, 8), 8)):
        b = synth.rhs(m.n, seed)
        r = oracle.gabp_steffensen(m, b, schedule, max_iter=2000, tol=1e-12)
        assert r["status"] == oracle.OK
        assert np.allclose(r["x"], np.linalg.solve(oracle.to_dense(m), b), rtol=1e-9, atol=1e-11)


def test_steffensen_serial_saves_sweeps():
    """The section's claim that the iterations converge faster: serial GaBP with Steffensen's
    iterations needs far fewer sweeps than plain serial GaBP on the 32 x 32 grid (measured 37 vs
    59) and on the paper's Poisson system with its smooth right-hand side (52-ish vs 167 to
    1e-12)."""
    for m, b in ((synth.grid2d(32, -1.0, 4.5), synth.rhs(1024, 1)),
                 (synth.poisson2d(10), np.full(100, (1.0 / 11) ** 2))):
        plain = oracle.gabp_serial(m, b, max_iter=2000, tol=1e-12)
        st = oracle.gabp_steffensen(m, b, "serial", max_iter=2000, tol=1e-12)
        assert plain["status"] == st["status"] == oracle.OK
        assert st["iters"] <= 0.7 * plain["iters"]


# ----------------------------------------------------------------------------- least squares (augmented system)
@pytest.mark.parametrize("m,k,per_row,gamma", [(300, 120, 4, 0.5), (600, 600, 6, 1.0), (200, 400, 5, 2.0)])
def test_lsq_matches_normal_equations(m, k, per_row, gamma):
    """Sec. "Extension to General Linear Systems" / the non-square chapter: the first k marginal
    means of the augmented system [[I, J^T], [J, -gamma I]] [x; z] = [0; y] are the regularised
    least-squares (MMSE) solution (J^T J + gamma I)^{-1} J^T y (dense Cholesky of the normal
    equations), for over-, square and under-determined J; the auxiliary block is
    z = (J x - y) / gamma (the second block row)."""
    J = synth.random_rect(m, k, per_row, 11)
    y = synth.rhs(m, 12)
    r = oracle.gabp_lsq(J, y, gamma, max_iter=5000, tol=1e-13)
    assert r["status"] == oracle.OK
    Jd = J.dense()
    xr = oracle.ridge_solve(Jd, y, gamma)
    assert np.linalg.norm(r["x"] - xr) <= 1e-10 * np.linalg.norm(xr)
    assert np.allclose(r["z"], (Jd @ r["x"] - y) / gamma, rtol=1e-9, atol=1e-11)


def test_lsq_cdma_mmse_detector():
    """The non-square chapter's MMSE detector x = (S^T S + Psi)^{-1} S^T y with Psi = sigma^-2 I,
    on a dense +-1/sqrt(N) spreading matrix (N = 16 chips, 8 users), as the dense textbook
    formula; naive and broadcast GaBP give it."""
    rng = np.random.default_rng(3)
    S = rng.choice([-1.0, 1.0], size=(16, 8)) / 4.0
    y = rng.standard_normal(16)
    psi = 0.5
    from scipy.sparse import csr_matrix
    c = csr_matrix(S)
    J = synth.RectCSR(16, 8, c.indptr.astype(np.int32), c.indices.astype(np.int32), c.data.copy())
    xr = np.linalg.solve(S.T @ S + psi * np.eye(8), S.T @ y)
    for variant in ("naive", "broadcast"):
        r = oracle.gabp_lsq(J, y, psi, max_iter=5000, tol=1e-13, variant=variant)
        assert r["status"] == oracle.OK
        assert np.allclose(r["x"], xr, rtol=1e-9, atol=1e-12)


def test_lsq_augmented_structure():
    """The augmented matrix is symmetric, has unit diagonal on the x block and -gamma on the z
    block, and J (resp. J^T) as its off-diagonal blocks -- checked against the dense J."""
    J = synth.random_rect(40, 25, 3, 4)
    Ja = oracle.to_dense(oracle.lsq_augmented(J, 0.7))
    Jd = J.dense()
    assert np.array_equal(Ja, Ja.T)
    assert np.array_equal(Ja[25:, :25], Jd) and np.array_equal(Ja[:25, 25:], Jd.T)
    assert np.array_equal(np.diag(Ja), np.concatenate([np.ones(25), np.full(40, -0.7)]))
    assert not np.any(Ja[:25, :25] - np.eye(25)) and not np.any(Ja[25:, 25:] + 0.7 * np.eye(40))


def test_timing_entries_equal_the_checked_oracle():
    """The host-baseline entries (Algorithm 2 without the input checks, on one thread and, where gcc
    has OpenMP, on all cores) run the same arithmetic per message as the checked call: identical
    marginal means and precisions after a fixed number of rounds (the residual sums may differ in
    order only), and the same stop round at a tolerance."""
    m = synth.random_sym(3000, 6, 1.1, 9)
    b = synth.rhs(m.n, 9)
    ref = oracle.gabp_broadcast(m, b, max_iter=7, tol=0.0)
    for threads in (False, True):
        if threads and oracle.host_threads() is None:
            continue
        r, dt = oracle.broadcast_timed(m, b, 7, threads=threads)
        assert r["status"] == ref["status"] and r["iters"] == 7 and dt > 0.0
        assert np.array_equal(r["x"], ref["x"]) and np.array_equal(r["P"], ref["P"])
    conv = oracle.gabp_broadcast(m, b, max_iter=500, tol=1e-12)
    r, _ = oracle.broadcast_timed(m, b, 500, threads=oracle.host_threads() is not None, tol=1e-12)
    assert r["status"] == conv["status"] == oracle.OK and r["iters"] == conv["iters"]
    assert np.allclose(r["x"], conv["x"], rtol=0, atol=1e-15 * np.max(np.abs(conv["x"])))
