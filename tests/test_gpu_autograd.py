"""Differentiable solve (torch.autograd.Function with a hand-written backward) on the GPU,
checked against the dense FP64 gradient of the oracle and central finite differences.

Loss 0.5 ||x - x*||^2, x = A^{-1} b, A random sparse symmetric (3 picks per row, degree ~6,
values U(-1,1), diagonal 1.2 x row abs-sum), n = 2048.  Tolerances: 1e-9 relative against the
dense gradient, 1e-6 against central finite differences (step 1e-5 relative, the loss
evaluated by dense LU)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ag():
    import __graft_entry__

    __graft_entry__.build()
    import paper_0811_2518_gb300 as gb
    from paper_0811_2518_gb300 import autograd

    return gb, autograd


def _setup(n=2048, seed=5):
    m = synth.random_sym(n, 3, 1.2, seed)
    b = synth.rhs(n, seed)
    xs = synth.rhs(n, seed + 100)
    return m, b, xs


def _grads(ag, m, b, xs, precision, save_x=True, tol=1e-12):
    gb, autograd = ag
    rp = torch.from_numpy(m.rowptr).cuda()
    cl = torch.from_numpy(m.col).cuda()
    vals = torch.from_numpy(m.val.copy()).cuda().requires_grad_(True)
    bt = torch.from_numpy(b.copy()).cuda().requires_grad_(True)
    x = autograd.gabp_solve_autograd(rp, cl, vals, bt, tol=tol, precision=precision, save_x=save_x)
    loss = 0.5 * torch.sum((x - torch.from_numpy(xs).cuda()) ** 2)
    loss.backward()
    return x.detach().cpu().numpy(), vals.grad.cpu().numpy(), bt.grad.cpu().numpy()


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", [0, 1])
def test_gradient_matches_dense(ag, precision):
    m, b, xs = _setup()
    x, gv, gbv = _grads(ag, m, b, xs, precision)
    A = oracle.to_dense(m)
    x0, lam, G = oracle.dense_gradient(A, b, xs)
    assert _relerr(x, x0) <= 1e-10
    assert _relerr(gbv, lam) <= 1e-9
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    assert _relerr(gv, G[rows, m.col]) <= 1e-9


def test_recompute_x_equals_saved(ag):
    m, b, xs = _setup(1024, 7)
    _, gv1, gb1 = _grads(ag, m, b, xs, 1, save_x=True)
    _, gv2, gb2 = _grads(ag, m, b, xs, 1, save_x=False)
    assert _relerr(gv2, gv1) <= 1e-10 and _relerr(gb2, gb1) <= 1e-10


def test_gradient_finite_differences(ag):
    gb, autograd = ag
    m, b, xs = _setup()
    x, gv, gbv = _grads(ag, m, b, xs, 1)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))

    def loss_of(vals, bb):
        # the loss itself, evaluated exactly (dense LU): finite differences of an
        # iterative solve would add the solve's own error divided by the step
        A = np.zeros((m.n, m.n))
        A[rows, m.col] = vals
        y = np.linalg.solve(A, bb)
        return 0.5 * np.sum((y - xs) ** 2)

    rng = np.random.default_rng(0)
    for i in rng.choice(m.n, 3, replace=False):  # dL/db_i
        h = 1e-5 * max(1.0, abs(b[i]))
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss_of(m.val, bp) - loss_of(m.val, bm)) / (2 * h)
        assert abs(fd - gbv[i]) <= 1e-6 * max(1.0, abs(fd))
    off = np.nonzero(rows < m.col)[0]
    for p in rng.choice(off, 4, replace=False):  # the symmetric pair A_ij = A_ji moved together
        i, j = rows[p], m.col[p]
        q = m.rowptr[j] + np.nonzero(m.col[m.rowptr[j]:m.rowptr[j + 1]] == i)[0][0]
        h = 1e-5 * abs(m.val[p])
        vp, vm = m.val.copy(), m.val.copy()
        vp[p] += h; vp[q] += h
        vm[p] -= h; vm[q] -= h
        fd = (loss_of(vp, b) - loss_of(vm, b)) / (2 * h)
        assert abs(fd - (gv[p] + gv[q])) <= 1e-6 * max(1.0, abs(fd))
    diag = np.nonzero(rows == m.col)[0]
    for p in rng.choice(diag, 2, replace=False):
        h = 1e-5 * abs(m.val[p])
        vp, vm = m.val.copy(), m.val.copy()
        vp[p] += h
        vm[p] -= h
        fd = (loss_of(vp, b) - loss_of(vm, b)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-6 * max(1.0, abs(fd))


def test_full_size_gradient_properties(ag):
    """n = 2^22, degree ~6 (the differentiable-solve workload): the adjoint solve satisfies
    A lambda = x - x* to the solve tolerance (host SpMV) and sampled dL/dA entries follow
    from lambda and x."""
    gb, autograd = ag
    m = synth.random_sym(1 << 22, 3, 1.2, 5)
    b = synth.rhs(m.n, 5)
    xs = synth.rhs(m.n, 105)
    x, gv, lam = _grads(ag, m, b, xs, 1, tol=1e-10)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    r = (x - xs) - np.bincount(rows, m.val * lam[m.col], minlength=m.n)
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(x - xs)
    rx = b - np.bincount(rows, m.val * x[m.col], minlength=m.n)
    assert np.linalg.norm(rx) <= 1.0001e-10 * np.linalg.norm(b)
    idx = np.random.default_rng(1).choice(m.nnz, 10000, replace=False)
    i, j = rows[idx], m.col[idx]
    want = np.where(i == j, -lam[i] * x[i], -0.5 * (lam[i] * x[j] + lam[j] * x[i]))
    scale = np.abs(lam[i] * x[j]) + np.abs(lam[j] * x[i])  # rounding of the two products and the sum
    assert np.all(np.abs(gv[idx] - want) <= 1e-15 * scale + 1e-300)


def test_shared_solver_training_loop(ag):
    """One Solver reused across steps whose parameters are A's values (gabp_set_values): each
    step's gradients equal those of a fresh handle, also when a second forward changes the
    values before the first backward runs (the backward puts its values back)."""
    gb, autograd = ag
    m, b, xs = _setup(n=2048, seed=7)
    rp = torch.from_numpy(m.rowptr).cuda()
    cl = torch.from_numpy(m.col).cuda()
    xst = torch.from_numpy(xs).cuda()
    shared = gb.Solver(m.n, rp, cl, torch.from_numpy(m.val).cuda(), precision=1)
    rng = np.random.default_rng(3)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    vals_steps = []
    for step in range(3):
        v = m.val.copy()
        off = rows != m.col
        v[off] *= 1.0 + 0.05 * step  # stays symmetric: the same factor on (i,j) and (j,i)
        v[~off] *= 1.0 + 0.08 * step + 0.01 * rng.random()
        vals_steps.append(v)

    def run(v, solver):
        vt = torch.from_numpy(v).cuda().requires_grad_(True)
        bt = torch.from_numpy(b).cuda().requires_grad_(True)
        x = autograd.gabp_solve_autograd(rp, cl, vt, bt, tol=1e-12, solver=solver)
        return vt, bt, 0.5 * torch.sum((x - xst) ** 2)

    for v in vals_steps:
        vt, bt, loss = run(v, shared)
        loss.backward()
        vf, bf, lf = run(v, None)
        lf.backward()
        assert torch.allclose(vt.grad, vf.grad, rtol=1e-9, atol=1e-14)
        assert torch.allclose(bt.grad, bf.grad, rtol=1e-9, atol=1e-14)
    # interleaved: forward(v0), forward(v2), backward(v0), backward(v2)
    v0t, b0t, l0 = run(vals_steps[0], shared)
    v2t, b2t, l2 = run(vals_steps[2], shared)
    l0.backward()
    l2.backward()
    for v, vt in ((vals_steps[0], v0t), (vals_steps[2], v2t)):
        A = oracle.to_dense(synth.CSR(m.n, m.rowptr, m.col, v, {}))
        x0, lam, G = oracle.dense_gradient(A, b, xs)
        assert _relerr(vt.grad.cpu().numpy(), G[np.repeat(np.arange(m.n), np.diff(m.rowptr)), m.col]) <= 1e-8
    shared.close()


def test_set_values_rejects_and_recovers(ag):
    gb, _ = ag
    m = synth.random_sym(512, 3, 1.2, 4)
    s = gb.Solver.from_csr(m, precision=1)
    b = torch.from_numpy(synth.rhs(m.n, 1)).cuda()
    bad = m.val.copy()
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    p = int(np.flatnonzero(rows != m.col)[0])
    bad[p] *= 1.5  # A_ij != A_ji
    with pytest.raises(gb.GaBPError):
        s.set_values(bad)
    x, st, it, rel = s.solve(b, tol=1e-10, check=False)
    assert st == gb.GABP_ERR_INVALID
    s.set_values(m.val)
    x, st, it, rel = s.solve(b, tol=1e-10)
    assert st == gb.GABP_OK
    ref = oracle.dense_solve(oracle.to_dense(m), synth.rhs(m.n, 1))
    assert _relerr(x.cpu().numpy(), ref) <= 1e-8
    s.close()
