"""gabp_solve_noalloc against gabp_solve (GPU, through the C ABI).

gabp_solve_noalloc serves callers that cannot call cudaMalloc at solve time
(latency-critical loops, processes whose device memory another allocator has
reserved, code under no-allocation rules): it keeps its working memory in a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also passes
on its own in a fresh process.

Two calls in a row on different systems check that the shared scratch carries
nothing from one call into the next.  The tolerance is the FP64 path's
(1e-12 relative, equal round counts).
"""
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


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _noalloc(gb, m, b, tol, max_iter):
    rp, col, val = _dev(m.rowptr, torch.int32), _dev(m.col, torch.int32), _dev(m.val, torch.float64)
    bd = _dev(b, torch.float64)
    x = torch.full_like(bd, float("nan"))
    stream = torch.cuda.current_stream()
    st, it, rel = gb.gabp_solve_noalloc(m.n, m.nnz, rp.data_ptr(), col.data_ptr(), val.data_ptr(), bd.data_ptr(),
                                        x.data_ptr(), tol, max_iter, stream.cuda_stream)
    return st, it, rel, x.cpu().numpy()


def _existing(gb, m, b, tol, max_iter):
    s = gb.Solver.from_csr(m)
    x, st, it, rel = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_iter=max_iter)
    s.close()
    return st, it, rel, x.cpu().numpy()


def test_noalloc_matches_gabp_solve_two_calls(gb):
    cases = [
        (synth.grid2d(32, -1.0, 4.5), 1),         # 32 x 32 grid, diagonal 4.5
        (synth.random_sym(9000, 6, 1.1, 12), 2),  # random symmetric, another size
    ]
    for m, seed in cases:
        b = synth.rhs(m.n, seed)
        st0, it0, rel0, x0 = _existing(gb, m, b, 1e-12, 1000)
        st1, it1, rel1, x1 = _noalloc(gb, m, b, 1e-12, 1000)
        assert st0 == st1 == gb.GABP_OK
        assert it0 == it1
        assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
        assert abs(rel1 - rel0) <= 1e-3 * rel0 + 1e-15


def test_noalloc_rejects_oversize(gb):
    m = synth.grid2d(130, -1.0, 4.5)  # n = 16900 > 16384
    st, it, rel, x = _noalloc(gb, m, synth.rhs(m.n, 3), 1e-10, 10)
    assert st == gb.GABP_ERR_INVALID
    assert "size out of range" in gb.gabp_last_error()


def test_noalloc_matches_oracle(gb):
    """The allocation-free path against the FP64 oracle (Algorithm 2): iterates after fixed rounds
    and the converged answer."""
    import oracle

    m = synth.random_sym(3000, 5, 1.1, 4)
    b = synth.rhs(m.n, 4)
    for rounds in (1, 6):
        ref = oracle.gabp_broadcast(m, b, max_iter=rounds, tol=0.0)
        st, it, rel, x = _noalloc(gb, m, b, 0.0, rounds)
        assert st == gb.GABP_NOT_CONVERGED and it == rounds
        assert np.max(np.abs(x - ref["x"])) <= 1e-13 * np.max(np.abs(ref["x"]))
    ref = oracle.gabp_broadcast(m, b, max_iter=1000, tol=1e-12)
    st, it, rel, x = _noalloc(gb, m, b, 1e-12, 1000)
    assert st == gb.GABP_OK and it == ref["iters"]
    assert np.max(np.abs(x - ref["x"])) <= 1e-12 * np.max(np.abs(ref["x"]))


def test_noalloc_status_cases(gb):
    """max_iter reached (NOT_CONVERGED, same rounds as gabp_solve), b = 0 (x = 0 after 0 rounds),
    and a larger call followed by a smaller one compared with gabp_solve (nothing of the larger
    call's scratch leaks into the smaller)."""
    m = synth.grid2d(32, -1.0, 4.5)
    b = synth.rhs(m.n, 5)
    st0, it0, rel0, x0 = _existing(gb, m, b, 1e-12, 5)
    st1, it1, rel1, x1 = _noalloc(gb, m, b, 1e-12, 5)
    assert st0 == st1 == gb.GABP_NOT_CONVERGED and it0 == it1 == 5
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
    st, it, rel, x = _noalloc(gb, m, np.zeros(m.n), 1e-12, 100)
    assert st == gb.GABP_OK and it == 0 and not np.any(x)
    big = synth.random_sym(9000, 6, 1.1, 12)
    _noalloc(gb, big, synth.rhs(big.n, 2), 1e-12, 1000)
    st0, it0, rel0, x0 = _existing(gb, m, b, 1e-12, 1000)
    st1, it1, rel1, x1 = _noalloc(gb, m, b, 1e-12, 1000)
    assert st0 == st1 == gb.GABP_OK and it0 == it1
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)


def test_noalloc_rejects_bad_matrix_on_the_device(gb):
    """An asymmetric value is found by the kernel itself and reported through the status word."""
    m = synth.grid2d(8, -1.0, 4.5)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    p = int(np.flatnonzero(rows < m.col)[3])
    m.val[p] = -1.5  # A_ij != A_ji
    st, it, rel, x = _noalloc(gb, m, synth.rhs(m.n, 1), 1e-10, 10)
    assert st == gb.GABP_ERR_INVALID
    assert "matrix rejected" in gb.gabp_last_error()


def test_noalloc_rejects_host_arrays(gb):
    """Host arrays are refused before any launch (the kernel would fault on them)."""
    m = synth.grid2d(4, -1.0, 4.5)
    rp = np.ascontiguousarray(m.rowptr)
    col = np.ascontiguousarray(m.col)
    val = np.ascontiguousarray(m.val)
    b = synth.rhs(m.n, 1)
    x = np.zeros(m.n)
    st, it, rel = gb.gabp_solve_noalloc(m.n, m.nnz, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                        b.ctypes.data, x.ctypes.data, 1e-10, 10, 0)
    assert st == gb.GABP_ERR_INVALID
    assert "device arrays" in gb.gabp_last_error()
    # one host array among device ones is refused too
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    rpd, cold, vald = (torch.from_numpy(a).cuda() for a in (rp, col, val))
    st, it, rel = gb.gabp_solve_noalloc(m.n, m.nnz, rpd.data_ptr(), cold.data_ptr(), vald.data_ptr(),
                                        b.ctypes.data, xd.data_ptr(), 1e-10, 10, 0)
    assert st == gb.GABP_ERR_INVALID
