"""FP64 CPU oracle for the GaBP solver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product (``paper_0811_2518_gb300``) never imports
it, and it never imports the product: the two share no code.

Paper: D. Bickson, "Gaussian Belief Propagation: Theory and Application".

Contents and the passage each follows:

* :func:`gabp_naive`      -- Algorithm 1, parallel (synchronous) schedule, in C.
* :func:`gabp_broadcast`  -- Algorithm 2 (broadcast variant), in C.
* :func:`gabp_serial`     -- Algorithm 1's rules under the serial schedule (one
  message store updated in place; Sec. "The Gaussian BP Algorithm", the
  paragraph on parallel vs serial scheduling), nodes firing colour by colour, in C.
* :func:`colour_greedy`   -- the colouring of those sweeps (index order, smallest
  colour unused by lower-indexed neighbours), in C.
* :func:`dense_solve`     -- x* = A^{-1} b by LU (Proposition "linear system =
  inference": the GaBP fixed point is the marginal-mean vector A^{-1} b).
* :func:`marginal_precisions_exact` -- 1/(A^{-1})_ii, the exact marginal
  precisions, which GaBP reaches on trees (Sec. "Convergence and Exactness").
* :func:`rho_abs_normalized` -- rho(|I - D^{-1/2} A D^{-1/2}|), the
  walk-summability quantity of the spectral-radius theorem.
* :func:`rate_bound_rounds` -- the round bound of Sec. "Upper Bound on
  Convergence Rate" for diagonally dominant A.
* :func:`diagonal_loading` / :func:`convergence_fix` -- Chapter "Fixing
  convergence of GaBP": J' = J + Gamma and the double loop
  x^(t+1) = (J + Gamma)^{-1} (h + Gamma x^(t)) whose inner solve is GaBP.
* :func:`convergence_fix_single_loop` -- the same chapter's single-loop form: one
  GaBP round per outer step with the damped potential update (numpy, FP64).
* :func:`aitken` / :func:`gabp_aitken` -- Sec. "Convergence Acceleration": Aitken's
  extrapolation of the marginal means of Algorithm 2 (numpy, FP64).
* :func:`steffensen_step` / :func:`gabp_steffensen` -- the same section's Steffensen
  iterations: two GaBP rounds (or serial sweeps), Aitken's extrapolation of the
  marginal-mean vector, the extrapolated vector replacing the iterate, GaBP continuing
  from it; parallel and serial schedules (numpy, FP64).
* :func:`lsq_augmented` / :func:`gabp_lsq` / :func:`ridge_solve` -- Sec. "Extension to
  General Linear Systems" and Chapter "Extending GaBP to support non-square matrices":
  the regularised least-squares (MMSE) solution x = (J^T J + gamma I)^{-1} J^T y of a
  rectangular J, read off the first k entries of the symmetric augmented system
  [[I_k, J^T], [J, -gamma I_m]] [x; z] = [0; y], which Algorithm 2 solves.
* :func:`dense_gradient`  -- gradients of 0.5 ||x - x*||^2 for x = A^{-1} b,
  written from the adjoint identity (no counterpart in the paper; it pins the
  differentiable solve).

Status codes: 0 converged, 1 not converged, 2 diverged, 3 breakdown, -1 invalid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gabp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgabp_oracle.so")
_OMP_PATH = os.path.join(_HERE, "_build", "libgabp_oracle_omp.so")
_lib = None
_omp = None
_lock = threading.Lock()

OK, NOT_CONVERGED, DIVERGED, BREAKDOWN, INVALID = 0, 1, 2, 3, -1


def _compile(path, extra, force):
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        # ISO C mode: no contraction of a * b + c into FMA, so x86-64 and aarch64 hosts give the
        # same results
        subprocess.run(["gcc", "-O3", "-std=c99", *extra, "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the C oracle with the host gcc (-O3, portable flags, one thread) and, where gcc
    has OpenMP, the same file built for all host cores (used only to time the host baseline)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    _compile(_LIB_PATH, [], force)
    try:
        _compile(_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _bind(lib):
    lib.orc_colour_greedy.restype = ctypes.c_int
    lib.orc_colour_greedy.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    for name in ("orc_gabp_naive", "orc_gabp_broadcast", "orc_gabp_serial", "orc_gabp_broadcast_unchecked"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                      ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_threads.argtypes = []
    return lib


def _load_omp():
    """The OpenMP build of the oracle, or None where gcc had no OpenMP."""
    global _omp
    _load()
    with _lock:
        if _omp is None and os.path.exists(_OMP_PATH):
            _omp = _bind(ctypes.CDLL(_OMP_PATH))
    return _omp


def host_threads():
    """Threads the all-cores build runs with (None when it was not built)."""
    lib = _load_omp()
    return lib.orc_threads() if lib is not None else None


def broadcast_timed(m, b, rounds, threads=False, checked=False, tol=0.0):
    """Timing entry of the host baseline: ``rounds`` synchronous rounds of Algorithm 2 (stops
    early only when tol > 0 is met), on one thread or, with ``threads``, on all host cores (the
    OpenMP build of the same file).  Without ``checked`` the input checks are skipped (run a
    checked call first).  Returns (result dict, seconds spent in the call)."""
    import time

    lib = _load_omp() if threads else _load()
    if lib is None:
        raise RuntimeError("the OpenMP build of the oracle is not available")
    rowptr = np.ascontiguousarray(m.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(m.col, dtype=np.int32)
    val = np.ascontiguousarray(m.val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(m.n)
    P = np.zeros(m.n)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    fn = lib.orc_gabp_broadcast if checked else lib.orc_gabp_broadcast_unchecked
    t0 = time.perf_counter()
    rc = fn(m.n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), int(rounds), float(tol), 0, _ptr(x), _ptr(P),
            ctypes.byref(it), ctypes.byref(rel), None, None)
    dt = time.perf_counter() - t0
    return {"status": rc, "x": x, "P": P, "iters": it.value, "relres": rel.value}, dt


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _run(name, m, b, max_iter, tol, stop_rule, messages):
    lib = _load()
    rowptr = np.ascontiguousarray(m.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(m.col, dtype=np.int32)
    val = np.ascontiguousarray(m.val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if b.shape != (m.n,):
        raise ValueError("b has the wrong shape")
    x = np.zeros(m.n)
    P = np.zeros(m.n)
    Pm = np.zeros(m.nnz) if messages else None
    Mm = np.zeros(m.nnz) if messages else None
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = getattr(lib, name)(m.n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), int(max_iter), float(tol),
                            int(stop_rule), _ptr(x), _ptr(P), ctypes.byref(it), ctypes.byref(rel),
                            _ptr(Pm) if messages else None, _ptr(Mm) if messages else None)
    out = {"status": rc, "x": x, "P": P, "iters": it.value, "relres": rel.value}
    if messages:
        out["Pmsg"] = Pm
        out["mumsg"] = Mm
    return out


def gabp_naive(m, b, max_iter=1000, tol=1e-12, stop_rule="residual", messages=False):
    """Algorithm 1 (naive GaBP), synchronous schedule, FP64.

    ``m`` is a full symmetric CSR (``synth.CSR``).  Returns a dict with
    ``status``, ``x`` (marginal means), ``P`` (marginal precisions), ``iters``,
    ``relres`` and, with ``messages=True``, ``Pmsg`` / ``mumsg``: for every CSR
    slot p of row i with col k != i, the message k -> i after the last round.
    ``stop_rule`` is "residual" (||b - A x_t|| <= tol ||b||) or "message"
    (max |message change| < tol, the rule of the paper's numerical examples).
    """
    return _run("orc_gabp_naive", m, b, max_iter, tol, 0 if stop_rule == "residual" else 1, messages)


def gabp_broadcast(m, b, max_iter=1000, tol=1e-12, stop_rule="residual", messages=False):
    """Algorithm 2 (broadcast GaBP), synchronous schedule, FP64; same interface as :func:`gabp_naive`."""
    return _run("orc_gabp_broadcast", m, b, max_iter, tol, 0 if stop_rule == "residual" else 1, messages)


def gabp_serial(m, b, max_iter=1000, tol=1e-12, stop_rule="residual", messages=False):
    """Algorithm 1's message rules, serial schedule (one store, in place): each sweep fires the
    nodes of colour 0, then colour 1, ... (:func:`colour_greedy`); ``iters`` counts sweeps.
    Same interface as :func:`gabp_naive`."""
    return _run("orc_gabp_serial", m, b, max_iter, tol, 0 if stop_rule == "residual" else 1, messages)


def colour_greedy(m):
    """(colour[n], number of colours): nodes in index order, each taking the smallest colour
    not used by a lower-indexed neighbour."""
    lib = _load()
    rowptr = np.ascontiguousarray(m.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(m.col, dtype=np.int32)
    colour = np.zeros(m.n, dtype=np.int32)
    nc = lib.orc_colour_greedy(m.n, _ptr(rowptr), _ptr(col), _ptr(colour))
    return colour, nc


# --------------------------------------------------------------------------- dense references
def to_dense(m) -> np.ndarray:
    A = np.zeros((m.n, m.n))
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    A[rows, m.col] = m.val
    return A


def dense_solve(A, b) -> np.ndarray:
    """x* = A^{-1} b (LAPACK LU with partial pivoting)."""
    return np.linalg.solve(np.asarray(A, dtype=np.float64), np.asarray(b, dtype=np.float64))


def marginal_precisions_exact(A) -> np.ndarray:
    """Exact marginal precisions P_i = 1 / (A^{-1})_ii."""
    return 1.0 / np.diag(np.linalg.inv(np.asarray(A, dtype=np.float64)))


def rho_abs_normalized(A) -> float:
    """rho(|I - D^{-1/2} A D^{-1/2}|) with D = diag(A) (spectral-radius theorem)."""
    A = np.asarray(A, dtype=np.float64)
    d = 1.0 / np.sqrt(np.diag(A))
    R = np.abs(np.eye(A.shape[0]) - d[:, None] * A * d[None, :])
    return float(np.max(np.abs(np.linalg.eigvalsh(R))))


def rate_bound_rounds(A, eps: float) -> int:
    """Sec. "Upper Bound on Convergence Rate": with eps_i = |a_ii| - sum_j |a_ij| > 0
    and gamma = max_ij 1 / (1 + eps_i / (|a_ij| |N(i)|)), GaBP reaches
    |x* - x_t| < eps ||b||_inf after at most ceil(log eps / log gamma) rounds."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    gamma = 0.0
    for i in range(n):
        off = [j for j in range(n) if j != i and A[i, j] != 0.0]
        e = abs(A[i, i]) - sum(abs(A[i, j]) for j in off)
        if e <= 0:
            raise ValueError("not strictly diagonally dominant")
        for j in off:
            gamma = max(gamma, 1.0 / (1.0 + e / (abs(A[i, j]) * len(off))))
    return int(np.ceil(np.log(eps) / np.log(gamma)))


def diagonal_loading(A, mode: str = "uniform", gamma: float = 0.25, delta: float = 0.0) -> np.ndarray:
    """Diagonal Gamma of the convergence fix.

    "uniform": Gamma = gamma * diag(A) -- the unit-diagonal model J = I - R loaded
    by gamma I, written back in A's scaling; walk-summable for gamma > rho(|R|) - 1.
    "dd": Gamma_ii = max(0, sum_j |A_ij| - A_ii) + delta * A_ii, which makes
    A + Gamma diagonally dominant (hence walk-summable) for delta > 0.
    """
    A = np.asarray(A, dtype=np.float64)
    d = np.diag(A).copy()
    if mode == "uniform":
        return gamma * d
    off = np.sum(np.abs(A), axis=1) - np.abs(d)
    return np.maximum(0.0, off - d) + delta * d


def convergence_fix(m, b, Gamma, tol=1e-10, inner_tol=1e-12, max_outer=500, inner_max_iter=2000,
                    variant="broadcast"):
    """Chapter "Fixing convergence of GaBP", iterative correction (double loop):
    x^(t+1) = (A + Gamma)^{-1} (b + Gamma x^(t)), x^(0) = 0, the inner solve being
    GaBP on A + Gamma.  Stops when ||b - A x|| <= tol ||b||.

    Returns dict(x, outer, inner_total, status, history) where history holds
    ||x^(t) - x*||_2 per outer step when the dense solution is cheap (n <= 4096).
    """
    Gamma = np.asarray(Gamma, dtype=np.float64)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    val = m.val.copy()
    diag_slots = np.nonzero(rows == m.col)[0]
    val[diag_slots] += Gamma[rows[diag_slots]]
    mp = SimpleNamespace(n=m.n, rowptr=m.rowptr, col=m.col, val=val, nnz=int(m.rowptr[-1]))
    A = to_dense(m) if m.n <= 4096 else None
    xs = dense_solve(A, b) if A is not None else None
    solve = gabp_broadcast if variant == "broadcast" else gabp_naive
    x = np.zeros(m.n)
    bn = np.linalg.norm(b)
    inner_total, hist, status = 0, [], NOT_CONVERGED
    for t in range(1, max_outer + 1):
        r = solve(mp, b + Gamma * x, max_iter=inner_max_iter, tol=inner_tol)
        if r["status"] not in (OK, NOT_CONVERGED):
            status = r["status"]
            break
        inner_total += r["iters"]
        x = r["x"]
        if xs is not None:
            hist.append(float(np.linalg.norm(x - xs)))
        ax = np.zeros(m.n)
        np.add.at(ax, rows, m.val * x[m.col])
        if np.linalg.norm(b - ax) <= tol * bn:
            status = OK
            break
    return {"x": x, "outer": t, "inner_total": inner_total, "status": status, "history": hist}


def aitken(x0, x1, x2):
    """Aitken's extrapolation of three consecutive iterates, element-wise (Sec. "Convergence
    Acceleration"): y = x0 - (x1 - x0)^2 / (x2 - 2 x1 + x0).  Where the second difference is
    zero or negligible (|D| <= 1e-14 |x2|: the component has stopped moving), y = x2."""
    x0, x1, x2 = (np.asarray(v, dtype=np.float64) for v in (x0, x1, x2))
    D = x2 - 2.0 * x1 + x0
    ok = np.abs(D) > 1e-14 * np.abs(x2)
    return np.where(ok, x0 - (x1 - x0) ** 2 / np.where(ok, D, 1.0), x2)


def gabp_aitken(m, b, max_iter=1000, tol=1e-12, history=False):
    """Algorithm 2 (parallel schedule, information form) with Aitken's method applied to the
    marginal means (Sec. "Convergence Acceleration"): after round t, y^(t) = aitken(x^(t-2),
    x^(t-1), x^(t)) per node, x^(0) = b_i / A_ii (no messages yet); y^(1) = x^(1).  The GaBP
    iteration itself is unchanged.  Stops when ||b - A y^(t)|| <= tol ||b||; returns dict(x=y,
    iters, status[, xs, ys])."""
    b = np.asarray(b, dtype=np.float64)
    n = m.n
    rows = np.repeat(np.arange(n), np.diff(m.rowptr))
    off = rows != m.col
    r, c, a = rows[off], m.col[off], m.val[off]
    diag = np.zeros(n)
    diag[rows[~off]] = m.val[~off]
    key = r.astype(np.int64) * n + c
    order = np.argsort(key)
    rev = order[np.searchsorted(key[order], c.astype(np.int64) * n + r)]
    P = np.zeros(len(a))
    H = np.zeros(len(a))
    hist = [b / diag]
    xs, ys = [], []
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return {"x": np.zeros(n), "iters": 0, "status": OK, "xs": xs, "ys": ys}
    status, y, t = NOT_CONVERGED, hist[0], 0
    for t in range(1, max_iter + 1):
        Pt = diag + np.bincount(r, P, minlength=n)
        Ht = b + np.bincount(r, H, minlength=n)
        d = Pt[c] - P[rev]
        if np.any(d == 0.0):
            status = BREAKDOWN
            break
        P, H = -a * a / d, -a * (Ht[c] - H[rev]) / d
        x = (b + np.bincount(r, H, minlength=n)) / (diag + np.bincount(r, P, minlength=n))
        hist.append(x)
        y = x if t < 2 else aitken(hist[-3], hist[-2], hist[-1])
        if history:
            xs.append(x)
            ys.append(y)
        if not np.all(np.isfinite(y)):
            status = DIVERGED
            break
        ax = np.bincount(rows, m.val * y[m.col], minlength=n)
        if np.linalg.norm(b - ax) <= tol * bn:
            status = OK
            break
    return {"x": y, "iters": t, "status": status, "xs": xs, "ys": ys}


def steffensen_step(x0, x1, x2):
    """Aitken's extrapolation of three consecutive marginal-mean VECTORS, as Steffensen's
    iterations use it (Sec. "Convergence Acceleration"): one scalar step along the newest
    difference, y = x2 - lam (x2 - x1) with lam = <x2 - x1, D> / <D, D>, D = x2 - 2 x1 + x0.
    For x_n = x* + c q^n (any vector c, scalar q != 1) it returns x* exactly, like the
    scalar formula; with D = 0 (nothing moves) lam = 0 and y = x2.  Returns (y, lam)."""
    x0, x1, x2 = (np.asarray(v, dtype=np.float64) for v in (x0, x1, x2))
    d = x2 - x1
    D = x2 - 2.0 * x1 + x0
    den = float(D @ D)
    lam = float(d @ D) / den if den > 0.0 else 0.0
    if not np.isfinite(lam):
        lam = 0.0
    return x2 - lam * d, lam


def gabp_steffensen(m, b, schedule="parallel", max_iter=1000, tol=1e-12, history=False):
    """Steffensen's iterations on GaBP (Sec. "Convergence Acceleration"), information form.

    A cycle starts from a message state whose marginal means are x_n, runs two GaBP rounds
    (Algorithm 2, parallel schedule) or two serial sweeps (nodes firing colour by colour, one
    store updated in place, as :func:`gabp_serial`), giving x_{n+1} and x_{n+2}, and forms
    y_n = :func:`steffensen_step` (x_n, x_{n+1}, x_{n+2}).  "y_n replaces x_n and GaBP runs
    again": the mean messages are moved by the same scalar step, h <- h_{n+2} - lam (h_{n+2} -
    h_{n+1}) (precision messages unchanged), which makes the marginal means of the new state
    exactly y_n when the precisions are stationary (x is affine in h), and the next cycle starts
    from that state.  Round t's iterate is x^(t) after the first round of a cycle and the
    extrapolated state's marginal means after the second; the run stops at the first t with
    ||b - A x|| <= tol ||b|| or at max_iter rounds (sweeps).  Returns dict(x, iters, status[,
    xs: the iterate of every round, pre: x_{n+2} of every cycle before the extrapolation,
    lams: the step of every cycle]).
    """
    b = np.asarray(b, dtype=np.float64)
    n = m.n
    rows = np.repeat(np.arange(n), np.diff(m.rowptr))
    off = rows != m.col
    r, c, a = rows[off], m.col[off], m.val[off]  # slot e of row r holds the message c -> r
    diag = np.zeros(n)
    diag[rows[~off]] = m.val[~off]
    key = r.astype(np.int64) * n + c
    order = np.argsort(key)
    rev = order[np.searchsorted(key[order], c.astype(np.int64) * n + r)]
    if schedule == "serial":
        colour, ncol = colour_greedy(m)
    elif schedule != "parallel":
        raise ValueError("schedule must be 'parallel' or 'serial'")

    def beliefs(P, H):
        return (b + np.bincount(r, H, minlength=n)) / (diag + np.bincount(r, P, minlength=n))

    def one_round(P, H):
        """Round (or sweep) from state (P, H); None on a zero cavity precision."""
        if schedule == "parallel":
            Pt = diag + np.bincount(r, P, minlength=n)
            Ht = b + np.bincount(r, H, minlength=n)
            d = Pt[c] - P[rev]
            if np.any(d == 0.0):
                return None
            return -a * a / d, -a * (Ht[c] - H[rev]) / d
        P, H = P.copy(), H.copy()
        for col in range(ncol):  # the nodes of one colour share no edge: they fire at once
            Pt = diag + np.bincount(r, P, minlength=n)
            Ht = b + np.bincount(r, H, minlength=n)
            f = colour[c] == col  # messages sent by the firing nodes
            d = Pt[c[f]] - P[rev[f]]
            if np.any(d == 0.0):
                return None
            P[f] = -a[f] ** 2 / d
            H[f] = -a[f] * (Ht[c[f]] - H[rev[f]]) / d
        return P, H

    xs, pre, lams = [], [], []
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return {"x": np.zeros(n), "iters": 0, "status": OK, "xs": xs, "pre": pre, "lams": lams}
    P = np.zeros(len(a))
    H = np.zeros(len(a))
    x = beliefs(P, H)
    xc, Hc = x, None  # the cycle's starting iterate; the state after its first round
    status, t = NOT_CONVERGED, 0
    for t in range(1, max_iter + 1):
        nxt = one_round(P, H)
        if nxt is None:
            status = BREAKDOWN
            break
        Pn, Hn = nxt
        x = beliefs(Pn, Hn)
        if t % 2 == 1:  # first round of a cycle
            x1, H1 = x, Hn
            P, H = Pn, Hn
        else:  # second round: extrapolate and move the mean messages by the same step
            _, lam = steffensen_step(xc, x1, x)
            lams.append(lam)
            if history:
                pre.append(x.copy())
            P, H = Pn, Hn - lam * (Hn - H1)
            x = beliefs(P, H)
            xc = x
        if history:
            xs.append(x.copy())
        if not np.all(np.isfinite(x)):
            status = DIVERGED
            break
        ax = np.bincount(rows, m.val * x[m.col], minlength=n)
        if np.linalg.norm(b - ax) <= tol * bn:
            status = OK
            break
    return {"x": x, "iters": t, "status": status, "xs": xs, "pre": pre, "lams": lams}


def convergence_fix_single_loop(m, b, Gamma, s=0.5, tol=1e-10, max_iter=100000, history=False):
    """Chapter "Fixing convergence of GaBP", the single-loop form: ONE GaBP round (Algorithm 2,
    information form, parallel schedule) on J' = A + Gamma per outer step, the node potentials
    moved by the damped update h^(t+1) = (1 - s) h^(t) + s (b + Gamma x^(t)); x^(0) = 0, so the
    first round runs with h^(1) = b.  The messages are never restarted.  Stops when
    ||b - A x^(t)|| <= tol ||b||.  Returns dict(x, iters, status[, xs: x^(t) per round]).
    """
    Gamma = np.asarray(Gamma, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = m.n
    rows = np.repeat(np.arange(n), np.diff(m.rowptr))
    off = rows != m.col
    r, c, a = rows[off], m.col[off], m.val[off]
    diag1 = np.zeros(n)
    diag1[rows[~off]] = m.val[~off]
    diag1 = diag1 + Gamma
    key = r.astype(np.int64) * n + c
    order = np.argsort(key)
    rev = order[np.searchsorted(key[order], c.astype(np.int64) * n + r)]  # slot of the reverse edge
    P = np.zeros(len(a))  # slot e = (i, k): message k -> i
    H = np.zeros(len(a))
    hpot = b.copy()
    x = np.zeros(n)
    bn = np.linalg.norm(b)
    xs = []
    status = NOT_CONVERGED
    t = 0
    if bn == 0.0:
        return {"x": x, "iters": 0, "status": OK, "xs": xs}
    for t in range(1, max_iter + 1):
        # one GaBP round on J' with the potentials h^(t): sender aggregates minus the reverse message
        Pt = diag1 + np.bincount(r, P, minlength=n)
        Ht = hpot + np.bincount(r, H, minlength=n)
        d = Pt[c] - P[rev]
        if np.any(d == 0.0):
            status = BREAKDOWN
            break
        P, H = -a * a / d, -a * (Ht[c] - H[rev]) / d
        Pt = diag1 + np.bincount(r, P, minlength=n)
        Ht = hpot + np.bincount(r, H, minlength=n)
        x = Ht / Pt
        if history:
            xs.append(x.copy())
        if not np.all(np.isfinite(x)):
            status = DIVERGED
            break
        hpot = (1.0 - s) * hpot + s * (b + Gamma * x)  # the damped potential of the next round
        ax = np.bincount(rows, m.val * x[m.col], minlength=n)
        if np.linalg.norm(b - ax) <= tol * bn:
            status = OK
            break
    return {"x": x, "iters": t, "status": status, "xs": xs}


def lsq_augmented(J, gamma: float):
    """The symmetric augmented matrix of a rectangular J (m x k, ``synth.RectCSR``):
    [[I_k, J^T], [J, -gamma I_m]] (the general-linear-systems construction with the -gamma I
    block that makes it invertible; the non-square chapter's matrix with Psi = gamma I), as a
    full symmetric CSR with n = k + m rows: variables x first, auxiliary z after them."""
    if not gamma > 0.0:
        raise ValueError("gamma must be positive")
    m, k = J.m, J.k
    jr = np.repeat(np.arange(m), np.diff(J.rowptr))
    rows = np.concatenate([np.arange(k), jr + k, J.col, np.arange(m) + k])
    cols = np.concatenate([np.arange(k), J.col, jr + k, np.arange(m) + k])
    vals = np.concatenate([np.ones(k), J.val, J.val, np.full(m, -float(gamma))])
    n = k + m
    key = rows.astype(np.int64) * n + cols
    order = np.argsort(key, kind="stable")
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return SimpleNamespace(n=n, rowptr=rowptr.astype(np.int32), col=cols[order].astype(np.int32),
                           val=vals[order], nnz=int(rowptr[-1]))


def ridge_solve(Jd, y, gamma: float) -> np.ndarray:
    """x = (J^T J + gamma I)^{-1} J^T y from the dense normal equations (Cholesky)."""
    Jd = np.asarray(Jd, dtype=np.float64)
    G = Jd.T @ Jd + gamma * np.eye(Jd.shape[1])
    L = np.linalg.cholesky(G)
    return np.linalg.solve(L.T, np.linalg.solve(L, Jd.T @ np.asarray(y, dtype=np.float64)))


def gabp_lsq(J, y, gamma: float, max_iter=1000, tol=1e-12, variant="broadcast"):
    """Regularised least squares by GaBP: Algorithm 2 (or 1) on :func:`lsq_augmented` with the
    right-hand side [0_k; y]; x is the first k marginal means, z the remaining m.  The stop rule
    is the augmented system's relative residual.  Returns the solver's dict plus x, z."""
    Ja = lsq_augmented(J, gamma)
    b = np.concatenate([np.zeros(J.k), np.asarray(y, dtype=np.float64)])
    r = (gabp_broadcast if variant == "broadcast" else gabp_naive)(Ja, b, max_iter=max_iter, tol=tol)
    r = dict(r)
    r["z"] = r["x"][J.k:]
    r["x"] = r["x"][:J.k]
    return r


def dense_gradient(A, b, xstar):
    """Gradients of L = 0.5 ||x - x*||^2 with x = A^{-1} b, A symmetric.

    lambda = A^{-T} (x - x*) = A^{-1} (x - x*);  dL/db = lambda;  dL/dA = -lambda x^T.
    Restricted to A's pattern and symmetrised (A stays symmetric): for a stored
    off-diagonal entry (i, j), g_ij = -(lambda_i x_j + lambda_j x_i) / 2; for the
    diagonal, g_ii = -lambda_i x_i.  Returns (x, dL/db, G) with G dense (zeros
    off the pattern).
    """
    A = np.asarray(A, dtype=np.float64)
    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, x - xstar)
    G = -0.5 * (np.outer(lam, x) + np.outer(x, lam))
    G[A == 0.0] = 0.0
    return x, lam, G
