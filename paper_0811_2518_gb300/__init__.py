"""GB300 (sm_103a) Gaussian belief propagation solver -- Python binding.

A thin ctypes layer over the C ABI declared in ``include/gabp.h``.  Functions
carry the C names (``gabp_create``, ``gabp_solve`` ...) and only marshal
arguments: every step of a solve runs in the CUDA kernels of ``libgabp.so``.
PyTorch supplies device memory and streams.  If the library has not been
built, importing the binding raises: there is no CPU fallback.

Paper: D. Bickson, "Gaussian Belief Propagation: Theory and Application"
(GaBP as a solver for A x = b, Algorithms 1 and 2).
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "GABP_OK", "GABP_NOT_CONVERGED", "GABP_DIVERGED", "GABP_BREAKDOWN", "GABP_TIMEOUT",
    "GABP_ERR_INVALID", "GABP_ERR_CUDA", "GABP_ERR_NOMEM",
    "GABP_PREC_FP64", "GABP_PREC_FP32_REFINE", "GABP_VARIANT_NODE", "GABP_VARIANT_EDGE",
    "Options", "lib", "library_path", "exported_symbols",
    "gabp_options_default", "gabp_create", "gabp_set_values", "gabp_set_options", "gabp_set_stream", "gabp_solve",
    "gabp_solve_host", "gabp_solve_batched", "gabp_marginal_precisions", "gabp_get_messages",
    "gabp_grad_values", "gabp_last_stats", "gabp_last_freeze", "gabp_profile_read", "gabp_solve_noalloc", "gabp_solve_systems", "gabp_tuned_shapes", "gabp_serial_colours", "gabp_set_messages", "gabp_residual_history", "gabp_destroy", "gabp_status_string", "gabp_last_error",
    "gabp_create_lsq", "gabp_solve_lsq", "gabp_create_dense",
    "Solver", "LSQSolver", "GaBPError",
]

GABP_OK, GABP_NOT_CONVERGED, GABP_DIVERGED, GABP_BREAKDOWN, GABP_TIMEOUT = 0, 1, 2, 3, 4
GABP_ERR_INVALID, GABP_ERR_CUDA, GABP_ERR_NOMEM = -1, -2, -3
GABP_PREC_FP64, GABP_PREC_FP32_REFINE = 0, 1
GABP_VARIANT_NODE, GABP_VARIANT_EDGE = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "_lib", "libgabp.so")


class Options(ctypes.Structure):
    """Mirror of ``gabp_options`` (include/gabp.h)."""
    _fields_ = [
        ("variant", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("freeze_precisions", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("inner_max_iter", ctypes.c_int),
        ("max_refine", ctypes.c_int),
        ("gamma_mode", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("lanes", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("reuse_precisions", ctypes.c_int),
        ("multi_split", ctypes.c_int),
        ("prec_stop_log2", ctypes.c_int),
        ("multi_mode", ctypes.c_int),
        ("overlap_precision", ctypes.c_int),
        ("device_loop", ctypes.c_int),
        ("schedule", ctypes.c_int),
        ("fix_single_loop", ctypes.c_int),
        ("accel", ctypes.c_int),
        ("unroll", ctypes.c_int),
        ("history", ctypes.c_int),
        ("fix_step", ctypes.c_double),
        ("warm_start", ctypes.c_int),
        ("initial_guess", ctypes.c_int),
        ("graphs", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class Profile(ctypes.Structure):
    """Mirror of ``gabp_profile``."""
    _fields_ = [("ms", ctypes.c_double * 6), ("rounds", ctypes.c_int64 * 6), ("launches", ctypes.c_int64)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "gabp_options_default": ([ctypes.POINTER(Options)], ctypes.c_int),
    "gabp_create": ([ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int64, _P, _P, _P, ctypes.c_int, _P,
                     ctypes.POINTER(Options)], ctypes.c_int),
    "gabp_set_values": ([_P, _P, ctypes.c_int], ctypes.c_int),
    "gabp_set_options": ([_P, ctypes.POINTER(Options)], ctypes.c_int),
    "gabp_set_stream": ([_P, _P], ctypes.c_int),
    "gabp_solve": ([_P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                    ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gabp_solve_host": ([_P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                         ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gabp_solve_batched": ([_P, ctypes.c_int32, _P, _P, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_int32), _P], ctypes.c_int),
    "gabp_marginal_precisions": ([_P, _P], ctypes.c_int),
    "gabp_get_messages": ([_P, _P, _P], ctypes.c_int),
    "gabp_grad_values": ([_P, _P, _P, _P], ctypes.c_int),
    "gabp_last_stats": ([_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "gabp_last_freeze": ([_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "gabp_solve_systems": ([_P, ctypes.c_int32, _P, _P, _P, ctypes.c_double, ctypes.c_int32, _P, _P, _P],
                           ctypes.c_int),
    "gabp_profile_read": ([_P, ctypes.POINTER(Profile), ctypes.c_int], ctypes.c_int),
    "gabp_solve_noalloc": ([ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int32,
                            _P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gabp_tuned_shapes": ([_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "gabp_serial_colours": ([_P, _P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "gabp_residual_history": ([_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "gabp_set_messages": ([_P, _P, _P], ctypes.c_int),
    "gabp_create_lsq": ([ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P, _P,
                         ctypes.c_double, ctypes.c_int, _P, ctypes.POINTER(Options)], ctypes.c_int),
    "gabp_solve_lsq": ([_P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gabp_create_dense": ([ctypes.POINTER(_P), ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_int, _P,
                           ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "gabp_destroy": ([_P], ctypes.c_int),
    "gabp_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gabp_last_error": ([], ctypes.c_char_p),
}


def _load():
    if not os.path.exists(library_path):
        raise ImportError(
            f"{library_path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()' or python paper_0811_2518_gb300/build.py)")
    L = ctypes.CDLL(library_path)
    for name, (args, res) in _SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def exported_symbols():
    """Names of every C entry point the binding declares (all must be exported)."""
    return list(_SIGNATURES)


class GaBPError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = gabp_status_string(status)
        err = gabp_last_error()
        super().__init__(f"{where}: {msg} ({status})" + (f" -- {err}" if err else ""))


# ----------------------------------------------------------------------------- C names
def gabp_options_default() -> Options:
    o = Options()
    lib.gabp_options_default(ctypes.byref(o))
    return o


def gabp_create(n, nnz, rowptr_ptr, col_ptr, val_ptr, mem_space, stream_ptr, options=None):
    """Returns (status, handle)."""
    h = _P()
    st = lib.gabp_create(ctypes.byref(h), int(n), int(nnz), _P(rowptr_ptr), _P(col_ptr), _P(val_ptr),
                         int(mem_space), _P(stream_ptr), ctypes.byref(options) if options is not None else None)
    return st, h


def gabp_create_dense(n, a_ptr, lda, mem_space, stream_ptr, options=None):
    """Handle for a dense symmetric n x n matrix (row-major, leading dimension lda); returns
    (status, handle, nnz kept)."""
    h, nnz = _P(), ctypes.c_int64(0)
    st = lib.gabp_create_dense(ctypes.byref(h), int(n), _P(a_ptr), int(lda), int(mem_space), _P(stream_ptr),
                               ctypes.byref(options) if options is not None else None, ctypes.byref(nnz))
    return st, h, nnz.value


def gabp_create_lsq(m, k, nnz, rowptr_ptr, col_ptr, val_ptr, gamma, mem_space, stream_ptr, options=None):
    """Least-squares handle for the m x k CSR J (augmented system [[I, J^T], [J, -gamma I]]);
    returns (status, handle)."""
    h = _P()
    st = lib.gabp_create_lsq(ctypes.byref(h), int(m), int(k), int(nnz), _P(rowptr_ptr), _P(col_ptr), _P(val_ptr),
                             float(gamma), int(mem_space), _P(stream_ptr),
                             ctypes.byref(options) if options is not None else None)
    return st, h


def gabp_solve_lsq(h, y_ptr, x_ptr, z_ptr, tol, max_iter):
    """x = (J^T J + gamma I)^{-1} J^T y on a least-squares handle (device arrays; z_ptr may be None);
    returns (status, iters, relres)."""
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = lib.gabp_solve_lsq(h, _P(y_ptr), _P(x_ptr), _P(z_ptr) if z_ptr else None, float(tol), int(max_iter),
                            ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def gabp_serial_colours(h, colour_ptr):
    """Colouring of the serial schedule into a device int32[n] array (pointer or None);
    returns (status, number of colours)."""
    nc = ctypes.c_int32(0)
    st = lib.gabp_serial_colours(h, colour_ptr, ctypes.byref(nc))
    return st, nc.value


def gabp_set_messages(h, P_ptr, hm_ptr):
    """Loads FP64 messages (input CSR layout, device arrays of nnz doubles) as the warm-start state."""
    return lib.gabp_set_messages(h, _P(P_ptr), _P(hm_ptr))


def gabp_residual_history(h, relres_ptr, cap):
    """Copies up to cap relative residuals of the last FP64 solve into a host float64 array;
    returns (status, entries recorded)."""
    c = ctypes.c_int32(0)
    st = lib.gabp_residual_history(h, relres_ptr, int(cap), ctypes.byref(c))
    return st, c.value


def gabp_set_values(h, val_ptr, mem_space):
    """New values on the handle's sparsity pattern (pointer to nnz doubles; mem_space 0 host, 1 device)."""
    return lib.gabp_set_values(h, val_ptr, mem_space)


def gabp_set_options(h, options):
    return lib.gabp_set_options(h, ctypes.byref(options))


def gabp_set_stream(h, stream_ptr):
    return lib.gabp_set_stream(h, _P(stream_ptr))


def _solve(fn, h, b_ptr, x_ptr, tol, max_iter):
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = fn(h, _P(b_ptr), _P(x_ptr), float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def gabp_solve(h, b_ptr, x_ptr, tol, max_iter):
    """Returns (status, iters, relres)."""
    return _solve(lib.gabp_solve, h, b_ptr, x_ptr, tol, max_iter)


def gabp_solve_host(h, b_ptr, x_ptr, tol, max_iter):
    return _solve(lib.gabp_solve_host, h, b_ptr, x_ptr, tol, max_iter)


def gabp_solve_batched(h, nrhs, B_ptr, X_ptr, ld, tol, max_iter, relres_host_ptr=None):
    it = ctypes.c_int32(0)
    st = lib.gabp_solve_batched(h, int(nrhs), _P(B_ptr), _P(X_ptr), int(ld), float(tol), int(max_iter),
                                ctypes.byref(it), _P(relres_host_ptr) if relres_host_ptr else None)
    return st, it.value


def gabp_marginal_precisions(h, Pi_ptr):
    return lib.gabp_marginal_precisions(h, _P(Pi_ptr))


def gabp_get_messages(h, P_ptr, hm_ptr):
    return lib.gabp_get_messages(h, _P(P_ptr), _P(hm_ptr))


def gabp_grad_values(h, lam_ptr, x_ptr, g_ptr):
    return lib.gabp_grad_values(h, _P(lam_ptr), _P(x_ptr), _P(g_ptr))


def gabp_last_stats(h):
    """Returns (status, rounds, num_edges, edge_updates, refine_steps)."""
    r, e, u, s = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
    st = lib.gabp_last_stats(h, ctypes.byref(r), ctypes.byref(e), ctypes.byref(u), ctypes.byref(s))
    return st, r.value, e.value, u.value, s.value


def gabp_last_freeze(h):
    """Returns (status, round whose precisions the last FP64 solve froze or 0, verification rounds)."""
    r, c = ctypes.c_int32(0), ctypes.c_int32(0)
    st = lib.gabp_last_freeze(h, ctypes.byref(r), ctypes.byref(c))
    return st, r.value, c.value


def gabp_solve_systems(h, nsys, offsets_host_ptr, b_ptr, x_ptr, tol, max_iter, status_ptr=None, iters_ptr=None,
                       relres_ptr=None):
    return lib.gabp_solve_systems(h, int(nsys), _P(offsets_host_ptr), _P(b_ptr), _P(x_ptr), float(tol),
                                  int(max_iter), _P(status_ptr), _P(iters_ptr), _P(relres_ptr))


def gabp_profile_read(h, reset=False):
    """Returns (status, dict) with per-phase ms / rounds and the launch count."""
    p = Profile()
    st = lib.gabp_profile_read(h, ctypes.byref(p), 1 if reset else 0)
    names = ("fp64", "prec32", "mean32", "refine64", "multi", "freeze32")
    return st, {"ms": dict(zip(names, list(p.ms))), "rounds": dict(zip(names, list(p.rounds))),
                "launches": p.launches}


def gabp_solve_noalloc(n, nnz, rowptr_ptr, col_ptr, val_ptr, b_ptr, x_ptr, tol, max_iter, stream_ptr):
    """Allocation-free FP64 solve of a small system (device arrays); returns (status, iters, relres)."""
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = lib.gabp_solve_noalloc(int(n), int(nnz), _P(rowptr_ptr), _P(col_ptr), _P(val_ptr), _P(b_ptr), _P(x_ptr),
                                float(tol), int(max_iter), _P(stream_ptr), ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def gabp_tuned_shapes(h):
    """Returns dict of the autotuner's choices: fp64 lanes, (lanes, unroll) of the FP32 kernels, multi-system
    split and kernel (1 grid-persistent, 2 teams), the grid-persistent kernel's (lanes, unroll) and whether
    it runs on the sliced layout."""
    a, b, c, d, e = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int32(0)
    lib.gabp_tuned_shapes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d), ctypes.byref(e))
    sh = lambda v: (v & 0xFF, v >> 8)
    return {"fp64_lanes": a.value, "prec32": sh(b.value), "mean32": sh(c.value), "multi_split": d.value,
            "multi_mode": e.value & 0xFF, "multi_grid": ((e.value >> 8) & 0xFF, (e.value >> 16) & 0xFF),
            "multi_grid_sliced": bool((e.value >> 24) & 1)}


def gabp_destroy(h):
    return lib.gabp_destroy(h)


def gabp_status_string(s) -> str:
    return lib.gabp_status_string(int(s)).decode()


def gabp_last_error() -> str:
    v = lib.gabp_last_error()
    return v.decode() if v else ""


# ----------------------------------------------------------------------------- torch convenience
def _check_out(t, shape, device, name):
    """An output tensor the library writes through its raw pointer: float64, contiguous, on the
    solver's device, of the expected shape (anything else would be written out of bounds)."""
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous() \
            or t.device != device or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of shape {tuple(shape)} on {device}")


def _check_host(a, n, name):
    import numpy as np

    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != n:
        raise ValueError(f"{name} must be a C-contiguous float64 numpy array of {n} entries")


class Solver:
    """A GaBP solver bound to one symmetric matrix A (full CSR, diagonal included).

    ``rowptr``/``col``/``val`` may be numpy arrays (host) or CUDA tensors
    (int32/int32/float64).  Solves take and return CUDA float64 tensors and run
    on ``stream`` (default: torch's current stream at construction; when that is
    the default stream, the library runs on a stream of its own, ordered after
    the default stream's pending work, so that its rounds can replay CUDA graphs).
    Every call returns with its results complete.
    """

    def __init__(self, n, rowptr, col, val, options: Options | None = None, stream=None, **opts):
        import numpy as np
        import torch

        self.n = int(n)
        self.options = options if options is not None else gabp_options_default()
        for k, v in opts.items():
            setattr(self.options, k, v)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = []
        if isinstance(rowptr, torch.Tensor):
            rp = rowptr.to(self.device, torch.int32).contiguous()
            cl = col.to(self.device, torch.int32).contiguous()
            vl = val.to(self.device, torch.float64).contiguous()
            self._keep += [rp, cl, vl]
            ptrs, mem = (rp.data_ptr(), cl.data_ptr(), vl.data_ptr()), 1
            nnz = int(cl.numel())
        else:
            rp = np.ascontiguousarray(rowptr, dtype=np.int32)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            vl = np.ascontiguousarray(val, dtype=np.float64)
            self._keep += [rp, cl, vl]
            ptrs, mem = (rp.ctypes.data, cl.ctypes.data, vl.ctypes.data), 0
            nnz = int(cl.size)
        self.nnz = nnz
        st, h = gabp_create(self.n, nnz, *ptrs, mem, self.stream.cuda_stream, self.options)
        self._keep = []
        if st != GABP_OK:
            raise GaBPError(st, "gabp_create")
        self.handle = h

    @classmethod
    def from_dense(cls, A, options: Options | None = None, stream=None, **opts):
        """Solver for a dense symmetric matrix (numpy array or CUDA float64 tensor, rows
        contiguous): ``gabp_create_dense`` keeps its nonzero entries in the row-CSR the
        broadcast rounds use."""
        import numpy as np
        import torch

        self = cls.__new__(cls)
        self.options = options if options is not None else gabp_options_default()
        for k, v in opts.items():
            setattr(self.options, k, v)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if isinstance(A, torch.Tensor):
            a = A.to(self.device, torch.float64)
            if a.dim() != 2 or a.shape[0] != a.shape[1] or a.stride(1) != 1:
                a = a.contiguous()
            ptr, lda, mem = a.data_ptr(), a.stride(0), 1
        else:
            a = np.asarray(A, dtype=np.float64)
            if a.ndim != 2 or a.shape[0] != a.shape[1] or a.strides[1] != 8:
                a = np.ascontiguousarray(a)
            ptr, lda, mem = a.ctypes.data, a.strides[0] // 8, 0
        if a.ndim != 2 or a.shape[0] != a.shape[1]:
            raise ValueError("A must be a square matrix")
        self.n = int(a.shape[0])
        self._keep = [a]
        st, h, nnz = gabp_create_dense(self.n, ptr, lda, mem, self.stream.cuda_stream, self.options)
        self._keep = []
        if st != GABP_OK:
            raise GaBPError(st, "gabp_create_dense")
        self.handle, self.nnz = h, nnz
        return self

    @classmethod
    def from_csr(cls, m, **kw):
        return cls(m.n, m.rowptr, m.col, m.val, **kw)

    def serial_colours(self):
        """(colour tensor int32[n] on the device, number of colours) of the serial schedule."""
        import torch

        c = torch.empty(self.n, dtype=torch.int32, device=self.device)
        st, nc = gabp_serial_colours(self.handle, c.data_ptr())
        if st != GABP_OK:
            raise GaBPError(st, "gabp_serial_colours")
        return c, nc

    def set_values(self, val):
        """New values (full CSR order, diagonal included) on the same pattern: a numpy array or a
        CUDA float64 tensor.  Raises GaBPError (and leaves the solver unusable) if they are invalid."""
        import numpy as np
        import torch

        if isinstance(val, torch.Tensor):
            v = val.detach().to(self.device, torch.float64).contiguous()
            if v.numel() != self.nnz:
                raise ValueError(f"{v.numel()} values for {self.nnz} stored entries")
            st = gabp_set_values(self.handle, v.data_ptr(), 1)
        else:
            v = np.ascontiguousarray(val, dtype=np.float64)
            if v.size != self.nnz:
                raise ValueError(f"{v.size} values for {self.nnz} stored entries")
            st = gabp_set_values(self.handle, v.ctypes.data, 0)
        if st != GABP_OK:
            raise GaBPError(st, "gabp_set_values")
        self.values_version = getattr(self, "values_version", 0) + 1

    def set_options(self, **opts):
        for k, v in opts.items():
            setattr(self.options, k, v)
        st = gabp_set_options(self.handle, self.options)
        if st != GABP_OK:
            raise GaBPError(st, "gabp_set_options")

    def solve(self, b, tol=1e-12, max_iter=1000, x=None, check=True):
        """x = A^{-1} b.  Returns (x, status, iters, relres).  With the option initial_guess=1, x
        (required then) holds the initial iterate on entry."""
        import torch

        b = b.to(self.device, torch.float64).contiguous()
        if b.numel() != self.n:
            raise ValueError(f"b has {b.numel()} entries, the matrix {self.n} rows")
        if x is None:
            if self.options.initial_guess:
                raise ValueError("initial_guess=1: pass the initial iterate as x")
            x = torch.empty_like(b)
        _check_out(x, b.shape, self.device, "x")
        st, it, rel = gabp_solve(self.handle, b.data_ptr(), x.data_ptr(), tol, max_iter)
        if check and st < 0:
            raise GaBPError(st, "gabp_solve")
        return x, st, it, rel

    def solve_host(self, b, x, tol=1e-12, max_iter=1000):
        """b, x: host numpy float64 arrays (pinned or pageable)."""
        _check_host(b, self.n, "b")
        _check_host(x, self.n, "x")
        st, it, rel = gabp_solve_host(self.handle, b.ctypes.data, x.ctypes.data, tol, max_iter)
        if st < 0:
            raise GaBPError(st, "gabp_solve_host")
        return st, it, rel

    def solve_batched(self, B, tol=1e-10, max_iter=5000, X=None, check=True):
        """Solve A X_r = B_r for every row r of the CUDA tensor B [R, n] (FP32 messages,
        FP64 refinement, shared precision messages).  Returns (X, status, inner_rounds, relres[R])."""
        import numpy as np
        import torch

        B = B.to(self.device, torch.float64).contiguous()
        if B.dim() != 2 or B.shape[1] != self.n:
            raise ValueError("B must be [R, n]")
        if X is None:
            X = torch.empty_like(B)
        _check_out(X, B.shape, self.device, "X")
        rel = np.zeros(B.shape[0])
        st, it = gabp_solve_batched(self.handle, B.shape[0], B.data_ptr(), X.data_ptr(), self.n, tol, max_iter,
                                    rel.ctypes.data)
        if check and st < 0:
            raise GaBPError(st, "gabp_solve_batched")
        return X, st, it, rel

    def marginal_precisions(self):
        import torch

        P = torch.empty(self.n, dtype=torch.float64, device=self.device)
        st = gabp_marginal_precisions(self.handle, P.data_ptr())
        if st != GABP_OK:
            raise GaBPError(st, "gabp_marginal_precisions")
        return P

    def messages(self):
        """(P, h) per input CSR slot: message col -> row of the last FP64 solve."""
        import torch

        P = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        hm = torch.empty_like(P)
        st = gabp_get_messages(self.handle, P.data_ptr(), hm.data_ptr())
        if st != GABP_OK:
            raise GaBPError(st, "gabp_get_messages")
        return P, hm

    def set_messages(self, P, hm):
        """Loads messages in the layout ``messages()`` returns (CUDA float64 tensors of nnz entries)
        as the state a solve with ``warm_start=1`` starts from: a checkpoint restored."""
        _check_out(P, (self.nnz,), self.device, "P")
        _check_out(hm, (self.nnz,), self.device, "hm")
        st = gabp_set_messages(self.handle, P.data_ptr(), hm.data_ptr())
        if st != GABP_OK:
            raise GaBPError(st, "gabp_set_messages")

    def grad_values(self, lam, x):
        import torch

        _check_out(lam, (self.n,), self.device, "lam")
        _check_out(x, (self.n,), self.device, "x")
        g = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        st = gabp_grad_values(self.handle, lam.data_ptr(), x.data_ptr(), g.data_ptr())
        if st != GABP_OK:
            raise GaBPError(st, "gabp_grad_values")
        return g

    def stats(self):
        st, rounds, E, eu, steps = gabp_last_stats(self.handle)
        return {"rounds": rounds, "edges": E, "edge_updates": eu, "refine_steps": steps,
                "freeze_round": gabp_last_freeze(self.handle)[1], "freeze_checks": gabp_last_freeze(self.handle)[2]}

    def solve_systems(self, b, offsets, tol=1e-10, max_iter=5000, x=None, check=True):
        """Independent systems of a block-diagonal A (row offsets ``offsets``, host ints) in one
        persistent launch.  Returns (x, worst status, per-system status, rounds, relres)."""
        import numpy as np
        import torch

        b = b.to(self.device, torch.float64).contiguous()
        if b.numel() != self.n:
            raise ValueError(f"b has {b.numel()} entries, the matrix {self.n} rows")
        if x is None:
            x = torch.empty_like(b)
        _check_out(x, b.shape, self.device, "x")
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        ns = off.size - 1
        sts = np.zeros(ns, dtype=np.int32)
        its = np.zeros(ns, dtype=np.int32)
        rel = np.zeros(ns)
        st = gabp_solve_systems(self.handle, ns, off.ctypes.data, b.data_ptr(), x.data_ptr(), tol, max_iter,
                                sts.ctypes.data, its.ctypes.data, rel.ctypes.data)
        if check and st < 0:
            raise GaBPError(st, "gabp_solve_systems")
        return x, st, sts, its, rel

    def tuned(self):
        return gabp_tuned_shapes(self.handle)

    def residual_history(self):
        """Relative residual of every recorded iterate of the last FP64 solve (numpy array; empty
        unless the solver was created with history > 0)."""
        import numpy as np

        st, cnt = gabp_residual_history(self.handle, None, 0)
        if st != GABP_OK:
            raise GaBPError(st, "gabp_residual_history")
        out = np.zeros(cnt)
        if cnt:
            st, cnt = gabp_residual_history(self.handle, out.ctypes.data, cnt)
            if st != GABP_OK:
                raise GaBPError(st, "gabp_residual_history")
        return out

    def profile(self, reset=False):
        st, p = gabp_profile_read(self.handle, reset)
        return p

    def close(self):
        if getattr(self, "handle", None):
            gabp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LSQSolver(Solver):
    """Regularised least squares x = (J^T J + gamma I)^{-1} J^T y for a rectangular sparse J
    (m x k CSR: numpy arrays or CUDA tensors), through the symmetric augmented system
    [[I, J^T], [J, -gamma I]] (``gabp_create_lsq``).  ``solve`` / ``solve_batched`` of the base
    class act on the augmented system of n = k + m unknowns; ``solve_lsq`` takes y and returns x."""

    def __init__(self, m, k, rowptr, col, val, gamma, options: Options | None = None, stream=None, **opts):
        import numpy as np
        import torch

        self.m, self.k, self.gamma = int(m), int(k), float(gamma)
        self.n = self.k + self.m
        self.options = options if options is not None else gabp_options_default()
        for key, v in opts.items():
            setattr(self.options, key, v)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if isinstance(rowptr, torch.Tensor):
            keep = [rowptr.to(self.device, torch.int32).contiguous(), col.to(self.device, torch.int32).contiguous(),
                    val.to(self.device, torch.float64).contiguous()]
            ptrs, mem = tuple(t.data_ptr() for t in keep), 1
        else:
            keep = [np.ascontiguousarray(rowptr, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32),
                    np.ascontiguousarray(val, dtype=np.float64)]
            ptrs, mem = tuple(a.ctypes.data for a in keep), 0
        if keep[0].shape[0] != self.m + 1 or keep[1].shape[0] != keep[2].shape[0]:
            raise ValueError("J must be a CSR of m rows: rowptr[m+1], col[nnz], val[nnz]")
        self.nnz_j = int(keep[1].shape[0])
        st, h = gabp_create_lsq(self.m, self.k, self.nnz_j, *ptrs, self.gamma, mem, self.stream.cuda_stream,
                                self.options)
        if st != GABP_OK:
            raise GaBPError(st, "gabp_create_lsq")
        self.handle = h

    @classmethod
    def from_rect(cls, J, gamma, **kw):
        return cls(J.m, J.k, J.rowptr, J.col, J.val, gamma, **kw)

    def solve_lsq(self, y, tol=1e-12, max_iter=1000, want_z=False, check=True):
        """x = (J^T J + gamma I)^{-1} J^T y.  Returns (x, z or None, status, iters, relres)."""
        import torch

        y = y.to(self.device, torch.float64).contiguous()
        if y.numel() != self.m:
            raise ValueError(f"y has {y.numel()} entries, J {self.m} rows")
        x = torch.empty(self.k, dtype=torch.float64, device=self.device)
        z = torch.empty(self.m, dtype=torch.float64, device=self.device) if want_z else None
        st, it, rel = gabp_solve_lsq(self.handle, y.data_ptr(), x.data_ptr(), z.data_ptr() if want_z else None,
                                     tol, max_iter)
        if check and st < 0:
            raise GaBPError(st, "gabp_solve_lsq")
        return x, z, st, it, rel
