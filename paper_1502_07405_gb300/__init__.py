"""GB300 (sm_103a) HSS-structured multifrontal sparse solver.

Thin Python binding of the C ABI declared in include/hssmf.h: argument
marshalling only, every step of the factorization and solve runs in the
CUDA kernels of libhssmf.so.  Importing this package loads the library and
fails loudly if it has not been built (``python -m
paper_1502_07405_gb300.build`` or ``__graft_entry__.build()``).

Matrix values, right-hand sides and solutions may be numpy arrays (host) or
CUDA torch tensors (device); device tensors are used in place on the
solver's stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhssmf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -m paper_1502_07405_gb300.build)")

lib = C.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_CUDA, ERR_SINGULAR, ERR_NOCONV, ERR_OOM, ERR_TIMEOUT = range(7)
PREC_FP64, PREC_FP32 = 0, 1
_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_SINGULAR", 4: "ERR_NOCONV",
           5: "ERR_OOM", 6: "ERR_TIMEOUT"}


class Options(C.Structure):
    _fields_ = [("hss_tol", C.c_double), ("d0", C.c_int), ("dd", C.c_int),
                ("oversample_p", C.c_int), ("hss_min_front", C.c_int), ("hss_leaf", C.c_int),
                ("nd_leaf", C.c_int), ("seed", C.c_uint64), ("precision", C.c_int),
                ("gmres_restart", C.c_int), ("maxit", C.c_int), ("rtol", C.c_double)]

    @classmethod
    def defaults(cls, **kw):
        o = cls()
        lib.hssmf_default_opts(C.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise AttributeError(k)
            setattr(o, k, v)
        return o

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("n", C.c_int), ("n_fronts", C.c_int), ("n_levels", C.c_int),
                ("n_hss_fronts", C.c_int), ("max_front", C.c_int), ("max_rank", C.c_int),
                ("max_d", C.c_int), ("adaptive_rounds", C.c_int), ("iterations", C.c_int),
                ("relres", C.c_double), ("factor_flops", C.c_double),
                ("factor_bytes", C.c_double), ("t_analyze_ms", C.c_double),
                ("t_factor_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("gpu_launches", C.c_int), ("id_launches", C.c_int), ("id_bytes", C.c_double),
                ("id_flops", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_I = C.c_int
_IP = C.POINTER(C.c_int)
lib.hssmf_default_opts.argtypes = [C.POINTER(Options)]
lib.hssmf_default_opts.restype = None
lib.hssmf_create.argtypes = [C.POINTER(_P), C.POINTER(Options), _P]
lib.hssmf_analyze_grid.argtypes = [_P, _I, _I, _I, _I, _IP, _IP]
lib.hssmf_analyze_grids.argtypes = [_P, _I, _IP, _I, _IP, _IP]
lib.hssmf_analyze_csr.argtypes = [_P, _I, _IP, _IP, _I, _IP, _IP, _IP]
lib.hssmf_factor.argtypes = [_P, _P]
lib.hssmf_solve.argtypes = [_P, _P, _P, _I, _I]
lib.hssmf_solve_T.argtypes = [_P, _P, _P, _I, _I]
lib.hssmf_get_stats.argtypes = [_P, C.POINTER(Stats)]
lib.hssmf_get_symbolic.argtypes = [_P, _IP, _IP, _IP, _IP, _IP]
lib.hssmf_get_upd.argtypes = [_P, _I, _IP]
lib.hssmf_get_phase_times.argtypes = [_P, C.POINTER(C.c_double), _I]
lib.hssmf_set_profiling.argtypes = [_P, _I]
lib.hssmf_get_id_trace.argtypes = [_P, _IP, _I]
lib.hssmf_pattern_grad.argtypes = [_P, _P, _P, _I, _I, _P]
lib.hssmf_pattern_grad.restype = C.c_int
lib.hssmf_get_id_trace.restype = C.c_int
lib.hssmf_get_id_launch_trace.argtypes = [_P, C.POINTER(C.c_double), _I]
lib.hssmf_get_id_launch_trace.restype = C.c_int
lib.hssmf_set_autotune.argtypes = [_P, _I]
lib.hssmf_set_autotune.restype = C.c_int
lib.hssmf_get_tuning.argtypes = [_P, _IP, _I]
lib.hssmf_get_tuning.restype = C.c_int
lib.hssmf_last_error.argtypes = [_P]
lib.hssmf_last_error.restype = C.c_char_p
lib.hssmf_destroy.argtypes = [_P]
lib.hssmf_destroy.restype = None
for _f in ("hssmf_create", "hssmf_analyze_grid", "hssmf_analyze_grids", "hssmf_analyze_csr", "hssmf_factor", "hssmf_solve", "hssmf_solve_T",
           "hssmf_get_stats", "hssmf_get_symbolic", "hssmf_get_upd", "hssmf_get_phase_times",
           "hssmf_set_profiling"):
    getattr(lib, _f).restype = C.c_int


class HssmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _int_ptr(a):
    return a.ctypes.data_as(_IP)


def _buf(x, writable=False):
    """(pointer, keep-alive) of a numpy array or a torch tensor (fp64)."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float64:
            raise TypeError("values, B and X must be float64")
        if not x.is_contiguous() and not x.t().is_contiguous():
            raise ValueError("tensors must be contiguous (column-major for 2-D: pass X.t())")
        return C.c_void_p(x.data_ptr()), x
    a = np.asarray(x)
    if a.dtype != np.float64:
        raise TypeError("values, B and X must be float64")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return C.c_void_p(a.ctypes.data), a


class Solver:
    """One hssmf context: analyze_grid -> factor -> solve / solve_T."""

    def __init__(self, opts: Options | None = None, stream=None, **kw):
        self.opts = opts if opts is not None else Options.defaults(**kw)
        self._h = C.c_void_p()
        s = C.c_void_p(0 if stream is None else int(stream))
        self._check(lib.hssmf_create(C.byref(self._h), C.byref(self.opts), s), ctx=False)
        self.n = 0
        self.nnz = 0
        self.factorizations = 0  # factor() calls made (the autograd wrapper checks it)

    def _check(self, st, ctx=True):
        if st != OK:
            msg = lib.hssmf_last_error(self._h).decode() if ctx and self._h else ""
            raise HssmfError(st, msg)

    def close(self):
        if self._h:
            lib.hssmf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def analyze_grid(self, dims, rowptr, colind):
        nx, ny, nz = (list(dims) + [1, 1])[:3]
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colind, dtype=np.int32)
        n = len(rp) - 1
        self._check(lib.hssmf_analyze_grid(self._h, nx, ny, nz, n, _int_ptr(rp), _int_ptr(ci)))
        self.n = n
        self.nnz = int(rp[-1])

    def analyze_grids(self, dims_list, rowptr, colind):
        """Several independent grids as one block-diagonal system (grid s
        owns the natural indices after grids 0..s-1)."""
        dims = np.ascontiguousarray([(list(d) + [1, 1])[:3] for d in dims_list], dtype=np.int32).reshape(-1)
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colind, dtype=np.int32)
        n = len(rp) - 1
        self._check(lib.hssmf_analyze_grids(self._h, len(dims_list), _int_ptr(dims), n, _int_ptr(rp),
                                            _int_ptr(ci)))
        self.n = n
        self.nnz = int(rp[-1])

    def analyze_csr(self, rowptr, colind, perm=None, sep_ptr=None, parent=None):
        """A general structurally symmetric pattern: algebraic nested
        dissection when perm is None, else the caller's ordering
        (perm[new] = old) and separator tree (sep_ptr, parent)."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colind, dtype=np.int32)
        n = len(rp) - 1
        if perm is None:
            st = lib.hssmf_analyze_csr(self._h, n, _int_ptr(rp), _int_ptr(ci), 0, None, None, None)
        else:
            pm = np.ascontiguousarray(perm, dtype=np.int32)
            sp = np.ascontiguousarray(sep_ptr, dtype=np.int32)
            pa = np.ascontiguousarray(parent, dtype=np.int32)
            st = lib.hssmf_analyze_csr(self._h, n, _int_ptr(rp), _int_ptr(ci), len(pa), _int_ptr(pm),
                                       _int_ptr(sp), _int_ptr(pa))
        self._check(st)
        self.n = n
        self.nnz = int(rp[-1])

    def factor(self, values):
        p, keep = _buf(values)
        self.factorizations += 1  # counted even if it fails: the old factors are gone
        self._check(lib.hssmf_factor(self._h, p))

    def _solve(self, fn, B, X, nrhs, ldb):
        pb, kb = _buf(B)
        px, kx = _buf(X, writable=True)
        self._check(fn(self._h, pb, px, int(nrhs), int(ldb)))
        return X

    def solve(self, B, X=None):
        """Solve A X = B.  B: (n,) or column-major (n, nrhs) numpy array, or a
        CUDA float64 tensor laid out column-major (e.g. an (nrhs, n) tensor
        viewed as its transpose)."""
        return self._solve_any(lib.hssmf_solve, B, X)

    def solve_T(self, B, X=None):
        return self._solve_any(lib.hssmf_solve_T, B, X)

    def _solve_any(self, fn, B, X):
        try:
            import torch
            is_t = isinstance(B, torch.Tensor)
        except ImportError:  # pragma: no cover
            is_t = False
        if is_t:
            nrhs = 1 if B.dim() == 1 else B.shape[1]
            if X is None:
                X = torch.empty_like(B)
            return self._solve(fn, B, X, nrhs, self.n)
        Bn = np.asfortranarray(B, dtype=np.float64)
        nrhs = 1 if Bn.ndim == 1 else Bn.shape[1]
        if X is None:
            X = np.zeros_like(Bn, order="F")
        return self._solve(fn, Bn, X, nrhs, self.n)

    def get_stats(self):
        s = Stats()
        self._check(lib.hssmf_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    PHASES = ("dense", "sample", "extract", "pre_id", "id", "post_id", "ulv", "schur", "solve",
              "outer", "id_kernels")

    def set_profiling(self, on=True):
        self._check(lib.hssmf_set_profiling(self._h, int(bool(on))))

    def get_phase_times(self):
        buf = (C.c_double * len(self.PHASES))()
        self._check(lib.hssmf_get_phase_times(self._h, buf, len(self.PHASES)))
        return dict(zip(self.PHASES, list(buf)))

    def pattern_grad(self, lam, x, out):
        """out[p] = -sum_c lam[row(p), c] x[col(p), c] on the CSR pattern (CUDA
        float64 tensors; lam and x column-major n x nrhs, out of length nnz)."""
        nrhs = 1 if lam.dim() == 1 else lam.shape[1]
        self._check(lib.hssmf_pattern_grad(self._h, C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()),
                                           int(nrhs), int(self.n), C.c_void_p(out.data_ptr())))
        return out

    ID_TRACE_FIELDS = ("front", "node", "round", "d", "m", "mc", "kr", "kc", "accepted", "kernel_r",
                       "kernel_c")

    def get_id_trace(self):
        """Per-node ID records of the last profiled factorization, an
        (records x 11) int array with columns ID_TRACE_FIELDS (kernel codes:
        100 * family + CTAs per ID; family 0 one CTA in L2, 1 shared memory,
        2 registers, 3 L2 cluster, 4 registers with one exchange per step)."""
        n = lib.hssmf_get_id_trace(self._h, None, 0)
        buf = np.zeros((max(n, 0), len(self.ID_TRACE_FIELDS)), dtype=np.int32)
        if n > 0:
            lib.hssmf_get_id_trace(self._h, _int_ptr(buf), n)
        return buf

    TUNING_FIELDS = ("dense_fronts", "panel_fronts", "bound", "threads", "tuned", "us")

    def set_autotune(self, on=True):
        self._check(lib.hssmf_set_autotune(self._h, int(bool(on))))

    def get_tuning(self):
        """Per-level split of the dense fronts between the panel path and the
        persistent kernel, a (levels x 6) int array with columns
        TUNING_FIELDS."""
        n = lib.hssmf_get_tuning(self._h, None, 0)
        buf = np.zeros((max(n, 0), 6), dtype=np.int32)
        if n > 0:
            lib.hssmf_get_tuning(self._h, _int_ptr(buf), n)
        return buf

    ID_LAUNCH_FIELDS = ("kernel", "ctas", "jobs", "max_d", "max_m", "ms")

    def get_id_launch_trace(self):
        """Per-launch records of the ID kernels of the last profiled
        factorization, a (launches x 6) float array with columns
        ID_LAUNCH_FIELDS."""
        n = lib.hssmf_get_id_launch_trace(self._h, None, 0)
        buf = np.zeros((max(n, 0), 6), dtype=np.float64)
        if n > 0:
            lib.hssmf_get_id_launch_trace(self._h, buf.ctypes.data_as(C.POINTER(C.c_double)), n)
        return buf

    def get_symbolic(self, n_fronts):
        perm = np.zeros(self.n, dtype=np.int32)
        sb, se, par, nu = (np.zeros(n_fronts, dtype=np.int32) for _ in range(4))
        self._check(lib.hssmf_get_symbolic(self._h, _int_ptr(perm), _int_ptr(sb), _int_ptr(se),
                                           _int_ptr(par), _int_ptr(nu)))
        return perm, sb, se, par, nu

    def get_upd(self, f, n_upd):
        out = np.zeros(n_upd, dtype=np.int32)
        self._check(lib.hssmf_get_upd(self._h, int(f), _int_ptr(out)))
        return out
