"""Thin ctypes binding of libamgc (include/amgc.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts NumPy / PyTorch
arguments to pointers and sizes.  Device vectors are torch CUDA tensors (float64); the
stream is torch's current CUDA stream unless one is given.  Importing works without a GPU;
any call that needs the library raises if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libamgc.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "amgc.h")

AMGC_OK, AMGC_EINVAL, AMGC_ESINGULAR, AMGC_NOT_CONVERGED = 0, -1, -2, -3
AMGC_BREAKDOWN, AMGC_TIMEOUT, AMGC_ECUDA, AMGC_ENOMEM = -4, -5, -6, -7

EXPORT = dict(agg=1, lagg=2, p_rowptr=3, p_col=4, p_val=5, k_rowptr=6, k_col=7, k_val=8, b1_rowptr=9,
              b1_col=10, b1_val=11, b2_rowptr=12, b2_col=13, b2_val=14, z=15, sinv=16, nullspace=17,
              pl_w=18, atinv=19, omega=20, coarse_inv=21, schur_rho=22, color=23)
_EXPORT_DTYPE = {k: (np.int32 if k in ("agg", "lagg", "color") or k.endswith(("rowptr", "col")) else np.float64)
                 for k in EXPORT}


class Bsr(C.Structure):
    _fields_ = [("n_brow", C.c_int32), ("n_bcol", C.c_int32), ("br", C.c_int32), ("bc", C.c_int32),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class Csr(C.Structure):
    _fields_ = [("n_row", C.c_int32), ("n_col", C.c_int32), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("levels_max", C.c_int32), ("coarse_max_rows", C.c_int32), ("transfer", C.c_int32),
                ("smoother_sweeps", C.c_int32), ("jacobi_sweeps", C.c_int32), ("simplec", C.c_int32),
                ("precision", C.c_int32), ("fgmres_restart", C.c_int32), ("fgmres_maxit", C.c_int32),
                ("seed", C.c_uint32), ("sa_omega", C.c_double), ("jacobi_omega", C.c_double),
                ("simple_alpha", C.c_double), ("tol", C.c_double), ("autotune", C.c_int32),
                ("schur_damping", C.c_int32), ("coarse_solver", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("rows", C.c_int32 * 16), ("disp_nodes", C.c_int32 * 16),
                ("lm_nodes", C.c_int32 * 16), ("dofs_per_node", C.c_int32 * 16), ("nnz", C.c_int64 * 16),
                ("operator_complexity", C.c_double), ("lambda_max", C.c_double * 16), ("setup_ms", C.c_double),
                ("last_iters", C.c_int32), ("last_relres", C.c_double), ("setup_phase_ms", C.c_double * 10)]


_lib = None

SETUP_PHASES = ("input_assembly", "aggregation", "lm_aggregation", "tentative_qr", "smoother_lambda_max",
                "smoothed_prolongator", "transpose", "galerkin", "coarsest_inverse", "sell_views")


class AmgcError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        super().__init__(f"{where}: {lib.amgc_strerror(code).decode()} ({code}): {lib.amgc_last_error().decode()}")
        self.code = code


def load():
    """Loads libamgc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"amgc CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.amgc_default_options.argtypes = [C.POINTER(Options)]
    lib.amgc_default_options.restype = None
    lib.amgc_setup.argtypes = [C.POINTER(Bsr), vp, C.POINTER(Csr), vp, vp, vp, vp, vp, vp, C.POINTER(Options), vp,
                               C.POINTER(vp)]
    lib.amgc_setup.restype = C.c_int
    for name in ("amgc_vcycle", "amgc_apply"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp]
        getattr(lib, name).restype = C.c_int
    lib.amgc_solve.argtypes = [vp, vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
    lib.amgc_solve.restype = C.c_int
    lib.amgc_solve_split.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
    lib.amgc_solve_split.restype = C.c_int
    lib.amgc_solve_host.argtypes = [vp, vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
    lib.amgc_solve_host.restype = C.c_int
    lib.amgc_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.amgc_stats.restype = C.c_int
    lib.amgc_export.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int64]
    lib.amgc_export.restype = C.c_int64
    lib.amgc_profile.argtypes = [vp, C.c_int32]
    lib.amgc_profile.restype = C.c_int
    lib.amgc_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
    lib.amgc_profile_read.restype = C.c_int
    for name in ("amgc_vcycle_transposed", "amgc_apply_transposed"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp]
        getattr(lib, name).restype = C.c_int
    lib.amgc_solve_transposed.argtypes = [vp, vp, vp, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
    lib.amgc_solve_transposed.restype = C.c_int
    lib.amgc_grad_scatter.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.amgc_grad_scatter.restype = C.c_int
    lib.amgc_grad_elements.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.amgc_grad_elements.restype = C.c_int
    lib.amgc_setup_batched.argtypes = [C.POINTER(Bsr), vp, C.POINTER(Csr), vp, vp, vp, vp, vp, vp, C.c_int32, vp, vp,
                                       C.POINTER(Options), vp, C.POINTER(vp)]
    lib.amgc_setup_batched.restype = C.c_int
    lib.amgc_solve_batched.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
    lib.amgc_solve_batched.restype = C.c_int
    lib.amgc_grad_elements_noalloc.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.amgc_grad_elements_noalloc.restype = C.c_int
    lib.amgc_set_row_mapping.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    lib.amgc_set_row_mapping.restype = C.c_int
    lib.amgc_set_wait_limit.argtypes = [vp, C.c_int64]
    lib.amgc_set_wait_limit.restype = C.c_int
    lib.amgc_set_smoother.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, C.c_double, vp]
    lib.amgc_set_smoother.restype = C.c_int
    lib.amgc_set_preconditioner.argtypes = [vp, C.c_int32, C.c_int32, C.c_double, vp]
    lib.amgc_set_preconditioner.restype = C.c_int
    lib.amgc_update_active_set.argtypes = [vp, vp, vp]
    lib.amgc_update_active_set.restype = C.c_int
    lib.amgc_pdass.argtypes = [vp, vp, vp, C.c_double, C.c_int32, vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               vp]
    lib.amgc_pdass.restype = C.c_int
    lib.amgc_destroy.argtypes = [vp]
    lib.amgc_destroy.restype = None
    lib.amgc_strerror.argtypes = [C.c_int]
    lib.amgc_strerror.restype = C.c_char_p
    lib.amgc_last_error.argtypes = []
    lib.amgc_last_error.restype = C.c_char_p
    lib.amgc_launch_count.argtypes = []
    lib.amgc_launch_count.restype = C.c_int64
    lib.amgc_trim_memory.argtypes = []
    lib.amgc_trim_memory.restype = C.c_int
    lib.amgc_f64_to_f32.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.amgc_f64_to_f32.restype = C.c_int
    _lib = lib
    return lib


def header_symbols(path: str = HEADER):
    """Names of the functions declared in include/amgc.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amgc_[a-z_]+)\s*\(", txt)))


def launch_count() -> int:
    """Kernels launched by libamgc in this process so far."""
    return int(load().amgc_launch_count())


def trim_memory():
    """Returns the unused device memory of the library's pool on the current device (amgc_trim_memory)."""
    _check(load().amgc_trim_memory(), "amgc_trim_memory")


def f64_to_f32(x, y, stream=None):
    """amgc_f64_to_f32: y = x rounded to FP32 (contiguous CUDA tensors, float64 -> float32)."""
    import torch
    if x.dtype != torch.float64 or y.dtype != torch.float32 or x.numel() != y.numel():
        raise TypeError("f64_to_f32: float64 input and float32 output of one size")
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise TypeError("f64_to_f32: contiguous CUDA tensors")
    _check(load().amgc_f64_to_f32(x.numel(), x.data_ptr(), y.data_ptr(), _stream_ptr(stream)), "amgc_f64_to_f32")


def default_options(**kw) -> Options:
    o = Options()
    load().amgc_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _check(code: int, where: str):
    if code != AMGC_OK:
        raise AmgcError(code, where)


class Hierarchy:
    """Owning handle of an amgc hierarchy (freed on close() or garbage collection)."""

    def __init__(self, handle: int, lib):
        self._h = C.c_void_p(handle)
        self._lib = lib

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h and self._h.value:
            self._lib.amgc_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        st = Stats()
        _check(self._lib.amgc_stats(self._h, C.byref(st)), "amgc_stats")
        n = st.n_levels
        return dict(n_levels=n, rows=list(st.rows[:n]), disp_nodes=list(st.disp_nodes[:n]),
                    lm_nodes=list(st.lm_nodes[:n]), dofs_per_node=list(st.dofs_per_node[:n]),
                    nnz=list(st.nnz[:n]), operator_complexity=st.operator_complexity,
                    lambda_max=list(st.lambda_max[:n]), setup_ms=st.setup_ms, last_iters=st.last_iters,
                    last_relres=st.last_relres, setup_phase_ms=dict(zip(SETUP_PHASES, st.setup_phase_ms)))

    def export(self, level: int, what: str) -> np.ndarray:
        code = EXPORT[what]
        nb = self._lib.amgc_export(self._h, level, code, None, 0)
        if nb < 0:
            raise AmgcError(int(nb), "amgc_export")
        out = np.empty(nb // np.dtype(_EXPORT_DTYPE[what]).itemsize, dtype=_EXPORT_DTYPE[what])
        if nb:
            r = self._lib.amgc_export(self._h, level, code, out.ctypes.data, nb)
            if r < 0:
                raise AmgcError(int(r), "amgc_export")
        return out

    def export_size(self, level: int, what: str) -> int:
        """Number of elements amgc_export would copy (no copy is made)."""
        nb = self._lib.amgc_export(self._h, level, EXPORT[what], None, 0)
        if nb < 0:
            raise AmgcError(int(nb), "amgc_export")
        return int(nb) // np.dtype(_EXPORT_DTYPE[what]).itemsize

    def profile(self, enable=True):
        """enable: True/3 = FP64 and FP32 applies, 1 = FP64 only, 2 = FP32 only, False/0 = off."""
        mask = 3 if enable is True else int(enable)
        _check(self._lib.amgc_profile(self._h, mask), "amgc_profile")

    def profile_read(self):
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        b = C.c_double(0.0)
        f = C.c_double(0.0)
        _check(self._lib.amgc_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(b), C.byref(f)),
               "amgc_profile_read")
        return ms.value, n.value, b.value, f.value

    ROW_MATRIX = dict(K=0, P=1, R=2, fuse=3)

    def set_row_mapping(self, level: int, matrix: str, precision: int, mapping: int):
        """amgc_set_row_mapping: matrix 'K', 'P' or 'R'; mapping -1 default, 0 warp per row,
        1 / 2 SELL threads per row, 3 staged FP32 kernel (level-0 K, precision 32).  matrix 'fuse':
        the level's smoother form, mapping 0 two launches, 1 fused, 2 split, -1 default."""
        _check(self._lib.amgc_set_row_mapping(self._h, int(level), self.ROW_MATRIX[matrix], int(precision),
                                              int(mapping)), "amgc_set_row_mapping")

    def set_wait_limit(self, polls: int):
        """amgc_set_wait_limit: tests per bounded device wait (< 0: the default; 0: every wait gives up)."""
        _check(self._lib.amgc_set_wait_limit(self._h, int(polls)), "amgc_set_wait_limit")

    # ------------------------------------------------------------ device-vector calls
    def vcycle(self, r, z, stream=None):
        _check(self._lib.amgc_vcycle(self._h, _ptr(r), _ptr(z), _stream_ptr(stream)), "amgc_vcycle")
        return z

    def apply(self, x, y, stream=None):
        _check(self._lib.amgc_apply(self._h, _ptr(x), _ptr(y), _stream_ptr(stream)), "amgc_apply")
        return y

    def solve(self, rhs, x, stream=None, check: bool = True):
        it = C.c_int32(0)
        rr = C.c_double(0.0)
        code = self._lib.amgc_solve(self._h, _ptr(rhs), _ptr(x), C.byref(it), C.byref(rr), _stream_ptr(stream))
        if check:
            _check(code, "amgc_solve")
        return it.value, rr.value, code

    def solve_split(self, rhs, u, lam, stream=None, check: bool = True):
        """amgc_solve_split: the solution's displacements into u and multipliers into lam."""
        it = C.c_int32(0)
        rr = C.c_double(0.0)
        code = self._lib.amgc_solve_split(self._h, _ptr(rhs), _ptr(u), _ptr(lam), C.byref(it), C.byref(rr),
                                          _stream_ptr(stream))
        if check:
            _check(code, "amgc_solve_split")
        return it.value, rr.value, code

    def apply_transposed(self, x, y, stream=None):
        _check(self._lib.amgc_apply_transposed(self._h, _ptr(x), _ptr(y), _stream_ptr(stream)),
               "amgc_apply_transposed")
        return y

    def vcycle_transposed(self, r, z, stream=None):
        _check(self._lib.amgc_vcycle_transposed(self._h, _ptr(r), _ptr(z), _stream_ptr(stream)),
               "amgc_vcycle_transposed")
        return z

    def solve_transposed(self, rhs, x, tol: float = 0.0, stream=None, check: bool = True):
        it = C.c_int32(0)
        rr = C.c_double(0.0)
        code = self._lib.amgc_solve_transposed(self._h, _ptr(rhs), _ptr(x), float(tol), C.byref(it), C.byref(rr),
                                               _stream_ptr(stream))
        if check:
            _check(code, "amgc_solve_transposed")
        return it.value, rr.value, code

    def grad_scatter(self, adj, x, gK, gB1=None, gB2=None, stream=None):
        _check(self._lib.amgc_grad_scatter(self._h, _ptr(adj), _ptr(x), _ptr(gK), _ptr(gB1), _ptr(gB2),
                                           _stream_ptr(stream)), "amgc_grad_scatter")
        return gK

    def solve_batched(self, rhs, x, n_sys: int, stream=None, check: bool = True):
        """rhs, x: device tensors (nrhs, rows); returns (iters, relres) per system q * nrhs + r."""
        nrhs = int(rhs.shape[0])
        it = np.zeros(n_sys, dtype=np.int32)
        rr = np.zeros(n_sys, dtype=np.float64)
        code = self._lib.amgc_solve_batched(self._h, nrhs, _ptr(rhs), _ptr(x), it.ctypes.data, rr.ctypes.data,
                                            _stream_ptr(stream))
        if check:
            _check(code, "amgc_solve_batched")
        return it, rr, code

    SMOOTHERS = dict(cheap_simple=0, uzawa=1, braess_sarazin=2, simple_sgs=3)

    def set_smoother(self, kind, omega: float = 0.7, sgs_sweeps: int = 1, sgs_omega: float = 0.7, stream=None):
        """amgc_set_smoother: kind 'cheap_simple', 'uzawa', 'braess_sarazin', 'simple_sgs' (or 0..3)."""
        k = self.SMOOTHERS[kind] if isinstance(kind, str) else int(kind)
        _check(self._lib.amgc_set_smoother(self._h, k, float(omega), int(sgs_sweeps), float(sgs_omega),
                                           _stream_ptr(stream)), "amgc_set_smoother")

    def set_preconditioner(self, kind: int, outer_sweeps: int = 1, omega: float = 0.8, stream=None):
        """amgc_set_preconditioner: 0 the coupled V-cycle, 1 nested multigrid (outer SIMPLE sweeps)."""
        _check(self._lib.amgc_set_preconditioner(self._h, int(kind), int(outer_sweeps), float(omega),
                                                 _stream_ptr(stream)), "amgc_set_preconditioner")

    def update_active_set(self, active, stream=None):
        """amgc_update_active_set: active is a host uint8 array (or a device tensor) of n_s flags."""
        if not hasattr(active, "data_ptr"):
            active = np.ascontiguousarray(active, dtype=np.uint8)
        _check(self._lib.amgc_update_active_set(self._h, _ptr(active), _stream_ptr(stream)), "amgc_update_active_set")

    def pdass(self, f, g0, x, c: float = 1.0, max_steps: int = 50, stream=None, check: bool = True):
        """amgc_pdass on device tensors f (3n), g0 (n_s) and x (rows); returns (final active set
        (host uint8), solves, total FGMRES iterations, status)."""
        n_s = int(g0.shape[0])
        act = np.zeros(n_s, dtype=np.uint8)
        steps = C.c_int32(0)
        its = C.c_int32(0)
        code = self._lib.amgc_pdass(self._h, _ptr(f), _ptr(g0), float(c), int(max_steps), _ptr(x), act.ctypes.data,
                                    C.byref(steps), C.byref(its), _stream_ptr(stream))
        if check:
            _check(code, "amgc_pdass")
        return act, steps.value, its.value, code

    def solve_host(self, rhs: np.ndarray, stream=None, check: bool = True, x: np.ndarray = None):
        """amgc_solve_host; x, when given, is the host output array (float64, contiguous, the size
        of rhs; page-locked memory makes the device-to-host copy direct), else a new array."""
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        if x is None:
            x = np.empty_like(rhs)
        elif x.dtype != np.float64 or not x.flags.c_contiguous or x.size != rhs.size:
            raise ValueError("solve_host: x must be a contiguous float64 array of the size of rhs")
        it = C.c_int32(0)
        rr = C.c_double(0.0)
        code = self._lib.amgc_solve_host(self._h, rhs.ctypes.data, x.ctypes.data, C.byref(it), C.byref(rr),
                                         _stream_ptr(stream))
        if check:
            _check(code, "amgc_solve_host")
        return x, it.value, rr.value, code


def grad_elements(conn, shape, Khat, node_free, adj, x, uD, E, gE, lift_mask=None, gt=None, stream=None):
    """amgc_grad_elements on device tensors (see include/amgc.h)."""
    lib = load()
    ne = int(conn.shape[0])
    _check(lib.amgc_grad_elements(ne, _ptr(conn), _ptr(shape), _ptr(Khat), _ptr(node_free), _ptr(adj), _ptr(x),
                                  _ptr(uD), _ptr(lift_mask), _ptr(E), _ptr(gE), _ptr(gt), _stream_ptr(stream)),
           "amgc_grad_elements")
    return gE, gt


def grad_elements_noalloc(conn, shape, Khat, node_free, adj, x, uD, E, gE, lift_mask=None, gt=None, stream=None):
    """amgc_grad_elements_noalloc: the element gradients with static device scratch (no allocation)."""
    lib = load()
    ne = int(conn.shape[0])
    _check(lib.amgc_grad_elements_noalloc(ne, _ptr(conn), _ptr(shape), _ptr(Khat), _ptr(node_free), _ptr(adj),
                                          _ptr(x), _ptr(uD), _ptr(lift_mask), _ptr(E), _ptr(gE), _ptr(gt),
                                          _stream_ptr(stream)), "amgc_grad_elements_noalloc")
    return gE, gt


def setup(prob, options: Optional[Options] = None, stream=None, node_ptr=None, lm_ptr=None, **opt_kw) -> Hierarchy:
    """amgc_setup on a ContactProblem (host or device arrays; the library copies them).

    With node_ptr / lm_ptr (host int32 arrays of n_inst + 1) the problem is a block-diagonal
    batch and amgc_setup_batched is called.
    """
    lib = load()
    o = options if options is not None else default_options(**opt_kw)
    keep = []

    def arr(a, dt):
        if hasattr(a, "data_ptr"):          # torch tensor (host or device): pass its pointer
            if not a.is_contiguous() or a.element_size() != np.dtype(dt).itemsize:
                raise TypeError("setup: tensors must be contiguous with the declared element type")
            keep.append(a)
            return a.data_ptr()
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data
    K = Bsr(prob.n_nodes, prob.n_nodes, 3, 3, arr(prob.K_rowptr, np.int32), arr(prob.K_col, np.int32),
            arr(prob.K_val, np.float64))
    M = Csr(prob.n_s, int(prob.master_node.shape[0]), arr(prob.M_rowptr, np.int32), arr(prob.M_col, np.int32),
            arr(prob.M_val, np.float64))
    out = C.c_void_p(0)
    if node_ptr is None:
        code = lib.amgc_setup(C.byref(K), arr(prob.D, np.float64), C.byref(M), arr(prob.slave_node, np.int32),
                              arr(prob.master_node, np.int32), arr(prob.triad, np.float64),
                              arr(prob.active, np.uint8), arr(prob.body_id, np.int32),
                              arr(prob.nullspace, np.float64), C.byref(o), _stream_ptr(stream), C.byref(out))
        _check(code, "amgc_setup")
    else:
        npt = np.ascontiguousarray(node_ptr, dtype=np.int32)
        lpt = np.ascontiguousarray(lm_ptr, dtype=np.int32)
        code = lib.amgc_setup_batched(C.byref(K), arr(prob.D, np.float64), C.byref(M),
                                      arr(prob.slave_node, np.int32), arr(prob.master_node, np.int32),
                                      arr(prob.triad, np.float64), arr(prob.active, np.uint8),
                                      arr(prob.body_id, np.int32), arr(prob.nullspace, np.float64),
                                      int(npt.size - 1), npt.ctypes.data, lpt.ctypes.data, C.byref(o),
                                      _stream_ptr(stream), C.byref(out))
        _check(code, "amgc_setup_batched")
    return Hierarchy(out.value, lib)
