"""Thin ctypes binding of librafem (include/rafem.h): argument marshalling only.

Every step of the computation runs in the CUDA library; if librafem.so is missing or cannot be loaded this
module raises, it never falls back to another implementation. Functions keep the C names
(rafem_create, rafem_assemble, rafem_solve_step, rafem_run, ...); `Context` wraps them for convenience.
Device pointers may be passed as integers (e.g. torch.Tensor.data_ptr()).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librafem.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rafem.h")

RAFEM_OK = 0
RAFEM_NOT_CONVERGED = 1
RAFEM_ERR_BAD_INPUT = -1
RAFEM_ERR_BAD_MESH = -2
RAFEM_ERR_OOM = -3
RAFEM_ERR_NONFINITE = -4
RAFEM_ERR_TIMEOUT = -5
RAFEM_ERR_CUDA = -6
RAFEM_ERR_INTERNAL = -7
RAFEM_ERR_BREAKDOWN = -8

RAFEM_SYS_V = 1
RAFEM_SYS_T = 2
RAFEM_PRECOND_JACOBI = 0
RAFEM_PRECOND_ILU0 = 1
RAFEM_PRECISION_FP64 = 0
RAFEM_PRECISION_MIXED = 1
RAFEM_SOLVER_PCG = 0
RAFEM_SOLVER_BICGSTAB = 1
RAFEM_SOLVER_GMRES = 2
RAFEM_SOLVER_PIPECG = 3
RAFEM_PREDICT_PROJECT = 4
RAFEM_COUPLING_STAGGERED = 0
RAFEM_COUPLING_MONOLITHIC = 1
RAFEM_COUPLED_FGMRES = 0
RAFEM_COUPLED_BICGSTAB = 1
RAFEM_LIFT_SYMMETRIC = 0
RAFEM_LIFT_ROW = 1
RAFEM_ILU_MULTICOLOR = 0
RAFEM_ILU_NATURAL = 1
RAFEM_ASSEMBLY_GATHER = 0
RAFEM_ASSEMBLY_COLOR = 1
RAFEM_ARITH_AUTO = 0
RAFEM_ARITH_FP64 = 1
RAFEM_ARITH_DW = 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class rafem_mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tets", ctypes.c_int32), ("coords", _dp), ("tets", _ip),
                ("bc_V", _u8p), ("g_V", _dp), ("bc_T", _u8p), ("g_T", _dp), ("sigma0", _dp), ("k", _dp)]


class rafem_params(ctypes.Structure):
    _fields_ = [("alpha_sigma", ctypes.c_double), ("rho_c", ctypes.c_double), ("perf", ctypes.c_double),
                ("T_a", ctypes.c_double), ("dt", ctypes.c_double), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("corrector_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("max_refine", ctypes.c_int32), ("n_corrector", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("precision", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("rows_per_tile", ctypes.c_int32), ("assembly", ctypes.c_int32),
                ("predictor", ctypes.c_int32), ("ilu_order", ctypes.c_int32), ("lift", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("coupling", ctypes.c_int32), ("arith", ctypes.c_int32),
                ("proj_basis", ctypes.c_int32), ("gmres_min_restart", ctypes.c_int32),
                ("coupled_solver", ctypes.c_int32)]


class rafem_step_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters_V", ctypes.c_int32), ("iters_T", ctypes.c_int32),
                ("refine_V", ctypes.c_int32), ("refine_T", ctypes.c_int32), ("correctors", ctypes.c_int32),
                ("relres_V", ctypes.c_double), ("relres_T", ctypes.c_double), ("step", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rafem_trace(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("iters_V", ctypes.c_int64), ("iters_T", ctypes.c_int64),
                ("solves", ctypes.c_int64), ("refine_V", ctypes.c_int64), ("ms_assemble_V", ctypes.c_double),
                ("ms_solve_V", ctypes.c_double), ("ms_assemble_T", ctypes.c_double), ("ms_solve_T", ctypes.c_double),
                ("ms_memcpy_h2d", ctypes.c_double), ("ms_memcpy_d2h", ctypes.c_double),
                ("ms_predict_V", ctypes.c_double), ("ms_predict_T", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rafem_adjoint_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("forward_status", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("segments", ctypes.c_int32), ("iters_V", ctypes.c_int64), ("iters_T", ctypes.c_int64),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rafem_advance_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("accepted", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("dt", ctypes.c_double), ("time", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load librafem.so (built in-tree). Raises if it is missing: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librafem.so not built ({LIB_PATH}); run python -m paper_2409_13036_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    sig = {
        "rafem_default_params": (None, [ctypes.POINTER(rafem_params)]),
        "rafem_create": (ctypes.c_int, [ctypes.POINTER(rafem_mesh), ctypes.POINTER(rafem_params), vp,
                                        ctypes.POINTER(vp)]),
        "rafem_assemble": (ctypes.c_int, [vp, ctypes.c_int]),
        "rafem_solve": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(rafem_step_stats)]),
        "rafem_solve_step": (ctypes.c_int, [vp, ctypes.POINTER(rafem_step_stats)]),
        "rafem_run": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.POINTER(rafem_step_stats)]),
        "rafem_get_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
        "rafem_set_state": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int64]),
        "rafem_pattern_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int32)]),
        "rafem_get_system": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp, vp]),
        "rafem_layout_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]),
        "rafem_solve_rhs": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, ctypes.POINTER(rafem_step_stats)]),
        "rafem_spmv": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "rafem_set_tracing": (ctypes.c_int, [vp, ctypes.c_int]),
        "rafem_get_trace": (ctypes.c_int, [vp, ctypes.POINTER(rafem_trace)]),
        "rafem_pcg_csr_noalloc": (ctypes.c_int, [ctypes.c_int32, vp, vp, vp, vp, vp, ctypes.c_double,
                                                 ctypes.c_int32, vp, ctypes.POINTER(rafem_step_stats)]),
        "rafem_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.POINTER(rafem_mesh)),
                                              ctypes.POINTER(rafem_params), vp, ctypes.POINTER(vp)]),
        "rafem_batch_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), vp]),
        "rafem_batch_stats": (ctypes.c_int, [vp, vp]),
        "rafem_batch_run": (ctypes.c_int, [vp, ctypes.c_int32, vp]),
        "rafem_set_schedule": (ctypes.c_int, [vp, ctypes.c_int32]),
        "rafem_get_schedule": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32)]),
        "rafem_precond_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int64), vp, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int32)]),
        "rafem_get_precond": (ctypes.c_int, [vp, ctypes.c_int, vp]),
        "rafem_precond_apply": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "rafem_set_dt": (ctypes.c_int, [vp, ctypes.c_double]),
        "rafem_set_tol": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double]),
        "rafem_step_host": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.POINTER(rafem_step_stats)]),
        "rafem_graph_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
        "rafem_advance": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(rafem_advance_stats)]),
        "rafem_reorder_rcm": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, vp, vp]),
        "rafem_get_coupled_system": (ctypes.c_int, [vp, vp, vp]),
        "rafem_reset": (ctypes.c_int, [vp]),
        "rafem_set_params": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "rafem_set_params_device": (ctypes.c_int, [vp, vp, vp]),
        "rafem_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int32]),
        "rafem_tape_begin": (ctypes.c_int, [vp, ctypes.c_int32]),
        "rafem_adjoint": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                         ctypes.POINTER(rafem_adjoint_stats)]),
        "rafem_destroy": (None, [vp]),
        "rafem_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_symbols() -> list[str]:
    """Names of every entry point declared in include/rafem.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rafem_[a-z0-9_]+)\s*\(", text)))


def status_string(s: int) -> str:
    return lib().rafem_status_string(int(s)).decode()


class RafemError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {status_string(status)} ({status})")
        self.status = status


def _check(s, where, soft_ok=True):
    if s < 0 or (s > 0 and not soft_ok):
        raise RafemError(s, where)
    return s


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_params(**kw) -> rafem_params:
    p = rafem_params()
    lib().rafem_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _dev(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _mesh_struct(mesh):
    keep = [np.ascontiguousarray(mesh.coords, dtype=np.float64), np.ascontiguousarray(mesh.tets, dtype=np.int32),
            np.ascontiguousarray(mesh.bc_V, dtype=np.uint8), np.ascontiguousarray(mesh.g_V, dtype=np.float64),
            np.ascontiguousarray(mesh.bc_T, dtype=np.uint8), np.ascontiguousarray(mesh.g_T, dtype=np.float64),
            np.ascontiguousarray(mesh.sigma0, dtype=np.float64), np.ascontiguousarray(mesh.k, dtype=np.float64)]
    c, t, bv, gv, bt, gt, s0, k = keep
    m = rafem_mesh(n_nodes=c.shape[0], n_tets=t.shape[0], coords=_ptr(c, ctypes.c_double),
                   tets=_ptr(t, ctypes.c_int32), bc_V=_ptr(bv, ctypes.c_uint8), g_V=_ptr(gv, ctypes.c_double),
                   bc_T=_ptr(bt, ctypes.c_uint8), g_T=_ptr(gt, ctypes.c_double), sigma0=_ptr(s0, ctypes.c_double),
                   k=_ptr(k, ctypes.c_double))
    return m, keep


class Context:
    """Owns one rafem_ctx (one problem instance, or a batch, on the current CUDA device)."""

    @classmethod
    def batch(cls, meshes, params: rafem_params | None = None, stream: int | None = None, **kw):
        """rafem_batch_create over a list of meshes."""
        self = cls.__new__(cls)
        structs, keeps = zip(*[_mesh_struct(m) for m in meshes])
        arr = (ctypes.POINTER(rafem_mesh) * len(structs))(*[ctypes.pointer(s) for s in structs])
        self.params = params if params is not None else default_params(**kw)
        self._ctx = ctypes.c_void_p()
        s = lib().rafem_batch_create(len(structs), arr, ctypes.byref(self.params), ctypes.c_void_p(stream or 0),
                                     ctypes.byref(self._ctx))
        _check(s, "rafem_batch_create")
        n = ctypes.c_int32()
        offs = np.zeros(len(structs) + 1, np.int32)
        _check(lib().rafem_batch_info(self._ctx, ctypes.byref(n), offs.ctypes.data), "rafem_batch_info")
        self.offsets = offs
        self.N = int(offs[-1])
        self.n_inst = int(n.value)
        self.n_tets = int(sum(int(np.asarray(m.tets).shape[0]) for m in meshes))
        return self

    def batch_stats(self):
        out = (rafem_step_stats * self.n_inst)()
        _check(lib().rafem_batch_stats(self._ctx, ctypes.cast(out, ctypes.c_void_p)), "rafem_batch_stats")
        return [o.as_dict() for o in out]

    def batch_run(self, n_steps: int):
        """rafem_batch_run: n_steps steps of every instance; returns (worst status, per-instance stats of the last
        step)."""
        out = (rafem_step_stats * self.n_inst)()
        s = lib().rafem_batch_run(self._ctx, int(n_steps), ctypes.cast(out, ctypes.c_void_p))
        return _check(s, "rafem_batch_run"), [o.as_dict() for o in out]

    def __init__(self, mesh, params: rafem_params | None = None, stream: int | None = None, **kw):
        self._keep = [np.ascontiguousarray(mesh.coords, dtype=np.float64),
                      np.ascontiguousarray(mesh.tets, dtype=np.int32),
                      np.ascontiguousarray(mesh.bc_V, dtype=np.uint8),
                      np.ascontiguousarray(mesh.g_V, dtype=np.float64),
                      np.ascontiguousarray(mesh.bc_T, dtype=np.uint8),
                      np.ascontiguousarray(mesh.g_T, dtype=np.float64),
                      np.ascontiguousarray(mesh.sigma0, dtype=np.float64),
                      np.ascontiguousarray(mesh.k, dtype=np.float64)]
        c, t, bv, gv, bt, gt, s0, k = self._keep
        m = rafem_mesh(n_nodes=c.shape[0], n_tets=t.shape[0], coords=_ptr(c, ctypes.c_double),
                       tets=_ptr(t, ctypes.c_int32), bc_V=_ptr(bv, ctypes.c_uint8), g_V=_ptr(gv, ctypes.c_double),
                       bc_T=_ptr(bt, ctypes.c_uint8), g_T=_ptr(gt, ctypes.c_double),
                       sigma0=_ptr(s0, ctypes.c_double), k=_ptr(k, ctypes.c_double))
        self.params = params if params is not None else default_params(**kw)
        self.N = int(c.shape[0])
        self._ctx = ctypes.c_void_p()
        s = lib().rafem_create(ctypes.byref(m), ctypes.byref(self.params), ctypes.c_void_p(stream or 0),
                               ctypes.byref(self._ctx))
        _check(s, "rafem_create")
        self._keep = None
        self.n_tets = int(t.shape[0])
        self.n_inst = 1
        self.offsets = np.array([0, self.N], np.int32)

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().rafem_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C-ABI calls ----------------------------------------------------------------------------------------
    def assemble(self, which: int):
        return _check(lib().rafem_assemble(self._ctx, which), "rafem_assemble")

    def solve(self, which: int):
        st = rafem_step_stats()
        s = lib().rafem_solve(self._ctx, which, ctypes.byref(st))
        return _check(s, "rafem_solve"), st

    def solve_step(self):
        st = rafem_step_stats()
        s = lib().rafem_solve_step(self._ctx, ctypes.byref(st))
        return _check(s, "rafem_solve_step"), st

    def run(self, n_steps: int):
        st = rafem_step_stats()
        s = lib().rafem_run(self._ctx, int(n_steps), ctypes.byref(st))
        return _check(s, "rafem_run"), st

    def get_field(self, which: int) -> np.ndarray:
        out = np.empty(self.N, dtype=np.float64)
        _check(lib().rafem_get_field(self._ctx, which, out.ctypes.data, 0), "rafem_get_field")
        return out

    def get_field_device(self, which: int, dst) -> None:
        _check(lib().rafem_get_field(self._ctx, which, _dev(dst), 1), "rafem_get_field")

    def set_state(self, T=None, V=None, step: int = 0):
        Ta = None if T is None else np.ascontiguousarray(T, dtype=np.float64)
        Va = None if V is None else np.ascontiguousarray(V, dtype=np.float64)
        s = lib().rafem_set_state(self._ctx, None if Ta is None else Ta.ctypes.data,
                                  None if Va is None else Va.ctypes.data, 0, int(step))
        _check(s, "rafem_set_state")

    def set_state_device(self, T=None, V=None, step: int = 0):
        _check(lib().rafem_set_state(self._ctx, _dev(T), _dev(V), 1, int(step)), "rafem_set_state")

    def pattern_info(self):
        n = ctypes.c_int32()
        nnz = ctypes.c_int64()
        nc = ctypes.c_int32()
        _check(lib().rafem_pattern_info(self._ctx, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nc)),
               "rafem_pattern_info")
        return n.value, nnz.value, nc.value

    def set_schedule(self, rows_per_tile: int):
        _check(lib().rafem_set_schedule(self._ctx, int(rows_per_tile)), "rafem_set_schedule")

    def get_schedule(self) -> dict:
        r, n, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rafem_get_schedule(self._ctx, ctypes.byref(r), ctypes.byref(n), ctypes.byref(g)),
               "rafem_get_schedule")
        return {"rows_per_tile": r.value, "n_tiles": n.value, "grid": g.value}

    def layout_info(self) -> dict:
        code, nst, cb, asm, ar = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rafem_layout_info(self._ctx, ctypes.byref(code), ctypes.byref(nst), ctypes.byref(cb),
                                       ctypes.byref(asm), ctypes.byref(ar)), "rafem_layout_info")
        return {"kernel_code": code.value, "nnz_stored": nst.value, "column_bytes": cb.value, "assembly": asm.value,
                "arith": ar.value}

    def get_system(self, which: int):
        """(row_ptr, col, vals, rhs) of the current lifted system, as host arrays."""
        n, nnz, _ = self.pattern_info()
        rp = np.empty(n + 1, np.int32)
        col = np.empty(nnz, np.int32)
        vals = np.empty(nnz, np.float64)
        rhs = np.empty(n, np.float64)
        _check(lib().rafem_get_system(self._ctx, which, rp.ctypes.data, col.ctypes.data, vals.ctypes.data,
                                      rhs.ctypes.data), "rafem_get_system")
        return rp, col, vals, rhs

    def solve_rhs(self, which: int, b_dev, x_dev):
        st = rafem_step_stats()
        s = lib().rafem_solve_rhs(self._ctx, which, _dev(b_dev), _dev(x_dev), ctypes.byref(st))
        return _check(s, "rafem_solve_rhs"), st

    def set_tracing(self, on: bool):
        _check(lib().rafem_set_tracing(self._ctx, 1 if on else 0), "rafem_set_tracing")

    def get_trace(self) -> dict:
        t = rafem_trace()
        _check(lib().rafem_get_trace(self._ctx, ctypes.byref(t)), "rafem_get_trace")
        return t.as_dict()

    def set_state_ptr(self, T_ptr=None, V_ptr=None, on_device=0, step=0):
        _check(lib().rafem_set_state(self._ctx, T_ptr, V_ptr, int(on_device), int(step)), "rafem_set_state")

    def get_field_ptr(self, which: int, dst_ptr: int, on_device=0):
        _check(lib().rafem_get_field(self._ctx, which, dst_ptr, int(on_device)), "rafem_get_field")

    def spmv(self, which: int, x_dev, y_dev):
        _check(lib().rafem_spmv(self._ctx, which, _dev(x_dev), _dev(y_dev)), "rafem_spmv")

    def get_coupled_system(self):
        """(blocks [nnz, 2, 2], residual [N, 2]) of the monolithic Newton system at the current state."""
        _, nnz, _ = self.pattern_info()
        blocks = np.empty((nnz, 2, 2), np.float64)
        res = np.empty((self.N, 2), np.float64)
        _check(lib().rafem_get_coupled_system(self._ctx, blocks.ctypes.data, res.ctypes.data), "rafem_get_coupled_system")
        return blocks, res

    # -- dynamic step size ------------------------------------------------------------------------------------
    def graph_info(self) -> dict:
        a, b, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rafem_graph_info(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)),
               "rafem_graph_info")
        return {"step_graph": a.value, "corrector_graph": b.value, "step_kernels": k.value}

    def set_dt(self, dt: float):
        _check(lib().rafem_set_dt(self._ctx, float(dt)), "rafem_set_dt")

    def step_host_ptr(self, T_in=None, V_in=None, T_out=None, V_out=None):
        """rafem_step_host on raw host addresses (ints or None)."""
        st = rafem_step_stats()
        s = lib().rafem_step_host(self._ctx, T_in, V_in, T_out, V_out, ctypes.byref(st))
        return _check(s, "rafem_step_host"), st

    def step_host(self, T=None, V=None):
        """One step from host state: numpy float64 arrays T, V (either may be None) are read before the step and
        overwritten with the fields after it."""
        Ta = None if T is None else np.ascontiguousarray(T, dtype=np.float64)
        Va = None if V is None else np.ascontiguousarray(V, dtype=np.float64)
        if Ta is not T and T is not None or Va is not V and V is not None:
            raise ValueError("T and V must be contiguous float64 arrays")
        return self.step_host_ptr(None if Ta is None else Ta.ctypes.data, None if Va is None else Va.ctypes.data,
                                  None if Ta is None else Ta.ctypes.data, None if Va is None else Va.ctypes.data)

    def set_tol(self, tol: float, inner_tol: float = 0.0):
        _check(lib().rafem_set_tol(self._ctx, float(tol), float(inner_tol)), "rafem_set_tol")

    def advance(self, duration: float, dt_min: float):
        st = rafem_advance_stats()
        s = lib().rafem_advance(self._ctx, float(duration), float(dt_min), ctypes.byref(st))
        return _check(s, "rafem_advance"), st.as_dict()

    # -- preconditioner ---------------------------------------------------------------------------------------
    def precond_info(self) -> dict:
        nl, npad, nz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        order = np.empty(self.N, np.int32)
        nf, cb = ctypes.c_int64(), ctypes.c_int32()
        _check(lib().rafem_precond_info(self._ctx, ctypes.byref(nl), ctypes.byref(npad), ctypes.byref(nz),
                                        order.ctypes.data, ctypes.byref(nf), ctypes.byref(cb)), "rafem_precond_info")
        return {"n_levels": nl.value, "padded_rows": npad.value, "nnz_stored": nz.value, "order": order,
                "factor_stored": nf.value, "column_bytes": cb.value}

    def get_precond(self, which: int) -> np.ndarray:
        _, nnz, _ = self.pattern_info()
        out = np.empty(nnz, np.float64)
        _check(lib().rafem_get_precond(self._ctx, which, out.ctypes.data), "rafem_get_precond")
        return out

    def precond_apply(self, which: int, r_dev, z_dev):
        _check(lib().rafem_precond_apply(self._ctx, which, _dev(r_dev), _dev(z_dev)), "rafem_precond_apply")

    # -- differentiation form -------------------------------------------------------------------------------
    def reset(self):
        _check(lib().rafem_reset(self._ctx), "rafem_reset")

    def set_params(self, sigma0=None, k=None):
        """Host arrays (numpy) or device tensors/pointers of E doubles, mesh element order."""
        if sigma0 is None and k is None:
            raise ValueError("nothing to set")
        host = [isinstance(x, np.ndarray) for x in (sigma0, k) if x is not None]
        if any(host) and not all(host):
            raise ValueError("sigma0 and k must both be host arrays or both device buffers")
        if host and host[0]:
            s0 = None if sigma0 is None else np.ascontiguousarray(sigma0, dtype=np.float64)
            kk = None if k is None else np.ascontiguousarray(k, dtype=np.float64)
            _check(lib().rafem_set_params(self._ctx, None if s0 is None else s0.ctypes.data,
                                          None if kk is None else kk.ctypes.data, 0), "rafem_set_params")
        else:
            _check(lib().rafem_set_params(self._ctx, _dev(sigma0), _dev(k), 1), "rafem_set_params")

    def set_params_device(self, sigma0=None, k=None):
        """rafem_set_params_device: FP32 device tensors (or pointers) of E floats, mesh element order."""
        if sigma0 is None and k is None:
            raise ValueError("nothing to set")
        _check(lib().rafem_set_params_device(self._ctx, _dev(sigma0), _dev(k)), "rafem_set_params_device")

    def set_wait_limit(self, limit_ns: int = 0, missing_arrivals: int = 0):
        """rafem_set_wait_limit: wall-clock limit of the solvers' device waits (0 = default 5 s); missing_arrivals
        > 0 makes the next solves' first grid barrier incomplete (tests of the timeout path)."""
        _check(lib().rafem_set_wait_limit(self._ctx, int(limit_ns), int(missing_arrivals)), "rafem_set_wait_limit")

    def tape_begin(self, checkpoint_every: int):
        _check(lib().rafem_tape_begin(self._ctx, int(checkpoint_every)), "rafem_tape_begin")

    def adjoint_ptr(self, dL_dT, dL_dV=None, in_on_device=1, dsigma0=None, dk=None, dT0=None, out_on_device=1):
        """rafem_adjoint with raw pointers (ints) or tensors; returns (status, stats dict)."""
        st = rafem_adjoint_stats()
        s = lib().rafem_adjoint(self._ctx, _dev(dL_dT), _dev(dL_dV), int(in_on_device), _dev(dsigma0), _dev(dk),
                                _dev(dT0), int(out_on_device), ctypes.byref(st))
        return _check(s, "rafem_adjoint"), st.as_dict()

    def adjoint(self, dL_dT, dL_dV=None, n_tets: int | None = None):
        """Host form: numpy dL/dT (and dL/dV) in, numpy (dL/dsigma0, dL/dk, dL/dT0, stats) out."""
        if n_tets is None:
            n_tets = self.n_tets
        gT = np.ascontiguousarray(dL_dT, dtype=np.float64)
        gV = None if dL_dV is None else np.ascontiguousarray(dL_dV, dtype=np.float64)
        gs = np.empty(n_tets)
        gk = np.empty(n_tets)
        g0 = np.empty(self.N)
        st = rafem_adjoint_stats()
        s = lib().rafem_adjoint(self._ctx, gT.ctypes.data, None if gV is None else gV.ctypes.data, 0,
                                gs.ctypes.data, gk.ctypes.data, g0.ctypes.data, 0, ctypes.byref(st))
        _check(s, "rafem_adjoint")
        return gs, gk, g0, st.as_dict()


def pcg_csr_noalloc(n_rows, row_ptr, col, vals, b, x, tol=1e-10, max_iter=20000, stream=None):
    """rafem_pcg_csr_noalloc: Jacobi-PCG on a caller-held device CSR system using only the library's fixed
    scratch array (no allocation). Arguments are device pointers (ints) or tensors; returns (status, stats)."""
    st = rafem_step_stats()
    s = lib().rafem_pcg_csr_noalloc(int(n_rows), _dev(row_ptr), _dev(col), _dev(vals), _dev(b), _dev(x), float(tol),
                                    int(max_iter), ctypes.c_void_p(stream or 0), ctypes.byref(st))
    return s, st


def reorder_rcm(mesh) -> np.ndarray:
    """rafem_reorder_rcm: reverse Cuthill-McKee node order of a mesh (perm[new] = old)."""
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    perm = np.empty(int(np.asarray(mesh.coords).shape[0]), np.int32)
    _check(lib().rafem_reorder_rcm(perm.shape[0], tets.shape[0], tets.ctypes.data, perm.ctypes.data),
           "rafem_reorder_rcm")
    return perm


# C names, for callers that prefer the flat API
def rafem_create(mesh, params=None, stream=None):
    return Context(mesh, params, stream)


def rafem_assemble(ctx: Context, which: int):
    return ctx.assemble(which)


def rafem_solve_step(ctx: Context):
    return ctx.solve_step()


def rafem_run(ctx: Context, n_steps: int):
    return ctx.run(n_steps)


def rafem_destroy(ctx: Context):
    ctx.close()
