"""ctypes binding to libdgjf.so, the C ABI declared in include/dg.h.

Argument marshalling only: every step of the method runs in the library's CUDA kernels. There is no
CPU fallback; if the shared library is missing or no sm_103a GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgjf.so")

DG_OK = 0
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_OOM", -3: "DG_ERR_BUDGET", -4: "DG_ERR_NONPHYSICAL",
          -5: "DG_ERR_TIMEOUT", -6: "DG_ERR_CUDA", -7: "DG_ERR_STATE", -8: "DG_ERR_UNSUPPORTED"}
EQ_ADVECTION, EQ_BURGERS, EQ_EULER = 0, 1, 2
FLUX_LLF = 0
BC_PERIODIC, BC_OUTFLOW = 0, 1
PREC_FP64, PREC_FP32_MIXED = 0, 1
BASIS_Q, BASIS_P = 0, 1
FILTER_JUMP, FILTER_GLOBAL, FILTER_OEDG = 0, 1, 2
IC_SINE, IC_RIEMANN1D, IC_ENTROPY1D, IC_QUADRANT2D, IC_VORTEX2D = range(5)

EXPORTED = ["dg_status_string", "dg_last_error", "dg_params_default", "dg_workspace_size", "dg_create",
            "dg_set_initial", "dg_state_size", "dg_write_state", "dg_write_state_device", "dg_read_state",
            "dg_read_state_device", "dg_step", "dg_advance_to", "dg_advance_steps", "dg_sync", "dg_mass",
            "dg_dims", "dg_kernel_launches", "dg_destroy", "dg_step_noalloc", "dg_set_target",
            "dg_batch_run", "dg_batch_run_persistent", "dg_probe_fma", "dg_probe_transform",
            "dg_probe_wait_timeout"]


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("bc", C.c_int * 4)]


class Params(C.Structure):
    _fields_ = [("enabled", C.c_int), ("cfl", C.c_double), ("gamma", C.c_double),
                ("adv_speed", C.c_double * 2), ("basis", C.c_int), ("nq", C.c_int), ("precision", C.c_int),
                ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t), ("tile_rows", C.c_int),
                ("tile_warps", C.c_int), ("positivity", C.c_int),
                ("hybrid", C.c_int), ("filter_kind", C.c_int)]


class DGError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = "%s failed: %s" % (where, STATUS.get(status, status))
        if detail:
            msg += " (%s)" % detail
        super().__init__(msg)


_lib = None


def load():
    """Load libdgjf.so (built by __graft_entry__.build() or paper_2407_19169_gb300/build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdgjf.so is not built (run paper_2407_19169_gb300/build.py); "
                          "there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    P, I, D, V, SZ, LL = C.POINTER, C.c_int, C.c_double, C.c_void_p, C.c_size_t, C.c_longlong
    dp = P(C.c_double)
    sig = {
        "dg_status_string": (C.c_char_p, [I]),
        "dg_last_error": (C.c_char_p, []),
        "dg_params_default": (I, [P(Params)]),
        "dg_workspace_size": (I, [P(Mesh), I, I, P(Params), P(SZ)]),
        "dg_create": (I, [P(Mesh), I, I, I, P(Params), V, P(V)]),
        "dg_set_initial": (I, [V, I, dp, I, I]),
        "dg_state_size": (I, [V, P(SZ)]),
        "dg_write_state": (I, [V, dp, SZ, D]),
        "dg_write_state_device": (I, [V, V, SZ, D]),
        "dg_read_state": (I, [V, dp, SZ, dp]),
        "dg_read_state_device": (I, [V, V, SZ, dp]),
        "dg_step": (I, [V, dp]),
        "dg_advance_to": (I, [V, D, LL, P(LL)]),
        "dg_advance_steps": (I, [V, LL]),
        "dg_sync": (I, [V, dp, P(LL)]),
        "dg_mass": (I, [V, dp]),
        "dg_dims": (I, [V, P(I), P(I), P(LL)]),
        "dg_kernel_launches": (I, [V, P(LL)]),
        "dg_destroy": (I, [V]),
        "dg_step_noalloc": (I, [P(Mesh), I, I, P(Params), V, V, dp, V]),
        "dg_set_target": (I, [V, D, LL]),
        "dg_batch_run": (I, [P(V), I, LL]),
        "dg_batch_run_persistent": (I, [P(V), I, LL]),
        "dg_probe_fma": (I, [I, I, dp]),
        "dg_probe_transform": (I, [I, LL, I, dp, dp]),
        "dg_probe_wait_timeout": (I, [C.c_uint, P(C.c_uint), dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int, where: str) -> int:
    if status != DG_OK:
        detail = load().dg_last_error().decode() if status == -6 else ""
        raise DGError(status, where, detail)
    return status


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def batch_run(solvers, steps: int, persistent: bool = False) -> int:
    """dg_batch_run (or dg_batch_run_persistent) over a list of Solver objects; returns the status
    (0 = all ok)."""
    arr = (C.c_void_p * len(solvers))(*[s.handle.value for s in solvers])
    f = load().dg_batch_run_persistent if persistent else load().dg_batch_run
    return f(arr, len(solvers), steps)


class Solver:
    """One DG solve on the current CUDA device (a handle from dg_create)."""

    def __init__(self, dim=1, nx=16, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(BC_PERIODIC,) * 4, k=2,
                 eq=EQ_BURGERS, filter=1, cfl=0.1, gamma=1.4, adv=(1.0, 0.0), basis=BASIS_Q,
                 precision=PREC_FP64, stream=None, tile_rows=0, workspace=None, tile_warps=0,
                 positivity=0, hybrid=0, filter_kind=FILTER_JUMP):
        L = load()
        self.mesh = Mesh(dim, nx, ny, x0, x1, y0, y1, (C.c_int * 4)(*bc))
        self.params = Params()
        check(L.dg_params_default(C.byref(self.params)), "dg_params_default")
        self.params.enabled = int(filter)
        self.params.cfl = cfl
        self.params.gamma = gamma
        self.params.adv_speed = (C.c_double * 2)(*adv)
        self.params.basis = basis
        self.params.precision = precision
        self.params.tile_rows = tile_rows
        self.params.tile_warps = tile_warps
        self.params.positivity = positivity
        self.params.hybrid = hybrid
        self.params.filter_kind = filter_kind
        self._workspace = workspace  # keep a caller tensor alive
        if workspace is not None:
            self.params.workspace = workspace.data_ptr()
            self.params.workspace_bytes = workspace.numel() * workspace.element_size()
        self.handle = C.c_void_p()
        self._stream = stream
        sptr = None if stream is None else C.c_void_p(stream)
        check(L.dg_create(C.byref(self.mesh), k, eq, FLUX_LLF, C.byref(self.params), sptr,
                          C.byref(self.handle)), "dg_create")
        nv, nm, nc = C.c_int(), C.c_int(), C.c_longlong()
        check(L.dg_dims(self.handle, C.byref(nv), C.byref(nm), C.byref(nc)), "dg_dims")
        self.shape = (nv.value, nm.value, nc.value)

    @staticmethod
    def workspace_size(dim=1, nx=16, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(BC_PERIODIC,) * 4, k=2,
                       eq=EQ_BURGERS, basis=BASIS_Q, precision=PREC_FP64, hybrid=0) -> int:
        L = load()
        mesh = Mesh(dim, nx, ny, x0, x1, y0, y1, (C.c_int * 4)(*bc))
        p = Params()
        check(L.dg_params_default(C.byref(p)), "dg_params_default")
        p.basis = basis
        p.precision = precision
        p.hybrid = hybrid
        n = C.c_size_t()
        check(L.dg_workspace_size(C.byref(mesh), k, eq, C.byref(p), C.byref(n)), "dg_workspace_size")
        return n.value

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))

    def set_initial(self, ic: int, params, nq_init: int = 0) -> None:
        prm = np.ascontiguousarray(params, dtype=np.float64)
        check(load().dg_set_initial(self.handle, ic, _dp(prm), len(prm), nq_init), "dg_set_initial")

    def write_state(self, u: np.ndarray, t: float = 0.0) -> None:
        u = np.ascontiguousarray(u, dtype=np.float64)
        check(load().dg_write_state(self.handle, _dp(u), u.size, t), "dg_write_state")

    def read_state(self):
        u = np.zeros(self.shape)
        t = C.c_double()
        check(load().dg_read_state(self.handle, _dp(u), u.size, C.byref(t)), "dg_read_state")
        return u, t.value

    def write_state_host_ptr(self, ptr: int, n: int, t: float = 0.0) -> None:
        """dg_write_state from a raw host pointer (e.g. a pinned torch tensor)."""
        check(load().dg_write_state(self.handle, C.cast(C.c_void_p(ptr), C.POINTER(C.c_double)), n, t),
              "dg_write_state")

    def read_state_host_ptr(self, ptr: int, n: int) -> float:
        t = C.c_double()
        check(load().dg_read_state(self.handle, C.cast(C.c_void_p(ptr), C.POINTER(C.c_double)), n,
                                   C.byref(t)), "dg_read_state")
        return t.value

    def write_state_device(self, ptr: int, n: int, t: float = 0.0) -> None:
        check(load().dg_write_state_device(self.handle, C.c_void_p(ptr), n, t), "dg_write_state_device")

    def read_state_device(self, ptr: int, n: int) -> float:
        t = C.c_double()
        check(load().dg_read_state_device(self.handle, C.c_void_p(ptr), n, C.byref(t)), "dg_read_state_device")
        return t.value

    def step(self) -> float:
        dt = C.c_double()
        check(load().dg_step(self.handle, C.byref(dt)), "dg_step")
        return dt.value

    def advance_to(self, T: float, max_steps: int = 1 << 62) -> int:
        n = C.c_longlong()
        st = load().dg_advance_to(self.handle, T, max_steps, C.byref(n))
        check(st, "dg_advance_to")
        return n.value

    def advance_toward(self, T: float, max_steps: int) -> int:
        """dg_advance_to with at most max_steps steps; returns its status without raising
        (DG_ERR_TIMEOUT = stopped at max_steps before T; dg_sync reports the solve's state)."""
        n = C.c_longlong()
        return load().dg_advance_to(self.handle, T, max_steps, C.byref(n))

    def advance_steps(self, n: int) -> None:
        check(load().dg_advance_steps(self.handle, n), "dg_advance_steps")

    def set_target(self, T_end: float, max_steps: int = 1 << 62) -> None:
        check(load().dg_set_target(self.handle, T_end, max_steps), "dg_set_target")

    def sync(self):
        t = C.c_double()
        n = C.c_longlong()
        st = load().dg_sync(self.handle, C.byref(t), C.byref(n))
        return st, t.value, n.value

    def mass(self) -> np.ndarray:
        m = np.zeros(self.shape[0])
        check(load().dg_mass(self.handle, _dp(m)), "dg_mass")
        return m

    def kernel_launches(self) -> int:
        n = C.c_longlong()
        check(load().dg_kernel_launches(self.handle, C.byref(n)), "dg_kernel_launches")
        return n.value

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().dg_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
