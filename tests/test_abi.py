"""CPU-only checks of the boundary: the CUDA library builds for sm_103a, loads, exports every entry
point the headers in include/ declare (dg.h, the method; dg_probes.h, the measurement probes), and
the binding's constants equal the header's enums. No kernel runs."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2407_19169_gb300 import _native as N
from paper_2407_19169_gb300 import build as B
from paper_2407_19169_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dg.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def declared():
    txt = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^DG_API\s+[\w\s\*]+?\b(dg_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_documented_api():
    names = declared()
    for must in ["dg_create", "dg_step", "dg_advance_to", "dg_read_state", "dg_destroy", "dg_set_initial",
                 "dg_write_state", "dg_advance_steps", "dg_sync"]:
        assert must in names
    assert sorted(N.EXPORTED) == names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r" T (dg_\w+)", out)))
    assert exported == declared()          # nothing else leaks out of the library


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_enums_match_header():
    txt = open(HEADER).read()

    def val(name):
        return int(re.search(r"\b%s\s*=\s*(-?\d+)" % name, txt).group(1))

    assert val("DG_EQ_EULER") == N.EQ_EULER and val("DG_EQ_BURGERS") == N.EQ_BURGERS
    assert val("DG_BC_OUTFLOW") == N.BC_OUTFLOW and val("DG_PREC_FP32_MIXED") == N.PREC_FP32_MIXED
    assert val("DG_BASIS_P") == N.BASIS_P and val("DG_IC_VORTEX2D") == N.IC_VORTEX2D
    assert val("DG_FILTER_GLOBAL") == N.FILTER_GLOBAL and val("DG_FILTER_OEDG") == N.FILTER_OEDG
    for code, name in N.STATUS.items():
        assert val(name) == code


def test_pure_calls_without_gpu(lib):
    L = N.load()
    assert L.dg_status_string(-4) == b"non-physical or non-finite cell average"
    p = N.Params()
    assert L.dg_params_default(ctypes.byref(p)) == 0
    assert p.enabled == 1 and abs(p.cfl - 0.1) < 1e-15 and abs(p.gamma - 1.4) < 1e-15
    mesh = N.Mesh(2, 2048, 2048, 0.0, 1.0, 0.0, 1.0, (ctypes.c_int * 4)(1, 1, 1, 1))
    n = ctypes.c_size_t()
    assert L.dg_workspace_size(ctypes.byref(mesh), 2, N.EQ_EULER, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value >= 3 * 8 * 4 * 9 * 2048 * 2048          # three FP64 state buffers
    bad = N.Mesh(2, 0, 5, 0.0, 1.0, 0.0, 1.0, (ctypes.c_int * 4)(1, 1, 1, 1))
    assert L.dg_workspace_size(ctypes.byref(bad), 2, N.EQ_EULER, ctypes.byref(p), ctypes.byref(n)) == -1
    assert L.dg_workspace_size(ctypes.byref(mesh), 5, N.EQ_EULER, ctypes.byref(p), ctypes.byref(n)) == -8
    # more than 2^31 cells: unsupported (the size is refused before anything is allocated)
    huge = N.Mesh(2, 65536, 32769, 0.0, 1.0, 0.0, 1.0, (ctypes.c_int * 4)(1, 1, 1, 1))
    assert L.dg_workspace_size(ctypes.byref(huge), 1, N.EQ_EULER, ctypes.byref(p), ctypes.byref(n)) == -8
    # one periodic and one outflow side on the same axis: invalid
    half = N.Mesh(1, 64, 1, 0.0, 1.0, 0.0, 1.0, (ctypes.c_int * 4)(0, 1, 0, 0))
    assert L.dg_workspace_size(ctypes.byref(half), 2, N.EQ_BURGERS, ctypes.byref(p), ctypes.byref(n)) == -1
    # the hybrid limiter needs the filter on and excludes the positivity limiter
    q = N.Params()
    L.dg_params_default(ctypes.byref(q))
    q.hybrid, q.positivity = 1, 1
    assert L.dg_workspace_size(ctypes.byref(mesh), 2, N.EQ_EULER, ctypes.byref(q), ctypes.byref(n)) == -8
    q.positivity, q.enabled = 0, 0
    assert L.dg_workspace_size(ctypes.byref(mesh), 2, N.EQ_EULER, ctypes.byref(q), ctypes.byref(n)) == -8
    q.enabled = 1
    assert L.dg_workspace_size(ctypes.byref(mesh), 2, N.EQ_EULER, ctypes.byref(q), ctypes.byref(n)) == 0
    # a non-positive CFL number or gamma <= 1: invalid
    q.cfl = 0.0
    assert L.dg_workspace_size(ctypes.byref(mesh), 2, N.EQ_EULER, ctypes.byref(q), ctypes.byref(n)) == -1


def test_splitmix64_reference_stream():
    # SplitMix64 seeded with 0: the published reference implementation's first outputs
    g = I.SplitMix64(0)
    assert g.next_u64() == 0xE220A8397B1DCDAF
    assert g.next_u64() == 0x6E789E6AA1B965F4
    h = I.SplitMix64(0)
    v = h.block_u64(2)
    assert int(v[0]) == 0xE220A8397B1DCDAF and int(v[1]) == 0x6E789E6AA1B965F4


def test_batch_and_probe_argument_checks_need_no_gpu(lib):
    """The batched entry points and the bounded-wait probe reject bad arguments before touching the
    device."""
    n = N.load()
    arr = (ctypes.c_void_p * 1)(None)
    assert n.dg_batch_run(None, 1, 1) == -1
    assert n.dg_batch_run_persistent(None, 1, 1) == -1
    assert n.dg_batch_run_persistent(arr, 0, 1) == -1
    assert n.dg_batch_run_persistent(arr, 1, -1) == -1
    assert n.dg_batch_run_persistent(arr, 1, 1) == -1        # a NULL solver
    assert n.dg_batch_run_persistent(arr, 1, (1 << 30) + 1) == -1   # beyond the 32-bit stage counters
    status, ms = ctypes.c_uint(0), ctypes.c_double(0.0)
    assert n.dg_probe_wait_timeout(1 << 25, ctypes.byref(status), ctypes.byref(ms)) == -1
    assert n.dg_probe_wait_timeout(10, None, ctypes.byref(ms)) == -1


def test_build_compiles_every_instantiation_unit():
    """The 2D stage kernel's (form, degree) objects and the batched kernels' per-degree objects are all
    in the build, each with its own defines, next to the dispatch object."""
    objs = {o: defs for _, o, defs in B.UNITS}
    for f in range(5):
        for k in (1, 2, 3):
            assert objs["stage2d_f%d_k%d.o" % (f, k)] == ["-DS2_FORM=%d" % f, "-DS2_K=%d" % k]
    assert objs["stage2d_dispatch.o"] == ["-DS2_DISPATCH"]
    for k in (1, 2, 3):
        assert objs["dg_batch_k%d.o" % k] == ["-DDG_BATCH_K=%d" % k]
    assert objs["dg_batch.o"] == [] and objs["dg_api.o"] == []
    assert len(objs) == len(B.UNITS)                       # no object built twice
