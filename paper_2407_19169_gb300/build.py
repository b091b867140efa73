"""Build the CUDA library libdgjf.so (sm_103a) in-tree.

Each translation unit is compiled by its own nvcc process, in parallel, then linked with
`nvcc -shared`. Nothing here falls back to a CPU implementation: without nvcc the build fails.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgjf.so")
# (source, object, defines): stage2d_units.cu is compiled once per (form, degree) of the 2D stage
# kernel and once for its dispatch tables, dg_batch.cu once for its host code and 1D kernels and once
# per degree of its 2D kernels, so that the slow instantiations compile in parallel.
UNITS = [(u, u.replace(".cu", ".o"), []) for u in
         ["dg_api.cu", "aux.cu", "stage1d.cu", "dg_noalloc.cu", "dg_batch.cu", "probes.cu"]] + \
        [("stage2d_units.cu", "stage2d_f%d_k%d.o" % (f, k), ["-DS2_FORM=%d" % f, "-DS2_K=%d" % k])
         for f in range(5) for k in (1, 2, 3)] + \
        [("stage2d_units.cu", "stage2d_dispatch.o", ["-DS2_DISPATCH"])] + \
        [("dg_batch.cu", "dg_batch_k%d.o" % k, ["-DDG_BATCH_K=%d" % k]) for k in (1, 2, 3)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -prec-div=false / -prec-sqrt=false: single-precision division and square root by the hardware
# approximations (a couple of ulp). They act only on FP32 arithmetic (the FP32 form's stage math);
# FP64 and the double-float cell averages are untouched.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-prec-div=false", "-prec-sqrt=false",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + \
        [os.path.join(os.path.dirname(HERE), "include", h) for h in ("dg.h", "dg_probes.h")] + \
        [os.path.abspath(__file__)]


def _stale(obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for src, o, defs in UNITS:
        obj = os.path.join(BUILD, o)
        if force or _stale(obj):
            cmd = [nvcc] + ARCH + FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
            jobs.append((o, cmd))
    if jobs:
        # the slowest units first, so that they start before the pool fills
        jobs.sort(key=lambda j: ("k3" not in j[0], "_f0" not in j[0] and "_f3" not in j[0]))
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(4, os.cpu_count() or 4))) as ex:
            futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): u for u, cmd in jobs}
            for f in cf.as_completed(futs):
                r = f.result()
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed for %s:\n%s" % (futs[f], r.stderr[-4000:]))
                if verbose and r.stderr:
                    print(r.stderr)
    objs = [os.path.join(BUILD, o) for _, o, _ in UNITS]
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
