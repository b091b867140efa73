"""Run the measurement probes of include/dg_probes.h on the current GPU and print one JSON line:
the FP32 / packed-FP32 / FP64 fused multiply-add throughput, and the Q2 modal -> volume-point
transform on the CUDA cores against the tensor cores (mma.sync TF32, one pass and 3xTF32) with its
relative L1 against FP64. Usage: python -m paper_2407_19169_gb300.probes [ncell]."""
import ctypes as C
import json
import sys

from . import _native as N


def run(ncell=1 << 22, reps=20):
    L = N.load()
    out = {}
    for kind, name in ((0, "fp32_ffma"), (1, "fp32_ffma2"), (2, "fp64_dfma")):
        t = C.c_double()
        iters = 20000 if kind != 2 else 400
        st = L.dg_probe_fma(kind, iters, C.byref(t))
        if st != 0:
            raise RuntimeError("dg_probe_fma(%d) returned %d" % (kind, st))
        out[name + "_tflops"] = t.value
    for var, name in ((0, "cuda_cores_fp32"), (1, "tensor_tf32"), (2, "tensor_3xtf32")):
        ms, err = C.c_double(), C.c_double()
        st = L.dg_probe_transform(var, ncell, reps, C.byref(ms), C.byref(err))
        if st != 0:
            raise RuntimeError("dg_probe_transform(%d) returned %d" % (var, st))
        out["transform_" + name] = {"ms_per_launch": ms.value, "rel_l1_vs_fp64": err.value,
                                    "cells": ncell, "bytes_moved": 2 * 36 * 4 * ncell,
                                    "gb_per_s": 2 * 36 * 4 * ncell / (ms.value * 1e-3) / 1e9}
    return out


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1 << 22
    print(json.dumps(run(n)))
