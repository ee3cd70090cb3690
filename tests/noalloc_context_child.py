"""Child process of tests/test_zz_no_alloc.py: lbm_observables_noalloc in a
CUDA context the caller created with the driver API (not the device's primary
context), then in the primary context, on the same synthetic fields.  The
fields are allocated and copied with the driver API in whichever context is
current, so every pointer the entry point gets belongs to that context.
Prints one JSON line {"own": {...}, "primary": {...}}.
"""
import ctypes as C
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

from paper_2512_21696_gb300 import _lib  # noqa: E402
from noalloc_fields import synthetic_fields  # noqa: E402

cu = C.CDLL("libcuda.so.1")
u64 = C.c_uint64


def ck(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} returned {rc}")


def run_in_current_context(lib, f):
    """Allocate, copy, call, free: all in the context current to this thread."""
    ptrs = {}
    try:
        for key in ("fields", "cell", "phi"):
            arr = np.ascontiguousarray(f[key])
            p = u64(0)
            ck(cu.cuMemAlloc_v2(C.byref(p), C.c_size_t(arr.nbytes)), "cuMemAlloc")
            ptrs[key] = p
            ck(cu.cuMemcpyHtoD_v2(p, arr.ctypes.data_as(C.c_void_p), C.c_size_t(arr.nbytes)), "cuMemcpyHtoD")
        out = _lib.lbm_obs()
        probe = (C.c_double * 5)(*f["probe"])
        nz, ny, nx = f["shape"]
        results = []
        for _ in range(2):
            rc = lib.lbm_observables_noalloc(C.c_void_p(ptrs["fields"].value), C.c_void_p(ptrs["cell"].value),
                                             C.c_void_p(ptrs["phi"].value), nx, ny, nz, f["G"], probe, None,
                                             C.byref(out))
            results.append(dict(rc=rc, mass=list(out.mass), sat=out.sat, flux_out=out.flux_out,
                                flux_vol=list(out.flux_vol), max_u=out.max_u, dp=out.dp, nan_count=out.nan_count))
        ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
        return results
    finally:
        for p in ptrs.values():
            cu.cuMemFree_v2(p)


def main():
    lib = _lib.load(build_if_needed=False)
    f = synthetic_fields((40, 37, 35), seed=77)
    ck(cu.cuInit(0), "cuInit")
    dev = C.c_int(0)
    ck(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")
    own = C.c_void_p()
    if hasattr(cu, "cuCtxCreate_v2"):
        ck(cu.cuCtxCreate_v2(C.byref(own), C.c_uint(0), dev), "cuCtxCreate")
    else:
        ck(cu.cuCtxCreate_v4(C.byref(own), None, C.c_uint(0), dev), "cuCtxCreate")
    try:
        res_own = run_in_current_context(lib, f)
    finally:
        ck(cu.cuCtxDestroy_v2(own), "cuCtxDestroy")
    prim = C.c_void_p()
    ck(cu.cuDevicePrimaryCtxRetain(C.byref(prim), dev), "cuDevicePrimaryCtxRetain")
    try:
        ck(cu.cuCtxSetCurrent(prim), "cuCtxSetCurrent")
        res_prim = run_in_current_context(lib, f)
    finally:
        cu.cuCtxSetCurrent(None)
        cu.cuDevicePrimaryCtxRelease_v2(dev)
    print(json.dumps({"own": res_own, "primary": res_prim}))


if __name__ == "__main__":
    main()
