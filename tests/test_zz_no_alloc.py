"""lbm_observables_noalloc against lbm_observables, through the C ABI.

Some callers cannot allocate device memory: code running in host callbacks or
allocator hooks, plug-ins whose host application owns the device memory pool,
and loops that must not risk an allocation's implicit synchronisation.  The
no-allocation entry point serves them by keeping the reduction's partial sums
in a file-scope device array.  Two calls in a row on the fields of a running
lattice must agree with the context's own observables; the second call also
shows that leftovers of the first in the shared array do not leak into it.
Synthetic fields on grids whose reductions span the largest block count, one
block and sixteen blocks (largest first, so that later calls start on an
array that an earlier call filled further) must agree with the FP64 oracle's
observables of the same fields.  In a separate process the entry point also
runs in a context the caller created with the driver API, where the array has
a device address of its own.  This file is collected last on purpose.
"""
import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import lbm_cases as LC
from noalloc_fields import synthetic_fields

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _close(a, b):
    return abs(a - b) <= TOL * max(abs(b), 1e-12)


def test_noalloc_observables_match_context_observables():
    import torch

    from paper_2512_21696_gb300 import _lib, lbm

    lib = _lib.load()
    case = LC.mixed_features(n=12, seed=21)
    nz, ny, nx = case.shape
    n = nx * ny * nz
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        for k, cv in enumerate(case.curves):
            lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
                kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
        thomeer_g=cv.get("thomeer_g", 0.0)))
        lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
        lbm.lbm_step(ctx, 6)
        ref = lbm.lbm_observables(ctx)
        fields = torch.empty(6 * n, dtype=torch.float32, device="cuda")
        lbm.lbm_get_fields(ctx, fields[0:n], fields[n:2 * n], fields[2 * n:5 * n], fields[5 * n:6 * n])
        torch.cuda.synchronize()
    finally:
        ctx.close()
    cell = torch.from_numpy(case.cell.reshape(-1).copy()).cuda()
    phi = torch.from_numpy(case.phi32.reshape(-1).copy()).cuda()
    probe = (C.c_double * 5)(*case.probe)
    for call in range(2):
        out = _lib.lbm_obs()
        rc = lib.lbm_observables_noalloc(fields.data_ptr(), cell.data_ptr(), phi.data_ptr(), nx, ny, nz,
                                         case.s["G"], probe, None, C.byref(out))
        assert rc == 0, f"call {call}: status {rc}"
        got = dict(mass=tuple(out.mass), sat=out.sat, flux_out=out.flux_out, flux_vol=tuple(out.flux_vol),
                   max_u=out.max_u, dp=out.dp)
        for a in range(2):
            assert _close(got["mass"][a], ref["mass"][a]), (call, got, ref)
        for d in range(3):
            assert abs(got["flux_vol"][d] - ref["flux_vol"][d]) <= TOL * max(abs(ref["flux_vol"][d]), 1e-9)
        for key in ("sat", "max_u", "dp"):
            assert _close(got[key], ref[key]), (call, key, got[key], ref[key])
        assert abs(got["flux_out"] - ref["flux_out"]) <= TOL * max(abs(ref["flux_out"]), 1e-9)
        assert out.nan_count == 0
    # the Python binding of the same entry point
    again = lbm.lbm_observables_noalloc(fields, cell, phi, case.shape, case.s["G"], case.probe)
    assert _close(again["mass"][0], ref["mass"][0])


def test_noalloc_rejects_oversized_grids():
    from paper_2512_21696_gb300 import _lib

    lib = _lib.load()
    out = _lib.lbm_obs()
    probe = (C.c_double * 5)(0, 0, 0, 0, 1)
    dummy = C.c_void_p(1)  # never dereferenced: the size check comes first
    rc = lib.lbm_observables_noalloc(dummy, dummy, dummy, 1 << 15, 1 << 14, 1, 0.0, probe, None, C.byref(out))
    assert rc == -1
    rc = lib.lbm_observables_noalloc(None, dummy, dummy, 4, 4, 4, 0.0, probe, None, C.byref(out))
    assert rc == -1


def _check_against_oracle(f, got, where):
    import oracle as O
    nz, ny, nx = f["shape"]
    n = nx * ny * nz
    fl = f["fields"]
    ref = O.observables_of(f["cell"].reshape(f["shape"]), f["phi"].reshape(f["shape"]), fl[0].reshape(f["shape"]),
                           fl[1].reshape(f["shape"]), fl[2:5].reshape((3,) + f["shape"]), fl[5].reshape(f["shape"]),
                           f["G"], f["probe"])
    umax = float(np.abs(fl[2:5]).max())
    for a in range(2):
        assert abs(got["mass"][a] - ref["mass"][a]) <= 1e-9 * ref["mass"][a], (where, a, got, ref)
    assert abs(got["sat"] - ref["sat"]) <= 1e-6 * ref["sat"], (where, got, ref)
    for d in range(3):
        assert abs(got["flux_vol"][d] - ref["flux_vol"][d]) <= 1e-9 * umax, (where, d, got, ref)
    assert abs(got["flux_out"] - ref["flux_out"]) <= 1e-9 * umax, (where, got, ref)
    assert abs(got["max_u"] - ref["max_u"]) <= 1e-6 * ref["max_u"], (where, got, ref)
    assert abs(got["dp"] - ref["dp"]) <= 1e-6, (where, got, ref)
    assert got["nan_count"] == ref["nan_count"] == 0


def _noalloc(lib, f, dev):
    out = _lib_obs()
    probe = (C.c_double * 5)(*f["probe"])
    nz, ny, nx = f["shape"]
    rc = lib.lbm_observables_noalloc(dev["fields"].data_ptr(), dev["cell"].data_ptr(), dev["phi"].data_ptr(), nx,
                                     ny, nz, f["G"], probe, None, C.byref(out))
    return rc, dict(mass=tuple(out.mass), sat=out.sat, flux_out=out.flux_out, flux_vol=tuple(out.flux_vol),
                    max_u=out.max_u, dp=out.dp, nan_count=out.nan_count)


def _lib_obs():
    from paper_2512_21696_gb300 import _lib
    return _lib.lbm_obs()


def test_noalloc_block_counts_largest_first():
    """112^3 cells reduce over the largest block count (the grid-stride cap of
    the shared array's rows), 12^3 over one block, 32^3 over sixteen; each
    twice in a row against the oracle's FP64 observables of the same fields."""
    import torch

    from paper_2512_21696_gb300 import _lib
    lib = _lib.load()
    for shape, seed in (((112, 112, 112), 1), ((12, 12, 12), 2), ((32, 32, 32), 3)):
        f = synthetic_fields(shape, seed)
        dev = dict(fields=torch.from_numpy(f["fields"]).cuda(), cell=torch.from_numpy(f["cell"]).cuda(),
                   phi=torch.from_numpy(f["phi"]).cuda())
        for call in range(2):
            rc, got = _noalloc(lib, f, dev)
            assert rc == 0, (shape, call, rc)
            _check_against_oracle(f, got, (shape, call))


def test_noalloc_in_a_context_the_caller_created():
    """A driver-API context that is not the device's primary one, then the
    primary context, in a fresh process: the array's address is resolved in
    each, and both give the oracle's observables, twice in a row."""
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "noalloc_context_child.py")
    res = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    f = synthetic_fields((40, 37, 35), seed=77)
    for where in ("own", "primary"):
        for call, got in enumerate(out[where]):
            assert got["rc"] == 0, (where, call, got)
            _check_against_oracle(f, got, (where, call))


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, so it cannot be captured: on a stream
    that is being captured it returns LBM_ERR_ARG before any work, and the
    capture itself stays valid."""
    import torch

    from paper_2512_21696_gb300 import _lib
    lib = _lib.load()
    f = synthetic_fields((8, 8, 8), seed=4)
    dev = dict(fields=torch.from_numpy(f["fields"]).cuda(), cell=torch.from_numpy(f["cell"]).cuda(),
               phi=torch.from_numpy(f["phi"]).cuda())
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    out = _lib.lbm_obs()
    probe = (C.c_double * 5)(*f["probe"])
    codes = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            y = dev["fields"] * 2.0
            codes.append(lib.lbm_observables_noalloc(dev["fields"].data_ptr(), dev["cell"].data_ptr(),
                                                     dev["phi"].data_ptr(), 8, 8, 8, f["G"], probe,
                                                     C.c_void_p(s.cuda_stream), C.byref(out)))
    assert codes == [-1]
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, dev["fields"] * 2.0)
