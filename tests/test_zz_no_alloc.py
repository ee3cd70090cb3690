"""lbm_observables_noalloc against lbm_observables, through the C ABI.

Some callers cannot allocate device memory: code running in host callbacks or
allocator hooks, plug-ins whose host application owns the device memory pool,
and loops that must not risk an allocation's implicit synchronisation.  The
no-allocation entry point serves them by keeping the reduction's partial sums
in a file-scope device array.  Two calls in a row on the fields of a running
lattice must agree with the context's own observables; the second call also
shows that leftovers of the first in the shared array do not leak into it.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import lbm_cases as LC

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
