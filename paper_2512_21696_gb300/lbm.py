"""Python binding of the C ABI: the same entry points, argument marshalling only.

Arrays may be NumPy arrays (host memory) or CUDA tensors exposing
``data_ptr()`` and ``is_cuda`` (device memory); all arrays of one call must be
of the same kind.  Per-cell arrays are indexed [z][y][x] (x fastest), vector
fields [3][z][y][x].  Errors raise :class:`LbmError` carrying the status code.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import (LBM_CELL_GRAY, LBM_CELL_INLET, LBM_CELL_OUTLET, LBM_CELL_PORE, LBM_CELL_SOLID,
                   LBM_MEM_DEVICE, LBM_MEM_HOST,
                   LBM_STORAGE_BF16S, LBM_STORAGE_F16S, LBM_STORAGE_F32, lbm_constitutive,
                   lbm_params)

__all__ = [
    "LbmError", "LbmContext", "lbm_default_params", "lbm_default_constitutive", "lbm_create",
    "lbm_destroy", "lbm_set_constitutive", "lbm_set_geometry", "lbm_init_fields", "lbm_step",
    "lbm_observables", "lbm_get_fields", "lbm_get_static", "lbm_save_state", "lbm_load_state",
    "lbm_profile", "lbm_profile_read", "lbm_launch_count", "lbm_abi_version", "lbm_observables_noalloc", "lbm_set_kernel",
    "lbm_get_kernel",
    "lbm_set_pressure", "lbm_pressure_levels", "LBM_CELL_INLET", "LBM_CELL_OUTLET", "lbm_set_mss",
    "lbm_mss_to_saturation", "lbm_batch_mss_to_saturation", "lbm_observables_async", "lbm_obs_decode",
    "LBM_OBS_RAW",
    "LBM_CELL_PORE", "LBM_CELL_SOLID", "LBM_CELL_GRAY", "LBM_STORAGE_F32", "LBM_STORAGE_F16S",
    "LBM_STORAGE_BF16S",
]


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = L.load()
        msg = lib.lbm_strerror(code).decode()
        cuda = lib.lbm_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})" + (f" [{cuda}]" if code in (L.LBM_ERR_CUDA, L.LBM_ERR_OOM) and cuda else ""))
        self.code = code


def _check(code: int, where: str) -> int:
    if code != L.LBM_OK:
        raise LbmError(code, where)
    return code


class LbmContext:
    """Owning handle of one lattice (``lbm_destroy`` on close / garbage collection)."""

    def __init__(self, handle: int, params: lbm_params):
        self.handle = C.c_void_p(handle)
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.ncell = params.nx * params.ny * params.nz
        self._keep = []

    def close(self):
        if getattr(self, "_view_of", None) is not None:  # a batch run: owned by its batch
            self.handle = C.c_void_p(None)
            return
        if self.handle and self.handle.value:
            L.load().lbm_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ----------------------------------------------------------------- marshalling
def _is_device(a) -> bool:
    return hasattr(a, "data_ptr") and bool(getattr(a, "is_cuda", False))


def _mem_kind(arrays) -> int:
    present = [a for a in arrays if a is not None]
    kinds = {_is_device(a) for a in present}
    if len(kinds) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return LBM_MEM_DEVICE if kinds == {True} else LBM_MEM_HOST


_TORCH_DTYPES = {np.float32: "float32", np.uint8: "uint8"}


def _ptr(a, dtype, count, keep):
    """Pointer of a host or device array holding `count` elements of `dtype`."""
    if a is None:
        return None
    if _is_device(a):
        want = _TORCH_DTYPES[dtype]
        if str(a.dtype).split(".")[-1] != want:
            raise TypeError(f"device array must be {want}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("device array must be contiguous")
        if a.numel() != count:
            raise ValueError(f"device array has {a.numel()} elements, expected {count}")
        return a.data_ptr()
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size != count:
        raise ValueError(f"array has {arr.size} elements, expected {count}")
    keep.append(arr)
    return arr.ctypes.data


# ----------------------------------------------------------------- entry points
def lbm_abi_version() -> int:
    return L.load().lbm_abi_version()


def lbm_default_params(nx: int, ny: int, nz: int, **overrides) -> lbm_params:
    p = lbm_params()
    _check(L.load().lbm_default_params(C.byref(p), int(nx), int(ny), int(nz)), "lbm_default_params")
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        if not hasattr(p, k):
            raise AttributeError(f"lbm_params has no field {k}")
        fld = getattr(p, k)
        if isinstance(fld, C.Array):
            for i, item in enumerate(v):
                if isinstance(fld[i], C.Array):
                    for j, x in enumerate(item):
                        fld[i][j] = x
                else:
                    fld[i] = item
        else:
            setattr(p, k, v)
    return p


def lbm_default_constitutive(**overrides) -> lbm_constitutive:
    c = lbm_constitutive()
    _check(L.load().lbm_default_constitutive(C.byref(c)), "lbm_default_constitutive")
    for k, v in overrides.items():
        setattr(c, "lambda_" if k in ("lambda", "lam") else k, float(v))
    return c


def lbm_create(params: lbm_params) -> LbmContext:
    h = C.c_void_p()
    _check(L.load().lbm_create(C.byref(h), C.byref(params)), "lbm_create")
    return LbmContext(h.value, params)


def lbm_destroy(ctx: LbmContext) -> None:
    ctx.close()


def lbm_set_constitutive(ctx: LbmContext, pore_type: int, c: lbm_constitutive) -> None:
    _check(L.load().lbm_set_constitutive(ctx.handle, int(pore_type), C.byref(c)), "lbm_set_constitutive")


def lbm_set_geometry(ctx: LbmContext, cell_type, phi, pore_type=None) -> None:
    keep = []
    mem = _mem_kind([cell_type, phi, pore_type])
    n = ctx.ncell
    _check(L.load().lbm_set_geometry(ctx.handle, _ptr(cell_type, np.uint8, n, keep),
                                     _ptr(phi, np.float32, n, keep),
                                     _ptr(pore_type, np.uint8, n, keep), mem), "lbm_set_geometry")


def lbm_init_fields(ctx: LbmContext, rhoA, rhoB, u=None) -> None:
    keep = []
    mem = _mem_kind([rhoA, rhoB, u])
    n = ctx.ncell
    _check(L.load().lbm_init_fields(ctx.handle, _ptr(rhoA, np.float32, n, keep),
                                    _ptr(rhoB, np.float32, n, keep),
                                    _ptr(u, np.float32, 3 * n, keep), mem), "lbm_init_fields")


def lbm_step(ctx: LbmContext, nsteps: int = 1) -> None:
    _check(L.load().lbm_step(ctx.handle, int(nsteps)), "lbm_step")


def lbm_set_pressure(ctx: LbmContext, rho_in, rho_out) -> None:
    """Densities (A, B) held in the inlet and in the outlet cells from the next step."""
    a = (C.c_double * 2)(*[float(v) for v in rho_in])
    b = (C.c_double * 2)(*[float(v) for v in rho_out])
    _check(L.load().lbm_set_pressure(ctx.handle, a, b), "lbm_set_pressure")


def lbm_set_mss(ctx: LbmContext, rate: float) -> None:
    """Mass-sink-source rate (wetting component gains rate * I per step) from the next step."""
    _check(L.load().lbm_set_mss(ctx.handle, float(rate)), "lbm_set_mss")


def lbm_mss_to_saturation(ctx: LbmContext, target: float, gain: float, max_rate: float, tol: float,
                          check_every: int, max_steps: int):
    """Drive the saturation to target with the mass-sink-source; returns (reached, steps)."""
    done = C.c_int()
    code = L.load().lbm_mss_to_saturation(ctx.handle, float(target), float(gain), float(max_rate), float(tol),
                                          int(check_every), int(max_steps), C.byref(done))
    if code not in (L.LBM_OK, L.LBM_ERR_TIMEOUT):
        _check(code, "lbm_mss_to_saturation")
    return code == L.LBM_OK, done.value


def lbm_batch_mss_to_saturation(batch, targets, gain: float, max_rate: float, tol: float, check_every: int,
                                max_steps: int):
    """Every run of a batch to its own target saturation; returns (reached, steps)."""
    t = (C.c_double * len(targets))(*[float(v) for v in targets])
    done = C.c_int()
    code = L.load().lbm_batch_mss_to_saturation(batch.handle, t, float(gain), float(max_rate), float(tol),
                                                int(check_every), int(max_steps), C.byref(done))
    if code not in (L.LBM_OK, L.LBM_ERR_TIMEOUT):
        _check(code, "lbm_batch_mss_to_saturation")
    return code == L.LBM_OK, done.value


def lbm_pressure_levels(ctx: LbmContext, levels, check_every: int, sat_tol: float, max_steps: int):
    """Stepped-pressure protocol: levels = [((rhoA_in, rhoB_in), (rhoA_out, rhoB_out)), ...].
    Returns (all_steady, saturation per level, steps per level)."""
    k = len(levels)
    rin = (C.c_double * (2 * k))(*[float(v) for lv in levels for v in lv[0]])
    rout = (C.c_double * (2 * k))(*[float(v) for lv in levels for v in lv[1]])
    sat, steps = (C.c_double * k)(), (C.c_int * k)()
    code = L.load().lbm_pressure_levels(ctx.handle, k, rin, rout, int(check_every), float(sat_tol),
                                        int(max_steps), sat, steps)
    if code not in (L.LBM_OK, L.LBM_ERR_TIMEOUT):
        _check(code, "lbm_pressure_levels")
    return code == L.LBM_OK, list(sat), list(steps)


LBM_OBS_RAW = L.LBM_OBS_RAW


def lbm_observables_async(ctx: LbmContext, raw_ptr: int) -> None:
    """Enqueue the observables into LBM_OBS_RAW doubles of (pinned) host memory at raw_ptr."""
    _check(L.load().lbm_observables_async(ctx.handle, C.c_void_p(int(raw_ptr))), "lbm_observables_async")


def lbm_obs_decode(ctx: LbmContext, raw_ptr: int, check: bool = True) -> dict:
    """Observables from raw sums written by lbm_observables_async (after the stream passed the copy)."""
    o = L.lbm_obs()
    code = L.load().lbm_obs_decode(ctx.handle, C.c_void_p(int(raw_ptr)), C.byref(o))
    if code not in (L.LBM_OK, L.LBM_ERR_NUMERIC) or (check and code != L.LBM_OK):
        raise LbmError(code, "lbm_obs_decode")
    return _obs_dict(o)


def _obs_dict(o) -> dict:
    return dict(mass=(o.mass[0], o.mass[1]), sat=o.sat, flux_out=o.flux_out,
                flux_vol=tuple(o.flux_vol), max_u=o.max_u, dp=o.dp, nan_count=o.nan_count, step=o.step)


def lbm_observables(ctx: LbmContext, check: bool = True) -> dict:
    o = L.lbm_obs()
    code = L.load().lbm_observables(ctx.handle, C.byref(o))
    if code not in (L.LBM_OK, L.LBM_ERR_NUMERIC) or (check and code != L.LBM_OK):
        raise LbmError(code, "lbm_observables")
    return _obs_dict(o)


def lbm_get_fields(ctx: LbmContext, rhoA=None, rhoB=None, u=None, sw=None):
    """Copy the current fields into the given arrays, or return host copies."""
    n, s = ctx.ncell, ctx.shape
    if rhoA is None and rhoB is None and u is None and sw is None:
        rhoA, rhoB = np.empty(s, np.float32), np.empty(s, np.float32)
        u, sw = np.empty((3,) + s, np.float32), np.empty(s, np.float32)
    mem = _mem_kind([rhoA, rhoB, u, sw])
    for a in (rhoA, rhoB, u, sw):
        if a is not None and not _is_device(a) and (not isinstance(a, np.ndarray) or a.dtype != np.float32
                                                    or not a.flags.c_contiguous):
            raise TypeError("host outputs must be C-contiguous float32 NumPy arrays")
    keep = []
    _check(L.load().lbm_get_fields(ctx.handle, _ptr(rhoA, np.float32, n, keep), _ptr(rhoB, np.float32, n, keep),
                                   _ptr(u, np.float32, 3 * n, keep), _ptr(sw, np.float32, n, keep), mem),
           "lbm_get_fields")
    return rhoA, rhoB, u, sw


def lbm_get_static(ctx: LbmContext):
    """Host copies of (K^-1 [6][...] as xx,yy,zz,xy,xz,yz; lamL*pd; Sw_irr; So_res)."""
    n, s = ctx.ncell, ctx.shape
    kinv = np.empty((6,) + s, np.float32)
    pcs, swirr, sores = (np.empty(s, np.float32) for _ in range(3))
    _check(L.load().lbm_get_static(ctx.handle, kinv.ctypes.data, pcs.ctypes.data, swirr.ctypes.data,
                                   sores.ctypes.data, LBM_MEM_HOST), "lbm_get_static")
    return kinv, pcs, swirr, sores


def lbm_save_state(ctx: LbmContext) -> bytes:
    lib = L.load()
    size = C.c_size_t()
    _check(lib.lbm_state_size(ctx.handle, C.byref(size)), "lbm_state_size")
    buf = C.create_string_buffer(size.value)
    _check(lib.lbm_save_state(ctx.handle, buf, size.value), "lbm_save_state")
    return buf.raw


def lbm_load_state(ctx: LbmContext, data: bytes) -> None:
    buf = C.create_string_buffer(data, len(data))
    _check(L.load().lbm_load_state(ctx.handle, buf, len(data)), "lbm_load_state")


def lbm_profile(ctx: LbmContext, enable: bool = True) -> None:
    _check(L.load().lbm_profile(ctx.handle, int(bool(enable))), "lbm_profile")


def lbm_profile_read(ctx: LbmContext) -> dict:
    arr = (L.lbm_kernel_stat * 32)()
    cnt = C.c_int()
    _check(L.load().lbm_profile_read(ctx.handle, arr, 32, C.byref(cnt)), "lbm_profile_read")
    return {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms) for k in range(min(cnt.value, 32))}


def lbm_set_kernel(ctx: LbmContext, path: int = 0, tile: int = 8) -> None:
    """Kernel path of lbm_step: 0 fused (default), 1 two launches; fused tile 0 = 32x8, 1 = 32x16,
    2 = 32x8 two CTAs per SM, 3 = 32x12, 4 = 64x8, 5 / 6 = the published-density march (32x8 / 32x7),
    7 = 64x7, 8 = chosen per grid among 2, 4 and 7 (default)."""
    _check(L.load().lbm_set_kernel(ctx.handle, int(path), int(tile)), "lbm_set_kernel")


def lbm_get_kernel(ctx: LbmContext) -> tuple:
    """(path, tile) a step of ctx runs, with tile 8 resolved to the shape chosen for the grid."""
    path, tile = C.c_int(), C.c_int()
    _check(L.load().lbm_get_kernel(ctx.handle, C.byref(path), C.byref(tile)), "lbm_get_kernel")
    return path.value, tile.value


def lbm_inject_launch_failures(ctx: LbmContext, count: int) -> None:
    """Testing hook: the next `count` step launches are rejected by the CUDA runtime on the host."""
    _check(L.load().lbm_inject_launch_failures(ctx.handle, int(count)), "lbm_inject_launch_failures")


def lbm_launch_count(ctx: LbmContext) -> int:
    c = C.c_longlong()
    _check(L.load().lbm_launch_count(ctx.handle, C.byref(c)), "lbm_launch_count")
    return c.value


def lbm_observables_noalloc(fields, cell_type, phi, shape, G, probe, stream=None, check: bool = True) -> dict:
    """Observables of caller-owned device fields without any device allocation.

    For callers that cannot allocate device memory (host callbacks, allocator
    hooks, plug-ins whose application owns the memory pool).  `fields` is a
    device float32 array of 6*ncell values (rhoA, rhoB, ux, uy, uz, Sw rows),
    `cell_type` uint8 and `phi` float32 device arrays of ncell values, `shape`
    (nz, ny, nx), `probe` (cx, cy, cz, r_in, r_out).  The library's shared
    device scratch is used, so concurrent calls on different streams race.
    """
    nz, ny, nx = shape
    n = nx * ny * nz
    for a in (fields, cell_type, phi):
        if not _is_device(a):
            raise TypeError("lbm_observables_noalloc takes device arrays only")
    keep = []
    pr = (C.c_double * 5)(*[float(v) for v in probe])
    o = L.lbm_obs()
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    code = L.load().lbm_observables_noalloc(_ptr(fields, np.float32, 6 * n, keep), _ptr(cell_type, np.uint8, n, keep),
                                            _ptr(phi, np.float32, n, keep), int(nx), int(ny), int(nz), float(G), pr,
                                            s, C.byref(o))
    if code not in (L.LBM_OK, L.LBM_ERR_NUMERIC) or (check and code != L.LBM_OK):
        raise LbmError(code, "lbm_observables_noalloc")
    return dict(mass=(o.mass[0], o.mass[1]), sat=o.sat, flux_out=o.flux_out,
                flux_vol=tuple(o.flux_vol), max_u=o.max_u, dp=o.dp, nan_count=o.nan_count, step=o.step)


# ---------------------------------------------------------------- batches
class LbmBatch:
    """Owning handle of a batch of lattices (``lbm_batch_destroy`` on close)."""

    def __init__(self, handle: int, runs):
        self.handle = C.c_void_p(handle)
        self.runs = list(runs)

    def close(self):
        if self.handle and self.handle.value:
            L.load().lbm_batch_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def lbm_batch_create(runs) -> LbmBatch:
    arr = (lbm_params * len(runs))(*runs)
    h = C.c_void_p()
    _check(L.load().lbm_batch_create(C.byref(h), len(runs), arr), "lbm_batch_create")
    return LbmBatch(h.value, runs)


def lbm_batch_run(batch: LbmBatch, run: int) -> LbmContext:
    """The context of one run (a view of the batch's buffers)."""
    h = C.c_void_p()
    _check(L.load().lbm_batch_run(batch.handle, int(run), C.byref(h)), "lbm_batch_run")
    ctx = LbmContext(h.value, batch.runs[run])
    ctx._view_of = batch
    return ctx


def lbm_batch_step(batch: LbmBatch, nsteps: int) -> None:
    _check(L.load().lbm_batch_step(batch.handle, int(nsteps)), "lbm_batch_step")


def lbm_batch_tune(batch: LbmBatch, trial_steps: int = 10):
    tiles = (C.c_int * len(batch.runs))()
    _check(L.load().lbm_batch_tune(batch.handle, int(trial_steps), tiles), "lbm_batch_tune")
    return list(tiles)


def lbm_batch_observables(batch: LbmBatch, check: bool = True) -> list:
    """lbm_observables of every run (one dict per run)."""
    arr = (L.lbm_obs * len(batch.runs))()
    code = L.load().lbm_batch_observables(batch.handle, arr)
    if code not in (L.LBM_OK, L.LBM_ERR_NUMERIC) or (check and code != L.LBM_OK):
        raise LbmError(code, "lbm_batch_observables")
    return [dict(mass=(o.mass[0], o.mass[1]), sat=o.sat, flux_out=o.flux_out, flux_vol=tuple(o.flux_vol),
                 max_u=o.max_u, dp=o.dp, nan_count=o.nan_count, step=o.step) for o in arr]


def lbm_batch_step_to_steady(batch: LbmBatch, check_every: int, rel_tol: float, max_steps: int):
    """(steady, steps taken): steps until every run's mean velocity settles."""
    done = C.c_int()
    code = L.load().lbm_batch_step_to_steady(batch.handle, int(check_every), float(rel_tol), int(max_steps),
                                             C.byref(done))
    if code not in (L.LBM_OK, L.LBM_ERR_TIMEOUT):
        raise LbmError(code, "lbm_batch_step_to_steady")
    return code == L.LBM_OK, done.value


def lbm_batch_info(batch: LbmBatch) -> dict:
    cells, steps, launches = C.c_longlong(), C.c_longlong(), C.c_longlong()
    groups = C.c_int()
    _check(L.load().lbm_batch_info(batch.handle, C.byref(cells), C.byref(steps), C.byref(launches),
                                   C.byref(groups)), "lbm_batch_info")
    return dict(cells=cells.value, steps=steps.value, launches=launches.value, groups=groups.value)


# ------------------------------------------------------ porosity gradient
def lbm_adjoint_run(ctx: LbmContext, q_target: float, s_target: float, nsteps: int, ckpt: int, out=None):
    """(L, q, S, dL/dphi) after nsteps from the current state (see lbm.h).

    out: optional float32 array (NumPy) or CUDA tensor of n cells receiving
    dL/dphi; a NumPy array is returned when it is None."""
    loss = L.lbm_loss(float(q_target), float(s_target))
    res = (C.c_double * 3)()
    if out is None:
        out = np.empty(ctx.shape, np.float32)
    if not _is_device(out) and (not isinstance(out, np.ndarray) or out.dtype != np.float32
                                or not out.flags.c_contiguous):
        raise TypeError("host output must be a C-contiguous float32 NumPy array")
    keep = []
    ptr = _ptr(out, np.float32, ctx.ncell, keep)
    _check(L.load().lbm_adjoint_run(ctx.handle, C.byref(loss), int(nsteps), int(ckpt), ptr, _mem_kind([out]), res),
           "lbm_adjoint_run")
    return res[0], res[1], res[2], out
