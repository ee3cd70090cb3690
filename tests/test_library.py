"""CPU checks of the C-ABI library: it builds, loads and exports what the
header declares; the host-only entry points behave as documented."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2512_21696_gb300 import _lib as L
from paper_2512_21696_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]*?\b(lbm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_set_geometry", "lbm_set_constitutive", "lbm_step",
                     "lbm_observables", "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = L.load()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/lbm.h but not exported"
    assert set(L.EXPORTS) <= set(declared_functions())


def test_struct_sizes_match_header_layout():
    lib = L.load()
    lib.lbm_struct_size.restype = C.c_size_t
    lib.lbm_struct_size.argtypes = [C.c_int]
    for which, cls in enumerate((L.lbm_params, L.lbm_constitutive, L.lbm_obs, L.lbm_kernel_stat)):
        assert lib.lbm_struct_size(which) == C.sizeof(cls), cls.__name__
    assert lib.lbm_struct_size(99) == 0


def test_host_only_entry_points():
    assert lbm.lbm_abi_version() == 1
    p = lbm.lbm_default_params(8, 9, 10)
    assert (p.nx, p.ny, p.nz) == (8, 9, 10)
    assert tuple(p.tau) == (1.0, 1.0) and p.rho_hi == 1.0 and p.rho_lo == 0.03
    assert p.storage == lbm.LBM_STORAGE_F32 and p.wet_idx == 1
    c = lbm.lbm_default_constitutive()
    assert (c.pd, c.lambda_, c.swr, c.nw, c.nn, c.phi_ref) == (0.02, 2.0, 0.15, 3.0, 2.0, 0.35)
    assert 3.0 <= c.pc_ref_max_f <= 4.0 and 0.5 <= c.pc_ref_min_f <= 0.65
    lib = L.load()
    assert lib.lbm_strerror(-1) == b"invalid argument"
    assert lib.lbm_default_params(None, 1, 1, 1) == -1
    assert lib.lbm_default_params(C.byref(L.lbm_params()), 0, 1, 1) == -1


def test_create_rejects_bad_parameters_before_touching_a_device():
    bad = lbm.lbm_default_params(4, 4, 4)
    bad.tau[1] = 0.4
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(bad)
    assert e.value.code == -1
    bad = lbm.lbm_default_params(4, 4, 4, storage=7)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(bad)
    # D2Q9 runs one plane with F32 storage; unknown lattices are refused
    for kw in (dict(nz=2, lattice=1), dict(nz=1, lattice=1, storage=3), dict(nz=1, lattice=2)):
        nz = kw.pop("nz")
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(lbm.lbm_default_params(4, 4, nz, **kw))
        assert e.value.code == -1


def test_null_handles_are_rejected():
    lib = L.load()
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_destroy(None) == 0
    assert lib.lbm_observables(None, None) == -1


def test_batch_create_rejects_mixed_physics_and_16bit_shift():
    """Checked before any device work, so this runs without a GPU."""
    import ctypes as C
    from paper_2512_21696_gb300 import _lib, lbm
    lib = _lib.load()
    a = lbm.lbm_default_params(8, 8, 8)
    b = lbm.lbm_default_params(12, 8, 8)
    b.G = a.G + 0.1
    arr = (lbm.lbm_params * 2)(a, b)
    h = C.c_void_p()
    assert lib.lbm_batch_create(C.byref(h), 2, arr) == -1
    assert lib.lbm_batch_create(C.byref(h), 0, arr) == -1
    c = lbm.lbm_default_params(8, 8, 8, storage=1)
    arr1 = (lbm.lbm_params * 1)(c)
    assert lib.lbm_batch_create(C.byref(h), 1, arr1) == -1
    assert lib.lbm_batch_destroy(None) == 0
