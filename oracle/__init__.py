"""FP64 CPU oracle of the two-component D3Q19 pseudo-potential LB step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the library never imports it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, OpenMP).  This module
compiles it with gcc and marshals NumPy arrays through ctypes; it holds no
physics of its own.  Parity of every oracle function is pinned by the
``-m "not gpu"`` tests against closed forms, invariants and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

TERM_SC, TERM_CSF, TERM_CAP, TERM_DRAG, TERM_BODY = range(5)


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("tau", C.c_double * 2),
        ("G", C.c_double),
        ("kappa", C.c_double),
        ("phi_avg", C.c_double * 2),
        ("phi_max", C.c_double * 2),
        ("csf_everywhere", C.c_int),
        ("rho_wall", C.c_double * 2),
        ("accel", (C.c_double * 3) * 2),
        ("wet", C.c_int),
        ("rho_hi", C.c_double), ("rho_lo", C.c_double),
        ("s_lo", C.c_double), ("s_hi", C.c_double), ("at_cut", C.c_double),
        ("eps_n", C.c_double), ("kr_min", C.c_double), ("c_g", C.c_double),
        ("rho_in", C.c_double * 2), ("rho_out", C.c_double * 2),
        ("lattice", C.c_int),
        ("mss", C.c_double),
        ("csf_div", C.c_int),
    ]


class OrcCurve(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("kc_d", "pd", "lambda_", "swr", "nw", "nn", "phi_ref", "f_max", "f_min", "aniso", "thomeer_g")]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcCurve), C.c_int, u8, dp, u8]
        lib.orc_destroy.argtypes = [P]
        lib.orc_init_fields.argtypes = [P, dp, dp, C.c_void_p]
        lib.orc_step.argtypes = [P, C.c_int]
        lib.orc_fields.argtypes = [P, dp, dp, dp, dp]
        lib.orc_force_term.argtypes = [P, C.c_int, C.c_int, dp]
        lib.orc_static.argtypes = [P, dp, dp, dp, dp, dp, ip]
        lib.orc_observables.argtypes = [P, dp, dp]
        lib.orc_observables_of.argtypes = [C.c_int, C.c_int, C.c_int, u8, dp, dp, dp, dp, dp, C.c_double, dp, dp]
        lib.orc_set_populations.argtypes = [P, dp]
        lib.orc_set_pressure.argtypes = [P, dp, dp]
        lib.orc_set_mss.argtypes = [P, C.c_double]
        lib.orc_get_populations.argtypes = [P, dp]
        lib.orc_set_residual.argtypes = [P, dp, dp, ip]
        lib.orc_get_residual.argtypes = [P, dp, dp, ip]
        lib.orc_collide_cell.argtypes = [dp, dp, dp, C.c_double, dp]
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_max_threads.restype = C.c_int
        lib.orc_q.restype = C.c_int
        lib.orc_q.argtypes = [P]
        lib.orc_steps.restype = C.c_long
        lib.orc_steps.argtypes = [P]
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def collide_cell(f, u, F, tau):
    """Post-collision populations of one component at one cell."""
    out = np.zeros(19)
    _load().orc_collide_cell(np.ascontiguousarray(f, dtype=np.float64),
                             np.ascontiguousarray(u, dtype=np.float64),
                             np.ascontiguousarray(F, dtype=np.float64), float(tau), out)
    return out


def observables_of(cell, phi, rhoA, rhoB, u, sw, G, probe=(0.0, 0.0, 0.0, 0.0, 1e30)):
    """Observables (the definitions of Oracle.observables) of given fields on a
    grid of shape (nz, ny, nx); u has shape (3, nz, ny, nx).  FP64."""
    nz, ny, nx = np.shape(cell)
    out = np.zeros(10)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    _load().orc_observables_of(nx, ny, nz, np.ascontiguousarray(cell, np.uint8).reshape(-1), f64(phi), f64(rhoA),
                               f64(rhoB), f64(u), f64(sw), float(G), np.asarray(probe, dtype=np.float64), out)
    return dict(mass=(out[0], out[1]), sat=out[2], flux_out=out[3], flux_vol=(out[4], out[5], out[6]),
                max_u=out[7], dp=out[8], nan_count=int(out[9]))


def make_params(shape, **kw) -> OrcParams:
    """Oracle parameters for a grid of shape (nz, ny, nx); keywords override."""
    nz, ny, nx = shape
    p = OrcParams()
    p.nx, p.ny, p.nz = nx, ny, nz
    per = kw.pop("periodic", (1, 1, 1))
    for d in range(3):
        p.periodic[d] = int(per[d])
    rho_hi = kw.pop("rho_hi", 1.0)
    rho_lo = kw.pop("rho_lo", 0.03)
    p.rho_hi, p.rho_lo = rho_hi, rho_lo
    tau = kw.pop("tau", (1.0, 1.0))
    p.tau[0], p.tau[1] = tau
    p.G = kw.pop("G", 0.0)
    p.kappa = kw.pop("kappa", 0.0)
    pav = kw.pop("phi_avg", (0.5 * (rho_hi + rho_lo),) * 2)
    pmx = kw.pop("phi_max", (rho_hi,) * 2)
    p.phi_avg[0], p.phi_avg[1] = pav
    p.phi_max[0], p.phi_max[1] = pmx
    p.csf_everywhere = int(kw.pop("csf_everywhere", 0))
    rw = kw.pop("rho_wall", (0.5 * (rho_hi + rho_lo),) * 2)
    p.rho_wall[0], p.rho_wall[1] = rw
    acc = kw.pop("accel", ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)))
    for a in range(2):
        for d in range(3):
            p.accel[a][d] = acc[a][d]
    p.wet = int(kw.pop("wet", 1))
    p.s_lo = kw.pop("s_lo", 0.1)
    p.s_hi = kw.pop("s_hi", 0.9)
    p.at_cut = kw.pop("at_cut", 0.95)
    p.eps_n = kw.pop("eps_n", 1e-4 * rho_hi)
    p.kr_min = kw.pop("kr_min", 1e-6)
    p.c_g = kw.pop("c_g", 1.0)
    p.lattice = {"d3q19": 0, "d2q9": 1}[kw.pop("lattice", "d3q19")]
    p.mss = kw.pop("mss", 0.0)
    p.csf_div = {"identity": 0, "neighbour_normals": 1}[kw.pop("csf_div", "identity")]
    rin = kw.pop("rho_in", (rho_hi, rho_lo))
    rout = kw.pop("rho_out", (rho_hi, rho_lo))
    for a in range(2):
        p.rho_in[a], p.rho_out[a] = rin[a], rout[a]
    if kw:
        raise TypeError(f"unknown oracle parameters {sorted(kw)}")
    return p


def make_curve(**kw) -> OrcCurve:
    c = OrcCurve()
    vals = dict(kc_d=1.0, pd=0.02, lambda_=2.0, swr=0.15, nw=3.0, nn=2.0, phi_ref=0.35,
                f_max=3.5, f_min=0.575, aniso=1.0, thomeer_g=0.0)
    if "lam" in kw:
        kw["lambda_"] = kw.pop("lam")
    vals.update(kw)
    for k, v in vals.items():
        setattr(c, k, float(v))
    return c


class Oracle:
    """One oracle lattice.  Arrays are NumPy, indexed [z][y][x] (x fastest)."""

    def __init__(self, params: OrcParams, cell, phi=None, ptype=None, curves=None):
        self.lib = _load()
        self.shape = (params.nz, params.ny, params.nx)
        self.n = int(params.nx) * params.ny * params.nz
        self.params = params
        cell = np.ascontiguousarray(cell, dtype=np.uint8).reshape(-1)
        assert cell.size == self.n
        phi = np.ones(self.n) if phi is None else np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        ptype = (np.zeros(self.n, np.uint8) if ptype is None
                 else np.ascontiguousarray(ptype, dtype=np.uint8).reshape(-1))
        curves = curves or [make_curve()]
        arr = (OrcCurve * len(curves))(*curves)
        self._h = self.lib.orc_create(C.byref(params), arr, len(curves), cell, phi, ptype)
        if not self._h:
            raise RuntimeError("orc_create failed")
        self.cell = cell
        self.Q = int(self.lib.orc_q(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init_fields(self, rhoA, rhoB, u=None):
        ra = np.ascontiguousarray(rhoA, dtype=np.float64).reshape(-1)
        rb = np.ascontiguousarray(rhoB, dtype=np.float64).reshape(-1)
        if u is None:
            self.lib.orc_init_fields(self._h, ra, rb, None)
        else:
            uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
            assert uu.size == 3 * self.n
            self.lib.orc_init_fields(self._h, ra, rb, uu.ctypes.data_as(C.c_void_p))
            self._keep = uu

    def step(self, n: int = 1):
        self.lib.orc_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(self.lib.orc_steps(self._h))

    def fields(self):
        """(rhoA, rhoB, u[3], Sw) of the last step, shaped like the grid."""
        n = self.n
        ra, rb, u, sw = np.zeros(n), np.zeros(n), np.zeros(3 * n), np.zeros(n)
        self.lib.orc_fields(self._h, ra, rb, u, sw)
        s = self.shape
        return ra.reshape(s), rb.reshape(s), u.reshape((3,) + s), sw.reshape(s)

    def force_term(self, term: int, comp: int):
        out = np.zeros(3 * self.n)
        self.lib.orc_force_term(self._h, int(term), int(comp), out)
        return out.reshape((3,) + self.shape)

    def static(self):
        n = self.n
        kinv, K0, lamL = np.zeros(9 * n), np.zeros(n), np.zeros(n)
        swirr, sores, iso = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
        self.lib.orc_static(self._h, kinv, K0, lamL, swirr, sores, iso)
        s = self.shape
        return dict(kinv=kinv.reshape((3, 3) + s), K0=K0.reshape(s), lamL=lamL.reshape(s),
                    swirr=swirr.reshape(s), sores=sores.reshape(s), iso=iso.reshape(s))

    def observables(self, probe=(0.0, 0.0, 0.0, 0.0, 1e30)):
        out = np.zeros(10)
        self.lib.orc_observables(self._h, np.asarray(probe, dtype=np.float64), out)
        return dict(mass=(out[0], out[1]), sat=out[2], flux_out=out[3],
                    flux_vol=(out[4], out[5], out[6]), max_u=out[7], dp=out[8],
                    nan_count=int(out[9]))

    def set_mss(self, rate):
        """Mass-sink-source rate (wetting gains m I per step) from the next step."""
        self.lib.orc_set_mss(self._h, float(rate))

    def set_pressure(self, rho_in, rho_out):
        """Densities (A, B) held in the inlet and outlet cells from the next step."""
        self.lib.orc_set_pressure(self._h, np.asarray(rho_in, dtype=np.float64),
                                  np.asarray(rho_out, dtype=np.float64))

    def populations(self):
        f = np.zeros(2 * self.Q * self.n)
        self.lib.orc_get_populations(self._h, f)
        return f.reshape((2, self.Q) + self.shape)

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert f.size == 2 * self.Q * self.n
        self.lib.orc_set_populations(self._h, f)

    def residual(self):
        n = self.n
        Rw, Ro, wet = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
        self.lib.orc_get_residual(self._h, Rw, Ro, wet)
        s = self.shape
        return Rw.reshape(s), Ro.reshape(s), wet.reshape(s)

    def set_residual(self, Rw, Ro, wet):
        self.lib.orc_set_residual(self._h, np.ascontiguousarray(Rw, np.float64).reshape(-1),
                                  np.ascontiguousarray(Ro, np.float64).reshape(-1),
                                  np.ascontiguousarray(wet, np.int32).reshape(-1))
