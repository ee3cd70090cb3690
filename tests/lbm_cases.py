"""Test cases run on both the CUDA library (through the C ABI) and the oracle.

A case is one dict of settings; `gpu_params` and `oracle_params` translate it
into the two independent parameter blocks.  All floating inputs are rounded
to FP32 first, because that is what the C ABI takes, and the oracle receives
exactly those values in FP64.
"""
from __future__ import annotations

import numpy as np

from paper_2512_21696_gb300 import synth

DEFAULTS = dict(G=0.0, kappa=0.0, tau=(1.0, 1.0), accel=((0, 0, 0), (0, 0, 0)), csf_everywhere=0,
                rho_wall=(0.515, 0.515), wet=1, rho_hi=1.0, rho_lo=0.03, periodic=(1, 1, 1),
                s_lo=0.1, s_hi=0.9, at_cut=0.95, kr_min=1e-6, c_g=1.0, phi_avg=(0.515, 0.515),
                phi_max=(1.0, 1.0), held=None, lattice="d3q19", mss=0.0)
CURVE = dict(kc_d=1.0, pd=0.02, lam=2.0, swr=0.15, nw=3.0, nn=2.0, phi_ref=0.35, f_max=3.5,
             f_min=0.575, aniso=1.0, thomeer_g=0.0)


class Case:
    def __init__(self, name, shape, cell, phi, rhoA, rhoB, u=None, ptype=None, curves=None, **settings):
        self.name = name
        self.shape = tuple(shape)
        self.cell = np.ascontiguousarray(cell, np.uint8)
        phi = np.where(self.cell == synth.GRAY, phi, np.where(self.cell == synth.SOLID, 0.0, 1.0))
        self.phi32 = np.ascontiguousarray(phi, np.float32)
        self.rhoA32 = np.ascontiguousarray(rhoA, np.float32)
        self.rhoB32 = np.ascontiguousarray(rhoB, np.float32)
        self.u32 = None if u is None else np.ascontiguousarray(u, np.float32)
        self.ptype = None if ptype is None else np.ascontiguousarray(ptype, np.uint8)
        self.curves = curves or [dict(CURVE)]
        self.s = dict(DEFAULTS)
        self.s.update(settings)
        self.s["eps_n"] = settings.get("eps_n", 1e-4 * self.s["rho_hi"])
        self.probe = settings.get("probe", (0.5 * (shape[2] - 1), 0.5 * (shape[1] - 1),
                                            0.5 * (shape[0] - 1), 0.0, 1e30))
        self.s.pop("probe", None)


def gpu_params(case: Case, **extra):
    from paper_2512_21696_gb300 import lbm
    nz, ny, nx = case.shape
    s = case.s
    p = lbm.lbm_default_params(nx, ny, nz)
    p.periodic[0], p.periodic[1], p.periodic[2] = s["periodic"]
    p.tau[0], p.tau[1] = s["tau"]
    p.G = s["G"]
    p.kappa_csf = s["kappa"]
    p.phi_avg[0], p.phi_avg[1] = s["phi_avg"]
    p.phi_max[0], p.phi_max[1] = s["phi_max"]
    p.csf_everywhere = s["csf_everywhere"]
    p.rho_wall[0], p.rho_wall[1] = s["rho_wall"]
    for a in range(2):
        for d in range(3):
            p.body_accel[a][d] = s["accel"][a][d]
    p.wet_idx = s["wet"]
    p.rho_hi, p.rho_lo = s["rho_hi"], s["rho_lo"]
    p.s_lo, p.s_hi, p.at_cut = s["s_lo"], s["s_hi"], s["at_cut"]
    p.eps_n, p.kr_min, p.c_g = s["eps_n"], s["kr_min"], s["c_g"]
    p.lattice = {"d3q19": 0, "d2q9": 1}[s["lattice"]]
    cx, cy, cz, rin, rout = case.probe
    p.probe_center[0], p.probe_center[1], p.probe_center[2] = cx, cy, cz
    p.probe_r_in, p.probe_r_out = rin, min(rout, 1e300)
    for k, v in extra.items():
        setattr(p, k, v)
    return p


def oracle_params(case: Case):
    import oracle as O
    s = case.s
    return O.make_params(case.shape, periodic=s["periodic"], tau=s["tau"], G=s["G"], kappa=s["kappa"],
                         phi_avg=s["phi_avg"], phi_max=s["phi_max"], csf_everywhere=s["csf_everywhere"],
                         rho_wall=s["rho_wall"], accel=s["accel"], wet=s["wet"], rho_hi=s["rho_hi"],
                         rho_lo=s["rho_lo"], s_lo=s["s_lo"], s_hi=s["s_hi"], at_cut=s["at_cut"],
                         eps_n=s["eps_n"], kr_min=s["kr_min"], c_g=s["c_g"], lattice=s["lattice"], mss=s["mss"])


def run_gpu(case: Case, steps: int, device_arrays=False, path=0, tile=0, **extra):
    """Fields (rhoA, rhoB, u, sw), observables and static data after `steps`."""
    from paper_2512_21696_gb300 import lbm
    ctx = lbm.lbm_create(gpu_params(case, **extra))
    try:
        lbm.lbm_set_kernel(ctx, path, tile)
        for k, cv in enumerate(case.curves):
            lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
                kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
                thomeer_g=cv["thomeer_g"]))
        if device_arrays:
            import torch
            dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
            lbm.lbm_set_geometry(ctx, dev(case.cell), dev(case.phi32), dev(case.ptype))
            lbm.lbm_init_fields(ctx, dev(case.rhoA32), dev(case.rhoB32), dev(case.u32))
        else:
            lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
            lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
        if case.s["held"] is not None:
            lbm.lbm_set_pressure(ctx, *case.s["held"])
        if case.s["mss"]:
            lbm.lbm_set_mss(ctx, case.s["mss"])
        lbm.lbm_step(ctx, steps)
        fields = lbm.lbm_get_fields(ctx)
        obs = lbm.lbm_observables(ctx, check=False)
        static = lbm.lbm_get_static(ctx)
        return fields, obs, static
    finally:
        ctx.close()


def make_oracle(case: Case):
    import oracle as O
    curves = [O.make_curve(**cv) for cv in case.curves]
    o = O.Oracle(oracle_params(case), case.cell, case.phi32.astype(np.float64), ptype=case.ptype,
                 curves=curves)
    o.init_fields(case.rhoA32.astype(np.float64), case.rhoB32.astype(np.float64),
                  None if case.u32 is None else case.u32.astype(np.float64))
    if case.s["held"] is not None:
        o.set_pressure(*case.s["held"])
    return o


def run_oracle(case: Case, steps: int):
    o = make_oracle(case)
    o.step(steps)
    return o.fields(), o.observables(probe=case.probe), o.static()


# ------------------------------------------------------------------- cases
def droplet(n=32, R=8, kappa=0.0, csf_everywhere=0, tau=(1.0, 1.0), G=1.1):
    """Static droplet, Sec. III.A in 3-D: sphere of A (rho 1.0/0.03) in B."""
    shape = (n, n, n)
    c = n // 2
    rA, rB = synth.droplet_fields(shape, R, (c, c, c), 1.0, 0.03)
    return Case(f"droplet{n}", shape, np.zeros(shape, np.uint8), np.ones(shape), rA, rB, G=G, kappa=kappa,
                csf_everywhere=csf_everywhere, tau=tau, probe=(c, c, c, R - 4, R + 4))


def mixed_features(n=8, seed=5, shape=None, periodic=(1, 1, 1), aniso=10.0, flip_flags=True, tau=(0.8, 1.3),
                   thomeer=0.0):
    """Solid, gray (two pore types, tensorial), walls with wetting densities,
    CSF in gray cells, body forces, both residual transitions; thomeer > 0
    gives the second pore type a Thomeer Pc curve with that factor."""
    rng = np.random.default_rng(seed)
    shape = shape or (n, n, n)
    cell = np.zeros(shape, np.uint8)
    cell[rng.random(shape) < 0.12] = synth.SOLID
    cell[(rng.random(shape) < 0.35) & (cell == 0)] = synth.GRAY
    phi = np.where(cell == synth.GRAY, 0.15 + 0.4 * rng.random(shape), 1.0)
    zz, yy, xx = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
    blocks = ((xx // 4 + yy // 4 + zz // 4) % 2) == 0
    ra = np.where(blocks, 1.0, 0.03) + 0.05 * rng.random(shape)
    rb = 1.06 - ra
    u0 = 0.01 * rng.standard_normal((3,) + shape)
    ptype = (rng.random(shape) < 0.5).astype(np.uint8)
    curves = [dict(CURVE, aniso=aniso), dict(CURVE, kc_d=1.5, pd=0.03, lam=1.5, swr=0.1, nw=2.5,
                                            nn=1.5, aniso=3.0, thomeer_g=thomeer)]
    return Case(f"mixed{shape}", shape, cell, phi, ra, rb, u=u0, ptype=ptype, curves=curves, G=1.1,
                kappa=-0.045, tau=tau, accel=((1e-4, 2e-5, 0), (0, -1e-4, 3e-5)), rho_wall=(0.7, 0.2),
                wet=1, periodic=periodic)


def drainage(n=128, seed=synth.SEED_BASE + 1):
    """Synthetic multiscale rock drainage: A injected from the x < 8 slab by a
    body force 1e-5 into wetting B; KC d = 1, Brooks-Corey Pd 0.02 lambda 2,
    Corey 3/2, Swr 0.15, CSF kappa = -0.045 in gray cells."""
    cell, phi, ptype = synth.drainage_geometry(n, seed)
    rA, rB = synth.drainage_fields(cell, 1.0, 0.03)
    return Case(f"drainage{n}", (n, n, n), cell, phi, rA, rB, ptype=ptype, G=1.1, kappa=-0.045,
                accel=((1e-5, 0, 0), (0, 0, 0)), rho_wall=(0.03, 1.0), wet=1)


def fiber_flow(n=24, axis=0, seed=synth.SEED_BASE + 2, ncyl=12, aniso=10.0, g=1e-5):
    """Fibre-bundle permeability (tensorial resistivity, anisotropy 10): wetting
    B at rho_hi everywhere with A dissolved at rho_lo, body acceleration g on
    B along `axis`.  Darcy: K_axis = <u_axis> nu / g with <u> over all cells."""
    cell, phi, ptype, _ = synth.fiber_bundle_geometry(n, seed, ncyl=ncyl)
    shape = cell.shape
    acc = [0.0, 0.0, 0.0]
    acc[axis] = g
    return Case(f"fiber{n}_{'xyz'[axis]}", shape, cell, phi, np.full(shape, 0.03), np.full(shape, 1.0),
                ptype=ptype, curves=[dict(CURVE, aniso=aniso)], G=1.1, accel=((0, 0, 0), tuple(acc)),
                rho_wall=(0.03, 1.0), wet=1)


def imbibition(n=32, seed=synth.SEED_BASE + 6, dp=0.02, tau=(1.0, 1.0), nz=None):
    """Pressure-driven imbibition (the set-ups of Sec. I and the Appendix):
    the synthetic multiscale rock between an inlet reservoir plane of wetting
    B (z = 0, rho_B = 1 + dp) and an outlet plane of non-wetting A
    (z = nz - 1), z not periodic.  The rock starts filled with A except a B
    slab next to the inlet.  Held densities are FP32-representable."""
    cell, phi, ptype = synth.drainage_geometry(n, seed)
    nz = nz or n
    cell, phi, ptype = cell[:nz].copy(), phi[:nz], ptype[:nz]
    cell[0], cell[-1] = synth.INLET, synth.OUTLET
    zz = np.arange(nz)[:, None, None] + np.zeros(cell.shape, np.int64)
    wet = zz < 4
    rA, rB = np.where(wet, 0.03, 1.0), np.where(wet, 1.0, 0.03)
    f32 = lambda v: float(np.float32(v))
    held = ((f32(0.03), f32(1.0 + dp)), (f32(1.0), f32(0.03)))
    return Case(f"imbibition{cell.shape}", cell.shape, cell, phi, rA, rB, ptype=ptype, G=1.1, kappa=-0.045,
                tau=tau, rho_wall=(0.03, 1.0), wet=1, periodic=(1, 1, 0), held=held)


def droplet2d(n=100, R=40, kappa=0.0, csf_everywhere=1, tau=(1.0, 1.0), G=1.1):
    """Sec. III.A on D2Q9: a droplet of A (radius R) in B on an n^2 periodic
    plane, rho 1.0 / 0.03."""
    shape = (1, n, n)
    c = n // 2
    rA, rB = synth.cylinder_droplet_fields(shape, R, (c, c), 1.0, 0.03)
    return Case(f"droplet2d{n}_R{R}", shape, np.zeros(shape, np.uint8), np.ones(shape), rA, rB, G=G, kappa=kappa,
                csf_everywhere=csf_everywhere, tau=tau, lattice="d2q9", probe=(c, c, 0, R - 4, R + 4))


def mixed2d(shape=(1, 13, 17), seed=9, periodic=(1, 1, 1), tau=(0.8, 1.3), thomeer=0.35):
    """D2Q9 counterpart of mixed_features: solid, gray (two pore types, one on
    a Thomeer curve, tensorial), wetting walls, CSF in gray cells, body
    forces, both residual transitions, open or periodic axes."""
    rng = np.random.default_rng(seed)
    cell = np.zeros(shape, np.uint8)
    cell[rng.random(shape) < 0.12] = synth.SOLID
    cell[(rng.random(shape) < 0.35) & (cell == 0)] = synth.GRAY
    phi = np.where(cell == synth.GRAY, 0.15 + 0.4 * rng.random(shape), 1.0)
    yy, xx = np.meshgrid(np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    blocks = (((xx // 4 + yy // 4) % 2) == 0)[None]
    ra = np.where(blocks, 1.0, 0.03) + 0.05 * rng.random(shape)
    rb = 1.06 - ra
    u0 = 0.01 * rng.standard_normal((3,) + shape)
    u0[2] = 0.0
    ptype = (rng.random(shape) < 0.5).astype(np.uint8)
    curves = [dict(CURVE, aniso=10.0), dict(CURVE, kc_d=1.5, pd=0.03, lam=1.5, swr=0.1, nw=2.5, nn=1.5, aniso=3.0,
                                           thomeer_g=thomeer)]
    return Case(f"mixed2d{shape}", shape, cell, phi, ra, rb, u=u0, ptype=ptype, curves=curves, G=1.1,
                kappa=-0.045, tau=tau, accel=((1e-4, 2e-5, 0), (0, -1e-4, 0)), rho_wall=(0.7, 0.2), wet=1,
                periodic=periodic, lattice="d2q9")


def imbibition2d(nx=64, ny=96, seed=synth.SEED_BASE + 9, dp=0.02):
    """The pressure-driven imbibition set-up on D2Q9: a plane of the
    multiscale-rock recipe between a wetting-B inlet row (y = 0) and a
    non-wetting-A outlet row (y = ny - 1), y not periodic."""
    cell3, phi3, ptype3 = synth.drainage_geometry(max(nx, ny), seed)
    cell, phi, ptype = cell3[:1, :ny, :nx].copy(), phi3[:1, :ny, :nx], ptype3[:1, :ny, :nx]
    cell[:, 0, :], cell[:, -1, :] = synth.INLET, synth.OUTLET
    yy = np.arange(ny)[None, :, None] + np.zeros(cell.shape, np.int64)
    wet = yy < 4
    rA, rB = np.where(wet, 0.03, 1.0), np.where(wet, 1.0, 0.03)
    f32 = lambda v: float(np.float32(v))
    held = ((f32(0.03), f32(1.0 + dp)), (f32(1.0), f32(0.03)))
    return Case(f"imbibition2d{cell.shape}", cell.shape, cell, phi, rA, rB, ptype=ptype, G=1.1, kappa=-0.045,
                rho_wall=(0.03, 1.0), wet=1, periodic=(1, 0, 1), held=held, lattice="d2q9")


def adjoint_case(n=8, seed=21, shape=None, steps_hint=None, thomeer=0.0):
    """Periodic lattice with solid, gray (one curve, tensorial, CSF, capillary)
    and both components, for the porosity gradient: A pushed along x."""
    rng = np.random.default_rng(seed)
    shape = shape or (n, n, n)
    cell = np.zeros(shape, np.uint8)
    cell[rng.random(shape) < 0.10] = synth.SOLID
    cell[(rng.random(shape) < 0.45) & (cell == 0)] = synth.GRAY
    phi = np.where(cell == synth.GRAY, 0.2 + 0.5 * rng.random(shape), 1.0)
    zz, yy, xx = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
    ra = np.where(xx < shape[2] // 2, 1.0, 0.03) + 0.02 * rng.random(shape)
    rb = 1.05 - ra
    return Case(f"adjoint{shape}", shape, cell, phi, ra, rb, curves=[dict(CURVE, aniso=10.0, thomeer_g=thomeer)], G=1.1,
                kappa=-0.045, tau=(0.8, 1.0), accel=((1e-4, 0, 0), (0, 0, 0)), rho_wall=(0.03, 1.0), wet=1)


def flat_blocks(lattice="d3q19", shape=None, periodic=(1, 1, 1), aniso=10.0, G=1.1, seed=2):
    """Blocks of uniform porosity (gray phi 0.35 and 0.2) between open pore
    and solid stripes: most gray cells see a flat neighbourhood (no axis),
    the block faces have an axis normal to the face."""
    shape = shape or ((1, 24, 30) if lattice == "d2q9" else (8, 16, 30))
    nz, ny, nx = shape
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    cell = np.zeros(shape, np.uint8)
    cell[...] = np.where((x % 15) >= 4, synth.GRAY, synth.PORE)
    cell = np.where(((x % 15) == 14) & (y % 8 < 3), synth.SOLID, cell).astype(np.uint8)
    phi = np.where(x < nx // 2, 0.35, 0.2) * np.ones(shape)
    rng = np.random.default_rng(seed)
    ra = np.where(x < nx // 3, 0.97, 0.03) * np.ones(shape) + 0.005 * rng.random(shape)
    rb = 1.0 - ra + 0.005 * rng.random(shape)
    return Case(f"flat_blocks_{lattice}{shape}", shape, cell, phi, ra, rb, lattice=lattice, periodic=periodic,
                G=G, tau=(0.8, 1.0), accel=((1e-5, 0, 0), (0, 0, 0)), curves=[dict(CURVE, aniso=aniso)])
