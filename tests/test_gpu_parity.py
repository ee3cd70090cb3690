"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

Tolerance: relative 1e-5 in the L2 norm over non-solid cells for rho^A,
rho^B, u and Sw (FP32 kernels against the FP64 oracle on identical FP32
inputs), and an element-wise bound max|x - x_or| / max|x_or| over the same
cells (TOL_MAX), which a wrong value in one cell of a large lattice cannot
pass.  TOL_MAX is per quantity: the densities and Sw are O(1) and carry a few
FP32 roundings per step (worst measured on a GB300 over every case here,
including 400 steps at 128^3: 5.2e-7); u is a small difference of O(1)
populations, so its error relative to max|u| is larger (worst measured 1.3e-5,
in the droplet, where max|u| is the ~1e-4 spurious current).  Each bound is
about 4x the worst measurement.  Geometry results of the FP64 precompute are compared at FP32
rounding (2e-6 relative).
"""
import numpy as np
import pytest

import lbm_cases as LC
from helpers import max_rel, rel_l2
from paper_2512_21696_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5
TOL_MAX = {"rhoA": 2e-6, "rhoB": 2e-6, "u": 5e-5, "sw": 2e-6}


def _compare(case, gpu, orc, tol=TOL, what=("rhoA", "rhoB", "u", "sw"), tol_max=TOL_MAX):
    (ga, gb, gu, gs), (oa, ob, ou, osw) = gpu, orc
    fl = case.cell != synth.SOLID
    errs = dict(rhoA=rel_l2(ga, oa, fl), rhoB=rel_l2(gb, ob, fl), u=rel_l2(gu, ou, fl), sw=rel_l2(gs, osw, fl))
    emax = dict(rhoA=max_rel(ga, oa, fl), rhoB=max_rel(gb, ob, fl), u=max_rel(gu, ou, fl), sw=max_rel(gs, osw, fl))
    print(f"parity {case.name}: L2 {errs} max {emax}")
    for k in what:
        assert errs[k] <= tol, f"{case.name}: {k} relative L2 error {errs[k]:.3e} > {tol:.0e} ({errs})"
        assert emax[k] <= tol_max[k], f"{case.name}: {k} element-wise error {emax[k]:.3e} > {tol_max[k]:.0e} ({emax})"
    return errs


def _compare_static(case, gstat, ostat):
    kinv, pcs, swirr, sores = gstat
    gray = case.cell == synth.GRAY
    if not gray.any():
        return
    ok = ostat["kinv"]
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    scale = np.abs(ok).max()
    for k, (a, b) in enumerate(pairs):
        np.testing.assert_allclose(kinv[k][gray], ok[a, b][gray], rtol=0, atol=2e-6 * scale)
    np.testing.assert_allclose(pcs[gray], (ostat["lamL"] * np.array([c["pd"] for c in case.curves])[
        case.ptype if case.ptype is not None else 0])[gray], rtol=2e-6)
    np.testing.assert_allclose(swirr[gray], ostat["swirr"][gray], rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(sores[gray], ostat["sores"][gray], rtol=2e-6, atol=1e-7)


# (path, tile): fused tiles 0-4 and 7, the published-density march (5, 6), the
# automatic choice (8), two launches
KERNELS = [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (0, 6), (0, 7), (0, 8), (1, 0)]


@pytest.mark.parametrize("path,tile", KERNELS)
@pytest.mark.parametrize("steps", [1, 10])
def test_mixed_features_small(steps, path, tile):
    case = LC.mixed_features()
    gf, gobs, gst = LC.run_gpu(case, steps, path=path, tile=tile)
    of, oobs, ost = LC.run_oracle(case, steps)
    _compare_static(case, gst, ost)
    _compare(case, gf, of)


@pytest.mark.parametrize("lattice,periodic", [("d3q19", (1, 1, 1)), ("d3q19", (0, 1, 0)), ("d2q9", (1, 1, 1)),
                                              ("d2q9", (0, 0, 1))])
def test_flat_gray_blocks_static_and_step(lattice, periodic):
    """Gray blocks of uniform porosity: the flat interiors carry no axis (an
    exactly zero gradient and Hessian), the faces an axis along the normal;
    the geometry precompute and 30 steps against the oracle."""
    case = LC.flat_blocks(lattice, periodic=periodic)
    gf, _, gst = LC.run_gpu(case, 30)
    of, _, ost = LC.run_oracle(case, 30)
    _compare_static(case, gst, ost)
    inner = (case.cell == synth.GRAY) & (ost["iso"] == 1)
    assert inner.sum() > 0.3 * (case.cell == synth.GRAY).sum()
    for k in range(3, 6):  # no off-diagonal term where the oracle has no axis
        assert np.all(gst[0][k][inner] == 0.0)
    _compare(case, gf, of)


@pytest.mark.parametrize("path,tile", [(0, 2), (1, 0)])
def test_mixed_features_thomeer_curve(path, tile):
    """The second pore type on a Thomeer Pc curve (capillary force, residual
    crossings of the geometry precompute)."""
    case = LC.mixed_features(thomeer=0.35, seed=11)
    gf, _, gst = LC.run_gpu(case, 10, path=path, tile=tile)
    of, _, ost = LC.run_oracle(case, 10)
    _compare_static(case, gst, ost)
    _compare(case, gf, of)


def test_mixed_features_device_arrays_and_tau():
    case = LC.mixed_features(seed=7, tau=(0.55, 0.7))
    gf, _, _ = LC.run_gpu(case, 20, device_arrays=True)
    of, _, _ = LC.run_oracle(case, 20)
    _compare(case, gf, of)


@pytest.mark.parametrize("path,tile", KERNELS)
@pytest.mark.parametrize("shape,periodic", [((5, 7, 13), (1, 1, 1)), ((9, 6, 11), (0, 1, 0)),
                                            ((1, 17, 33), (1, 0, 1)), ((3, 3, 3), (0, 0, 0)),
                                            ((20, 37, 70), (1, 1, 0))])
def test_ragged_and_open_boundaries(shape, periodic, path, tile):
    case = LC.mixed_features(shape=shape, periodic=periodic, seed=sum(shape))
    gf, _, gst = LC.run_gpu(case, 12, path=path, tile=tile)
    of, _, ost = LC.run_oracle(case, 12)
    _compare_static(case, gst, ost)
    _compare(case, gf, of)


def test_droplet_400_steps():
    """32^3 static droplet (G = 1.1), 400 FP32 steps against the FP64 oracle."""
    case = LC.droplet()
    gf, gobs, _ = LC.run_gpu(case, 400)
    of, oobs, _ = LC.run_oracle(case, 400)
    errs = _compare(case, gf, of)
    assert abs(gobs["mass"][0] - oobs["mass"][0]) < 1e-5 * oobs["mass"][0]
    assert abs(gobs["dp"] - oobs["dp"]) < 1e-4 * abs(oobs["dp"])
    assert abs(gobs["max_u"] - oobs["max_u"]) < 1e-4 * oobs["max_u"]
    print("droplet errors", errs)


def test_droplet_csf_everywhere_400_steps():
    case = LC.droplet(kappa=-0.045, csf_everywhere=1)
    gf, gobs, _ = LC.run_gpu(case, 400)
    of, oobs, _ = LC.run_oracle(case, 400)
    _compare(case, gf, of)
    assert abs(gobs["dp"] - oobs["dp"]) < 1e-3 * abs(oobs["dp"])


def test_droplet_regularised_tau():
    case = LC.droplet(n=24, R=6, tau=(0.55, 0.8))
    gf, _, _ = LC.run_gpu(case, 200)
    of, _, _ = LC.run_oracle(case, 200)
    _compare(case, gf, of)


def test_drainage_full_size_two_steps():
    """The 128^3 multiscale-rock workload of the benchmark, two steps."""
    case = LC.drainage(128)
    gf, gobs, gst = LC.run_gpu(case, 2)
    of, oobs, ost = LC.run_oracle(case, 2)
    _compare_static(case, gst, ost)
    _compare(case, gf, of)
    assert gobs["nan_count"] == 0
    assert abs(gobs["sat"] - oobs["sat"]) < 1e-6


@pytest.mark.parametrize("tile", [5, 2])
def test_drainage_full_size_400_steps(tile):
    """The 128^3 multiscale-rock workload of the benchmark, 400 FP32 steps
    against 400 FP64 oracle steps (the benchmark's kernel, the march, and the
    rolling-window kernel; the oracle run is shared)."""
    case = LC.drainage(128)
    of, oobs = _drainage128_oracle_400()
    gf, gobs, _ = LC.run_gpu(case, 400, tile=tile)
    _compare(case, gf, of)
    assert gobs["nan_count"] == 0
    assert abs(gobs["sat"] - oobs["sat"]) < 1e-6
    for a in range(2):
        assert abs(gobs["mass"][a] - oobs["mass"][a]) < 1e-6 * oobs["mass"][a]


_DRAINAGE128 = {}


def _drainage128_oracle_400():
    if not _DRAINAGE128:
        f, obs, _ = LC.run_oracle(LC.drainage(128), 400)
        _DRAINAGE128["v"] = (f, obs)
    return _DRAINAGE128["v"]


def test_drainage_small_many_steps():
    case = LC.drainage(32)
    gf, _, _ = LC.run_gpu(case, 200)
    of, _, _ = LC.run_oracle(case, 200)
    _compare(case, gf, of)


def test_degenerate_cases():
    from paper_2512_21696_gb300 import lbm
    # zero steps: fields are the initial ones
    case = LC.mixed_features(seed=3)
    gf, _, _ = LC.run_gpu(case, 0)
    np.testing.assert_array_equal(gf[0], case.rhoA32 * (case.cell != synth.SOLID))
    # a single cell
    one = LC.Case("one", (1, 1, 1), np.zeros((1, 1, 1)), np.ones((1, 1, 1)), np.full((1, 1, 1), 0.7),
                  np.full((1, 1, 1), 0.2), G=1.1)
    gf, gobs, _ = LC.run_gpu(one, 5)
    of, oobs, _ = LC.run_oracle(one, 5)
    _compare(one, gf, of)
    # all solid: nothing moves, nothing is non-finite
    shape = (4, 4, 4)
    solid = LC.Case("solid", shape, np.full(shape, synth.SOLID), np.zeros(shape), np.ones(shape), np.ones(shape))
    gf, gobs, _ = LC.run_gpu(solid, 3)
    assert gobs["nan_count"] == 0 and gobs["mass"] == (0.0, 0.0)
    # one component only (rho^B = 0)
    single = LC.Case("single", (6, 6, 6), np.zeros((6, 6, 6)), np.ones((6, 6, 6)), np.ones((6, 6, 6)),
                     np.zeros((6, 6, 6)), accel=((1e-5, 0, 0), (0, 0, 0)), wet=0)
    gf, _, _ = LC.run_gpu(single, 30)
    of, _, _ = LC.run_oracle(single, 30)
    _compare(single, gf, of, what=("rhoA", "u"))


def test_invalid_inputs_are_rejected():
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed_features()
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(ctx, 1)
        assert e.value.code == -6
        bad = case.cell.copy()
        bad[0, 0, 0] = 7
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_geometry(ctx, bad, case.phi32)
        badphi = case.phi32.copy()
        badphi[case.cell == synth.GRAY] = 1.5
        if (case.cell == synth.GRAY).any():
            with pytest.raises(lbm.LbmError):
                lbm.lbm_set_geometry(ctx, case.cell, badphi)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_constitutive(ctx, 16, lbm.lbm_default_constitutive())
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive(aniso=0.5))
    finally:
        ctx.close()
    p = LC.gpu_params(case)
    p.tau[0] = 0.5
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(p)


def test_checkpoint_roundtrip_is_bit_exact():
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed_features(seed=11)
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        for k, cv in enumerate(case.curves):
            lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
                kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
        thomeer_g=cv.get("thomeer_g", 0.0)))
        lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
        lbm.lbm_step(ctx, 7)
        state = lbm.lbm_save_state(ctx)
        lbm.lbm_step(ctx, 9)
        a = [x.copy() for x in lbm.lbm_get_fields(ctx)]
        lbm.lbm_load_state(ctx, state)
        lbm.lbm_step(ctx, 9)
        b = lbm.lbm_get_fields(ctx)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
        assert lbm.lbm_observables(ctx)["step"] == 16
    finally:
        ctx.close()


def test_mass_conservation_fp32():
    case = LC.drainage(48)
    gf0, g0, _ = LC.run_gpu(case, 0)
    gf, g1, _ = LC.run_gpu(case, 300)
    for a in range(2):
        assert abs(g1["mass"][a] - g0["mass"][a]) < 2e-6 * g0["mass"][a]


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5, 6])
def test_fused_matches_two_launch_path(tile):
    """The fused kernel and the two-launch path share the per-cell arithmetic."""
    case = LC.drainage(48)
    a, _, _ = LC.run_gpu(case, 25, path=0, tile=tile)
    b, _, _ = LC.run_gpu(case, 25, path=1)
    for x, y in zip(a, b):
        assert np.all(np.isfinite(x)) and np.all(np.isfinite(y))
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-6 * max(1.0, np.abs(y).max()))


def test_host_injected_faults_are_reported():
    """Faults made on the host: a NaN porosity is rejected by the geometry
    call; a NaN density in the initial fields is counted by the observables,
    which then return LBM_ERR_NUMERIC (the context stays usable)."""
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed_features(seed=9)
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        badphi = case.phi32.copy()
        badphi[case.cell == synth.GRAY] = np.nan
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_geometry(ctx, case.cell, badphi, case.ptype)
        assert e.value.code == -1
        lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
        ra = case.rhoA32.copy()
        ra[case.cell != synth.SOLID] = np.where(np.arange((case.cell != synth.SOLID).sum()) == 3, np.nan,
                                                ra[case.cell != synth.SOLID])
        lbm.lbm_init_fields(ctx, ra, case.rhoB32, case.u32)
        lbm.lbm_step(ctx, 2)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_observables(ctx)
        assert e.value.code == -4
        assert lbm.lbm_observables(ctx, check=False)["nan_count"] > 0
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
        lbm.lbm_step(ctx, 2)
        assert lbm.lbm_observables(ctx)["nan_count"] == 0
    finally:
        ctx.close()


def test_async_observables_equal_the_synchronous_ones():
    """lbm_observables_async + lbm_obs_decode: the same values as
    lbm_observables for every step of a loop that never synchronises."""
    import torch
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed_features(seed=31)
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        for k, cv in enumerate(case.curves):
            lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
                kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"]))
        lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
        state = lbm.lbm_save_state(ctx)
        raw = torch.zeros((6, lbm.LBM_OBS_RAW), dtype=torch.float64).pin_memory()
        row = raw.stride(0) * raw.element_size()
        for k in range(6):
            lbm.lbm_step(ctx, 1)
            lbm.lbm_observables_async(ctx, raw.data_ptr() + k * row)
        torch.cuda.synchronize()
        got = [lbm.lbm_obs_decode(ctx, raw.data_ptr() + k * row) for k in range(6)]
        lbm.lbm_load_state(ctx, state)
        for k in range(6):
            lbm.lbm_step(ctx, 1)
            assert lbm.lbm_observables(ctx) == got[k]
    finally:
        ctx.close()


@pytest.mark.parametrize("tile", [5, 6])
@pytest.mark.parametrize("shape,periodic,steps", [((48, 48, 48), (1, 1, 1), 25), ((40, 37, 70), (1, 0, 1), 12),
                                                  ((9, 6, 11), (0, 1, 0), 12), ((128, 128, 128), (1, 1, 1), 3)])
def test_march_is_bit_identical_to_rolling_window(shape, periodic, steps, tile):
    """The published-density march reads the ring densities its neighbours
    computed instead of recomputing them, with the same per-cell arithmetic
    in the same order: the states equal the rolling-window kernel's bit for bit
    (periodic and open faces, ragged tiles, the 128^3 benchmark lattice)."""
    if shape == (48, 48, 48) or shape == (128, 128, 128):
        case = LC.drainage(shape[0])
    else:
        case = LC.mixed_features(shape=shape, periodic=periodic, seed=sum(shape))
    a, ga, _ = LC.run_gpu(case, steps, path=0, tile=tile)
    b, gb, _ = LC.run_gpu(case, steps, path=0, tile=2)
    assert ga["nan_count"] == 0 and gb["nan_count"] == 0  # equal arrays of NaN would compare equal
    for x, y in zip(a, b):
        assert np.all(np.isfinite(y))
        np.testing.assert_array_equal(x, y)
    assert ga == gb


@pytest.mark.parametrize("tile", [4, 7, 8])
@pytest.mark.parametrize("shape,periodic,steps", [((48, 48, 48), (1, 1, 1), 25), ((40, 37, 70), (1, 0, 1), 12),
                                                  ((9, 6, 11), (0, 1, 0), 12), ((128, 128, 128), (1, 1, 1), 3),
                                                  ((8, 192, 192), (1, 1, 1), 6)])
def test_tile_shapes_are_bit_identical(shape, periodic, steps, tile):
    """The 64-wide tiles (64x8, 64x7 with a ragged last band of rows) and the
    automatic choice among the tile shapes compute the default tile's
    states bit for bit (fields and observables), on lattices where the
    choice falls on different shapes."""
    if shape[0] == shape[1] == shape[2]:
        case = LC.drainage(shape[0])
    else:
        case = LC.mixed_features(shape=shape, periodic=periodic, seed=sum(shape))
    a, ga, _ = LC.run_gpu(case, steps, path=0, tile=tile)
    b, gb, _ = LC.run_gpu(case, steps, path=0, tile=2)
    assert ga["nan_count"] == 0 and gb["nan_count"] == 0
    for x, y in zip(a, b):
        assert np.all(np.isfinite(y))
        np.testing.assert_array_equal(x, y)
    assert ga == gb


@pytest.mark.parametrize("lattice,storage,path,tile", [("d3q19", 0, 0, 2), ("d3q19", 0, 0, 5), ("d3q19", 0, 1, 0),
                                                        ("d3q19", 3, 0, 2), ("d3q19", 1, 0, 2), ("d2q9", 0, 0, 2)])
def test_failed_launch_keeps_the_previous_state(lattice, storage, path, tile):
    """A step whose launch the runtime rejects (host-injected: a zero-size
    block, no device work) returns LBM_ERR_CUDA and leaves the buffer parity,
    the step count and the fields where the last good step left them; the
    next steps continue from there as if the failure had not happened."""
    from paper_2512_21696_gb300 import lbm
    if lattice == "d2q9":
        case = LC.mixed2d(shape=(1, 17, 23), seed=5)
    else:
        case = LC.mixed_features(seed=21)

    def run(fail_after):
        ctx = lbm.lbm_create(LC.gpu_params(case, storage=storage))
        try:
            lbm.lbm_set_kernel(ctx, path, tile)
            for k, cv in enumerate(case.curves):
                lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
                    kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                    phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"]))
            lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
            lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
            lbm.lbm_step(ctx, 3)
            before = [x.copy() for x in lbm.lbm_get_fields(ctx)]
            if fail_after:
                for count in (1, 2):  # the first or the second launch of a step fails
                    lbm.lbm_inject_launch_failures(ctx, count)
                    with pytest.raises(lbm.LbmError) as e:
                        lbm.lbm_step(ctx, 1)
                    assert e.value.code == -2
                    lbm.lbm_inject_launch_failures(ctx, 0)
                    assert lbm.lbm_observables(ctx, check=False)["step"] == 3
                    for x, y in zip(lbm.lbm_get_fields(ctx), before):
                        np.testing.assert_array_equal(x, y)
            lbm.lbm_step(ctx, 4)
            return lbm.lbm_get_fields(ctx), lbm.lbm_observables(ctx, check=False)["step"]
        finally:
            ctx.close()

    (fa, sa), (fb, sb) = run(True), run(False)
    assert sa == sb == 7
    for x, y in zip(fa, fb):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fibre_bundle_tensorial_400_steps(axis):
    """The tensorial fibre bundle (Eqs. 6-7, anisotropy 10; the 192^3
    workload's cylinder density, 25 cylinders at 48^3), body force along each
    axis, 400 FP32 steps against the oracle field by field."""
    case = LC.fiber_flow(48, axis, ncyl=25)
    gf, gobs, gst = LC.run_gpu(case, 400, tile=5)
    of, oobs, ost = LC.run_oracle(case, 400)
    _compare_static(case, gst, ost)
    _compare(case, gf, of)


@pytest.mark.parametrize("shape,storage,want", [((128, 128, 128), 0, 7), ((8, 192, 192), 0, 4), ((96, 96, 96), 0, 2),
                                                ((24, 24, 24), 0, 2), ((128, 128, 128), 3, 7), ((128, 128, 128), 1, 7),
                                                ((8, 192, 192), 1, 2)])
def test_tile_choice_per_grid(shape, storage, want):
    """The default tile (8) resolves per grid on the 152-SM GB300: 64x7 where
    its 38 columns x 4 chunks fill the 152 one-CTA slots (128^3), 64x8 where
    both 64-wide shapes fill them (192 x 192 planes), 32x8 on widths that are
    not a multiple of 64; the shifted 16-bit kernel has 32x8 and 64x7 only."""
    import torch

    from paper_2512_21696_gb300 import lbm
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the expected shapes are those of a 152-SM GB300")
    nz, ny, nx = shape
    ctx = lbm.lbm_create(lbm.lbm_default_params(nx, ny, nz, storage=storage))
    try:
        assert lbm.lbm_get_kernel(ctx) == (0, want)
        lbm.lbm_set_kernel(ctx, 0, 3)
        assert lbm.lbm_get_kernel(ctx) == (0, 3 if storage == 0 else 2)
        lbm.lbm_set_kernel(ctx, 0, 4)
        assert lbm.lbm_get_kernel(ctx) == (0, 2 if storage == 1 else 4)
        lbm.lbm_set_kernel(ctx, 1, 5)
        assert lbm.lbm_get_kernel(ctx) == (1, 5)
    finally:
        ctx.close()
