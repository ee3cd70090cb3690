"""The D2Q9 variant of the CUDA step against the FP64 oracle's D2Q9 mode.

Parity as for D3Q19: relative 1e-5 in the L2 norm over non-solid cells for
rho^A, rho^B, u and Sw (FP32 kernels against the FP64 oracle on identical
FP32 inputs), plus the observables the paper reports for its 2-D droplet
(Sec. III.A: Laplace pressure jump, maximum spurious velocity).
"""
import numpy as np
import pytest

import lbm_cases as LC
from helpers import rel_l2
from paper_2512_21696_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _assert_parity(case, gpu, orc, tol=TOL):
    (ga, gb, gu, gs), (oa, ob, ou, osw) = gpu, orc
    fl = case.cell != synth.SOLID
    e = dict(rhoA=rel_l2(ga, oa, fl), rhoB=rel_l2(gb, ob, fl), u=rel_l2(gu, ou, fl), sw=rel_l2(gs, osw, fl))
    assert max(e.values()) <= tol, f"{case.name}: {e}"
    return e


@pytest.mark.parametrize("kappa", [0.0, -0.045])
def test_droplet_sec3a_400_steps(kappa):
    """The paper's 2-D droplet: R = 40 on a 100^2 periodic plane."""
    case = LC.droplet2d(kappa=kappa)
    gf, gobs, _ = LC.run_gpu(case, 400)
    of, oobs, _ = LC.run_oracle(case, 400)
    e = _assert_parity(case, gf, of)
    assert abs(gobs["dp"] - oobs["dp"]) < 1e-4 * abs(oobs["dp"])
    assert abs(gobs["max_u"] - oobs["max_u"]) < 1e-4 * oobs["max_u"]
    assert abs(gobs["mass"][0] - oobs["mass"][0]) < 1e-6 * oobs["mass"][0]
    print(f"kappa {kappa}: errors {e}, dp {gobs['dp']:.6e} (oracle {oobs['dp']:.6e}), "
          f"max|u| {gobs['max_u']:.4e} (oracle {oobs['max_u']:.4e})")


@pytest.mark.parametrize("shape,periodic", [((1, 13, 17), (1, 1, 1)), ((1, 9, 31), (0, 1, 1)),
                                            ((1, 40, 7), (1, 0, 1)), ((1, 5, 5), (0, 0, 1))])
@pytest.mark.parametrize("steps", [1, 25])
def test_mixed_features_2d(shape, periodic, steps):
    case = LC.mixed2d(shape=shape, periodic=periodic, seed=sum(shape))
    gf, _, _ = LC.run_gpu(case, steps)
    of, _, _ = LC.run_oracle(case, steps)
    _assert_parity(case, gf, of)


def test_mixed_features_2d_regularised_long():
    case = LC.mixed2d(shape=(1, 24, 30), tau=(0.6, 0.9), seed=3)
    gf, _, _ = LC.run_gpu(case, 300)
    of, _, _ = LC.run_oracle(case, 300)
    _assert_parity(case, gf, of)


def test_imbibition_2d_with_reservoirs():
    case = LC.imbibition2d()
    gf, gobs, _ = LC.run_gpu(case, 300)
    of, oobs, _ = LC.run_oracle(case, 300)
    _assert_parity(case, gf, of)
    assert abs(gobs["sat"] - oobs["sat"]) < 1e-6


def test_checkpoint_roundtrip_2d():
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed2d()
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        for k, cv in enumerate(case.curves):
            lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
                kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
                thomeer_g=cv["thomeer_g"]))
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
    finally:
        ctx.close()


def test_d2q9_is_refused_where_not_built():
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed2d()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([LC.gpu_params(case), LC.gpu_params(case)])
    assert e.value.code == -1
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_adjoint_run(ctx, 1e-3, 0.5, 4, 2)
        assert e.value.code == -1
    finally:
        ctx.close()


def test_degenerate_planes():
    """An all-solid plane steps and reports zero mass; a one-cell periodic
    plane keeps its uniform state; a one-cell-wide channel with walls."""
    from paper_2512_21696_gb300 import lbm
    shape = (1, 6, 5)
    solid = LC.Case("solid2d", shape, np.full(shape, synth.SOLID, np.uint8), np.ones(shape),
                    np.full(shape, 0.5), np.full(shape, 0.5), lattice="d2q9", G=1.1)
    _, gobs, _ = LC.run_gpu(solid, 3)
    assert gobs["mass"] == (0.0, 0.0) and gobs["nan_count"] == 0
    for shape, periodic in (((1, 1, 1), (1, 1, 1)), ((1, 7, 1), (1, 0, 1))):
        rng = np.random.default_rng(3)
        case = LC.Case(f"tiny2d{shape}", shape, np.zeros(shape, np.uint8), np.ones(shape),
                       0.5 + 0.4 * rng.random(shape), 0.5 + 0.4 * rng.random(shape), lattice="d2q9", G=1.1,
                       periodic=periodic, accel=((1e-4, 0, 0), (0, 0, 0)))
        gf, _, _ = LC.run_gpu(case, 20)
        of, _, _ = LC.run_oracle(case, 20)
        _assert_parity(case, gf, of)
