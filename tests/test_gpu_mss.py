"""Mass-sink-source term and the saturation controllers on the GPU.

The term itself is compared with the FP64 oracle (relative 1e-5 in the L2
norm over non-solid cells, as the other parity tests) on every kernel path;
the controllers are host logic around it and are checked against the
observables they steer by."""
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


def _with_mss(case, rate):
    case.s["mss"] = rate
    return case


@pytest.mark.parametrize("path,tile", [(0, 0), (0, 2), (0, 4), (1, 0)])
def test_mss_term_matches_oracle(path, tile):
    case = _with_mss(LC.mixed_features(seed=13), 2e-3)
    gf, gobs, _ = LC.run_gpu(case, 30, path=path, tile=tile)
    of, oobs, _ = LC.run_oracle(case, 30)
    _assert_parity(case, gf, of)
    assert abs(gobs["mass"][1] - oobs["mass"][1]) < 1e-6 * oobs["mass"][1]


def test_mss_with_reservoirs_and_on_d2q9():
    for case in (_with_mss(LC.imbibition(16), -1e-3), _with_mss(LC.mixed2d(), 2e-3)):
        gf, _, _ = LC.run_gpu(case, 40)
        of, _, _ = LC.run_oracle(case, 40)
        _assert_parity(case, gf, of)


@pytest.mark.parametrize("storage", [1, 3])
def test_mss_on_16bit_storages_moves_the_same_mass(storage):
    case = _with_mss(LC.mixed_features(seed=13), 2e-3)
    _, gobs, _ = LC.run_gpu(case, 30, storage=storage)
    _, oobs, _ = LC.run_oracle(case, 30)
    assert abs(gobs["mass"][1] - oobs["mass"][1]) < 2e-3 * oobs["mass"][1]


def _setup(ctx, case):
    from paper_2512_21696_gb300 import lbm
    for k, cv in enumerate(case.curves):
        lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
            kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
            phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
            thomeer_g=cv["thomeer_g"]))
    lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
    lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)


def test_batch_runs_with_their_own_rates_match_single_lattices():
    from paper_2512_21696_gb300 import lbm
    cases = [LC.mixed_features(seed=13), LC.mixed_features(shape=(6, 9, 11), seed=14),
             LC.mixed_features(shape=(8, 7, 5), seed=15)]
    rates = [2e-3, -1e-3, 0.0]
    b = lbm.lbm_batch_create([LC.gpu_params(c) for c in cases])
    try:
        views = [lbm.lbm_batch_run(b, r) for r in range(len(cases))]
        for v, c, m in zip(views, cases, rates):
            _setup(v, c)
            lbm.lbm_set_mss(v, m)
        lbm.lbm_batch_step(b, 12)
        lbm.lbm_set_mss(views[2], 1.5e-3)  # a rate change between steps: no new capture needed
        lbm.lbm_batch_step(b, 12)
        got = [[x.copy() for x in lbm.lbm_get_fields(v)] for v in views]
    finally:
        b.close()
    for r, (c, g) in enumerate(zip(cases, got)):
        o = LC.make_oracle(c)
        o.set_mss(rates[r])
        o.step(12)
        if r == 2:
            o.set_mss(1.5e-3)
        o.step(12)
        _assert_parity(c, g, o.fields())


@pytest.mark.parametrize("delta", [0.06, -0.05])
def test_saturation_controller_reaches_its_target(delta):
    from paper_2512_21696_gb300 import lbm
    case = LC.drainage(32)
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        _setup(ctx, case)
        lbm.lbm_step(ctx, 20)
        obs0 = lbm.lbm_observables(ctx)
        s0, m0 = obs0["sat"], sum(obs0["mass"])
        target = s0 + delta
        ok, steps = lbm.lbm_mss_to_saturation(ctx, target, 0.05, 5e-3, 2e-3, 20, 20000)
        obs = lbm.lbm_observables(ctx)
        print(f"S0 {s0:.4f} target {target:.4f} reached {ok} after {steps} steps: S {obs['sat']:.4f}")
        assert ok and abs(obs["sat"] - target) <= 2e-3 and obs["nan_count"] == 0
        assert abs(sum(obs["mass"]) - m0) < 1e-5 * m0  # the term moves mass between components only
    finally:
        ctx.close()


def test_batch_saturation_controller_reaches_every_target():
    from paper_2512_21696_gb300 import lbm
    cases = [LC.drainage(24, seed=synth.SEED_BASE + 20 + k) for k in range(3)]
    b = lbm.lbm_batch_create([LC.gpu_params(c) for c in cases])
    try:
        views = [lbm.lbm_batch_run(b, r) for r in range(len(cases))]
        for v, c in zip(views, cases):
            _setup(v, c)
        lbm.lbm_batch_step(b, 20)
        s0 = [o["sat"] for o in lbm.lbm_batch_observables(b)]
        targets = [s0[0] + 0.05, s0[1] - 0.04, s0[2] + 0.02]
        ok, steps = lbm.lbm_batch_mss_to_saturation(b, targets, 0.05, 5e-3, 2e-3, 20, 20000)
        sat = [o["sat"] for o in lbm.lbm_batch_observables(b)]
        print("targets", targets, "reached", ok, "after", steps, "steps:", sat)
        assert ok and all(abs(s - t) <= 2e-3 for s, t in zip(sat, targets))
    finally:
        b.close()


def test_adjoint_refuses_a_mass_source():
    from paper_2512_21696_gb300 import lbm
    case = LC.adjoint_case()
    ctx = lbm.lbm_create(LC.gpu_params(case))
    try:
        _setup(ctx, case)
        lbm.lbm_set_mss(ctx, 1e-3)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_adjoint_run(ctx, 1e-3, 0.5, 4, 2)
        assert e.value.code == -1
    finally:
        ctx.close()
