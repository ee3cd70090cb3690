"""The hand-written adjoint (lbm_adjoint_run) against the oracle's discrete
adjoint, central differences of the FP32 forward, and itself under other
checkpoint intervals; the autograd wrapper."""
import numpy as np
import pytest

import lbm_cases as LC
from paper_2512_21696_gb300 import synth

pytestmark = pytest.mark.gpu
TARGETS = (2e-3, 0.45)


def _ctx(case):
    from paper_2512_21696_gb300 import lbm
    ctx = lbm.lbm_create(LC.gpu_params(case))
    cv = case.curves[0]
    lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive(
        kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
        phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
        thomeer_g=cv.get("thomeer_g", 0.0)))
    return ctx


def _gpu_grad(case, steps, ckpt, phi=None):
    from paper_2512_21696_gb300 import lbm
    ctx = _ctx(case)
    try:
        lbm.lbm_set_geometry(ctx, case.cell, case.phi32 if phi is None else phi.astype(np.float32))
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32)
        L, q, S, g = lbm.lbm_adjoint_run(ctx, *TARGETS, steps, ckpt)
        fields = [x.copy() for x in lbm.lbm_get_fields(ctx)]
    finally:
        ctx.close()
    return L, q, S, g, fields


def _oracle_grad(case, steps):
    from oracle import adjoint as A
    return A.loss_and_gradient(case.s, case.cell, case.curves[0], case.phi32.astype(np.float64),
                               case.rhoA32.astype(np.float64), case.rhoB32.astype(np.float64), steps, *TARGETS)


@pytest.mark.parametrize("steps,ckpt,thomeer", [(6, 4, 0.0), (40, 16, 0.0), (40, 16, 0.3)])
def test_adjoint_matches_oracle_discrete_adjoint(steps, ckpt, thomeer):
    case = LC.adjoint_case(thomeer=thomeer)
    L, q, S, g, _ = _gpu_grad(case, steps, ckpt)
    Lo, qo, So, go = _oracle_grad(case, steps)
    gray = case.cell == synth.GRAY
    err = np.linalg.norm((g - go)[gray]) / np.linalg.norm(go[gray])
    print(f"steps {steps}: L {L:.6e} (oracle {Lo:.6e}), relative L2 gradient error {err:.3e}")
    assert abs(L - Lo) <= 1e-5 * abs(Lo)
    assert np.count_nonzero(g[~gray]) == 0
    assert err <= 3e-4  # measured 5e-5 (6 steps) and 9e-5 (40 steps)


@pytest.mark.parametrize("steps", [1, 2])
def test_adjoint_single_steps_element_by_element(steps):
    """One and two steps, where a wrong transposed term cannot hide behind
    accumulation: every gray cell's gradient against the oracle's discrete
    adjoint, within 1e-4 of the largest."""
    case = LC.adjoint_case(seed=25)
    L, q, S, g, _ = _gpu_grad(case, steps, 1)
    Lo, qo, So, go = _oracle_grad(case, steps)
    gray = case.cell == synth.GRAY
    scale = np.abs(go[gray]).max()
    err = np.abs(g - go)[gray].max() / scale
    print(f"{steps} step(s): max |grad - oracle| / max |oracle| = {err:.3e}")
    assert scale > 0 and err <= 1e-4
    assert np.count_nonzero(g[~gray]) == 0


def test_adjoint_is_independent_of_the_checkpoint_interval():
    case = LC.adjoint_case(seed=22)
    _, _, _, g1, f1 = _gpu_grad(case, 24, 24)
    _, _, _, g2, f2 = _gpu_grad(case, 24, 5)
    gray = case.cell == synth.GRAY
    # same recomputed states, and the neighbour adjoints are gathered in a
    # fixed order: only the FP64 sums of the geometry adjoint may differ
    err = np.linalg.norm((g1 - g2)[gray]) / np.linalg.norm(g1[gray])
    print(f"checkpoint interval 24 vs 5: relative L2 gradient difference {err:.3e}")
    assert err <= 1e-12
    for x, y in zip(f1, f2):
        np.testing.assert_array_equal(x, y)


def test_adjoint_matches_central_differences_of_the_fp32_forward():
    from paper_2512_21696_gb300 import lbm
    case = LC.adjoint_case(n=10, seed=23)
    steps = 30
    _, _, _, g, _ = _gpu_grad(case, steps, 10)
    gray = np.argwhere(case.cell == synth.GRAY)
    rng = np.random.default_rng(7)
    h = 2e-3
    scale = np.abs(g).max()
    errs = []
    for k in rng.choice(len(gray), 16, replace=False):
        idx = tuple(gray[k])
        Ls = []
        for sgn in (1, -1):
            phi = case.phi32.astype(np.float64).copy()
            phi[idx] += sgn * h
            ctx = _ctx(case)
            try:
                lbm.lbm_set_geometry(ctx, case.cell, phi.astype(np.float32))
                lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32)
                lbm.lbm_step(ctx, steps)
                o = lbm.lbm_observables(ctx)
            finally:
                ctx.close()
            Ls.append((o["flux_out"] - TARGETS[0]) ** 2 / TARGETS[0] ** 2 + (o["sat"] - TARGETS[1]) ** 2)
        fd = (Ls[0] - Ls[1]) / (2 * h)
        errs.append(abs(fd - g[idx]) / scale)
    print("max |fd - adjoint| / max|grad| =", max(errs))
    assert max(errs) <= 0.02


def test_autograd_function_and_final_state():
    import torch
    from paper_2512_21696_gb300 import adjoint, lbm
    case = LC.adjoint_case(seed=24)
    ctx = _ctx(case)
    try:
        phi = torch.tensor(case.phi32, requires_grad=True)
        loss = adjoint.porosity_loss(phi, ctx, case.cell, case.rhoA32, case.rhoB32, nsteps=12, ckpt=5,
                                     q_target=TARGETS[0], s_target=TARGETS[1])
        loss.backward()
        after = [x.copy() for x in lbm.lbm_get_fields(ctx)]
    finally:
        ctx.close()
    L, q, S, g, _ = _gpu_grad(case, 12, 5)
    assert abs(float(loss) - L) <= 1e-12 * abs(L)  # the forward is deterministic
    gray = case.cell == synth.GRAY
    assert np.linalg.norm((phi.grad.numpy() - g)[gray]) <= 5e-4 * np.linalg.norm(g[gray])
    plain, _, _ = LC.run_gpu(case, 12, tile=2)  # the kernel the context ran
    for x, y in zip(after, plain):
        np.testing.assert_array_equal(x, y)


def test_adjoint_at_the_96_cubed_drainage_scale():
    """The 96^3 multiscale-rock drainage, 2000 FP32 steps, checkpoints every
    100: directional derivatives of the loss against central differences of
    the FP32 forward.  One cell's gradient is ~1e-7, so moving one cell's phi
    changes the loss by ~1e-9, below the rounding of a 2000-step FP32 run
    (single-cell differences are checked on small lattices above); along a
    direction v over all gray cells the change is sum_c g_c v_c, ~1e5 times
    larger.  Directions: the sign of the gradient, and that sign on a random
    half of the gray cells (|v| = 1 per cell), with h = 1e-3 in phi."""
    from paper_2512_21696_gb300 import lbm
    case = LC.drainage(96)
    steps, ckpt, h = 2000, 100, 1e-3

    def ctx_for(phi):
        ctx = lbm.lbm_create(LC.gpu_params(case))
        lbm.lbm_set_constitutive(ctx, 0, lbm.lbm_default_constitutive())
        lbm.lbm_set_geometry(ctx, case.cell, phi.astype(np.float32), case.ptype)
        lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32)
        return ctx

    ctx = ctx_for(case.phi32)
    try:
        L, q, S, g = lbm.lbm_adjoint_run(ctx, *TARGETS, steps, ckpt)
    finally:
        ctx.close()
    gray = case.cell == synth.GRAY
    assert np.count_nonzero(g[~gray]) == 0 and np.abs(g[gray]).max() > 0
    rng = np.random.default_rng(11)
    half = rng.random(case.shape) < 0.5
    dirs = {"sign": np.where(gray, np.sign(g), 0.0), "half": np.where(gray & half, np.sign(g), 0.0)}
    for name, v in dirs.items():
        Ls = []
        for sgn in (1, -1):
            ctx = ctx_for(case.phi32.astype(np.float64) + sgn * h * v)
            try:
                lbm.lbm_step(ctx, steps)
                o = lbm.lbm_observables(ctx)
            finally:
                ctx.close()
            Ls.append((o["flux_out"] - TARGETS[0]) ** 2 / TARGETS[0] ** 2 + (o["sat"] - TARGETS[1]) ** 2)
        fd = (Ls[0] - Ls[1]) / (2 * h)
        ad = float((g.astype(np.float64) * v).sum())
        print(f"96^3, 2000 steps, direction {name}: adjoint {ad:.6e}, central difference {fd:.6e}, "
              f"relative {abs(fd - ad) / abs(ad):.3e}")
        assert abs(fd - ad) <= 0.02 * abs(ad)
