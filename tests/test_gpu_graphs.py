"""CUDA-graph replay of lbm_step on small lattices against direct launches.

lbm_step replays captured graphs of a fixed, even number of steps when a
lattice is small enough for its steps to be launch-bound.  The replayed
kernels are the directly launched ones with the same arguments, so a run
stepped in long calls must equal, bit for bit, the same run stepped one step
per call (which never replays): for both lattices, the 16-bit storages, the
two-launch path, reservoirs whose pressure changes between calls (the
graphs must be re-captured) and both buffer parities.
"""
import numpy as np
import pytest

import lbm_cases as LC

pytestmark = pytest.mark.gpu


def _open(case, path=0, tile=2, storage=0):
    from paper_2512_21696_gb300 import lbm
    extra = {"storage": storage} if storage else {}
    ctx = lbm.lbm_create(LC.gpu_params(case, **extra))
    lbm.lbm_set_kernel(ctx, path, tile)
    for k, cv in enumerate(case.curves):
        lbm.lbm_set_constitutive(ctx, k, lbm.lbm_default_constitutive(
            kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
            phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
            thomeer_g=cv["thomeer_g"]))
    lbm.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
    lbm.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
    if case.s["held"] is not None:
        lbm.lbm_set_pressure(ctx, *case.s["held"])
    return ctx


def _run(case, calls, one_by_one, between=None, **kw):
    """Steps `calls` (a list of step counts), either as given or one step per
    call; `between(ctx, k)` runs after call k.  Returns the fields, the
    population state and the launch count."""
    from paper_2512_21696_gb300 import lbm
    ctx = _open(case, **kw)
    try:
        for k, m in enumerate(calls):
            if one_by_one:
                for _ in range(m):
                    lbm.lbm_step(ctx, 1)
            else:
                lbm.lbm_step(ctx, m)
            if between:
                between(ctx, k)
        fields = [np.array(x, copy=True) for x in lbm.lbm_get_fields(ctx)]
        state = bytes(lbm.lbm_save_state(ctx))
        return fields, state, lbm.lbm_launch_count(ctx)
    finally:
        ctx.close()


def _same(case, calls, between=None, **kw):
    fa, sa, la = _run(case, calls, False, between, **kw)
    fb, sb, lb = _run(case, calls, True, between, **kw)
    for x, y in zip(fa, fb):
        assert np.all(np.isfinite(x))  # equal arrays of NaN would compare equal
        np.testing.assert_array_equal(x, y)
    assert sa == sb
    assert la == lb  # every replayed launch is counted
    assert all(np.isfinite(x).all() for x in fa)


# 35 steps: one direct, one replay, two direct (odd: the next call replays the
# other parity's graph); 34: the shortest call that replays; 100: three replays
CALLS = [35, 100, 34, 33, 67]


def test_graph_replay_d3q19_tiles_and_paths():
    case = LC.mixed_features(seed=4)
    for path, tile in ((0, 2), (0, 0), (1, 0)):
        _same(case, CALLS, path=path, tile=tile)


@pytest.mark.parametrize("storage", [1, 3, 4])
def test_graph_replay_16bit_storages(storage):
    _same(LC.mixed_features(seed=6), [35, 70], storage=storage)


def test_graph_replay_d2q9():
    _same(LC.mixed2d(shape=(1, 24, 30), seed=5), CALLS)


def test_graph_replay_reservoirs_with_pressure_and_mss_changes():
    """Parameters the kernels take by value change between calls: each change
    must reach the replayed steps."""
    from paper_2512_21696_gb300 import lbm
    levels = [((0.0, 1.03), (0.5, 0.5)), ((0.0, 1.05), (0.6, 0.4)), ((0.0, 1.02), (0.5, 0.5))]

    def between(ctx, k):
        if k < len(levels):
            lbm.lbm_set_pressure(ctx, *levels[k])
        if k == 1:
            lbm.lbm_set_mss(ctx, 2e-5)
        if k == 2:
            lbm.lbm_set_mss(ctx, 0.0)

    _same(LC.imbibition(n=16), [40, 40, 40, 40], between)
    _same(LC.imbibition2d(nx=24, ny=32), [40, 40, 40, 40], between)


def test_graph_replay_matches_the_oracle():
    """A long call (replayed) against the FP64 oracle, as the parity tests do
    for direct steps."""
    from helpers import rel_l2
    from paper_2512_21696_gb300 import synth
    case = LC.drainage(32)
    ctx = _open(case)
    try:
        from paper_2512_21696_gb300 import lbm
        lbm.lbm_step(ctx, 200)
        ga, gb, gu, gs = lbm.lbm_get_fields(ctx)
    finally:
        ctx.close()
    (oa, ob, ou, osw), _, _ = LC.run_oracle(case, 200)
    fl = case.cell != synth.SOLID
    for g, o in ((ga, oa), (gb, ob), (gu, ou), (gs, osw)):
        assert rel_l2(g, o, fl) <= 1e-5


def test_lbm_step_inside_a_callers_graph_capture():
    """A caller capturing its own stream gets plain launches inside its graph
    (no nested capture of ours): two direct steps, 40 steps captured by the
    caller and replayed twice equal 82 steps stepped directly."""
    import torch
    from paper_2512_21696_gb300 import lbm
    case = LC.mixed2d(shape=(1, 24, 30), seed=7)
    s = torch.cuda.Stream()
    ref = _open(case)
    try:
        lbm.lbm_step(ref, 82)
        want = [np.array(x, copy=True) for x in lbm.lbm_get_fields(ref)]
    finally:
        ref.close()
    p = LC.gpu_params(case)
    p.stream = s.cuda_stream
    from paper_2512_21696_gb300 import lbm as L
    ctx = L.lbm_create(p)
    try:
        for k, cv in enumerate(case.curves):
            L.lbm_set_constitutive(ctx, k, L.lbm_default_constitutive(
                kc_d=cv["kc_d"], pd=cv["pd"], lam=cv["lam"], swr=cv["swr"], nw=cv["nw"], nn=cv["nn"],
                phi_ref=cv["phi_ref"], pc_ref_max_f=cv["f_max"], pc_ref_min_f=cv["f_min"], aniso=cv["aniso"],
                thomeer_g=cv["thomeer_g"]))
        L.lbm_set_geometry(ctx, case.cell, case.phi32, case.ptype)
        L.lbm_init_fields(ctx, case.rhoA32, case.rhoB32, case.u32)
        L.lbm_step(ctx, 2)  # both kernel variants resolve their launch configuration outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            L.lbm_step(ctx, 40)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        got = L.lbm_get_fields(ctx)
        for x, y in zip(want, got):
            assert np.all(np.isfinite(x))
            np.testing.assert_array_equal(x, y)
    finally:
        ctx.close()
