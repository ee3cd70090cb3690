"""The zigzag pathway between two wavy-fibre bundles (Sec. I.B, Sec. III.E)
on D2Q9: parity with the FP64 oracle on the full 120 x 180 case, and the
effect the paper reports.  With the isotropic resistivity of the phi = 0.95
bundles the flow spreads into them; with the tensorial one (least component
1e-4 K0, Eq. 7) the bundle faces become barriers and the pathway carries
most of the flux.
"""
import numpy as np
import pytest

import lbm_cases as LC
from helpers import rel_l2
from paper_2512_21696_gb300 import synth

pytestmark = pytest.mark.gpu
RHO_IN = 0.740 / 0.733  # the paper's pressure ratio, p = rho_B / 3


def _case(aniso):
    cell, phi, path = synth.zigzag_pathway_geometry()
    shape = cell.shape
    case = LC.Case(f"zigzag_aniso{aniso:g}", shape, cell, phi, np.zeros(shape), np.ones(shape), lattice="d2q9",
                   periodic=(0, 0, 1), G=1.1, tau=(0.55, 0.55), rho_wall=(0.03, 1.0), wet=1,
                   held=((0.0, RHO_IN), (0.0, 1.0)), curves=[dict(LC.CURVE, aniso=aniso)])
    return case, path


@pytest.mark.parametrize("aniso", [1.0, 1e4])
def test_zigzag_parity_300_steps(aniso):
    case, _ = _case(aniso)
    (ga, gb, gu, gs), gobs, gst = LC.run_gpu(case, 300)
    (oa, ob, ou, osw), oobs, ost = LC.run_oracle(case, 300)
    fl = case.cell != synth.SOLID
    e = dict(rhoB=rel_l2(gb, ob, fl), u=rel_l2(gu, ou, fl))
    assert max(e.values()) <= 1e-5, e
    assert np.abs(ga).max() == 0.0 and np.abs(oa).max() == 0.0  # component A stays absent
    # the flat bundle interiors carry no axis, the faces next to the pathway do
    if aniso > 1:
        gray = case.cell == synth.GRAY
        assert (ost["iso"][gray] == 1).mean() > 0.5
        assert (ost["iso"][gray] == 0).any()


def test_zigzag_tensorial_resistivity_confines_the_flow():
    """Steady state (30 000 steps; the shares are the same at 120 000): the
    pathway, a sixth of the width, carries under 60 % of the flux with the
    isotropic resistivity and over 80 % with the tensorial one."""
    from paper_2512_21696_gb300 import lbm
    share = {}
    for aniso in (1.0, 1e4):
        case, path = _case(aniso)
        (ga, gb, gu, gs), gobs, _ = LC.run_gpu(case, 30000)
        assert gobs["nan_count"] == 0
        uy = -gu[1, 0, 1:-1, :]  # downwards, inlet on top
        rows = uy.sum(axis=1)
        assert np.all(rows > 0)
        share[aniso] = float(((uy * path[0, 1:-1, :]).sum(axis=1) / rows).mean())
    assert share[1.0] < 0.6 and share[1e4] > 0.8, share
