"""How strongly the method amplifies rounding-sized changes of its inputs,
measured on the FP64 oracle alone (no GPU): the limit below which no
implementation of other precision or summation order can agree with it.

A relative perturbation of 6e-8 (one FP32 rounding) is applied to the initial
densities of both components, and the perturbed and unperturbed runs are
compared.  Two readings and workloads decide what the parity tests can ask:

* Eq. 4's unit-normal floor.  With eps_n = 1e-8 rho_hi the normal in a bulk
  phase, where |grad rho| is at round-off level, is itself a function of
  round-off, and the CSF force there follows it: the droplet's velocity field
  moves by 2e-3 of its norm.  With eps_n = 1e-4 rho_hi it moves by 8e-7; the
  floor changes the Sec. III.A droplet relations by 0.1 % (test_oracle_pins).
* A fibre bundle driven across its fibres.  The 24^3 bundle of the
  permeability tests, driven along z at g = 1e-5, flows 250 times slower than
  along x (mean u_z 4.5e-8): density rounding then moves K_z by up to 7e-6
  and the velocity field by 6e-5.  At g = 1e-3 (still Darcy flow, Re < 1e-3)
  the same perturbation moves K_z by 7e-8.
"""
import numpy as np
import pytest

import lbm_cases as LC
import oracle as O
from helpers import rel_l2
from paper_2512_21696_gb300 import synth


def _perturbed_pair(case, steps, seed=1):
    a = LC.make_oracle(case)
    a.step(steps)
    rng = np.random.default_rng(seed)
    pert = 1.0 + 6e-8 * rng.standard_normal(case.shape)
    b = O.Oracle(LC.oracle_params(case), case.cell, case.phi32.astype(np.float64), ptype=case.ptype,
                 curves=[O.make_curve(**cv) for cv in case.curves])
    b.init_fields(case.rhoA32.astype(np.float64) * pert, case.rhoB32.astype(np.float64) * pert)
    b.step(steps)
    return a, b


@pytest.mark.parametrize("eps,lo,hi", [(1e-8, 1e-4, 1.0), (1e-4, 0.0, 3e-6)])
def test_unit_normal_floor_conditions_the_csf_droplet(eps, lo, hi):
    """24^3 droplet (R = 6, G = 1.1) with Eq. 4 everywhere (kappa = -0.045),
    300 steps: the velocity change under a rounding-sized input change is at
    least 1e-4 with eps_n = 1e-8 (measured 2.1e-3) and at most 3e-6 with
    eps_n = 1e-4 (measured 7.9e-7)."""
    case = LC.droplet(n=24, R=6, kappa=-0.045, csf_everywhere=1)
    case.s["eps_n"] = eps * case.s["rho_hi"]
    a, b = _perturbed_pair(case, 300)
    fl = case.cell != synth.SOLID
    du = rel_l2(b.fields()[2], a.fields()[2], fl)
    print(f"eps_n {eps:.0e}: velocity change {du:.3e}")
    assert lo <= du <= hi


_FIBRE = {}


def _fibre_sensitivity():
    if not _FIBRE:
        for gg in (1e-5, 1e-3):
            case = LC.fiber_flow(24, 2, g=gg)
            a, b = _perturbed_pair(case, 600)
            fl = case.cell != synth.SOLID
            qa, qb = a.observables()["flux_vol"][2], b.observables()["flux_vol"][2]
            _FIBRE[gg] = (abs(qb - qa) / abs(qa), rel_l2(b.fields()[2], a.fields()[2], fl))
    return _FIBRE


@pytest.mark.parametrize("g,hi_k,hi_u", [(1e-5, 3e-5, 3e-4), (1e-3, 3e-7, 3e-6)])
def test_slow_cross_fibre_flow_amplifies_rounding(g, hi_k, hi_u):
    """The permeability-test bundle driven along z: the relative change of K_z
    and of the velocity field under a rounding-sized input change, bounded at
    about 4x what is measured (g = 1e-5: 6.8e-6 and 5.8e-5; g = 1e-3: 7.3e-8
    and 5.2e-7), and the slow case at least 10x the fast one."""
    res = _fibre_sensitivity()
    dk, du = res[g]
    print(f"g {g:.0e}: K_z change {dk:.3e}, velocity change {du:.3e}")
    assert dk <= hi_k and du <= hi_u
    assert res[1e-5][1] >= 10 * res[1e-3][1]
