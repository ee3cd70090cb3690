"""Pins of the oracle's discrete adjoint (oracle/adjoint.py), no GPU.

The PyTorch statement of the step must reproduce the C oracle to round-off
(so it is the same forward map), and its reverse-mode gradient must match
central differences of its own FP64 loss (so the reverse pass, including the
eigenvector derivative of the principal axis, is wired correctly)."""
import numpy as np
import pytest
import torch

import lbm_cases as LC
from oracle import adjoint as A

STEPS = 6
TARGETS = (2e-3, 0.45)


def _args(case):
    return (case.s, case.cell, case.curves[0])


@pytest.mark.parametrize("thomeer", [0.0, 0.3])
def test_torch_forward_matches_c_oracle(thomeer):
    case = LC.adjoint_case(thomeer=thomeer)
    of, oobs, _ = LC.run_oracle(case, STEPS)
    m, st, out, geo = A.run(case.s, case.cell, case.curves[0], torch.tensor(case.phi32.astype(np.float64)),
                            case.rhoA32.astype(np.float64), case.rhoB32.astype(np.float64), STEPS)
    fl = case.cell != 1
    ra, rb, u, sw = of
    assert np.abs(out["rho"][0].numpy() - ra)[fl].max() < 1e-13
    assert np.abs(out["rho"][1].numpy() - rb)[fl].max() < 1e-13
    assert np.abs(out["u"].numpy() - u)[:, fl].max() < 1e-14
    assert np.abs(out["sw"].numpy() - sw)[fl].max() < 1e-13
    L, q, S = A.loss_of(case.cell, geo, out, *TARGETS)
    assert abs(float(q) - oobs["flux_out"]) < 1e-15 and abs(float(S) - oobs["sat"]) < 1e-14


@pytest.mark.parametrize("thomeer", [0.0, 0.3])
def test_reverse_mode_gradient_matches_central_differences(thomeer):
    case = LC.adjoint_case(thomeer=thomeer)
    phi = case.phi32.astype(np.float64)
    rA, rB = case.rhoA32.astype(np.float64), case.rhoB32.astype(np.float64)
    L, q, S, g = A.loss_and_gradient(*_args(case), phi, rA, rB, STEPS, *TARGETS)
    assert np.count_nonzero(g[case.cell != LC.synth.GRAY]) == 0
    gray = np.argwhere(case.cell == LC.synth.GRAY)
    rng = np.random.default_rng(3)
    h = 1e-4  # the FD error is round-off below ~1e-5, truncation (h^2) above

    def central(idx, hh):
        pp, pm = phi.copy(), phi.copy()
        pp[idx] += hh
        pm[idx] -= hh
        return (A.loss_only(*_args(case), pp, rA, rB, STEPS, *TARGETS)[0]
                - A.loss_only(*_args(case), pm, rA, rB, STEPS, *TARGETS)[0]) / (2 * hh)

    for k in rng.choice(len(gray), 6, replace=False):
        idx = tuple(gray[k])
        # Richardson: (4 D(h/2) - D(h))/3 cancels the h^2 term of the central
        # difference (the Thomeer curve bends strongly enough for it to show)
        fd = (4.0 * central(idx, h / 2) - central(idx, h)) / 3.0
        assert abs(g[idx] - fd) <= 1e-4 * abs(fd) + 1e-9 * np.abs(g).max(), (idx, g[idx], fd)


def test_eigenvector_derivative_formula():
    """d e1 from the perturbation formula against differences of eigh."""
    rng = np.random.default_rng(5)
    B = rng.standard_normal((3, 3))
    M = torch.tensor(B @ B.T, requires_grad=True)
    e = A.TopEigvec.apply(M)
    wvec = torch.tensor(rng.standard_normal(3))
    (e @ wvec).backward()
    D = rng.standard_normal((3, 3))
    D = D + D.T
    h = 1e-6

    def top(Mx):
        w, V = np.linalg.eigh(Mx)
        v = V[:, 2]
        return v * np.sign(v @ e.detach().numpy())

    fd = (top(B @ B.T + h * D) - top(B @ B.T - h * D)) / (2 * h) @ wvec.numpy()
    assert abs((M.grad.numpy() * D).sum() - fd) < 1e-6 * max(1.0, abs(fd))
