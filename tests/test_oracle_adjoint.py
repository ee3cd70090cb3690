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


def test_torch_geometry_matches_c_oracle_on_flat_blocks():
    """The geometry of the PyTorch statement (Eqs. 5-7) against the C oracle
    on uniform-porosity blocks: no axis in the flat interiors, the same
    tensor everywhere (the two sum the gradient stencil independently)."""
    case = LC.flat_blocks("d3q19", shape=(6, 10, 30))
    _, _, ost = LC.run_oracle(case, 0)
    cv = case.curves[0]
    geo = A.geometry(case.cell, torch.tensor(case.phi32.astype(np.float64)), cv, case.s["c_g"])
    kinv = geo["kinv"].detach().numpy()  # [z, y, x, 3, 3]
    gray = case.cell == 2
    ok = np.moveaxis(ost["kinv"], (0, 1), (-2, -1))
    assert np.abs(kinv - ok)[gray].max() <= 1e-12 * np.abs(ok[gray]).max()
    flat = gray & (ost["iso"] == 1)
    assert flat.sum() > 0.3 * gray.sum()
    off = ~np.eye(3, dtype=bool)
    assert np.all(kinv[flat][:, off] == 0.0)


def test_zigzag_pathway_geometry():
    """The Sec. I.B / III.E input: a connected open pathway a sixth of the
    width, gray bundles of phi = 0.95 out to the walls, reservoir rows."""
    from paper_2512_21696_gb300 import synth
    cell, phi, path = synth.zigzag_pathway_geometry()
    assert cell.shape == phi.shape == path.shape == (1, 182, 120)
    assert np.all(cell[0, 0] == synth.OUTLET) and np.all(cell[0, -1] == synth.INLET)
    inner = cell[0, 1:-1]
    assert set(np.unique(inner)) == {synth.PORE, synth.GRAY}
    assert np.all(path[0, 1:-1] == (inner == synth.PORE)) and not path[0, [0, -1]].any()
    assert np.all(phi[cell == synth.GRAY] == np.float32(0.95)) and np.all(phi[cell != synth.GRAY] == 1.0)
    rows = path[0, 1:-1]
    assert np.all(rows.sum(axis=1) == 20)  # every row: the same width
    assert all((rows[k] & rows[k + 1]).any() for k in range(rows.shape[0] - 1))  # connected top to bottom
    assert not rows[:, 0].any() and not rows[:, -1].any()  # the bundles reach both walls
