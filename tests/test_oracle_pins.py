"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes part of the oracle by something other than the oracle itself:
an analytic solution, an exact discrete identity, a conservation law, a
library routine, or the independent NumPy evaluator in ``naive_lbm``.
"""
import os

import numpy as np
import pytest

import oracle as O
import naive_lbm as N
from helpers import (cosine_hessian_matrix, rest_only_populations, stencil_sine_vector)
from paper_2512_21696_gb300 import synth

VEL = N.VEL
CS2 = 1.0 / 3.0


def kc(phi, d=1.0):
    return d * d * phi ** 3 / (180.0 * (1.0 - phi) ** 2)


# --------------------------------------------------------------------------
# Collision: Hermite-regularised operator with the Eq. 3 force term
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [0.55, 0.8, 1.0, 1.7])
def test_collision_moments_match_bgk_with_force(tau):
    """Zeroth, first and second moments equal those of BGK with the same force.

    For BGK, f* = f - (f - feq)/tau + (1 - 1/(2 tau)) F_i, whose moments are
    rho, (1-1/tau) j + rho u/tau + (1-1/(2tau)) F and
    (1-1/tau) S + (rho(I/3 + uu))/tau + (1-1/(2tau))(uF + Fu), S = sum c c f.
    With u = (j + F/2)/rho the regularised operator must reproduce them.
    """
    rng = np.random.default_rng(7)
    for _ in range(20):
        f = N.WGT * (1.0 + 0.2 * rng.standard_normal(19)) * rng.uniform(0.1, 1.5)
        F = 1e-3 * rng.standard_normal(3)
        rho = f.sum()
        j = VEL.T @ f
        u = (j + 0.5 * F) / rho
        out = O.collide_cell(f, u, F, tau)
        assert abs(out.sum() - rho) < 1e-14
        mom = VEL.T @ out
        bgk_mom = (1 - 1 / tau) * j + rho * u / tau + (1 - 1 / (2 * tau)) * F
        np.testing.assert_allclose(mom, bgk_mom, rtol=0, atol=1e-14)
        S = np.einsum("ia,ib,i->ab", VEL, VEL, f)
        S_out = np.einsum("ia,ib,i->ab", VEL, VEL, out)
        Seq = rho * (np.eye(3) / 3 + np.outer(u, u))
        bgk_S = (1 - 1 / tau) * S + Seq / tau + (1 - 1 / (2 * tau)) * (np.outer(u, F) + np.outer(F, u))
        np.testing.assert_allclose(S_out, bgk_S, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
# Flow pins: shear-wave viscosity, Poiseuille, Darcy, Brinkman
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
@pytest.mark.parametrize("tau", [0.6, 1.0, 1.4])
def test_shear_wave_decay_gives_lattice_viscosity(tau, lattice):
    """u_x = U sin(k y) decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3."""
    ny = 64
    shape = (1, ny, 1)
    p = O.make_params(shape, tau=(tau, tau), wet=0, lattice=lattice)
    cell = np.zeros(shape, np.uint8)
    k = 2 * np.pi / ny
    y = np.arange(ny)
    u = np.zeros((3,) + shape)
    u[0, 0, :, 0] = 1e-4 * np.sin(k * y)
    o = O.Oracle(p, cell)
    o.init_fields(np.ones(shape), np.zeros(shape), u)
    amps, ts = [], []
    for t in range(1, 301):
        o.step(1)
        if t >= 30 and t % 10 == 0:
            ux = o.fields()[2][0, 0, :, 0]
            amps.append(2.0 / ny * np.dot(ux, np.sin(k * y)))
            ts.append(t)
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (k * k) - nu) / nu < 5e-3


def _channel(ny_fluid, periodic_y, **kw):
    """Walls normal to y: solid rows (periodic y) or the outside (non-periodic)."""
    ny = ny_fluid + (2 if periodic_y else 0)
    shape = (1, ny, 1)
    cell = np.zeros(shape, np.uint8)
    if periodic_y:
        cell[0, 0, 0] = cell[0, -1, 0] = synth.SOLID
    p = O.make_params(shape, periodic=(1, int(periodic_y), 1), **kw)
    return shape, cell, p


def test_poiseuille_profile():
    """Body-force channel: u(y) = g/(2 nu) (y - y0)(y1 - y), walls halfway."""
    W, g = 32, 1e-6
    shape, cell, p = _channel(W, True, accel=((g, 0, 0), (0, 0, 0)), wet=0)
    o = O.Oracle(p, cell)
    o.init_fields(np.ones(shape), np.zeros(shape))
    o.step(20000)
    ux = o.fields()[2][0, 0, 1:-1, 0]
    y = np.arange(1, W + 1)
    nu = 1.0 / 6.0
    exact = g / (2 * nu) * (y - 0.5) * (W + 0.5 - y)
    assert np.max(np.abs(ux - exact)) / exact.max() < 1e-2


def test_d2q9_is_the_plane_projection_of_d3q19_at_unit_tau():
    """On a z-invariant state D3Q19 populations summed over c_z obey the D2Q9
    step: the projected weights are 4/9, 1/9, 1/36, and equilibrium, force
    term and every isotropic stencil project linearly.  At tau = 1 the
    regularised part, whose projection would carry the zz moment, vanishes.
    So the D2Q9 oracle and the D3Q19 oracle on one periodic plane agree to
    round-off, with solid, gray (tensorial, capillary, residual switches),
    Shan-Chen, walls and body forces (Eq. 4 is left out: its moment Hessian
    has a zz entry on D3Q19)."""
    rng = np.random.default_rng(8)
    shape = (1, 12, 10)
    cell = np.zeros(shape, np.uint8)
    cell[rng.random(shape) < 0.1] = synth.SOLID
    cell[(rng.random(shape) < 0.4) & (cell == 0)] = synth.GRAY
    phi = np.where(cell == synth.GRAY, 0.15 + 0.4 * rng.random(shape), 1.0)
    xx = np.arange(shape[2])[None, None, :] + np.zeros(shape)
    ra = np.where(xx < 5, 1.0, 0.03) + 0.05 * rng.random(shape)
    rb = 1.06 - ra
    u0 = 0.01 * rng.standard_normal((3,) + shape)
    u0[2] = 0.0
    common = dict(G=1.1, tau=(1.0, 1.0), accel=((1e-4, 2e-5, 0), (0, -1e-4, 0)), rho_wall=(0.7, 0.2), wet=1)
    curves = [O.make_curve(aniso=10.0)]
    o3 = O.Oracle(O.make_params(shape, **common), cell, phi, curves=curves)
    o2 = O.Oracle(O.make_params(shape, lattice="d2q9", **common), cell, phi, curves=curves)
    # flipped residual flags, so that both hysteresis transitions occur
    s = np.clip((rb / (ra + rb) - 0.03 / 1.03) / (1.0 / 1.03 - 0.03 / 1.03), 0, 1)
    wet0 = np.where(cell == synth.GRAY, s < 0.5, s >= 0.5).astype(np.int32)
    for o in (o3, o2):
        o.init_fields(ra, rb, u0)
        o.set_residual(np.zeros(shape), np.zeros(shape), wet0)
    assert o2.Q == 9 and o3.Q == 19
    vel19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0),
             (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1),
             (0, -1, -1), (0, 1, -1), (0, -1, 1)]
    vel9 = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]
    proj = np.zeros((9, 19))
    for i, c in enumerate(vel19):
        proj[vel9.index(c[:2]), i] = 1.0
    for _ in range(25):
        o3.step(1)
        o2.step(1)
    f3, f2 = o3.populations(), o2.populations()
    np.testing.assert_allclose(np.einsum("qi,ai...->aq...", proj, f3), f2, rtol=0, atol=1e-13)
    for x, y in zip(o3.fields(), o2.fields()):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)
    Rw, Ro, _ = o2.residual()
    assert (Rw > 0).any() and (Ro > 0).any()


def test_open_axis_equals_solid_rows():
    """A non-periodic axis behaves exactly like solid rows just outside it."""
    W, g = 12, 1e-5
    shape_a, cell_a, pa = _channel(W, True, accel=((g, 0, 0), (0, 0, 0)), G=1.1)
    shape_b, cell_b, pb = _channel(W, False, accel=((g, 0, 0), (0, 0, 0)), G=1.1)
    rng = np.random.default_rng(3)
    rA = 0.5 + 0.4 * rng.random((1, W, 1))
    rB = 1.03 - rA
    oa, ob = O.Oracle(pa, cell_a), O.Oracle(pb, cell_b)
    pad = lambda a: np.pad(a, ((0, 0), (1, 1), (0, 0)), constant_values=0.5)
    oa.init_fields(pad(rA), pad(rB))
    ob.init_fields(rA, rB)
    oa.step(50)
    ob.step(50)
    fa, fb = oa.fields(), ob.fields()
    np.testing.assert_allclose(fa[0][:, 1:-1], fb[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(fa[2][:, :, 1:-1], fb[2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("phi", [0.3, 0.5])
def test_darcy_uniform_gray(phi):
    """Uniform gray domain, one component: steady u = g K0(phi)/nu exactly."""
    g = 1e-6
    shape = (4, 4, 4)
    cell = np.full(shape, synth.GRAY, np.uint8)
    p = O.make_params(shape, accel=((g, 0, 0), (0, 0, 0)), wet=0)
    curves = [O.make_curve(kc_d=2.0), O.make_curve(kc_d=1.0)]
    ptype = np.ones(shape, np.uint8)  # second curve: kc_d = 1
    o = O.Oracle(p, cell, np.full(shape, phi), ptype=ptype, curves=curves)
    o.init_fields(np.ones(shape), np.zeros(shape))
    o.step(6000)
    ux = o.fields()[2][0]
    expected = g * kc(phi) / (1.0 / 6.0)
    # The stiff semi-implicit update contracts by (rho - R/2)/(rho + R/2) ~ -0.993
    # per step, so FP64 round-off in j is amplified ~1/(1 - 0.993) and the
    # iteration settles in a 2-cycle ~4e-9 (relative) around the fixed point.
    np.testing.assert_allclose(ux, expected, rtol=1e-7)


def test_two_component_darcy_with_corey_permeabilities():
    """A uniform mixture in a uniform gray domain under one body acceleration:
    steady u = K0 (rho_A + rho_B) g / coef with the Eq. 1 drag coefficient
    coef = rho_n nu_n / kr_n + rho_w nu_w / kr_w, Corey kr_w = Se^nw,
    kr_n = (1 - Se)^nn at the local saturation (no interface, so no capillary,
    Shan-Chen or Eq. 4 force)."""
    g, phi, kd = 1e-6, 0.5, 10.0
    shape = (4, 4, 4)
    cell = np.full(shape, synth.GRAY, np.uint8)
    p = O.make_params(shape, accel=((g, 0, 0), (g, 0, 0)), wet=1, tau=(1.0, 0.8))
    curve = O.make_curve(kc_d=kd, swr=0.15, nw=3.0, nn=2.0)
    o = O.Oracle(p, cell, np.full(shape, phi), curves=[curve])
    ra, rb = 0.4, 0.6  # B wets
    o.init_fields(np.full(shape, ra), np.full(shape, rb))
    o.step(200)
    r_lo, r_hi = 0.03 / 1.03, 1.0 / 1.03
    s_w = (rb / (ra + rb) - r_lo) / (r_hi - r_lo)
    se = (s_w - 0.15) / 0.85
    kr_w, kr_n = se ** 3.0, (1.0 - se) ** 2.0
    nu_a, nu_b = (1.0 - 0.5) / 3.0, (0.8 - 0.5) / 3.0
    coef = ra * nu_a / kr_n + rb * nu_b / kr_w
    expected = kc(phi, kd) * (ra + rb) * g / coef
    u = o.fields()[2]
    np.testing.assert_allclose(u[0], expected, rtol=1e-10)
    assert np.abs(u[1:]).max() < 1e-20
    assert abs(kr_w - kr_n) > 0.05 and abs(se ** 2 - (1 - se) ** 3) > 0.1  # the exponents matter here


def test_shan_chen_force_next_to_a_wall():
    """Beside a solid plane the other component's density stencil sees the
    virtual wall density (the wetting control): for uniform fluid densities,
    F_SC^A = -G rho^A (rho^B - rho_wall^B) / 2 towards the wall's normal, and
    symmetrically for B; no force one cell further in."""
    shape = (6, 4, 4)
    cell = np.zeros(shape, np.uint8)
    cell[0] = synth.SOLID
    G, rw = 1.1, (0.2, 0.7)
    p = O.make_params(shape, G=G, rho_wall=rw)
    ra, rb = 0.3, 0.6
    fl = cell != synth.SOLID
    o = _rest_state(p, cell, np.where(fl, ra, 0.0), np.where(fl, rb, 0.0))
    FA, FB = o.force_term(O.TERM_SC, 0), o.force_term(O.TERM_SC, 1)
    # z = 1 has the wall below (-z), z = 5 above (+z, periodic): the stencil's
    # z component is (rho(+z side) - rho(-z side)) / 2
    np.testing.assert_allclose(FA[2, 1], -G * ra * (rb - rw[1]) / 2, rtol=1e-13)
    np.testing.assert_allclose(FB[2, 1], -G * rb * (ra - rw[0]) / 2, rtol=1e-13)
    np.testing.assert_allclose(FA[2, 5], -G * ra * (rw[1] - rb) / 2, rtol=1e-13)
    assert np.abs(FA[:2]).max() < 1e-15 and np.abs(FA[2, 2:5]).max() < 1e-15


@pytest.mark.parametrize("phi", [0.6, 0.4])
def test_darcy_between_pressure_reservoirs(phi):
    """One component through a uniform gray column between an inlet and an
    outlet reservoir (Eq. 1 drag, the reservoir reading of the pressure
    boundaries).  At steady state the interior density is linear in x, the
    mass flux rho u is the same at every cell and obeys Darcy's law
    rho u = -(K0/nu) dp/dx with p = rho/3 and the local slope; the linear
    profile reaches the held densities between the reservoir node and the
    face half a cell beyond it (the same place as halfway bounce-back), and
    the reservoirs keep their densities with u = 0."""
    L = 16
    shape = (1, 1, L)
    cell = np.full(shape, synth.GRAY, np.uint8)
    cell[..., 0], cell[..., -1] = synth.INLET, synth.OUTLET
    r_in, r_out = 1.005, 0.995
    p = O.make_params(shape, periodic=(0, 1, 1), wet=0, rho_in=(r_in, 0.0), rho_out=(r_out, 0.0))
    o = O.Oracle(p, cell, np.full(shape, phi))
    o.init_fields(np.ones(shape), np.zeros(shape))
    o.step(60000)
    a, b, u, sw = o.fields()
    assert a[0, 0, 0] == r_in and a[0, 0, -1] == r_out and np.all(u[:, 0, 0, [0, -1]] == 0.0)
    x = np.arange(1, L - 1)
    r = a[0, 0, 1:-1]
    slope, icpt = np.polyfit(x, r, 1)
    assert np.abs(r - (slope * x + icpt)).max() < 1e-8 * abs(slope)
    J = (a * u[0])[0, 0, 1:-1]
    assert np.ptp(J) < 1e-8 * J.mean()
    nu = 1.0 / 6.0
    np.testing.assert_allclose(J.mean(), -kc(phi) / nu * slope / 3.0, rtol=1e-6)
    x_in, x_out = (r_in - icpt) / slope, (r_out - icpt) / slope
    assert 0.4 < x_in <= 0.5 and 0.4 < (L - 1) - x_out <= 0.5
    assert abs(x_in - ((L - 1) - x_out)) < 1e-3  # the offset depends weakly on the local density


def test_tensorial_resistivity_direction():
    """phi varying along z only puts the principal axis on z (Eq. 7).

    Driving along x must not feel the anisotropy (same flux for a = 1 and
    a = 10).  Driving along z the steady one-dimensional flux J = rho u_z is
    uniform and the period average of the momentum balance
    rho g = R_zz u_z + dp/dz gives J = <rho> g / (nu a <1/K0>).
    """
    nz = 32
    shape = (nz, 1, 1)
    z = np.arange(nz)
    phi = (0.85 + 0.05 * np.cos(2 * np.pi * z / nz))[:, None, None]
    cell = np.full(shape, synth.GRAY, np.uint8)
    g = 1e-6

    def run(aniso, d):
        acc = [0.0, 0.0, 0.0]
        acc[d] = g
        p = O.make_params(shape, accel=(tuple(acc), (0, 0, 0)), wet=0)
        o = O.Oracle(p, cell, phi, curves=[O.make_curve(aniso=aniso)])
        o.init_fields(np.ones(shape), np.zeros(shape))
        o.step(8000)
        ra, rb, u, sw = o.fields()
        return (ra * u[d]).mean(), ra.mean(), o.static()

    qx1, _, st = run(1.0, 0)
    qx10, _, st10 = run(10.0, 0)
    assert abs(qx1 - qx10) < 1e-9 * abs(qx1)
    kinv = st10["kinv"][:, :, :, 0, 0]
    K0 = kc(phi[:, 0, 0])
    np.testing.assert_allclose(kinv[2, 2], 10.0 / K0, rtol=1e-12)
    np.testing.assert_allclose(kinv[0, 0], 1.0 / K0, rtol=1e-12)
    assert np.abs(kinv[0, 2]).max() < 1e-9 / K0.min()
    for a in (1.0, 10.0):
        J, rho_mean, _ = run(a, 2)
        closed = rho_mean * g / ((1.0 / 6.0) * a * np.mean(1.0 / K0))
        assert abs(J / closed - 1.0) < 1e-4


def test_brinkman_channel():
    """Uniform gray channel: u = (gK/nu)[1 - cosh((y-yc)/sqrt K)/cosh(W/(2 sqrt K))]."""
    W, g, phi = 32, 1e-6, 0.97
    shape, cell, p = _channel(W, True, accel=((g, 0, 0), (0, 0, 0)), wet=0)
    cell[0, 1:-1, 0] = synth.GRAY
    o = O.Oracle(p, cell, np.full(shape, phi))
    o.init_fields(np.ones(shape), np.zeros(shape))
    o.step(20000)
    ux = o.fields()[2][0, 0, 1:-1, 0]
    K = kc(phi)
    nu = 1.0 / 6.0
    y = np.arange(1, W + 1)
    yc = 0.5 * (0.5 + W + 0.5)
    exact = g * K / nu * (1 - np.cosh((y - yc) / np.sqrt(K)) / np.cosh(W / (2 * np.sqrt(K))))
    assert np.max(np.abs(ux - exact)) / exact.max() < 2e-2


# --------------------------------------------------------------------------
# Inter-component forces on analytic density fields
# --------------------------------------------------------------------------
def _rest_state(p, cell, rhoA, rhoB, phi=None, curves=None):
    o = O.Oracle(p, cell, phi, curves=curves)
    o.init_fields(rhoA, rhoB)
    o.set_populations(rest_only_populations(rhoA, rhoB, o.Q))
    o.step(1)
    return o


def test_shan_chen_force_on_cosine_field():
    """F_SC^A = -G rho^A (1/cs^2) sum w_i rho^B(x+c_i) c_i, exact for cosines."""
    n = 12
    shape = (n, n, n)
    k = 2 * np.pi * np.array([1, 2, 1]) / n
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    th = k[0] * x + k[1] * y + k[2] * z
    rhoA = 0.6 + 0.3 * np.cos(th + 0.4)
    rhoB = 0.5 + 0.2 * np.cos(th)
    G = 1.1
    o = _rest_state(O.make_params(shape, G=G), np.zeros(shape, np.uint8), rhoA, rhoB)
    FA = o.force_term(O.TERM_SC, 0)
    v = stencil_sine_vector(k)
    gradB = -0.2 * np.sin(th)[None] * v[:, None, None, None] / CS2
    np.testing.assert_allclose(FA, -G * rhoA[None] * gradB, rtol=0, atol=1e-15)
    FB = o.force_term(O.TERM_SC, 1)
    gradA = -0.3 * np.sin(th + 0.4)[None] * v[:, None, None, None] / CS2
    np.testing.assert_allclose(FB, -G * rhoB[None] * gradA, rtol=0, atol=1e-15)


def test_capillary_force_flat_interface_telescopes():
    """Sum over an interface of -Pc rho_r n H equals -(Pc/4) times the At jump.

    With H = |grad At|/2 the capillary force density is -Pc grad(At)/2 and the
    central difference telescopes: sum_{z=a..b} grad_z At = [At(b+1) + At(b)
    - At(a) - At(a-1)]/2.  Pc is made constant by a huge Brooks-Corey lambda
    and phi = phi_ref (Leverett factor 1).
    """
    nz = 32
    shape = (nz, 2, 2)
    z = np.arange(nz)
    A = (-0.99 * np.cos(2 * np.pi * z / nz))[:, None, None] * np.ones(shape)
    c = 1.0
    rw, rn = 0.5 * c * (1 + A), 0.5 * c * (1 - A)
    p = O.make_params(shape, at_cut=1.0, wet=1)
    cell = np.full(shape, synth.GRAY, np.uint8)
    curve = O.make_curve(lam=1e9, phi_ref=0.35)
    o = _rest_state(p, cell, rn, rw, phi=np.full(shape, 0.35), curves=[curve])
    Fz = o.force_term(O.TERM_CAP, 0)[2] + o.force_term(O.TERM_CAP, 1)[2]
    a, b = 0, 16
    Az = A[:, 0, 0]
    jump = 0.25 * (Az[b + 1] + Az[b] - Az[a] - Az[a - 1])
    total = Fz[a:b + 1, 0, 0].sum()
    # Se^(-1/lambda) with lambda = 1e9 and Se >= 1e-2 keeps Pc within 5e-9 of pd
    assert abs(total - (-0.02 * jump)) < 1e-8 * 0.02
    assert np.abs(o.force_term(O.TERM_CAP, 0)[0]).max() < 1e-18
    # Thomeer: Pc = Pe 10^(-G / ln(1 - Se)) tends to the entry pressure Pe as
    # G -> 0 (|ln(1 - Se)| >= 0.01 for Se >= 1e-2) and, for Se < 1, is capped
    # at 10 Pe (an amplitude 0.9 keeps s, hence Se, below 1 in every cell)
    for g, scale, amp, tol in ((1e-9, 1.0, 0.99, 1e-6), (1e3, 10.0, 0.9, 1e-12)):
        A = (-amp * np.cos(2 * np.pi * z / nz))[:, None, None] * np.ones(shape)
        Az = A[:, 0, 0]
        jump = 0.25 * (Az[b + 1] + Az[b] - Az[a] - Az[a - 1])
        o = _rest_state(p, cell, 0.5 * c * (1 - A), 0.5 * c * (1 + A), phi=np.full(shape, 0.35),
                        curves=[O.make_curve(thomeer_g=g, phi_ref=0.35)])
        Fz = o.force_term(O.TERM_CAP, 0)[2] + o.force_term(O.TERM_CAP, 1)[2]
        total = Fz[a:b + 1, 0, 0].sum()
        assert abs(total - (-0.02 * scale * jump)) < tol * 0.02 * scale


def test_thomeer_capillary_pressure_inside_the_curve():
    """Cell by cell, the capillary force of Eq. 1 summed over the components is
    -Pc(Sw) grad(At) / 2 (H = |grad At| / 2, the rho_r / rho_t weights sum to
    one), so Pc can be read off and set against Thomeer's hyperbola
    Pc = Pe 10^min(-G / ln(1 - Se), 1) at interior saturations, on both sides
    of the cap (phi = phi_ref: Pe = Pd)."""
    nz = 32
    shape = (nz, 2, 2)
    z = np.arange(nz)
    A = (-0.9 * np.cos(2 * np.pi * z / nz))[:, None, None] * np.ones(shape)
    p = O.make_params(shape, at_cut=1.0, wet=1)
    cell = np.full(shape, synth.GRAY, np.uint8)
    g, pd, swr = 0.5, 0.02, 0.15
    o = _rest_state(p, cell, 0.5 * (1 - A), 0.5 * (1 + A), phi=np.full(shape, 0.35),
                    curves=[O.make_curve(thomeer_g=g, phi_ref=0.35, pd=pd, swr=swr)])
    Fz = (o.force_term(O.TERM_CAP, 0)[2] + o.force_term(O.TERM_CAP, 1)[2])[:, 0, 0]
    Az = A[:, 0, 0]
    dAt = 0.5 * (np.roll(Az, -1) - np.roll(Az, 1))  # the isotropic stencil on a z-only field
    r_lo, r_hi = 0.03 / 1.03, 1.0 / 1.03
    s = np.clip(((1 + Az) / 2 - r_lo) / (r_hi - r_lo), 0.0, 1.0)  # wetting B at rho_B / rho_t
    se = np.clip((s - swr) / (1 - swr), 1e-2, 1.0)
    expect = pd * 10.0 ** np.minimum(-g / np.log(1.0 - se), 1.0)
    use = np.abs(dAt) > 1e-3
    got = -2.0 * Fz[use] / dAt[use]
    np.testing.assert_allclose(got, expect[use], rtol=1e-10)
    e = -g / np.log(1.0 - se[use])
    assert (e < 1.0).sum() >= 4 and (e > 1.0).sum() >= 4  # both branches are exercised


@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
def test_csf_force_on_cylinder_matches_continuum(lattice):
    """Eq. 4 on a smooth cylindrical interface: div n = 1/r in two dimensions.

    phi^A = rho^B = b0 + b1 tanh((r - R)/w) rises outward, so n^A = r-hat and
    F_csf^A,r = kappa (-1/r) (d rho^B/dr / phi_avg) (rho^A / phi_max).  The
    lattice stencils carry an O((1/w)^2) truncation error (0.8 % at w = 8).
    """
    n, R, w = 128, 40.0, 8.0
    shape = (1, n, n)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cx = cy = n / 2 - 0.5
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    b0, b1 = 0.5, 0.45
    rhoB = (b0 + b1 * np.tanh((r - R) / w))[None]
    rhoA = (0.6 - 0.2 * np.tanh((r - R) / w))[None]
    kappa = -0.045
    p = O.make_params(shape, kappa=kappa, csf_everywhere=1, phi_avg=(0.515, 0.515), phi_max=(1.0, 1.0),
                      lattice=lattice)
    o = _rest_state(p, np.zeros(shape, np.uint8), rhoA, rhoB)
    F = o.force_term(O.TERM_CSF, 0)[:2, 0]
    rh = np.stack([(x - cx) / r, (y - cy) / r])
    Fr = (F * rh).sum(axis=0)
    dBdr = b1 / w / np.cosh((r - R) / w) ** 2
    cont = kappa * (-1.0 / r) * (dBdr / 0.515) * (rhoA[0] / 1.0)
    band = np.abs(r - R) < 1.0
    rel = np.abs(Fr[band] - cont[band]) / np.abs(cont[band])
    assert rel.max() < 0.02
    assert np.all(np.sign(Fr[band]) == np.sign(cont[band]))


def test_csf_acts_in_gray_cells_only_unless_everywhere():
    """Eq. 4 is the under-resolved regions' surface-tension control: with
    csf_everywhere = 0 its force is exactly zero in pore cells and, in gray
    cells, equal to the force of the same densities with Eq. 4 applied
    everywhere (it depends on the densities only)."""
    n, R, w = 64, 20.0, 4.0
    shape = (1, n, n)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
    rhoB = (0.5 + 0.45 * np.tanh((r - R) / w))[None]
    rhoA = (0.6 - 0.2 * np.tanh((r - R) / w))[None]
    cell = np.where(x < n // 2, synth.GRAY, synth.PORE).astype(np.uint8)[None]
    phi = np.where(cell == synth.GRAY, 0.5, 1.0)
    F = {}
    for everywhere in (0, 1):
        p = O.make_params(shape, kappa=-0.045, csf_everywhere=everywhere, lattice="d2q9")
        o = _rest_state(p, cell, rhoA, rhoB, phi=phi)
        F[everywhere] = np.stack([o.force_term(O.TERM_CSF, a) for a in range(2)])
    gray = cell == synth.GRAY
    assert np.all(F[0][..., ~gray] == 0.0)
    np.testing.assert_array_equal(F[0][..., gray], F[1][..., gray])
    assert np.abs(F[1][..., ~gray]).max() > 1e-6  # the pore cells do carry a force when applied everywhere


# --------------------------------------------------------------------------
# Conservation
# --------------------------------------------------------------------------
def test_mass_and_momentum_conservation_periodic():
    n = 16
    shape = (n, n, n)
    rng = np.random.default_rng(11)
    rA, rB = synth.droplet_fields(shape, 5, (8, 8, 8), 1.0, 0.03)
    rA = rA + 0.01 * rng.random(shape)
    u = 1e-3 * rng.standard_normal((3,) + shape)
    o = O.Oracle(O.make_params(shape, G=1.1, tau=(0.8, 1.2)), np.zeros(shape, np.uint8))
    o.init_fields(rA, rB, u)
    m0 = (rA.sum(), rB.sum())
    o.step(1)
    a, b, uu, _ = o.fields()
    p1 = ((a + b)[None] * uu).sum(axis=(1, 2, 3))
    o.step(60)
    a, b, uu, _ = o.fields()
    assert abs(a.sum() - m0[0]) < 1e-12 * m0[0]
    assert abs(b.sum() - m0[1]) < 1e-12 * m0[1]
    p2 = ((a + b)[None] * uu).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(p2, p1, rtol=0, atol=1e-13)


def test_mass_conserved_with_walls_and_gray_cells():
    n = 12
    shape = (n, n, n)
    rng = np.random.default_rng(5)
    cell = np.zeros(shape, np.uint8)
    cell[rng.random(shape) < 0.15] = synth.SOLID
    cell[(rng.random(shape) < 0.3) & (cell == 0)] = synth.GRAY
    phi = 0.2 + 0.3 * rng.random(shape)
    rA, rB = synth.droplet_fields(shape, 4, (6, 6, 6), 1.0, 0.03)
    p = O.make_params(shape, G=1.1, kappa=-0.045, accel=((1e-5, 0, 0), (0, 0, 0)), tau=(0.7, 1.0))
    o = O.Oracle(p, cell, phi, curves=[O.make_curve(aniso=10.0)])
    o.init_fields(rA, rB)
    fl = cell != synth.SOLID
    m0 = (rA[fl].sum(), rB[fl].sum())
    o.step(40)
    a, b, _, _ = o.fields()
    assert abs(a[fl].sum() - m0[0]) < 1e-12 * m0[0]
    assert abs(b[fl].sum() - m0[1]) < 1e-12 * m0[1]


# --------------------------------------------------------------------------
# Laplace's law (2-D droplets, Sec. III.A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
def test_laplace_law_two_dimensional(lattice):
    """Delta p = sigma / R (Sec. III.A): Delta p * R is nearly the same for every R.

    R is the mass-equivalent radius of the droplet.  Diffuse-interface
    pseudo-potential droplets slowly dissolve and carry a curvature
    (Tolman-like) correction, so sigma = Delta p R varies by a few percent
    over R = 10..18 on a 64^2 grid; a wrong sign of G, a wrong stencil
    normalisation or a missing component would break the 1/R law outright.
    """
    n = 64
    shape = (1, n, n)
    dps, radii = [], []
    for R in (10.0, 14.0, 18.0):
        rA, rB = synth.cylinder_droplet_fields(shape, R, (32, 32), 1.0, 0.03)
        o = O.Oracle(O.make_params(shape, G=1.1, lattice=lattice), np.zeros(shape, np.uint8))
        o.init_fields(rA, rB)
        o.step(3000)
        a = o.fields()[0]
        radii.append(np.sqrt((a.sum() - a.min() * a.size) / (a.max() - a.min()) / np.pi))
        dps.append(o.observables(probe=(32, 32, 0, R - 4, R + 4))["dp"])
    dps, radii = np.array(dps), np.array(radii)
    sig = dps * radii
    assert np.all(dps > 0) and np.all(np.diff(dps) < 0)
    assert (sig.max() - sig.min()) / sig.mean() < 0.08
    slope, icpt = np.polyfit(1.0 / radii, dps, 1)
    assert abs(icpt) < 0.10 * dps.max()


def test_laplace_law_three_dimensional():
    """Delta p = 2 sigma / R for spherical droplets (Sec. III.A's law in 3-D).

    Droplets of A with R = 5, 6.5, 8, 9.5 in a 32^3 periodic box (G = 1.1,
    600 steps; R is the mass-equivalent radius).  Measured: Delta p 0.0282,
    0.0214, 0.0181, 0.0153 and sigma = Delta p R / 2 from 0.064 to 0.070 (the
    diffuse interface dissolves the droplet by about half a cell and carries
    a curvature correction); a linear fit against 1/R has slope 0.117 and
    intercept 0.0025, 9 % of the largest Delta p.  A cylinder of the same
    interface (R = 10 on a 48^2 periodic plane) gives sigma = Delta p R
    within 15 % of the spheres' Delta p R / 2: the factor 2 of the 3-D law.
    A wrong sign of G or a missing component would break the linear law
    outright.
    """
    n = 32
    shape = (n, n, n)
    c = n // 2
    dps, radii = [], []
    for R in (5.0, 6.5, 8.0, 9.5):
        rA, rB = synth.droplet_fields(shape, R, (c, c, c), 1.0, 0.03)
        o = O.Oracle(O.make_params(shape, G=1.1), np.zeros(shape, np.uint8))
        o.init_fields(rA, rB)
        o.step(600)
        a = o.fields()[0]
        radii.append(((a.sum() - a.min() * a.size) / (a.max() - a.min()) * 3.0 / (4.0 * np.pi)) ** (1.0 / 3.0))
        dps.append(o.observables(probe=(c, c, c, R - 4, R + 4))["dp"])
    dps, radii = np.array(dps), np.array(radii)
    sig = dps * radii / 2.0
    assert np.all(dps > 0) and np.all(np.diff(dps) < 0)
    assert (sig.max() - sig.min()) / sig.mean() < 0.12
    slope, icpt = np.polyfit(1.0 / radii, dps, 1)
    assert abs(icpt) < 0.12 * dps.max()
    assert abs(slope / 2.0 / sig.mean() - 1.0) < 0.15
    # the factor 2 of the sphere: the same interface bent into a cylinder (the
    # same D3Q19 model on one periodic plane, Delta p = sigma / R) gives the
    # same sigma (measured 0.063 against the spheres' 0.064 - 0.070)
    shape2 = (1, 48, 48)
    rA, rB = synth.cylinder_droplet_fields(shape2, 10.0, (24, 24), 1.0, 0.03)
    o = O.Oracle(O.make_params(shape2, G=1.1), np.zeros(shape2, np.uint8))
    o.init_fields(rA, rB)
    o.step(1500)
    a = o.fields()[0]
    rc = np.sqrt((a.sum() - a.min() * a.size) / (a.max() - a.min()) / np.pi)
    sig_cyl = o.observables(probe=(24, 24, 0, 6.0, 14.0))["dp"] * rc
    assert abs(sig_cyl / sig.mean() - 1.0) < 0.15, (sig_cyl, sig)


# --------------------------------------------------------------------------
# Geometry precompute: Hessian axis, Leverett scaling, residual amounts
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
@pytest.mark.parametrize("phi0", [0.35, 0.1, 1 / 3, 0.7])
def test_flat_porosity_has_no_axis(lattice, phi0):
    """A region of uniform phi has zero gradient and Hessian (Eqs. 6-7), so M = 0
    and no axis: K^-1 = I / K0 exactly, in a periodic block and in the interior
    of a flat gray slab that borders open pore."""
    shape = (1, 10, 12) if lattice == "d2q9" else (6, 10, 12)
    aniso = 10.0
    for slab in (False, True):
        cell = np.full(shape, synth.GRAY, np.uint8)
        if slab:
            cell[..., :3] = synth.PORE
        phi = np.where(cell == synth.GRAY, np.float32(phi0), 1.0).astype(np.float32).astype(np.float64)
        o = O.Oracle(O.make_params(shape, lattice=lattice), cell, phi, curves=[O.make_curve(aniso=aniso)])
        st = o.static()
        gray = cell == synth.GRAY
        # cells whose whole 3x3(x3) neighbourhood is gray with the same phi
        inner = gray.copy()
        if slab:
            inner[..., :5] = False
            inner[..., -1] = False  # periodic in x: its +x neighbour is pore
        assert inner.any()
        assert np.all(st["iso"][inner] == 1)
        K0 = kc(float(np.float32(phi0)))
        for idx in zip(*np.nonzero(inner)):
            got = st["kinv"][(slice(None), slice(None)) + idx]
            np.testing.assert_allclose(got, np.eye(3) / K0, rtol=1e-14)
            assert np.all(got[~np.eye(3, dtype=bool)] == 0.0)
        if slab:  # next to the pore the gradient is along x: the axis is x
            edge = np.zeros(shape, bool)
            edge[..., 3] = True
            assert np.all(st["iso"][edge] == 0)
            e = st["kinv"][0, 0][edge] * K0
            np.testing.assert_allclose(e, aniso, rtol=1e-12)


@pytest.mark.parametrize("delta", [1e-6, 1e-4])
def test_tiny_porosity_wave_keeps_its_axis(delta):
    """A real but tiny porosity variation phi0 + delta sin(2 pi x / n) has its
    gradient and Hessian along x at every cell, so every cell is anisotropic
    with e1 = x: the tie test's floor swallows round-off, not real gradients."""
    n, aniso = 16, 5.0
    shape = (4, 4, n)
    x = np.arange(n)
    phi = (0.35 + delta * np.sin(2 * np.pi * x / n))[None, None, :] * np.ones(shape)
    phi = phi.astype(np.float32).astype(np.float64)
    cell = np.full(shape, synth.GRAY, np.uint8)
    st = O.Oracle(O.make_params(shape), cell, phi, curves=[O.make_curve(aniso=aniso)]).static()
    assert np.all(st["iso"] == 0)
    K0 = kc(phi)
    np.testing.assert_allclose(st["kinv"][0, 0] * K0, aniso, rtol=1e-9)
    np.testing.assert_allclose(st["kinv"][1, 1] * K0, 1.0, rtol=1e-9)
    np.testing.assert_allclose(st["kinv"][2, 2] * K0, 1.0, rtol=1e-9)
    assert np.abs(st["kinv"][0, 1] * K0).max() < 1e-9


@pytest.mark.parametrize("c_g", [1.0, 4.0])
@pytest.mark.parametrize("m", [(1, 0, 0), (0, 1, 0), (1, 1, 0), (1, 1, 1), (1, 2, 3), (2, 0, 1)])
def test_principal_axis_on_cosine_porosity(m, c_g):
    """Closed-form Hessian and gradient of phi0 + a cos(k.x), eigh for e1 of
    M = H H + c_g grad(phi) grad(phi)^T (two weights of the gradient term)."""
    n = 12
    shape = (n, n, n)
    k = 2 * np.pi * np.array(m, float) / n
    amp, phi0, aniso = 0.1, 0.4, 7.0
    phi = synth.cosine_porosity(shape, phi0, amp, k)
    cell = np.full(shape, synth.GRAY, np.uint8)
    o = O.Oracle(O.make_params(shape, c_g=c_g), cell, phi, curves=[O.make_curve(aniso=aniso)])
    st = o.static()
    Mk = cosine_hessian_matrix(k)
    v = stencil_sine_vector(k) / CS2
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    th = k[0] * x + k[1] * y + k[2] * z
    checked = 0
    for idx in zip(*[a.ravel() for a in (z, y, x)]):
        H = -amp * np.cos(th[idx]) * Mk
        g = -amp * np.sin(th[idx]) * v
        M = H @ H + c_g * np.outer(g, g)
        wv, V = np.linalg.eigh(M)
        K0 = kc(phi[idx])
        got = st["kinv"][(slice(None), slice(None)) + idx]
        if wv[2] - wv[1] <= 1e-12 * max(wv[2], 1e-30):
            assert st["iso"][idx] == 1
            np.testing.assert_allclose(got, np.eye(3) / K0, rtol=1e-12)
            continue
        if wv[2] - wv[1] < 1e-6 * wv[2]:
            continue  # ill-conditioned axis; not a meaningful comparison
        e1 = V[:, 2]
        exp_kinv = (np.eye(3) + (aniso - 1) * np.outer(e1, e1)) / K0
        np.testing.assert_allclose(got, exp_kinv, rtol=0, atol=1e-9 / K0)
        checked += 1
    assert checked > n ** 3 // 2
    if m in [(1, 0, 0), (0, 1, 0)]:
        d = m.index(1)
        K0 = kc(phi)
        np.testing.assert_allclose(st["kinv"][d, d], aniso / K0, rtol=1e-12)


def test_leverett_invariance_and_residual_crossings():
    """Eq. 5: Pc sqrt(K0/phi) is phi-independent; Sw_irr/So_res invert Pc(Sw).

    The residual amounts also jump from cell to cell: cells whose scaled entry
    pressure lies above Pc_ref,min hold no residual oil (Fig. 6 discussion).
    """
    n = 10
    shape = (n, n, n)
    rng = np.random.default_rng(2)
    phi = 0.1 + 0.5 * rng.random(shape)
    cell = np.full(shape, synth.GRAY, np.uint8)
    cv = dict(pd=0.02, lam=2.0, swr=0.15, phi_ref=0.35, f_max=3.5, f_min=0.575)
    o = O.Oracle(O.make_params(shape), cell, phi, curves=[O.make_curve(**cv)])
    st = o.static()
    K0 = kc(phi)
    J = st["lamL"] * np.sqrt(K0 / phi)
    np.testing.assert_allclose(J, np.sqrt(kc(0.35) / 0.35), rtol=1e-13)

    def pc_fwd(sw, lamL):
        se = (sw - cv["swr"]) / (1 - cv["swr"])
        return lamL * cv["pd"] * se ** (-1.0 / cv["lam"])

    for key, pref in (("swirr", cv["f_max"] * cv["pd"]), ("sores", cv["f_min"] * cv["pd"])):
        sw = st[key] if key == "swirr" else 1.0 - st[key]
        below = pref <= st["lamL"] * cv["pd"]
        assert np.all(sw[below] == 1.0)
        np.testing.assert_allclose(pc_fwd(sw[~below], st["lamL"][~below]), pref, rtol=1e-12)
    assert np.any(st["sores"] == 0.0) and np.any(st["sores"] > 0.1)


@pytest.mark.parametrize("g", [0.1, 0.4, 1.5])
def test_thomeer_residual_crossings(g):
    """Thomeer curve (the Appendix's Pc form): the residual amounts sit where
    Thomeer's hyperbola log10(Pc/Pe) * ln(1 - Se) = -G crosses Pc_ref,max and
    Pc_ref,min (Pe = lamL Pd, Se normalised); cells whose entry pressure is at
    or above a reference pressure have Sw = 1 there; a larger G (more
    gradual pore throats) leaves more residual water at the same pressure."""
    n = 8
    shape = (n, n, n)
    rng = np.random.default_rng(4)
    phi = 0.1 + 0.5 * rng.random(shape)
    cell = np.full(shape, synth.GRAY, np.uint8)
    cv = dict(pd=0.02, swr=0.15, phi_ref=0.35, f_max=3.5, f_min=0.575, thomeer_g=g)
    st = O.Oracle(O.make_params(shape), cell, phi, curves=[O.make_curve(**cv)]).static()
    for key, f in (("swirr", cv["f_max"]), ("sores", cv["f_min"])):
        sw = st[key] if key == "swirr" else 1.0 - st[key]
        x = f / st["lamL"]  # Pc_ref / Pe
        below = x <= 1.0
        assert np.all(sw[below] == 1.0)
        se = (sw[~below] - cv["swr"]) / (1 - cv["swr"])
        # 1 - Se is formed from Sw here, so cells just above entry, where the
        # non-wetting fraction is tiny, are checked only for being tiny
        ok = (1.0 - se) > 1e-5
        np.testing.assert_allclose(np.log10(x[~below][ok]) * np.log(1.0 - se[ok]), -g, rtol=1e-9)
        assert np.all(np.exp(-g / np.log10(x[~below][~ok])) <= 2e-5)
    assert np.any(st["sores"] == 0.0) and np.any(st["sores"] > 0.0)
    st2 = O.Oracle(O.make_params(shape), cell, phi, curves=[O.make_curve(**dict(cv, thomeer_g=2 * g))]).static()
    assert np.all(st2["swirr"] >= st["swirr"]) and np.any(st2["swirr"] > st["swirr"])


@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
def test_mass_sink_source_special_cases(lattice):
    """The mass-sink-source term moves mass from the non-wetting to the
    wetting component in rest equilibrium: from a uniform 50/50 mixture at
    rest (the middle of an interface, indicator 1) one step moves exactly m
    per cell, the total and the momentum stay unchanged; from the bulk state
    (rho_hi, rho_lo) (indicator 0) nothing moves."""
    shape = (1, 6, 7) if lattice == "d2q9" else (5, 6, 7)
    n = int(np.prod(shape))
    m = 3e-3
    for (rw, rn), moved in (((0.515, 0.515), m), ((1.0, 0.03), 0.0)):
        out = []
        for rate in (0.0, m):
            o = O.Oracle(O.make_params(shape, G=1.1, wet=1, mss=rate, lattice=lattice), np.zeros(shape, np.uint8))
            o.init_fields(np.full(shape, rn), np.full(shape, rw))
            o.step(1)
            out.append((o.observables(), o.populations()))
        (ob0, f0), (ob1, f1) = out
        # the post-collision populations carry it (the fields of the step do not yet)
        mass0, mass1 = f0.reshape(2, -1).sum(axis=1), f1.reshape(2, -1).sum(axis=1)
        assert abs((mass1[1] - mass0[1]) - n * moved) < 1e-12 * n
        assert abs((mass1[0] - mass0[0]) + n * moved) < 1e-12 * n
        # the added populations are the rest equilibrium: no momentum
        df = f1 - f0
        assert np.allclose(df.sum(axis=1)[1], moved, atol=1e-14) and np.allclose(df.sum(axis=1)[0], -moved, atol=1e-14)
        # every opposite pair gains the same amount (i odd and i + 1 are opposites in both sets)
        assert np.abs(df[:, 1::2] - df[:, 2::2]).max() < 1e-15
        if moved:  # in every cell the added populations are w_i dm: the lattice's weights as a multiset
            W = ([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12) if lattice == "d3q19" else ([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
            per_cell = df.reshape(2, df.shape[1], -1)
            for c in range(per_cell.shape[2]):
                np.testing.assert_allclose(np.sort(per_cell[1, :, c]) / moved, np.sort(W), rtol=1e-9)
                np.testing.assert_allclose(np.sort(-per_cell[0, :, c]) / moved, np.sort(W), rtol=1e-9)


def test_residual_hysteresis_switches():
    """Wet cells with s < s_lo take residual water; dry cells with s > s_hi take residual oil."""
    n = 8
    shape = (1, 1, n)
    cell = np.full(shape, synth.GRAY, np.uint8)
    phi = np.full(shape, 0.3)
    rw = np.array([0.03, 0.05, 0.5, 0.95, 0.99, 1.0, 0.3, 0.02])[None, None, :]
    rn = 1.03 - rw
    p = O.make_params(shape, wet=1)
    o = O.Oracle(p, cell, phi)
    o.init_fields(rn, rw)
    st = o.static()
    wet0 = np.array([1, 1, 1, 0, 0, 1, 0, 0])[None, None, :]
    o.set_residual(np.zeros(shape), np.zeros(shape), wet0)
    o.set_populations(rest_only_populations(rn, rw))
    o.step(1)
    Rw, Ro, wet = o.residual()
    s = np.clip((rw / 1.03 - 0.03 / 1.03) / (1.0 / 1.03 - 0.03 / 1.03), 0, 1)
    to_dry = (wet0 == 1) & (s < 0.1)
    to_wet = (wet0 == 0) & (s > 0.9)
    np.testing.assert_array_equal(wet, np.where(to_dry, 0, np.where(to_wet, 1, wet0)))
    np.testing.assert_array_equal(Rw, np.where(to_dry, st["swirr"], 0.0))
    np.testing.assert_array_equal(Ro, np.where(to_wet, st["sores"], 0.0))
    sw = o.fields()[3]
    np.testing.assert_allclose(sw, Rw + (1 - Rw - Ro) * s, rtol=1e-14)
    assert to_dry.sum() >= 2 and to_wet.sum() >= 2


# --------------------------------------------------------------------------
# Brute force: the C oracle against the independent NumPy evaluator
# --------------------------------------------------------------------------
def _bruteforce_case(seed, csf_everywhere, tau, pressure=False, thomeer=0.0, mss=0.0):
    rng = np.random.default_rng(seed)
    n = 8
    shape = (n, n, n)
    cell = np.zeros(shape, np.uint8)
    cell[rng.random(shape) < 0.12] = synth.SOLID
    cell[(rng.random(shape) < 0.35) & (cell == 0)] = synth.GRAY
    bc = {}
    if pressure:
        # an inlet plane and an outlet plane (with holes of solid) inside the periodic box
        cell[:, :, 0] = np.where(cell[:, :, 0] == synth.SOLID, synth.SOLID, synth.INLET)
        cell[:, :, 4] = np.where(cell[:, :, 4] == synth.SOLID, synth.SOLID, synth.OUTLET)
        bc = dict(rho_in=(0.08, 1.02), rho_out=(0.97, 0.05))
    phi = np.where(cell == synth.GRAY, 0.15 + 0.4 * rng.random(shape), 1.0)
    zz, yy, xx = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    blocks = ((xx // 4 + yy // 4 + zz // 4) % 2) == 0
    ra = np.where(blocks, 1.0, 0.03) + 0.05 * rng.random(shape)
    rb = 1.06 - ra
    u0 = 0.01 * rng.standard_normal((3,) + shape)
    common = dict(G=1.1, kappa=-0.045, tau=tau, accel=((1e-4, 2e-5, 0), (0, -1e-4, 3e-5)),
                  c_g=1.0, rho_wall=(0.7, 0.2), wet=1, csf_everywhere=csf_everywhere, mss=mss, **bc)
    curve = dict(kc_d=1.0, pd=0.02, swr=0.15, nw=3.0, nn=2.0, phi_ref=0.35, f_max=3.5,
                 f_min=0.575, aniso=10.0, thomeer_g=thomeer)
    o = O.Oracle(O.make_params(shape, **common), cell, phi, curves=[O.make_curve(lam=2.0, **curve)])
    pd = dict(common, rho_hi=1.0, rho_lo=0.03, phi_avg=(0.515, 0.515), phi_max=(1.0, 1.0),
              s_lo=0.1, s_hi=0.9, at_cut=0.95, eps_n=1e-4, kr_min=1e-6)
    nv = N.NaiveLBM(pd, cell, phi, curve={**curve, "lambda": 2.0})
    o.init_fields(ra, rb, u0)
    nv.init(ra, rb, u0)
    # flip the initial flags so that both transitions occur in the first step
    s = nv.s_of(rb, ra)
    wet0 = np.where(cell == synth.GRAY, s < 0.5, s >= 0.5)
    o.set_residual(np.zeros(shape), np.zeros(shape), wet0.astype(np.int32))
    nv.wet = wet0 & (cell != synth.SOLID)
    return o, nv, cell


@pytest.mark.parametrize("csf_everywhere,tau,pressure,thomeer,mss", [(0, (0.8, 1.3), False, 0.0, 0.0),
                                                                     (1, (1.0, 1.0), False, 0.0, 0.0),
                                                                     (0, (0.8, 1.3), True, 0.0, 0.0),
                                                                     (0, (0.8, 1.3), False, 0.35, 0.0),
                                                                     (0, (0.8, 1.3), True, 0.0, 2e-3)])
def test_bruteforce_against_numpy_evaluator(csf_everywhere, tau, pressure, thomeer, mss):
    o, nv, cell = _bruteforce_case(5, csf_everywhere, tau, pressure, thomeer, mss)
    st = o.static()
    np.testing.assert_allclose(np.moveaxis(st["kinv"], (0, 1), (-2, -1)), nv.geo["kinv"],
                               rtol=1e-12, atol=0)
    for k in range(10):
        o.step(1)
        nv.step()
        a, b, u, sw = o.fields()
        np.testing.assert_allclose(a, nv.rho[0], rtol=0, atol=1e-13)
        np.testing.assert_allclose(b, nv.rho[1], rtol=0, atol=1e-13)
        np.testing.assert_allclose(u, nv.u, rtol=0, atol=1e-14)
        np.testing.assert_allclose(sw, nv.sw, rtol=0, atol=1e-13)
        if k == 0:
            Rw, Ro, wet = o.residual()
            assert (Rw > 0).sum() > 0 and (Ro > 0).sum() > 0
            for t, name in ((O.TERM_SC, "sc"), (O.TERM_CSF, "csf"), (O.TERM_CAP, "cap"),
                            (O.TERM_DRAG, "drag"), (O.TERM_BODY, "body")):
                for comp in range(2):
                    np.testing.assert_allclose(o.force_term(t, comp), nv.terms[comp][name],
                                               rtol=0, atol=1e-15)
    np.testing.assert_allclose(o.populations(), nv.f, rtol=0, atol=1e-14)


@pytest.mark.parametrize("pressure", [False, True])
def test_observables_are_plain_sums(pressure):
    o, nv, cell = _bruteforce_case(9, 0, (1.0, 1.0), pressure)
    o.step(3)
    a, b, u, sw = o.fields()
    ob = o.observables(probe=(4, 4, 4, 2.5, 3.5))
    fl = cell != synth.SOLID
    assert abs(ob["mass"][0] - a[fl].sum()) < 1e-12
    phic = np.where(cell == synth.GRAY, o.static()["K0"] * 0 + nv.geo["phi"], 1.0)
    inner = fl & (cell != synth.INLET) & (cell != synth.OUTLET)  # saturation leaves reservoirs out
    assert abs(ob["sat"] - (phic * sw)[inner].sum() / phic[inner].sum()) < 1e-13
    assert abs(ob["flux_out"] - u[0, :, :, -1].sum() / 64) < 1e-15
    assert abs(ob["max_u"] - np.sqrt((u ** 2).sum(axis=0))[fl].max()) < 1e-15
    # the probe: mean mixture pressure within r_in of the centre minus the mean
    # beyond r_out, over fluid cells (the reservoirs included)
    zz, yy, xx = np.meshgrid(*(np.arange(k) for k in cell.shape), indexing="ij")
    r2 = (xx - 4) ** 2 + (yy - 4) ** 2 + (zz - 4) ** 2
    pr = (a + b) / 3.0 + o.params.G * a * b
    inside, outside = fl & (r2 < 2.5 ** 2), fl & (r2 > 3.5 ** 2)
    assert inside.any() and outside.any()
    assert abs(ob["dp"] - (pr[inside].mean() - pr[outside].mean())) < 1e-14


# --------------------------------------------------------------------------
# Eq. 4 against the relations of the paper's printed droplet results
# --------------------------------------------------------------------------
def _golden(name):
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].split()
        if line:
            rows[(line[0], float(line[1]))] = float(line[2])
    return rows


def test_csf_lowers_surface_tension_like_sec3a():
    """tests/golden/csf_droplet_sec3a.txt (Sec. III.A): a negative kappa lowers
    sigma (the paper: by a factor of 35 at kappa = -0.045) while the spurious
    velocity changes by well under a few percent (the paper: 0.3 %).  The
    oracle's 2-D droplet (R = 14 on 64^2, G = 1.1) must show sigma decreasing
    monotonically with kappa, by more than a factor of 2 at kappa = -0.045,
    with max|u| within 5 % and the 10-90 % interface width unchanged."""
    gold = _golden("csf_droplet_sec3a.txt")
    assert gold[("sigma", -0.045)] < gold[("sigma", 0.0)]
    assert abs(gold[("max_ux", -0.045)] / gold[("max_ux", 0.0)] - 1) < 0.05
    n, R = 64, 14.0
    shape = (1, n, n)
    sig, umax, width = [], [], []
    for kappa in (0.0, -0.02, -0.045):
        rA, rB = synth.cylinder_droplet_fields(shape, R, (32, 32), 1.0, 0.03)
        o = O.Oracle(O.make_params(shape, G=1.1, kappa=kappa, csf_everywhere=1), np.zeros(shape, np.uint8))
        o.init_fields(rA, rB)
        o.step(3000)
        a = o.fields()[0]
        rad = np.sqrt((a.sum() - a.min() * a.size) / (a.max() - a.min()) / np.pi)
        ob = o.observables(probe=(32, 32, 0, R - 4, R + 4))
        sig.append(ob["dp"] * rad)
        umax.append(ob["max_u"])
        f = (a[0, 32, 32:] - a.min()) / (a.max() - a.min())
        width.append(int(np.argmax(f < 0.1) - np.argmax(f < 0.9)))
    assert sig[0] > sig[1] > sig[2] > 0
    assert sig[2] < 0.5 * sig[0]
    assert max(abs(u / umax[0] - 1) for u in umax) < 0.05
    assert max(width) - min(width) <= 1


# --------------------------------------------------------------------------
# How much the Eq. 4 reading moves the results: the unit-normal floor eps_n
# and the discretisation of the divergence of the unit normal
# --------------------------------------------------------------------------
EQ4_READINGS = [("identity", 1e-8), ("identity", 1e-4), ("neighbour_normals", 1e-8), ("neighbour_normals", 1e-4)]


def _cylinder_csf(div, eps):
    n, R, w = 128, 40.0, 8.0
    shape = (1, n, n)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cx = cy = n / 2 - 0.5
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    rhoB = (0.5 + 0.45 * np.tanh((r - R) / w))[None]
    rhoA = (0.6 - 0.2 * np.tanh((r - R) / w))[None]
    kappa = -0.045
    p = O.make_params(shape, kappa=kappa, csf_everywhere=1, phi_avg=(0.515, 0.515), phi_max=(1.0, 1.0),
                      eps_n=eps, csf_div=div)
    o = _rest_state(p, np.zeros(shape, np.uint8), rhoA, rhoB)
    F = o.force_term(O.TERM_CSF, 0)[:2, 0]
    Fr = (F * np.stack([(x - cx) / r, (y - cy) / r])).sum(axis=0)
    cont = kappa * (-1.0 / r) * (0.45 / w / np.cosh((r - R) / w) ** 2 / 0.515) * rhoA[0]
    band = np.abs(r - R) < 1.0
    return F, float((np.abs(Fr[band] - cont[band]) / np.abs(cont[band])).max())


def test_eq4_cylinder_under_both_floors_and_discretisations():
    """Eq. 4 leaves the divergence of the unit normal undiscretised and its
    unit normal unregularised.  The two discretisations (the curvature
    identity tr(H)/s - g.H.g/s^3 of the cell's own neighbourhood, and the
    isotropic divergence of the neighbours' unit normals g/max(|g|, eps)) and
    the two floors (eps_n = 1e-8 and 1e-4 rho_hi) all give the continuum
    force on a smooth cylindrical interface, kappa (-1/r) (d rho^B/dr /
    phi_avg) rho^A / phi_max, within 1 % at the interface (measured: 0.79 %
    identity, 0.52 % neighbour normals, equal for both floors).  Across the
    whole field the floor moves the force by at most 2.3 % of its maximum
    (identity) and 1.1 % (neighbour normals)."""
    F = {}
    for div, eps in EQ4_READINGS:
        F[(div, eps)], err = _cylinder_csf(div, eps)
        assert err < 0.01, (div, eps, err)
    for div in ("identity", "neighbour_normals"):
        a, b = F[(div, 1e-8)], F[(div, 1e-4)]
        assert np.abs(a - b).max() < 0.03 * np.abs(a).max(), div


def test_eq4_droplet_relations_under_both_floors_and_discretisations():
    """The Sec. III.A relations (tests/golden/csf_droplet_sec3a.txt) under the
    four readings of Eq. 4: the 2-D droplet of R = 14 on 64^2 (G = 1.1, 3000
    steps) at kappa = -0.045 against kappa = 0.  Measured: sigma(-0.045) /
    sigma(0) = 0.1734 / 0.1736 (identity, eps_n 1e-8 / 1e-4) and 0.1608 /
    0.1603 (neighbour normals); max|u| ratio 0.993 / 0.994 and 0.981 / 0.981;
    10-90 % width 4 cells in every run.  So the floor moves sigma by 0.1 %
    and max|u| by 0.1 % under either discretisation; the discretisation moves
    sigma by 7.5 % and max|u| by 1.2 %, with the same qualitative result (a
    six-fold drop of sigma, spurious currents within 2 %)."""
    n, R = 64, 14.0
    shape = (1, n, n)

    def run(kappa, div="identity", eps=1e-4):
        rA, rB = synth.cylinder_droplet_fields(shape, R, (32, 32), 1.0, 0.03)
        o = O.Oracle(O.make_params(shape, G=1.1, kappa=kappa, csf_everywhere=1, eps_n=eps, csf_div=div),
                     np.zeros(shape, np.uint8))
        o.init_fields(rA, rB)
        o.step(3000)
        a = o.fields()[0]
        rad = np.sqrt((a.sum() - a.min() * a.size) / (a.max() - a.min()) / np.pi)
        ob = o.observables(probe=(32, 32, 0, R - 4, R + 4))
        f = (a[0, 32, 32:] - a.min()) / (a.max() - a.min())
        return ob["dp"] * rad, ob["max_u"], int(np.argmax(f < 0.1) - np.argmax(f < 0.9))

    s0, u0, w0 = run(0.0)
    got = {k: run(-0.045, *k) for k in EQ4_READINGS}
    ratio = {k: (v[0] / s0, v[1] / u0) for k, v in got.items()}
    for k, (sr, ur) in ratio.items():
        assert 0.12 < sr < 0.22 and abs(ur - 1) < 0.025, (k, sr, ur)
        assert got[k][2] == w0, k
    for div in ("identity", "neighbour_normals"):
        (sa, ua), (sb, ub) = ratio[(div, 1e-8)], ratio[(div, 1e-4)]
        assert abs(sa / sb - 1) < 0.005 and abs(ua / ub - 1) < 0.002, div
    (si, ui), (sn, un) = ratio[("identity", 1e-8)], ratio[("neighbour_normals", 1e-8)]
    assert abs(si / sn - 1) < 0.10 and abs(ui / un - 1) < 0.02
