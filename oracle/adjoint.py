"""FP64 PyTorch statement of the step and its discrete adjoint.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests use it to
check the library's hand-written adjoint; the library never imports it.

The forward map is the same time step as ``lbm_oracle.c`` (pull streaming with
halfway bounce-back at solid cells, moments, residual hysteresis, Shan-Chen,
Eq. 4 curvature force, Eq. 1 capillary and tensorial viscous forces with the
semi-implicit velocity, regularised collision with the Eq. 3 force term),
written over whole periodic arrays with ``torch.roll``; the tests pin it to
the C oracle to round-off.  The porosity enters through the geometry
precompute (Eqs. 5-7): Kozeny-Carman K0, the Leverett factor, the residual
amounts and the principal axis e1 of M = H H + c_g grad(phi) grad(phi)^T.
The discrete adjoint is reverse-mode differentiation of this forward map by
``torch.autograd`` (a library primitive used as one step), except for the
top eigenvector, whose derivative is the perturbation formula
d e1 = sum_{k != 1} e_k (e_k^T dM e1) / (mu1 - mu_k), which stays finite
when the two smaller eigenvalues coincide.  Piecewise-constant parts (the
residual hysteresis, the H(At) cut-off, clamps and floors) contribute their
active branch only.

Loss (outlet flux and saturation mismatch):
    L = (q - q*)^2 / q*^2 + (S - S*)^2,
    q = mean of u_x over the plane x = nx - 1 (solid cells count 0),
    S = sum(phi_c Sw) / sum(phi_c) over non-solid cells (phi_c = 1 in pores).
"""
from __future__ import annotations

import numpy as np
import torch

PORE, SOLID, GRAY = 0, 1, 2
_V = [(0, 0, 0)]
for _d in range(3):
    for _s in (1, -1):
        _v = [0, 0, 0]
        _v[_d] = _s
        _V.append(tuple(_v))
for (_a, _b) in ((0, 1), (0, 2), (1, 2)):
    for (_sa, _sb) in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
        _v = [0, 0, 0]
        _v[_a], _v[_b] = _sa, _sb
        _V.append(tuple(_v))
VEL = _V                                              # c_i as (cx, cy, cz)
WGT = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
OPP = [VEL.index(tuple(-x for x in c)) for c in VEL]
CS2 = 1.0 / 3.0


def _to(f, c):
    """Value at x + c (periodic); arrays end in [z, y, x]."""
    return torch.roll(f, shifts=(-c[2], -c[1], -c[0]), dims=(-3, -2, -1))


def _from(f, c):
    """Value at x - c (periodic)."""
    return torch.roll(f, shifts=(c[2], c[1], c[0]), dims=(-3, -2, -1))


def iso_grad(field):
    """(1/cs^2) sum_i w_i field(x + c_i) c_i as [3, z, y, x]; summed as central
    differences over the opposite pairs, so a flat field gives exactly 0."""
    comps = [torch.zeros_like(field) for _ in range(3)]
    for i in range(1, 19):
        if OPP[i] < i:
            continue
        sh = _to(field, VEL[i]) - _to(field, [-x for x in VEL[i]])
        for d in range(3):
            if VEL[i][d]:
                comps[d] = comps[d] + WGT[i] * VEL[i][d] * sh / CS2
    return torch.stack(comps)


def moment_hessian(seen, center):
    """(1/cs^4) sum_i w_i (c_i c_i - cs^2 I)(seen(x + c_i) - center(x)), [3, 3, z, y, x]."""
    H = [[torch.zeros_like(seen) for _ in range(3)] for _ in range(3)]
    for i in range(1, 19):
        c = VEL[i]
        diff = _to(seen, c) - center
        for a in range(3):
            for b in range(3):
                q = c[a] * c[b] - (CS2 if a == b else 0.0)
                if q != 0.0:
                    H[a][b] = H[a][b] + WGT[i] * q * diff / (CS2 * CS2)
    return torch.stack([torch.stack(r) for r in H])


class TopEigvec(torch.autograd.Function):
    """Top eigenvector of symmetric 3x3 matrices [..., 3, 3] (ties need not
    be excluded: tied cells are masked by the caller)."""

    @staticmethod
    def forward(ctx, M):
        w, V = torch.linalg.eigh(M)
        ctx.save_for_backward(w, V)
        return V[..., :, 2]

    @staticmethod
    def backward(ctx, g):
        w, V = ctx.saved_tensors
        e1 = V[..., :, 2]
        lam = torch.zeros_like(V)
        for k in (0, 1):
            ek = V[..., :, k]
            gap = w[..., 2] - w[..., k]
            ck = torch.where(gap > 0, (g * ek).sum(-1) / torch.where(gap > 0, gap, torch.ones_like(gap)),
                             torch.zeros_like(gap))
            outer = ek[..., :, None] * e1[..., None, :]
            lam = lam + ck[..., None, None] * 0.5 * (outer + outer.transpose(-1, -2))
        return lam


def _kc(d, phi):
    return d * d * phi ** 3 / (180.0 * (1.0 - phi) ** 2)


def geometry(cell, phi_gray, curve, c_g):
    """Gray-cell constants as differentiable functions of phi (gray cells).

    Returns K^-1 [z, y, x, 3, 3], the Leverett capillary scale lamL*pd and the
    residual amounts Sw_irr, So_res (zero outside gray cells)."""
    gray = torch.as_tensor(cell == GRAY)
    pore = torch.as_tensor(cell == PORE)
    phi = torch.where(gray, phi_gray, torch.where(pore, torch.ones_like(phi_gray), torch.zeros_like(phi_gray)))
    g = iso_grad(phi)
    Hr = [[None] * 3 for _ in range(3)]
    for a in range(3):
        ea = [0, 0, 0]
        ea[a] = 1
        ma = [-x for x in ea]
        Hr[a][a] = _to(phi, ea) - 2 * phi + _to(phi, ma)
        for b in range(a + 1, 3):
            eb = [0, 0, 0]
            eb[b] = 1
            pp = [ea[k] + eb[k] for k in range(3)]
            pm = [ea[k] - eb[k] for k in range(3)]
            mp = [eb[k] - ea[k] for k in range(3)]
            mm = [-ea[k] - eb[k] for k in range(3)]
            Hr[a][b] = Hr[b][a] = 0.25 * (_to(phi, pp) - _to(phi, pm) - _to(phi, mp) + _to(phi, mm))
    H = torch.stack([torch.stack(r, -1) for r in Hr], -2)          # [z, y, x, 3, 3]
    gc = torch.stack(list(g), -1)                                   # [z, y, x, 3]
    M = H @ H + c_g * gc[..., :, None] * gc[..., None, :]
    w = torch.linalg.eigvalsh(M.detach())
    mu1, mu2 = w[..., 2], w[..., 1]
    iso = ((mu1 - mu2) <= 1e-12 * torch.clamp(mu1, min=1e-30)) | ~gray
    safe = torch.where(iso[..., None, None], torch.diag(torch.tensor([0.0, 1.0, 2.0], dtype=M.dtype)), M)
    e1 = TopEigvec.apply(safe)
    outer = torch.where(iso[..., None, None], torch.zeros_like(safe), e1[..., :, None] * e1[..., None, :])
    phis = torch.where(gray, phi, torch.full_like(phi, 0.5))
    K0 = _kc(curve["kc_d"], phis)
    kinv = (torch.eye(3, dtype=phi.dtype) + (curve["aniso"] - 1.0) * outer) / K0[..., None, None]
    kinv = torch.where(gray[..., None, None], kinv, torch.zeros_like(kinv))
    kref = _kc(curve["kc_d"], curve["phi_ref"])
    lamL = torch.sqrt((kref / curve["phi_ref"]) / (K0 / phis))

    def sw_at(f):
        x = f / lamL
        if curve.get("thomeer_g", 0.0) > 0.0:
            # Thomeer: log10(x) ln(1 - Se) = -G above entry (x > 1), Se = 1 below
            xs = torch.where(x > 1.0, x, torch.full_like(x, 2.0))
            se = torch.where(x > 1.0, -torch.expm1(-curve["thomeer_g"] / torch.log10(xs)), torch.ones_like(x))
        else:
            se = torch.clamp(x ** (-curve["lam"]), max=1.0)
        return curve["swr"] + (1 - curve["swr"]) * se

    z = lambda v: torch.where(gray, v, torch.zeros_like(v))
    return dict(kinv=kinv, pcs=z(lamL * curve["pd"]), swirr=z(sw_at(curve["f_max"])),
                sores=z(1.0 - sw_at(curve["f_min"])), phi=phi)


def _equilibrium(rho, u):
    uu = (u * u).sum(0)
    out = []
    for i in range(19):
        c = VEL[i]
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        out.append(WGT[i] * rho * (1 + cu / CS2 + (cu * cu - CS2 * uu) / (2 * CS2 * CS2)))
    return torch.stack(out)


def _collide(fs, u, F, tau):
    rho = fs.sum(0)
    fne = fs - _equilibrium(rho, u)
    P = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            P[a][b] = sum(VEL[i][a] * VEL[i][b] * fne[i] for i in range(19) if VEL[i][a] * VEL[i][b] != 0) \
                + 0.5 * (u[a] * F[b] + F[a] * u[b])
    feq = _equilibrium(rho, u)
    out = []
    uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2]
    for i in range(19):
        c = VEL[i]
        QP = sum((c[a] * c[b] - (CS2 if a == b else 0.0)) * P[a][b] for a in range(3) for b in range(3))
        cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2]
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        Fi = WGT[i] * (cF / CS2 + (2 * cu * cF - 2 * CS2 * uF) / (2 * CS2 * CS2))
        out.append(feq[i] + (1 - 1 / tau) * WGT[i] * QP / (2 * CS2 * CS2) + 0.5 * Fi)
    return torch.stack(out)


class Model:
    """Fully periodic lattice (walls as solid cells), one constitutive curve."""

    def __init__(self, settings: dict, cell, curve: dict):
        self.p = dict(settings)
        self.cell = np.asarray(cell, np.uint8)
        self.solid = torch.as_tensor(self.cell == SOLID)
        self.gray = torch.as_tensor(self.cell == GRAY)
        self.curve = dict(curve)

    def s_of(self, rw, rn):
        p = self.p
        r_lo = p["rho_lo"] / (p["rho_hi"] + p["rho_lo"])
        r_hi = p["rho_hi"] / (p["rho_hi"] + p["rho_lo"])
        return torch.clamp((rw / (rw + rn) - r_lo) / (r_hi - r_lo), 0.0, 1.0)

    def init(self, rhoA, rhoB, u=None):
        shape = self.cell.shape
        u = torch.zeros((3,) + shape, dtype=torch.float64) if u is None else torch.as_tensor(u, dtype=torch.float64)
        u = torch.where(self.solid[None], torch.zeros_like(u), u)
        rho = [torch.as_tensor(rhoA, dtype=torch.float64), torch.as_tensor(rhoB, dtype=torch.float64)]
        f = torch.stack([torch.where(self.solid[None], torch.zeros(1, dtype=torch.float64), _equilibrium(r, u))
                         for r in rho])
        w = self.p["wet"]
        s = self.s_of(rho[w], rho[1 - w])
        wet = torch.where(self.solid, torch.zeros_like(s, dtype=torch.bool), s >= 0.5)
        z = torch.zeros(shape, dtype=torch.float64)
        return dict(f=f, wet=wet, Rw=z, Ro=z)

    def step(self, st, geo):
        p, cv = self.p, self.curve
        f = st["f"]
        solid, gray = self.solid, self.gray
        fs = []
        for i in range(19):
            wall_src = _from(solid, VEL[i])
            fs.append(torch.where(wall_src[None], f[:, OPP[i]], _from(f[:, i], VEL[i])))
        fs = torch.stack(fs, 1)
        fs = torch.where(solid[None, None], torch.zeros_like(fs), fs)
        rho = fs.sum(1)
        j = torch.stack([sum(VEL[i][d] * (fs[0, i] + fs[1, i]) for i in range(19) if VEL[i][d]) for d in range(3)])
        w = p["wet"]
        one = torch.ones_like(rho[0])
        rt = torch.where(solid, one, rho[0] + rho[1])
        s = self.s_of(rho[w], torch.where(solid, one, rho[1 - w]))
        to_dry = gray & st["wet"] & (s < p["s_lo"])
        to_wet = gray & ~st["wet"] & (s > p["s_hi"])
        Rw = torch.where(to_dry, geo["swirr"], torch.where(to_wet, torch.zeros_like(s), st["Rw"]))
        Ro = torch.where(to_wet, geo["sores"], torch.where(to_dry, torch.zeros_like(s), st["Ro"]))
        wet = torch.where(to_dry, torch.zeros_like(st["wet"]), torch.where(to_wet, torch.ones_like(st["wet"]),
                                                                           st["wet"]))
        sw = torch.where(gray, Rw + (1 - Rw - Ro) * s, s)
        seen = [torch.where(solid, torch.full_like(rho[a], p["rho_wall"][a]), rho[a]) for a in range(2)]
        grad = [iso_grad(seen[1 - a]) for a in range(2)]
        Fo = torch.zeros_like(j)
        parts = []
        for a in range(2):
            sc = -p["G"] * rho[a][None] * grad[a]
            body = rho[a][None] * torch.tensor(p["accel"][a], dtype=torch.float64)[:, None, None, None]
            csf = torch.zeros_like(sc)
            if p["kappa"] != 0.0:
                H = moment_hessian(seen[1 - a], rho[1 - a])
                g = grad[a]
                sn = torch.sqrt((g ** 2).sum(0) + p["eps_n"] ** 2)
                gHg = torch.einsum("a...,ab...,b...->...", g, H, g)
                div = (H[0, 0] + H[1, 1] + H[2, 2]) / sn - gHg / sn ** 3
                mask = torch.ones_like(gray) if p["csf_everywhere"] else gray
                csf = torch.where(mask[None], p["kappa"] * (-div)[None] * (grad[a] / p["phi_avg"][a])
                                  * (rho[a] / p["phi_max"][a])[None], torch.zeros_like(sc))
            parts.append(sc + body + csf)
        den = seen[w] + seen[1 - w]
        At = torch.where(den > 0, (seen[w] - seen[1 - w]) / torch.where(den > 0, den, torch.ones_like(den)),
                         torch.zeros_like(den))
        dAt = iso_grad(At)
        mag = torch.sqrt((dAt ** 2).sum(0))
        Hc = torch.where(torch.abs(At) <= p["at_cut"], 0.5 * mag, torch.zeros_like(mag))
        se_c = torch.clamp((sw - cv["swr"]) / (1 - cv["swr"]), 1e-2, 1.0)
        if cv.get("thomeer_g", 0.0) > 0.0:
            # Thomeer: Pc = Pe 10^min(-G / ln(1 - Se), 1)
            open_ = se_c < 1.0
            ss = torch.where(open_, se_c, torch.full_like(se_c, 0.5))
            ex = torch.where(open_, cv["thomeer_g"] / -torch.log1p(-ss), torch.zeros_like(se_c))
            Pc = geo["pcs"] * torch.pow(10.0, torch.clamp(ex, max=1.0))
        else:
            Pc = geo["pcs"] * se_c ** (-1.0 / cv["lam"])
        nvec = dAt / torch.clamp(mag, min=p["eps_n"])
        for a in range(2):
            cap = -Pc[None] * (rho[a] / rt)[None] * nvec * Hc[None]
            parts[a] = parts[a] + torch.where((gray & (Hc > 0))[None], cap, torch.zeros_like(cap))
            Fo = Fo + parts[a]
        se_k = torch.clamp((sw - cv["swr"]) / (1 - cv["swr"]), 0.0, 1.0)
        kr = [None, None]
        kr[w] = se_k ** cv["nw"]
        kr[1 - w] = (1 - se_k) ** cv["nn"]
        coef = sum(rho[b] * ((p["tau"][b] - 0.5) / 3.0) / torch.clamp(kr[b], min=p["kr_min"]) for b in range(2))
        R = coef[..., None, None] * geo["kinv"]
        eye = torch.eye(3, dtype=torch.float64)
        A = rt[..., None, None] * eye + 0.5 * R
        rhs = torch.stack(list(j + 0.5 * Fo), -1)
        gmask = gray[..., None, None]
        ug = torch.linalg.solve(torch.where(gmask, A, eye.expand_as(A)),
                                torch.where(gray[..., None], rhs, torch.zeros_like(rhs))[..., None])[..., 0]
        ug = torch.stack([ug[..., d] for d in range(3)])
        un = (j + 0.5 * Fo) / rt[None]
        u = torch.where(gray[None], ug, un)
        u = torch.where(solid[None], torch.zeros_like(u), u)
        Ru = torch.einsum("...ab,b...->a...", R, u)
        F = [parts[a] + torch.where(gray[None], -(rho[a] / rt)[None] * Ru, torch.zeros_like(Ru)) for a in range(2)]
        fnew = torch.stack([_collide(fs[a], u, F[a], p["tau"][a]) for a in range(2)])
        fnew = torch.where(solid[None, None], torch.zeros_like(fnew), fnew)
        return dict(f=fnew, wet=wet, Rw=Rw, Ro=Ro), dict(rho=rho, u=u, sw=sw)


def run(settings, cell, curve, phi_gray, rhoA, rhoB, steps, u0=None):
    """Forward run; returns the model, final state and the last step's fields."""
    m = Model(settings, cell, curve)
    geo = geometry(m.cell, phi_gray, curve, settings["c_g"])
    st = m.init(rhoA, rhoB, u0)
    out = None
    for _ in range(steps):
        st, out = m.step(st, geo)
    return m, st, out, geo


def loss_of(cell, geo, out, q_target, s_target):
    """L, q, S of the last step's fields."""
    nz, ny, nx = cell.shape
    solid = torch.as_tensor(cell == SOLID)
    q = torch.where(solid[:, :, nx - 1], torch.zeros_like(out["u"][0, :, :, nx - 1]), out["u"][0, :, :, nx - 1]).sum() \
        / (ny * nz)
    phic = torch.where(solid, torch.zeros_like(geo["phi"]), geo["phi"])
    S = (phic * out["sw"]).sum() / phic.sum()
    L = (q - q_target) ** 2 / q_target ** 2 + (S - s_target) ** 2
    return L, q, S


def loss_and_gradient(settings, cell, curve, phi, rhoA, rhoB, steps, q_target, s_target, u0=None):
    """(L, q, S, dL/dphi) with dL/dphi zero outside gray cells (FP64)."""
    ph = torch.tensor(np.asarray(phi, np.float64), requires_grad=True)
    m, st, out, geo = run(settings, cell, curve, ph, rhoA, rhoB, steps, u0)
    L, q, S = loss_of(m.cell, geo, out, q_target, s_target)
    L.backward()
    g = ph.grad.detach().numpy().copy()
    g[np.asarray(cell) != GRAY] = 0.0
    return float(L.detach()), float(q.detach()), float(S.detach()), g


def loss_only(settings, cell, curve, phi, rhoA, rhoB, steps, q_target, s_target, u0=None):
    with torch.no_grad():
        ph = torch.tensor(np.asarray(phi, np.float64))
        m, st, out, geo = run(settings, cell, curve, ph, rhoA, rhoB, steps, u0)
        L, q, S = loss_of(m.cell, geo, out, q_target, s_target)
    return float(L), float(q), float(S), out
