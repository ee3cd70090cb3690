"""Whole-array NumPy evaluator of the same LB step, used to pin the C oracle.

This is a second, independent statement of the step (whole-array shifts with
``np.roll`` instead of the oracle's per-cell neighbour loops, ``numpy.linalg``
for the 3x3 eigenproblem and the linear solve instead of the oracle's Jacobi
rotations and Gaussian elimination).  The brute-force tests run both on tiny
periodic grids with every branch active and require agreement to round-off,
so an indexing, sign or transposition slip in either shows up.  The dtype is
a parameter, which also lets the tests estimate how FP32 rounding alone moves
the results.

Equations: Eq. 2-3 (LB equation, force term), Eq. 4 (CSF), Eq. 1 (capillary
and viscous multiscale force), Eq. 5 and Fig. 6 (Leverett scaling, residual
components), Eq. 6-7 (tensorial resistivity), and the reservoir reading of
the pressure boundaries of the imbibition set-ups (Sec. I, Appendix); see the
oracle's header for the readings of the points the paper leaves open.
"""
from __future__ import annotations

import numpy as np

PORE, SOLID, GRAY, INLET, OUTLET = 0, 1, 2, 3, 4

_VEL = [(0, 0, 0)]
for d in range(3):
    for s in (1, -1):
        v = [0, 0, 0]
        v[d] = s
        _VEL.append(tuple(v))
for (a, b) in ((0, 1), (0, 2), (1, 2)):
    for (sa, sb) in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
        v = [0, 0, 0]
        v[a], v[b] = sa, sb
        _VEL.append(tuple(v))
VEL = np.array(_VEL, dtype=np.int64)             # (19, 3) as (cx, cy, cz)
WGT = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
OPP = np.array([int(np.nonzero((VEL == -VEL[i]).all(axis=1))[0][0]) for i in range(19)])
CS2 = 1.0 / 3.0


def shift_from(field, c):
    """Value at x - c for every x (periodic); arrays are [..., z, y, x]."""
    return np.roll(field, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(-3, -2, -1))


def shift_to(field, c):
    """Value at x + c for every x (periodic)."""
    return np.roll(field, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(-3, -2, -1))


def iso_grad(field):
    """(1/cs^2) sum_i w_i field(x + c_i) c_i, returned as [3][z][y][x]; summed
    as central differences over the opposite pairs, so a flat field gives 0."""
    out = np.zeros((3,) + field.shape, dtype=field.dtype)
    for i in range(1, 19):
        if OPP[i] < i:
            continue
        sh = shift_to(field, VEL[i]) - shift_to(field, -VEL[i])
        for d in range(3):
            if VEL[i][d]:
                out[d] += WGT[i] * VEL[i][d] * sh / CS2
    return out


def moment_hessian(field_seen, field_center):
    """(1/cs^4) sum_i w_i (c_i c_i - cs^2 I)(field(x + c_i) - field(x))."""
    H = np.zeros((3, 3) + field_seen.shape, dtype=field_seen.dtype)
    for i in range(1, 19):
        c = VEL[i]
        diff = shift_to(field_seen, c) - field_center
        for a in range(3):
            for b in range(3):
                q = c[a] * c[b] - (CS2 if a == b else 0.0)
                if q != 0.0:
                    H[a, b] += WGT[i] * q * diff / (CS2 * CS2)
    return H


def kozeny_carman(d, phi):
    return d * d * phi ** 3 / (180.0 * (1.0 - phi) ** 2)


def geometry(cell, phi_in, curve, c_g=1.0):
    """Gray-cell constants: K^-1 (3x3 per cell), Leverett factor, residual bounds."""
    phi = np.where(cell == SOLID, 0.0, np.where(cell == GRAY, phi_in, 1.0)).astype(np.float64)
    g = iso_grad(phi)
    H = np.zeros((3, 3) + phi.shape)
    for a in range(3):
        ea = np.zeros(3, int)
        ea[a] = 1
        H[a, a] = shift_to(phi, ea) - 2 * phi + shift_to(phi, -ea)
        for b in range(a + 1, 3):
            eb = np.zeros(3, int)
            eb[b] = 1
            v = 0.25 * (shift_to(phi, ea + eb) - shift_to(phi, ea - eb)
                        - shift_to(phi, -ea + eb) + shift_to(phi, -ea - eb))
            H[a, b] = H[b, a] = v
    Hc = np.moveaxis(H, (0, 1), (-2, -1))
    gc = np.moveaxis(g, 0, -1)
    M = Hc @ Hc + c_g * gc[..., :, None] * gc[..., None, :]
    w, V = np.linalg.eigh(M)
    mu1, mu2 = w[..., 2], w[..., 1]
    e1 = V[..., :, 2]
    iso = (mu1 - mu2) <= 1e-12 * np.maximum(mu1, 1e-30)
    kd = curve["kc_d"]
    gray = cell == GRAY
    phis = np.where(gray, phi, 0.5)
    K0 = kozeny_carman(kd, phis)
    a1 = curve["aniso"] - 1.0
    eye = np.eye(3)
    outer = e1[..., :, None] * e1[..., None, :]
    kinv = (eye + np.where(iso[..., None, None], 0.0, a1 * outer)) / K0[..., None, None]
    kref = kozeny_carman(kd, curve["phi_ref"])
    lamL = np.sqrt((kref / curve["phi_ref"]) / (K0 / phis))

    def sw_at(p):
        x = p / (lamL * curve["pd"])
        if curve.get("thomeer_g", 0.0) > 0.0:
            # Thomeer hyperbola: log10(x) ln(non-wetting fraction) = -G
            se = np.where(x > 1.0, -np.expm1(-curve["thomeer_g"] / np.log10(np.where(x > 1.0, x, 2.0))), 1.0)
        else:
            se = np.minimum(x ** (-curve["lambda"]), 1.0)
        return curve["swr"] + (1 - curve["swr"]) * se

    swirr = sw_at(curve["f_max"] * curve["pd"])
    sores = 1.0 - sw_at(curve["f_min"] * curve["pd"])
    z = lambda v: np.where(gray, v, 0.0)
    kinv = np.where(gray[..., None, None], kinv, 0.0)
    return dict(kinv=kinv, K0=z(K0), lamL=z(lamL), swirr=z(swirr), sores=z(sores), phi=phi, iso=iso & gray)


def equilibrium(rho, u):
    uu = (u * u).sum(axis=0)
    out = []
    for i in range(19):
        cu = VEL[i, 0] * u[0] + VEL[i, 1] * u[1] + VEL[i, 2] * u[2]
        out.append(WGT[i] * rho * (1 + cu / CS2 + (cu * cu - CS2 * uu) / (2 * CS2 * CS2)))
    return np.stack(out)


def collide(fs, u, F, tau):
    rho = fs.sum(axis=0)
    feq = equilibrium(rho, u)
    fne = fs - feq
    P = np.zeros((3, 3) + rho.shape, dtype=fs.dtype)
    for a in range(3):
        for b in range(3):
            P[a, b] = np.tensordot(VEL[:, a] * VEL[:, b], fne, axes=(0, 0)) + 0.5 * (u[a] * F[b] + F[a] * u[b])
    out = np.empty_like(fs)
    for i in range(19):
        c = VEL[i]
        QP = sum((c[a] * c[b] - (CS2 if a == b else 0.0)) * P[a, b] for a in range(3) for b in range(3))
        cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2]
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2]
        Fi = WGT[i] * (cF / CS2 + (2 * cu * cF - 2 * CS2 * uF) / (2 * CS2 * CS2))
        out[i] = feq[i] + (1 - 1 / tau) * WGT[i] * QP / (2 * CS2 * CS2) + 0.5 * Fi
    return out


class NaiveLBM:
    """State and step on a fully periodic grid (walls only as solid cells)."""

    def __init__(self, p: dict, cell, phi=None, curve=None, dtype=np.float64):
        self.p = p
        self.dt = dtype
        self.cell = np.asarray(cell, dtype=np.uint8)
        self.solid = self.cell == SOLID
        self.gray = self.cell == GRAY
        self.pres = (self.cell == INLET) | (self.cell == OUTLET)
        curve = curve or dict(kc_d=1.0, pd=0.02, **{"lambda": 2.0}, swr=0.15, nw=3.0, nn=2.0,
                              phi_ref=0.35, f_max=3.5, f_min=0.575, aniso=1.0)
        self.curve = curve
        self.geo = geometry(self.cell, np.ones(self.cell.shape) if phi is None else phi, curve, p["c_g"])
        self.kinv = self.geo["kinv"].astype(dtype)

    def s_of(self, rw, rn):
        p = self.p
        r_lo = p["rho_lo"] / (p["rho_hi"] + p["rho_lo"])
        r_hi = p["rho_hi"] / (p["rho_hi"] + p["rho_lo"])
        return np.clip((rw / (rw + rn) - r_lo) / (r_hi - r_lo), 0.0, 1.0)

    def init(self, rhoA, rhoB, u=None):
        dt = self.dt
        u = np.zeros((3,) + self.cell.shape) if u is None else np.asarray(u)
        u = np.where(self.solid[None], 0.0, u).astype(dt)
        rho = [np.asarray(rhoA, dt), np.asarray(rhoB, dt)]
        self.f = np.stack([np.where(self.solid[None], 0.0, equilibrium(r, u)) for r in rho]).astype(dt)
        w = self.p["wet"]
        s = self.s_of(rho[w], rho[1 - w])
        self.wet = np.where(self.solid, False, s >= 0.5)
        self.Rw = np.zeros(self.cell.shape, dt)
        self.Ro = np.zeros(self.cell.shape, dt)

    def step(self):
        p, dt = self.p, self.dt
        f = self.f
        fs = np.empty_like(f)
        for i in range(19):
            wall_src = shift_from(self.solid, VEL[i])
            fs[:, i] = np.where(wall_src[None], f[:, OPP[i]], shift_from(f[:, i], VEL[i]))
        fs = np.where(self.solid[None, None], 0.0, fs)
        rho = fs.sum(axis=1)
        j = np.tensordot(VEL.T.astype(dt), fs.sum(axis=0), axes=(1, 0))
        # reservoirs: the held densities, no momentum
        held = np.stack([np.where(self.cell == INLET, p.get("rho_in", (0, 0))[a], p.get("rho_out", (0, 0))[a])
                         for a in range(2)]).astype(dt)
        rho = np.where(self.pres[None], held, rho)
        j = np.where(self.pres[None], 0.0, j)
        w = p["wet"]
        fluid = ~self.solid
        rt = np.where(fluid, rho[0] + rho[1], 1.0)
        s = self.s_of(rho[w], np.where(fluid, rho[1 - w], 1.0))
        # residual hysteresis in gray cells
        to_dry = self.gray & self.wet & (s < p["s_lo"])
        to_wet = self.gray & ~self.wet & (s > p["s_hi"])
        self.Rw = np.where(to_dry, self.geo["swirr"], np.where(to_wet, 0.0, self.Rw)).astype(dt)
        self.Ro = np.where(to_wet, self.geo["sores"], np.where(to_dry, 0.0, self.Ro)).astype(dt)
        self.wet = np.where(to_dry, False, np.where(to_wet, True, self.wet))
        sw = np.where(self.gray, self.Rw + (1 - self.Rw - self.Ro) * s, s)
        seen = [np.where(self.solid, p["rho_wall"][a], rho[a]).astype(dt) for a in range(2)]
        grad = [iso_grad(seen[1 - a]) for a in range(2)]
        F = []
        terms = {}
        for a in range(2):
            sc = -p["G"] * rho[a][None] * grad[a]
            body = rho[a][None] * np.asarray(p["accel"][a], dt)[:, None, None, None]
            csf = np.zeros_like(sc)
            if p["kappa"] != 0.0:
                # div of g/sqrt(|g|^2 + eps^2) = tr(H)/s - g.H.g/s^3, H = Hessian of phi^a
                H = moment_hessian(seen[1 - a], rho[1 - a])
                g = grad[a]
                s = np.sqrt((g ** 2).sum(axis=0) + p["eps_n"] ** 2)
                gHg = np.einsum("a...,ab...,b...->...", g, H, g)
                div = (H[0, 0] + H[1, 1] + H[2, 2]) / s - gHg / s ** 3
                mask = np.ones(self.cell.shape, bool) if p["csf_everywhere"] else self.gray
                csf = np.where(mask[None], p["kappa"] * (-div)[None] * (grad[a] / p["phi_avg"][a])
                               * (rho[a] / p["phi_max"][a])[None], 0.0)
            terms[a] = dict(sc=sc, body=body, csf=csf)
        # capillary force in gray cells
        den = seen[w] + seen[1 - w]
        At_field = np.where(den > 0, (seen[w] - seen[1 - w]) / np.where(den > 0, den, 1.0), 0.0)
        dAt = iso_grad(At_field)
        mag = np.sqrt((dAt ** 2).sum(axis=0))
        H = np.where(np.abs(At_field) <= p["at_cut"], 0.5 * mag, 0.0)
        cv = self.curve
        se_c = np.clip((sw - cv["swr"]) / (1 - cv["swr"]), 1e-2, 1.0)
        if cv.get("thomeer_g", 0.0) > 0.0:
            with np.errstate(divide="ignore"):
                expo = np.minimum(cv["thomeer_g"] / -np.log1p(-se_c), 1.0)
            Pc = self.geo["lamL"] * cv["pd"] * np.exp(np.log(10.0) * expo)
        else:
            Pc = self.geo["lamL"] * cv["pd"] * se_c ** (-1.0 / cv["lambda"])
        nvec = dAt / np.maximum(mag, p["eps_n"])
        for a in range(2):
            cap = -Pc[None] * (rho[a] / rt)[None] * nvec * H[None]
            terms[a]["cap"] = np.where((self.gray & (H > 0))[None], cap, 0.0)
        Fo = sum(terms[a][k] for a in range(2) for k in ("sc", "body", "csf", "cap"))
        # semi-implicit velocity
        se_k = np.clip((sw - cv["swr"]) / (1 - cv["swr"]), 0.0, 1.0)
        kr = [None, None]
        kr[w] = se_k ** cv["nw"]
        kr[1 - w] = (1 - se_k) ** cv["nn"]
        coef = sum(rho[b] * ((p["tau"][b] - 0.5) / 3.0) / np.maximum(kr[b], p["kr_min"]) for b in range(2))
        R = coef[..., None, None] * self.kinv
        A = rt[..., None, None] * np.eye(3) + 0.5 * R
        rhs = np.moveaxis(j + 0.5 * Fo, 0, -1)
        ug = np.linalg.solve(np.where(self.gray[..., None, None], A, np.eye(3)),
                             np.where(self.gray[..., None], rhs, 0.0)[..., None])[..., 0]
        ug = np.moveaxis(ug, -1, 0)
        un = (j + 0.5 * Fo) / rt[None]
        u = np.where(self.gray[None], ug, un)
        u = np.where((self.solid | self.pres)[None], 0.0, u).astype(dt)
        Ru = np.einsum("...ab,b...->a...", R, u)
        for a in range(2):
            terms[a]["drag"] = np.where(self.gray[None], -(rho[a] / rt)[None] * Ru, 0.0)
            for k in terms[a]:
                terms[a][k] = np.where(self.pres[None], 0.0, terms[a][k])
            F.append(sum(terms[a].values()))
        fnew = np.stack([collide(fs[a], u, F[a], p["tau"][a]) for a in range(2)])
        if p.get("mss", 0.0):
            # mass-sink-source: rest equilibrium of +dm (wetting) and -dm (other)
            rw, rn = rho[w] / rt, rho[1 - w] / rt
            r_lo = p["rho_lo"] / (p["rho_hi"] + p["rho_lo"])
            ib = 4 * r_lo * (1 - r_lo)
            dm = p["mss"] * np.maximum((4 * rw * rn - ib) / (1 - ib), 0.0)
            dm = np.where(self.solid | self.pres, 0.0, dm)
            fnew[w] = fnew[w] + WGT[:, None, None, None] * dm[None]
            fnew[1 - w] = fnew[1 - w] - WGT[:, None, None, None] * dm[None]
        rest = np.zeros((3,) + self.cell.shape, dt)
        fnew = np.where(self.pres[None, None], np.stack([equilibrium(rho[a], rest) for a in range(2)]), fnew)
        self.f = np.where(self.solid[None, None], 0.0, fnew).astype(dt)
        self.rho, self.u, self.sw, self.terms = rho, u, sw, terms
        return self
