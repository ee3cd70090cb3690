"""Seeded synthetic inputs: geometries and initial density fields.

This module only draws and shapes random inputs (cell types, porosity maps,
initial densities).  It holds none of the lattice Boltzmann arithmetic, so both
the CUDA path and the FP64 oracle can be fed from it without sharing any of the
method's code.

The recipes stand in for the paper's inputs that are not available here: the
scanned rock images of its ref. [14] (Sec. III.C, III.D, Appendix) and the REV
library runs of the Appendix.  Every generator takes an explicit seed and uses
NumPy's PCG64, so a given (recipe, size, seed) always yields the same arrays.

Cell type codes (shared vocabulary of the C-ABI and the oracle):
  0 = resolved pore, 1 = solid, 2 = gray (under-resolved porous cell).
"""
from __future__ import annotations

import numpy as np

PORE, SOLID, GRAY, INLET, OUTLET = 0, 1, 2, 3, 4

# Base seed of the synthetic workloads; workload k uses SEED_BASE + k.
SEED_BASE = 2512216960


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- random fields
def gaussian_random_field(shape, ell: float, rng: np.random.Generator) -> np.ndarray:
    """White N(0,1) noise convolved periodically with a Gaussian of std `ell` cells.

    Arrays are indexed [z][y][x].  The convolution is done in Fourier space with
    the Gaussian's transfer function, i.e. a periodised Gaussian kernel.
    """
    white = rng.standard_normal(shape)
    spec = np.fft.rfftn(white)
    freqs = [np.fft.fftfreq(n) for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    grids = np.meshgrid(*freqs, indexing="ij")
    k2 = sum((2.0 * np.pi * g) ** 2 for g in grids)
    spec *= np.exp(-0.5 * k2 * ell * ell)
    field = np.fft.irfftn(spec, s=shape)
    field -= field.mean()
    sd = field.std()
    return field / sd if sd > 0 else field


def top_fraction(field: np.ndarray, frac: float) -> np.ndarray:
    """Boolean mask of the cells whose value lies in the top `frac` quantile."""
    if frac <= 0:
        return np.zeros(field.shape, dtype=bool)
    thr = np.quantile(field, 1.0 - frac)
    return field > thr


def box_average_periodic(values: np.ndarray, mask: np.ndarray, half: int = 1) -> np.ndarray:
    """Mean of `values` over the masked cells of each (2*half+1)^3 periodic box."""
    num = np.zeros_like(values, dtype=np.float64)
    den = np.zeros_like(values, dtype=np.float64)
    v = np.where(mask, values, 0.0)
    m = mask.astype(np.float64)
    for dz in range(-half, half + 1):
        for dy in range(-half, half + 1):
            for dx in range(-half, half + 1):
                num += np.roll(v, (dz, dy, dx), axis=(0, 1, 2))
                den += np.roll(m, (dz, dy, dx), axis=(0, 1, 2))
    out = np.where(den > 0, num / np.maximum(den, 1.0), values)
    return out


# ------------------------------------------------------------------ droplets
def droplet_fields(shape, radius: float, center, rho_hi: float, rho_lo: float,
                   inside_component: int = 0):
    """Sphere of one component (density rho_hi) in the other (rho_hi outside).

    Cell centres sit at integer coordinates; a cell is inside when its squared
    distance to `center` is <= radius^2.  Returns (rhoA, rhoB) indexed [z][y][x].
    """
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cz, cy, cx = center[2], center[1], center[0]
    inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= radius * radius
    a = np.where(inside, rho_hi, rho_lo).astype(np.float64)
    b = np.where(inside, rho_lo, rho_hi).astype(np.float64)
    return (a, b) if inside_component == 0 else (b, a)


def cylinder_droplet_fields(shape, radius: float, center_xy, rho_hi: float, rho_lo: float):
    """Infinite cylinder along z (a 2-D droplet when nz == 1)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = (x - center_xy[0]) ** 2 + (y - center_xy[1]) ** 2 <= radius * radius
    a = np.where(inside, rho_hi, rho_lo).astype(np.float64)
    b = np.where(inside, rho_lo, rho_hi).astype(np.float64)
    return a, b


# ------------------------------------------------- multiscale rock (drainage)
def drainage_geometry(n: int, seed: int, solid_frac=0.20, gray_frac=0.25,
                      ell_solid=6.0, ell_gray=2.0, reservoir=8):
    """Synthetic multiscale rock on an n^3 periodic grid.

    Solid = top `solid_frac` of a Gaussian field (length `ell_solid`); gray =
    top `gray_frac` of a second field (length `ell_gray`) minus the solid;
    gray porosity = 0.1 + 0.5*U, averaged over gray cells of each 3^3 box and
    clipped to [0.1, 0.6]; the slab x < `reservoir` is forced to open pore so
    the injected component has an inlet reservoir.

    Returns (type u8, phi f64, pore_type u8), each indexed [z][y][x].
    """
    rng = rng_for(seed)
    shape = (n, n, n)
    f1 = gaussian_random_field(shape, ell_solid, rng)
    f2 = gaussian_random_field(shape, ell_gray, rng)
    solid = top_fraction(f1, solid_frac)
    gray = top_fraction(f2, gray_frac) & ~solid
    cell = np.full(shape, PORE, dtype=np.uint8)
    cell[solid] = SOLID
    cell[gray] = GRAY
    phi_raw = 0.1 + 0.5 * rng.random(shape)
    phi_s = box_average_periodic(phi_raw, gray, 1)
    phi = np.where(gray, np.clip(phi_s, 0.1, 0.6), np.where(solid, 0.0, 1.0))
    if reservoir > 0:
        cell[:, :, :reservoir] = PORE
        phi[:, :, :reservoir] = 1.0
    ptype = np.zeros(shape, dtype=np.uint8)
    return cell, phi.astype(np.float64), ptype


def drainage_fields(cell: np.ndarray, rho_hi: float, rho_lo: float, reservoir=8,
                    injected: int = 0):
    """Injected component fills the inlet slab x < reservoir, the other the rest."""
    inj = np.zeros(cell.shape, dtype=bool)
    inj[:, :, :reservoir] = True
    a = np.where(inj, rho_hi, rho_lo).astype(np.float64)
    b = np.where(inj, rho_lo, rho_hi).astype(np.float64)
    if injected == 1:
        a, b = b, a
    return a, b


# ------------------------------------------------------------- fibre bundle
def vmf_sample(mu: np.ndarray, kappa: float, size: int, rng: np.random.Generator) -> np.ndarray:
    """Unit vectors from the von Mises-Fisher distribution on S^2 (Wood, 1994).

    In three dimensions the cosine w to the mean direction has the closed-form
    inverse CDF w = 1 + log(u + (1-u) exp(-2 kappa)) / kappa.
    """
    mu = np.asarray(mu, dtype=np.float64)
    mu = mu / np.linalg.norm(mu)
    u = rng.random(size)
    w = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * kappa)) / kappa
    ang = 2.0 * np.pi * rng.random(size)
    helper = np.array([1.0, 0.0, 0.0]) if abs(mu[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    t1 = np.cross(mu, helper)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(mu, t1)
    s = np.sqrt(np.clip(1.0 - w * w, 0.0, None))
    return (w[:, None] * mu[None, :]
            + s[:, None] * (np.cos(ang)[:, None] * t1[None, :] + np.sin(ang)[:, None] * t2[None, :]))


def fiber_bundle_geometry(n: int, seed: int, ncyl=400, radius=1.5, kappa=20.0,
                          length_frac=0.5, smooth=2.0, gray_cut=0.99):
    """Gray fibre bundle: 400 seeded cylinders, vMF axes about a random direction.

    The fibre indicator is smoothed by a periodic Gaussian (std `smooth`),
    porosity phi = 1 - 0.9*density/max(density); cells with phi < gray_cut are
    gray, all others open pore.  Segments have length length_frac*n.
    Returns (type u8, phi f64, pore_type u8, mean_axis).
    """
    rng = rng_for(seed)
    shape = (n, n, n)
    axis0 = rng.standard_normal(3)
    axis0 /= np.linalg.norm(axis0)
    axes = vmf_sample(axis0, kappa, ncyl, rng)
    centres = rng.random((ncyl, 3)) * n
    ind = np.zeros(shape, dtype=np.float64)
    half = 0.5 * length_frac * n
    off = np.arange(-2, 3)
    oz, oy, ox = np.meshgrid(off, off, off, indexing="ij")
    block = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1)  # (125, 3) as x,y,z
    for c, a in zip(centres, axes):
        ts = np.arange(-half, half + 0.5, 0.5)
        pts = c[None, :] + ts[:, None] * a[None, :]
        base = np.floor(pts).astype(np.int64)
        cand = (base[:, None, :] + block[None, :, :]).reshape(-1, 3)
        cand = np.unique(cand, axis=0)
        d = cand.astype(np.float64) - c[None, :]
        d -= n * np.round(d / n)
        t = np.clip(d @ a, -half, half)
        perp = d - t[:, None] * a[None, :]
        hit = np.einsum("ij,ij->i", perp, perp) <= radius * radius
        cw = np.mod(cand[hit], n)
        ind[cw[:, 2], cw[:, 1], cw[:, 0]] = 1.0
    spec = np.fft.rfftn(ind)
    freqs = [np.fft.fftfreq(n), np.fft.fftfreq(n), np.fft.rfftfreq(n)]
    grids = np.meshgrid(*freqs, indexing="ij")
    k2 = sum((2.0 * np.pi * g) ** 2 for g in grids)
    dens = np.fft.irfftn(spec * np.exp(-0.5 * k2 * smooth * smooth), s=shape)
    dens = np.clip(dens, 0.0, None)
    phi = 1.0 - 0.9 * dens / max(dens.max(), 1e-300)
    cell = np.where(phi < gray_cut, GRAY, PORE).astype(np.uint8)
    phi = np.where(cell == GRAY, phi, 1.0)
    return cell, phi, np.zeros(shape, dtype=np.uint8), axis0


# ------------------------------------------------------ REV pore-type library
def rev_geometry(edge: int, kind: str, seed: int):
    """Fully resolved (pore/solid only) REV of one of four pore types.

    kind: 'spheres' (overlapping sphere pack), 'grf' (Gaussian field, 50%),
    'fibers' (solid cylinders), 'slits' (solid matrix cut by planar cracks).
    Returns (type u8, phi f64, pore_type u8) on an edge^3 periodic grid.
    """
    rng = rng_for(seed)
    shape = (edge, edge, edge)
    z, y, x = np.meshgrid(np.arange(edge), np.arange(edge), np.arange(edge), indexing="ij")
    solid = np.zeros(shape, dtype=bool)
    if kind == "spheres":
        target = 0.6
        while solid.mean() < target:
            c = rng.random(3) * edge
            r = rng.uniform(0.08, 0.16) * edge
            d = [x - c[0], y - c[1], z - c[2]]
            d = [dd - edge * np.round(dd / edge) for dd in d]
            solid |= d[0] ** 2 + d[1] ** 2 + d[2] ** 2 <= r * r
    elif kind == "grf":
        solid = top_fraction(gaussian_random_field(shape, max(2.0, edge / 12.0), rng), 0.5)
    elif kind == "fibers":
        nfib = max(4, edge // 4)
        axes = vmf_sample(np.array([0.0, 0.0, 1.0]), 5.0, nfib, rng)
        cen = rng.random((nfib, 3)) * edge
        r = max(1.5, edge / 16.0)
        for c, a in zip(cen, axes):
            d = np.stack([x - c[0], y - c[1], z - c[2]], axis=-1)
            d -= edge * np.round(d / edge)
            t = d @ a
            perp = d - t[..., None] * a
            solid |= np.einsum("...i,...i->...", perp, perp) <= r * r
    elif kind == "slits":
        solid[:] = True
        for _ in range(3):
            nrm = rng.standard_normal(3)
            nrm /= np.linalg.norm(nrm)
            off = rng.random() * edge
            ap = rng.uniform(1.0, 2.0)
            dist = (x * nrm[0] + y * nrm[1] + z * nrm[2] - off)
            dist = np.abs(dist - edge * np.round(dist / edge))
            solid &= dist > ap
    else:
        raise ValueError(kind)
    cell = np.where(solid, SOLID, PORE).astype(np.uint8)
    phi = np.where(solid, 0.0, 1.0)
    return cell, phi, np.zeros(shape, dtype=np.uint8)


def cosine_porosity(shape, phi0: float, amp: float, k) -> np.ndarray:
    """phi = phi0 + amp*cos(k . x) on integer cell centres (x, y, z)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return phi0 + amp * np.cos(k[0] * x + k[1] * y + k[2] * z)


def zigzag_pathway_geometry(nx=120, ny=180, half_width=10.0, amp=20.0, period=90.0, phi_bundle=0.95):
    """The two-dimensional fibre-bundle case of Sec. I.B / Sec. III.E on one
    plane: an open pathway (pore cells within half_width in x of the
    sinusoidal centre line x_c(y) = nx/2 + amp sin(2 pi y / period)) between
    two gray bundles of porosity phi_bundle that reach the walls, with a row
    of inlet cells above (y = ny + 1) and of outlet cells below (y = 0).
    Returns (cell, phi, path): shape (1, ny + 2, nx) each, path marking the
    pathway's pore cells."""
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    xc = nx / 2.0 - 0.5 + amp * np.sin(2.0 * np.pi * y / period)
    inner = np.abs(x - xc) <= half_width
    cell = np.full((1, ny + 2, nx), GRAY, np.uint8)
    cell[0, 1:-1, :][inner] = PORE
    cell[0, -1, :], cell[0, 0, :] = INLET, OUTLET
    phi = np.where(cell == GRAY, phi_bundle, 1.0).astype(np.float32)
    path = np.zeros(cell.shape, bool)
    path[0, 1:-1, :] = inner
    return cell, phi, path
