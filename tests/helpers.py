"""Closed forms and small utilities shared by the tests (no method arithmetic)."""
from __future__ import annotations

import numpy as np


def stencil_sine_vector(k):
    """Exact sum_i w_i c_i sin(k . c_i) over the D3Q19 set, written out.

    Faces contribute 2*(1/18) sin(k_d); the eight edges with c_d = +-1
    contribute 2*(1/36) [sin(k_d + k_e) + sin(k_d - k_e)] for both e != d.
    """
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros(3)
    for d in range(3):
        acc = (2.0 / 18.0) * np.sin(k[d])
        for e in range(3):
            if e != d:
                acc += (2.0 / 36.0) * (np.sin(k[d] + k[e]) + np.sin(k[d] - k[e]))
        out[d] = acc
    return out


def cosine_hessian_matrix(k):
    """M_k with H = -amp cos(theta) M_k for the face/cross difference stencils."""
    k = np.asarray(k, dtype=np.float64)
    M = np.zeros((3, 3))
    for a in range(3):
        M[a, a] = 2.0 * (1.0 - np.cos(k[a]))
        for b in range(3):
            if b != a:
                M[a, b] = np.sin(k[a]) * np.sin(k[b])
    return M


def rel_l2(a, b, mask=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_rel(a, b, mask=None):
    """Element-wise error max|a - b| / max|b| (over the masked cells, all
    components): the bound that a wrong value in a single cell cannot hide
    under, where the L2 norm of a large lattice averages it away."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    mb = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0)) if b.size else 0.0


def rest_only_populations(rhoA, rhoB, Q=19):
    """Post-collision state whose streamed densities equal (rhoA, rhoB) exactly.

    All mass sits in the rest population, which streams onto itself, so the
    first step sees exactly these densities and zero momentum.
    """
    shape = np.shape(rhoA)
    f = np.zeros((2, Q) + shape)
    f[0, 0] = rhoA
    f[1, 0] = rhoB
    return f
