"""Synthetic potentials v on the periodic grid hJ, h = 1/n (Section 2 of the paper).

The paper's Section 5 fields (a Gaussian bump or a cross in c(x), random Gaussian wells) are not
fully specified there, so these seeded generators stand in for them with the same structure:

* Helmholtz: v(x) = -(omega / c(x))^2 with c(x) = 1 + sum_j a_j exp(-|x - x_j|^2 / (2 sigma_j^2)).
* Schroedinger-type: v(x) = alpha * (sum_j -b_j exp(-|x - x_j|^2 / (2 w^2)) - E), with alpha
  scaled so that max |v| h^2 hits a target.

Distances are periodic (minimum image per axis). Arrays are float64, row-major, with the last
axis fastest, index j = (j_1, ..., j_d) sampling x = h j.
"""

from __future__ import annotations

import math

import numpy as np


def grid_coords(n: int, d: int) -> list[np.ndarray]:
    """Coordinates of hJ as d broadcastable float64 arrays (x_i = j_i / n)."""
    x1 = np.arange(n, dtype=np.float64) / n
    out = []
    for axis in range(d):
        shape = [1] * d
        shape[axis] = n
        out.append(x1.reshape(shape))
    return out


def periodic_sqdist(coords: list[np.ndarray], centre) -> np.ndarray:
    """|x - centre|^2 on the unit torus, minimum image per axis."""
    acc = None
    for xi, ci in zip(coords, centre):
        delta = np.mod(xi - ci + 0.5, 1.0) - 0.5
        term = delta * delta
        acc = term if acc is None else acc + term
    return acc


def helmholtz_gaussian_bump(n: int, omega: float, amp: float = 0.2, width: float = 0.1,
                            d: int = 2) -> np.ndarray:
    """v = -(omega/c)^2, c = 1 + amp * exp(-|x - 1/2|^2 / (2 width^2)) (one centred bump)."""
    coords = grid_coords(n, d)
    r2 = periodic_sqdist(coords, [0.5] * d)
    c = 1.0 + amp * np.exp(-r2 / (2.0 * width * width))
    c = np.broadcast_to(c, (n,) * d)
    return np.ascontiguousarray(-(omega / c) ** 2)


def helmholtz_random_bumps(n: int, omega: float, nbumps: int, seed: int, d: int = 2,
                           amp: float = 0.3, sig_lo: float = 0.02, sig_hi: float = 0.08
                           ) -> np.ndarray:
    """v = -(omega/c)^2 with c = 1 + sum of nbumps seeded Gaussians.

    a_j ~ U(-amp, amp), x_j ~ U[0,1)^d, sigma_j ~ U(sig_lo, sig_hi), drawn in that order from
    numpy.random.default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    a = rng.uniform(-amp, amp, nbumps)
    xc = rng.uniform(0.0, 1.0, (nbumps, d))
    sig = rng.uniform(sig_lo, sig_hi, nbumps)
    coords = grid_coords(n, d)
    c = np.ones((n,) * d)
    for j in range(nbumps):
        r2 = periodic_sqdist(coords, xc[j])
        c += a[j] * np.exp(-r2 / (2.0 * sig[j] * sig[j]))
    if not float(c.min()) > 0.0:
        raise ValueError("velocity field is not positive for this seed")
    return np.ascontiguousarray(-(omega / c) ** 2)


def schrodinger_random_wells(n: int, nwells: int, seed: int, d: int = 3, energy: float = 0.3,
                             width: float = 0.05, target_h2v: float = 0.6) -> np.ndarray:
    """v = alpha * (sum_j -b_j exp(-|x - x_j|^2 / (2 width^2)) - energy), max|v| h^2 = target.

    b_j ~ U(0.5, 1.5) then x_j ~ U[0,1)^d, from numpy.random.default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    b = rng.uniform(0.5, 1.5, nwells)
    xc = rng.uniform(0.0, 1.0, (nwells, d))
    coords = grid_coords(n, d)
    base = np.full((n,) * d, -energy)
    for j in range(nwells):
        r2 = periodic_sqdist(coords, xc[j])
        base -= b[j] * np.exp(-r2 / (2.0 * width * width))
    h = 1.0 / n
    alpha = target_h2v / (float(np.abs(base).max()) * h * h)
    return np.ascontiguousarray(alpha * base)


def gaussian_source(n: int, d: int, sigma_cells: float = 2.0) -> np.ndarray:
    """Right-hand side f: a Gaussian point source at the centre, width sigma = sigma_cells * h."""
    coords = grid_coords(n, d)
    r2 = periodic_sqdist(coords, [0.5] * d)
    sig = sigma_cells / n
    f = np.exp(-r2 / (2.0 * sig * sig))
    return np.ascontiguousarray(np.broadcast_to(f, (n,) * d).copy())


# The workloads: name -> (d, n, builder). Seeds are fixed per workload; `seed` overrides them.
WORKLOADS = {
    # 2D Helmholtz, one centred bump, 4 points per wavelength (omega = 2 pi 8, n = 32).
    "helm2d_n32": dict(d=2, n=32, kind="bump", omega=2 * math.pi * 8, seed=1),
    # 2D Helmholtz, 16 random bumps, omega = 2 pi 64, n = 256.
    "helm2d_n256": dict(d=2, n=256, kind="bumps", omega=2 * math.pi * 64, nb=16, seed=2),
    # 2D Helmholtz, 64 random bumps, omega = 2 pi 256, n = 1024.
    "helm2d_n1024": dict(d=2, n=1024, kind="bumps", omega=2 * math.pi * 256, nb=64, seed=3),
    # 3D Schroedinger-type, 8 random wells, max|v| h^2 = 0.6, n = 64.
    "schr3d_n64": dict(d=3, n=64, kind="wells", nb=8, seed=4),
    # 1D Helmholtz, one centred bump, 4 points per wavelength (omega = 2 pi 64, n = 256).
    "helm1d_n256": dict(d=1, n=256, kind="bump", omega=2 * math.pi * 64, seed=5),
}


def make_workload(name: str, seed: int | None = None, n: int | None = None) -> np.ndarray:
    """Potential v for a named workload. `n` rescales the grid (omega keeps 4 points/wavelength)."""
    spec = dict(WORKLOADS[name])
    if seed is not None:
        spec["seed"] = seed
    if n is not None and n != spec["n"]:
        if "omega" in spec:
            spec["omega"] = spec["omega"] * n / spec["n"]
        spec["n"] = n
    kind = spec["kind"]
    if kind == "bump":
        return helmholtz_gaussian_bump(spec["n"], spec["omega"], d=spec["d"])
    if kind == "bumps":
        return helmholtz_random_bumps(spec["n"], spec["omega"], spec["nb"], spec["seed"],
                                     d=spec["d"])
    if kind == "wells":
        return schrodinger_random_wells(spec["n"], spec["nb"], spec["seed"], d=spec["d"])
    raise ValueError(kind)
