"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method itself: only random draws and
the closed-form synthetic fields the workloads are built from. Every generator
takes an explicit seed and uses numpy's ``default_rng``.

* ``uniform_vector``  - U(-1, 1) DoF vectors (operator-apply inputs).
* ``sinker``          - random sphere centres U(0.1, 0.9)^3 for the piecewise
                        "sinker" viscosity field (radius 0.1, 8 spheres).
* ``fourier_modes`` / ``fourier_field`` - a divergence-free velocity
                        u(x) = sum_m c_m cos(2 pi k_m . x + phi_m) with integer
                        wave vectors k_m (components in -3..3, k_m != 0),
                        c_m = (k_m x a_m) / |k_m x a_m|, a_m ~ N(0, I),
                        phi_m ~ U(0, 2 pi): unit amplitude per mode and
                        exactly divergence-free because c_m . k_m = 0.
* ``bfs_channel``     - the grid and active-cell flags of the backward-facing
                        step channel (geometry only); ``bfs_vertices`` its
                        vertices with the 5 % seeded jitter inside the fluid.
"""
import numpy as np


def uniform_vector(n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=int(n))


def sinker(seed, count=8, radius=0.1, nu_max=1e4, nu_matrix=1.0):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.1, 0.9, size=(count, 3))
    return {'law': 'sinker', 'centers': centers, 'radius': float(radius),
            'nu_max': float(nu_max), 'nu_matrix': float(nu_matrix)}


def carreau_blood_like():
    """Carreau-Yasuda parameters of the 32^3 throughput workload."""
    return {'law': 'carreau', 'eta0': 1.0, 'eta_inf': 1e-3, 'kappa': 1.0, 'lam': 1.0,
            'a': 2.0, 'b': 0.5}


def fourier_modes(seed, count=8, kmax=3):
    rng = np.random.default_rng(seed)
    ks, cs, phis = [], [], []
    while len(ks) < count:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not np.any(k):
            continue
        a = rng.standard_normal(3)
        c = np.cross(k.astype(np.float64), a)
        norm = np.linalg.norm(c)
        if norm < 1e-12:
            continue
        ks.append(k.astype(np.float64))
        cs.append(c / norm)
        phis.append(rng.uniform(0.0, 2.0 * np.pi))
    return np.array(ks), np.array(cs), np.array(phis)


def fourier_field(points, modes):
    """Evaluate the Fourier velocity at points (P, 3) -> (P, 3)."""
    ks, cs, phis = modes
    pts = np.asarray(points, dtype=np.float64)
    arg = 2.0 * np.pi * pts @ ks.T + phis          # (P, m)
    return np.cos(arg) @ cs


def fourier_field_gradient(points, modes):
    """d u_i / d x_j of ``fourier_field`` (P, 3, 3), for input checks."""
    ks, cs, phis = modes
    pts = np.asarray(points, dtype=np.float64)
    arg = 2.0 * np.pi * pts @ ks.T + phis
    return -2.0 * np.pi * np.einsum('pm,mi,mj->pij', np.sin(arg), cs, ks)


def bfs_channel(cells_per_unit, inlet_length=5.0, outlet_length=30.0, step=1.0, height=2.0, depth=4.0):
    """Grid of the backward-facing-step channel: the inlet [-inlet_length, 0] x [step, height]
    feeds the outlet [0, outlet_length] x [0, height] (expansion ratio height / (height - step)),
    z in [0, depth] periodic; cubes of side 1 / cells_per_unit. Returns the grid over the
    bounding box and its active flags (nz, ny, nx): the block [-inlet_length, 0] x [0, step]
    is removed. Boundary ids of the grid: -x the inflow, +x the outflow, -y / +y and the faces
    against the removed block no-slip walls."""
    m = int(cells_per_unit)
    nx, ny, nz = round((inlet_length + outlet_length) * m), round(height * m), round(depth * m)
    lo = (-float(inlet_length), 0.0, 0.0)
    xc = lo[0] + (np.arange(nx) + 0.5) / m
    yc = (np.arange(ny) + 0.5) / m
    removed = (xc[None, :] < 0.0) & (yc[:, None] < step)
    active = np.broadcast_to(~removed, (nz, ny, nx)).copy()
    return {"dims": (nx, ny, nz), "extent": (inlet_length + outlet_length, float(height), float(depth)),
            "lo": lo, "active": active, "periodic": (False, False, True)}


def bfs_vertices(channel, amp=0.05, seed=4):
    """Vertices (nz+1, ny+1, nx+1, 3) of the channel grid with the vertices inside the fluid
    moved by U(-amp h, amp h) per direction (seed 4): a vertex moves when all 8 cells around
    it are active and it is not on the grid's outer surface, so the walls, the step, the
    inflow and outflow planes and the periodic end planes stay planar."""
    nx, ny, nz = channel["dims"]
    ext, lo = channel["extent"], channel["lo"]
    h = np.array([ext[0] / nx, ext[1] / ny, ext[2] / nz])
    xs = [lo[d] + h[d] * np.arange(n + 1) for d, n in enumerate((nx, ny, nz))]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing='ij')
    V = np.stack([X, Y, Z], axis=-1)
    act = np.asarray(channel["active"], dtype=bool)
    free = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    inner = np.ones((nz - 1, ny - 1, nx - 1), dtype=bool)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                inner &= act[dz:dz + nz - 1, dy:dy + ny - 1, dx:dx + nx - 1]
    free[1:nz, 1:ny, 1:nx] = inner
    J = np.random.default_rng(seed).uniform(-amp, amp, size=V.shape) * h
    return V + J * free[..., None]
