"""Seeded synthetic inputs for the bond-based peridynamic time step.

This module only *generates inputs*: lattice coordinates, nodal volumes,
boundary-condition masks, planar notch/pre-crack rectangles, per-instance
material draws and Gaussian-random-field parameters.  It holds none of the
method's arithmetic (no family search, no stretch, no force, no micromodulus
formula, no integrator); the CUDA library and the CPU oracle each implement
those on their own and both consume what is generated here.

The shapes follow the workloads of the paper's benchmarks (regular cubic
tensor-grid beams of hundreds of thousands to tens of millions of nodes,
Section 4, Fig. "profile_regular") and its examples (notched beams under
displacement-controlled three-point bending, Sections 6-7).  The paper's
meshes and experimental data are not available, so every geometry here is a
synthetic stand-in with the stated sizes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


@dataclasses.dataclass
class Workload:
    """One synthetic problem: geometry, material, boundary conditions, run length.

    Arrays are in the caller's node order (row-major lattice order, z fastest).
    ``cuts`` are planar rectangles ``(axis, pos, lo_a, hi_a, lo_b, hi_b)``: the
    plane ``x[axis] == pos`` restricted to ``lo_a <= x[a] <= hi_a`` and
    ``lo_b <= x[b] <= hi_b`` where ``(a, b)`` are the two other axes in ascending
    order.  A bond whose segment crosses such a rectangle is absent from the start
    (the paper's initial-notch rule, Section 6).
    """

    name: str
    coords: np.ndarray            # (n, 3) float64, metres
    volumes: np.ndarray           # (n,) float64, m^3
    horizon: float                # delta, metres
    bulk_modulus: float           # K, Pa  (micromodulus is derived by each consumer)
    sc: float                     # constant critical stretch (used when sc_hash is None)
    sc_hash: Optional[Tuple[int, float, float]]  # (seed, lo, hi): per-bond U[lo, hi) draw
    bc_type: np.ndarray           # (n, 3) uint8: 1 = displacement-controlled component
    bc_disp: np.ndarray           # (n, 3) float64: displacement per unit of the load scale
    bc_force: np.ndarray          # (n, 3) float64: body-force density per unit of load
    disp_rate: float              # displacement scale after step k is disp_rate * k
    load: float                   # body-force scale
    no_fail: Optional[np.ndarray]  # (n,) uint8 or None
    cuts: List[Tuple[int, float, float, float, float, float]]
    dt: float
    damping: float                # eta, kg m^-3 s^-1
    density: float                # rho, kg m^-3
    steps: int
    shape: Tuple[int, int, int]
    dx: float
    ramp_steps: int = 0       # 0: displacement scale rate*k; T: smooth start over T steps
    kr: float = 0.0           # > 1: bilinear softening with s_0 = s_c / kr
    state_based: object = None  # (K, G): ordinary state-based linear solid instead of PMB
    trilinear: object = None    # (s_1 / s_0, kink force / peak force) with kr: trilinear law

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])

    def cuts_array(self) -> np.ndarray:
        if not self.cuts:
            return np.zeros((0, 6), dtype=np.float64)
        return np.asarray(self.cuts, dtype=np.float64).reshape(-1, 6)


def lattice(nx: int, ny: int, nz: int, dx: float, jitter: float = 0.0,
            seed: int = 0) -> np.ndarray:
    """Simple cubic lattice, node (ix, iy, iz) at dx*(ix, iy, iz), z fastest.

    ``jitter`` > 0 displaces every node by U(-jitter, jitter)*dx per axis
    (the irregular-mesh stand-in).
    """
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * dx
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        x += rng.uniform(-jitter, jitter, size=x.shape) * dx
    return x


def _grid_index(shape):
    nx, ny, nz = shape
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return ix.ravel(), iy.ravel(), iz.ravel()


def _empty_bc(n):
    return (np.zeros((n, 3), np.uint8), np.zeros((n, 3), np.float64),
            np.zeros((n, 3), np.float64))


def tensile_bar(nx: int = 40, ny: int = 10, nz: int = 10, dx: float = 1e-3,
                rate: float = 1e-7, slab: int = 3, steps: int = 1000,
                K: float = 5e9, sc: float = 5e-3) -> Workload:
    """Plain tensile bar: x-end slabs of ``slab`` layers pulled apart at +-rate m/step.

    Default is the 40x10x10 = 4000-node bar, dx = 1 mm, delta = 3.01 dx,
    K = 5 GPa, s_c = 5e-3, rho = 2400, dt = 1e-7 s, eta = 2.5e6, 1000 steps.
    Only the x component of the end slabs is prescribed.
    """
    x = lattice(nx, ny, nz, dx)
    n = x.shape[0]
    ix, _, _ = _grid_index((nx, ny, nz))
    t, g, b = _empty_bc(n)
    left = ix < slab
    right = ix >= nx - slab
    t[left, 0] = 1
    t[right, 0] = 1
    g[left, 0] = -rate
    g[right, 0] = rate
    return Workload(
        name=f"tensile_bar_{nx}x{ny}x{nz}", coords=x, volumes=np.full(n, dx ** 3),
        horizon=3.01 * dx, bulk_modulus=K, sc=sc, sc_hash=None,
        bc_type=t, bc_disp=g, bc_force=b, disp_rate=1.0, load=0.0, no_fail=None,
        cuts=[], dt=1e-7, damping=2.5e6, density=2400.0, steps=steps,
        shape=(nx, ny, nz), dx=dx)


def notched_beam(nx: int = 300, ny: int = 58, nz: int = 58, length: float = 0.5,
                 rate: float = 1e-8, steps: int = 5000, K: float = 3e10,
                 sc_lo: float = 9e-5, sc_hi: float = 1.1e-4,
                 seed: int = 2105041502, horizon_factor: float = math.pi,
                 notch_depth: float = 0.3) -> Workload:
    """Notched three-point-bend beam on an nx x ny x nz lattice (default 1,009,200 nodes).

    dx = length/nx, delta = pi*dx.  Bonds crossing the mid-span plane
    x = (nx-1)/2*dx below ``notch_depth`` of the height (z from the bottom face)
    are absent from the start.  Supports: 2-node-wide bottom strips at both ends,
    all components fixed.  Load: the 2-node-wide top-centre strip is moved in -z
    at ``rate`` m/step.  Per-bond s_c ~ U[sc_lo, sc_hi) from a counter-based
    draw keyed on the unordered pair of caller node ids (seed ``seed``).
    """
    dx = length / nx
    x = lattice(nx, ny, nz, dx)
    n = x.shape[0]
    ix, iy, iz = _grid_index((nx, ny, nz))
    t, g, b = _empty_bc(n)
    sup = (iz == 0) & ((ix < 2) | (ix >= nx - 2))
    t[sup, :] = 1
    mid = nx // 2
    load = (iz == nz - 1) & ((ix == mid - 1) | (ix == mid))
    t[load, 2] = 1
    g[load, 2] = -rate
    xm = 0.5 * (nx - 1) * dx
    eps = 0.25 * dx
    # the notch rectangle spans the full width (y) and the bottom notch_depth*H (z)
    ztop = (notch_depth * nz - 0.5) * dx
    cuts = [(0, xm, -eps, (ny - 1) * dx + eps, -eps, ztop)]
    return Workload(
        name=f"notched_beam_{nx}x{ny}x{nz}", coords=x, volumes=np.full(n, dx ** 3),
        horizon=horizon_factor * dx, bulk_modulus=K, sc=0.5 * (sc_lo + sc_hi),
        sc_hash=(seed, sc_lo, sc_hi), bc_type=t, bc_disp=g, bc_force=b,
        disp_rate=1.0, load=0.0, no_fail=None, cuts=cuts, dt=1e-7, damping=2.5e6,
        density=2400.0, steps=steps, shape=(nx, ny, nz), dx=dx)


def plate(nx: int = 1000, ny: int = 400, nz: int = 40, dx: float = 1e-3,
          rate: float = 1e-8, slab: int = 3, steps: int = 500, K: float = 3e10,
          sc: float = 1e-4) -> Workload:
    """Pre-cracked plate: edge slit on the plane y = W/2 over x <= Lx/4, through
    the thickness; the y-end slabs (``slab`` layers) are pulled apart in y at
    +-rate m/step.  Default 1000x400x40 = 16M nodes, delta = 3.01 dx."""
    x = lattice(nx, ny, nz, dx)
    n = x.shape[0]
    _, iy, _ = _grid_index((nx, ny, nz))
    t, g, b = _empty_bc(n)
    lo = iy < slab
    hi = iy >= ny - slab
    t[lo, 1] = 1
    t[hi, 1] = 1
    g[lo, 1] = -rate
    g[hi, 1] = rate
    ym = 0.5 * (ny - 1) * dx
    eps = 0.25 * dx
    cuts = [(1, ym, -eps, 0.25 * (nx - 1) * dx + 0.5 * dx, -eps, (nz - 1) * dx + eps)]
    return Workload(
        name=f"plate_{nx}x{ny}x{nz}", coords=x, volumes=np.full(n, dx ** 3),
        horizon=3.01 * dx, bulk_modulus=K, sc=sc, sc_hash=None, bc_type=t, bc_disp=g,
        bc_force=b, disp_rate=1.0, load=0.0, no_fail=None, cuts=cuts, dt=1e-7,
        damping=2.5e6, density=2400.0, steps=steps, shape=(nx, ny, nz), dx=dx)


def cracked_plate_force(nx: int = 250, ny: int = 100, nz: int = 4, dx: float = 1e-3,
                        load: float = 1.0, steps: int = 2000, K: float = 3e10,
                        sc: float = 1e-4, edge: int = 2) -> Workload:
    """Force-loaded pre-cracked plate (the sensitivity workload, default 100k nodes).

    Edge crack on the plane y = W/2 over x <= Lx/4 (mouth at x = 0).  The y-end
    strips (``edge`` layers) carry an opposing body-force density in +-y of unit
    magnitude per unit ``load``; ``load`` is the scalar whose sensitivity is
    sought.  No component is displacement-controlled.
    """
    x = lattice(nx, ny, nz, dx)
    n = x.shape[0]
    _, iy, _ = _grid_index((nx, ny, nz))
    t, g, b = _empty_bc(n)
    b[iy < edge, 1] = -1.0
    b[iy >= ny - edge, 1] = 1.0
    ym = 0.5 * (ny - 1) * dx
    eps = 0.25 * dx
    cuts = [(1, ym, -eps, 0.25 * (nx - 1) * dx + 0.5 * dx, -eps, (nz - 1) * dx + eps)]
    return Workload(
        name=f"cracked_plate_{nx}x{ny}x{nz}", coords=x, volumes=np.full(n, dx ** 3),
        horizon=3.01 * dx, bulk_modulus=K, sc=sc, sc_hash=None, bc_type=t, bc_disp=g,
        bc_force=b, disp_rate=0.0, load=load, no_fail=None, cuts=cuts, dt=1e-7,
        damping=2.5e6, density=2400.0, steps=steps, shape=(nx, ny, nz), dx=dx)


def mouth_nodes(w: Workload, layers: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    """Nodes at x = 0 just above / just below the slit plane y = W/2 (crack mouth)."""
    nx, ny, nz = w.shape
    ix, iy, _ = _grid_index(w.shape)
    mid = ny // 2
    above = np.nonzero((ix == 0) & (iy >= mid) & (iy < mid + layers))[0]
    below = np.nonzero((ix == 0) & (iy < mid) & (iy >= mid - layers))[0]
    return above, below


def batch_instances(count: int = 256, n_lo: int = 2000, n_hi: int = 60000,
                    seed: int = 2105041504, dx: float = 1e-3) -> List[Workload]:
    """Independent bars (4:1:1) and notched beams (5:1:1), alternating, with node
    counts log-uniform in [n_lo, n_hi], K ~ lognormal(ln 3e10, 0.2),
    s_c ~ lognormal(ln 1e-4, 0.15); delta = 3.01 dx."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        K = float(math.exp(rng.normal(math.log(3e10), 0.2)))
        sc = float(math.exp(rng.normal(math.log(1e-4), 0.15)))
        if k % 2 == 0:
            a = (target / 4.0) ** (1.0 / 3.0)   # 4a x a x a nodes
            nx, ny, nz = max(4, round(4 * a)), max(2, round(a)), max(2, round(a))
            w = tensile_bar(nx, ny, nz, dx=dx, rate=1e-9, slab=min(3, nx // 4), K=K, sc=sc,
                            steps=2000)
        else:
            a = (target / 5.0) ** (1.0 / 3.0)   # 5a x a x a nodes
            nx, ny, nz = max(5, round(5 * a)), max(2, round(a)), max(2, round(a))
            w = notched_beam(nx, ny, nz, length=nx * dx, rate=1e-9, K=K, steps=2000,
                             horizon_factor=3.01)
            w.sc_hash = None
            w.sc = sc
        w.name = f"inst{k:03d}_" + w.name
        out.append(w)
    return out


def grf_params(seed: int, corr_len: float, features: int = 256):
    """Random-Fourier-feature parameters of a unit-variance Gaussian random field
    with squared-exponential correlation of length ``corr_len``."""
    rng = np.random.default_rng(seed)
    omega = rng.normal(0.0, 1.0 / corr_len, size=(features, 3))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=features)
    return omega, phase


def grf_eval(points: np.ndarray, omega: np.ndarray, phase: np.ndarray) -> np.ndarray:
    """Evaluate the random-feature field at ``points`` (m, 3)."""
    m = omega.shape[0]
    out = np.empty(points.shape[0], dtype=np.float64)
    step = 1 << 16
    for s in range(0, points.shape[0], step):
        p = points[s:s + step]
        out[s:s + step] = math.sqrt(2.0 / m) * np.cos(p @ omega.T + phase).sum(axis=1)
    return out


def sensitivity_plate(load: float = 8e6, steps: int = 2000) -> Workload:
    """The 250 x 100 x 4 pre-cracked plate of the sensitivity runs (100,000 nodes)
    with the y-edge body-force density scaled by ``load``.  The largest bond
    stretch over 2000 steps from rest is about 3.8e-12 per unit load, so the
    default keeps every bond near 0.3 s_c (s_c = 1e-4): nothing breaks."""
    return cracked_plate_force(250, 100, 4, load=load, steps=steps)


def bond_stiffness_grf(w: Workload, off: np.ndarray, idx: np.ndarray, c0: float,
                       seed: int = 2105041505, rel: float = 0.1,
                       corr_dx: float = 5.0) -> np.ndarray:
    """Per directed bond stiffness c0 (1 + rel g(m_ij)), g a unit-variance random
    field (correlation length corr_dx * dx) at the bond midpoint m_ij.  The field
    is evaluated once per distinct midpoint, so (i, j) and (j, i) get the same
    value exactly."""
    omega, phase = grf_params(seed, corr_dx * w.dx)
    rows = np.repeat(np.arange(w.n), np.diff(off))
    twice = np.rint((w.coords[rows] + w.coords[idx]) / w.dx).astype(np.int64)
    lo = twice.min(axis=0)
    span = twice.max(axis=0) - lo + 1
    t = twice - lo
    key = (t[:, 0] * span[1] + t[:, 1]) * span[2] + t[:, 2]
    uniq, inv = np.unique(key, return_inverse=True)
    pts = np.stack([uniq // (span[1] * span[2]), (uniq // span[2]) % span[1], uniq % span[2]],
                   axis=1)
    g = grf_eval(0.5 * (pts + lo) * w.dx, omega, phase)
    return c0 * (1.0 + rel * g[inv])


def reverse_bond(n: int, off: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Position of (j, i) for every directed bond (i, j) of a CSR family with
    ascending rows (for building symmetric per-bond fields)."""
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    key = rows * n + idx
    return np.searchsorted(key, idx.astype(np.int64) * n + rows)


def random_state(n: int, seed: int, u_scale: float, v_scale: float):
    """Seeded random displacement and velocity fields (n, 3)."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-u_scale, u_scale, size=(n, 3)),
            rng.uniform(-v_scale, v_scale, size=(n, 3)))
