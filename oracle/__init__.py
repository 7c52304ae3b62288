"""FP64 CPU oracle of the bond-based peridynamic time step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over nodes,
ascending neighbour order).  This wrapper only marshals numpy arrays.

What pins each function (tests in ``tests/test_oracle_pins.py``):

* ``micromodulus`` (Eq. 5): the printed worked value c = 2.32e18 of the
  optimised-parameters table (Section 6) from E = 37.0 GPa, nu = 1/4,
  delta = 15.7 mm; and the continuum strain-energy identity behind it
  (W = 9/2 K eps^2 under uniform dilation) via the lattice quadrature ratio,
  which tends to 1 as delta/dx grows.
* ``family_*`` (Eq. 9): brute force equals the cell grid; interior nodes have
  the 122 offsets with |o|^2 <= 9; directed-bond totals equal closed-form
  counts of lattice offset pairs.
* ``step`` (Eqs. 4-6, 10-11, damped Euler-Cromer reading): zero force under
  rigid translation, near-zero under rotation; antisymmetry (sum V_i F_i = 0);
  momentum decays by exactly (1 - dt eta / rho) per step; forces equal minus
  the energy gradient (finite differences of ``energy_density``); a two-node
  bond reproduces the closed-form linear recurrence and breaks at the
  analytic step; displacement BCs follow the prescribed ramp.
* ``damage`` (Eq. 8): zero at the start, in [0, 1], monotone, and equal to the
  fraction of crossing offsets for a node next to a full planar cut; with
  unequal volumes, phi_i of a star-shaped family computed by hand in exact
  fractions (each bond weighted by the neighbour's volume V_j).
* no-fail nodes (Section 6): a two-node bond pulled past s_c with the flag on
  either end alone stays intact in both directions and keeps its force.
* body force (Eqs. 10-11): a node without bonds under load * b follows the
  damped Euler-Cromer recurrence in exact rationals (bond-based and
  state-based steps).
* ``splitmix64``: the published reference outputs of the generator.
* ``stiffness_factors`` (micromodulus functions, surface correction): the
  conical function reproduces the lattice quadrature ratio computed directly
  from the stencil offsets and tends to the continuum W = 9/2 K eps^2; the
  volume correction is symmetric, 1 between bulk nodes when V0 is the bulk
  family volume, and equals 2 V0 / (V_i + V_j) with V_i counted directly from
  the stencil for nodes on a free face (``tests/test_oracle_stiffness.py``).
* bilinear softening (``kr`` > 1): reduces to the PMB law bit for bit at
  kr = 1; a two-node bond follows the closed-form bilinear envelope under
  loading, unloads along the secant to the origin and reloads onto the
  envelope; the remembered stretch never decreases (``tests/test_oracle_soft.py``).
* ordinary state-based linear solid (``state_based=(K, G)``): uniform dilation
  gives theta = 3 eps and W = (9/2) K eps^2 at every node; simple shear gives
  G gamma^2 / 2 times the stencil quadrature ratio (-> 1 for large horizons);
  force = minus the energy gradient; rigid motions are force free; momentum is
  conserved (``tests/test_oracle_osb.py``).
* ``critical_stretch`` (Eq. 7) in 3D, plane stress and plane strain: the
  fracture-energy derivation by quadrature (micromodulus from the
  strain-energy match, energy of the bonds crossing a unit area);
  ``youngs_modulus``: the Lame-parameter forms.
* ``adjoint`` (Euler-Cromer and velocity-Verlet reverse modes): central
  differences of the pinned forward runs; the dot-product test of the bond
  Jacobian (``tests/test_oracle_adjoint.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into an in-tree shared library (gcc, FP64, OpenMP).

    ``-ffp-contract=off`` keeps results identical on x86-64 and aarch64."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Model(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("vol", ctypes.c_void_p),
        ("rows", ctypes.c_void_p), ("nrows", ctypes.c_int64),
        ("off", ctypes.c_void_p), ("idx", ctypes.c_void_p),
        ("c", ctypes.c_double), ("c_bond", ctypes.c_void_p),
        ("sc", ctypes.c_double), ("sc_mode", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("sc_seed", ctypes.c_uint64), ("sc_lo", ctypes.c_double), ("sc_hi", ctypes.c_double),
        ("no_fail", ctypes.c_void_p), ("bc_type", ctypes.c_void_p),
        ("bc_disp", ctypes.c_void_p), ("bc_force", ctypes.c_void_p),
        ("disp_rate", ctypes.c_double), ("load", ctypes.c_double),
        ("dt", ctypes.c_double), ("damping", ctypes.c_double), ("density", ctypes.c_double),
        ("ramp_steps", ctypes.c_int64),
        ("kr", ctypes.c_double), ("kappa", ctypes.c_void_p),
        ("model", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("K", ctypes.c_double), ("G", ctypes.c_double),
        ("wvol", ctypes.c_void_p), ("theta", ctypes.c_void_p),
        ("k1", ctypes.c_double), ("beta", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.or_micromodulus.restype = ctypes.c_double
        L.or_micromodulus.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_critical_stretch_3d.restype = ctypes.c_double
        L.or_critical_stretch_3d.argtypes = [ctypes.c_double] * 3
        L.or_critical_stretch_2d.restype = ctypes.c_double
        L.or_critical_stretch_2d.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int]
        L.or_youngs_modulus.restype = ctypes.c_double
        L.or_youngs_modulus.argtypes = [ctypes.c_double] * 2
        L.or_splitmix64.restype = ctypes.c_uint64
        L.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_sc_bond.restype = ctypes.c_double
        L.or_sc_bond.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int64, ctypes.c_int64]
        for name in ("or_family_bruteforce", "or_family_cells"):
            f = getattr(L, name)
            f.restype = ctypes.c_int64
            f.argtypes = [P, ctypes.c_int64, ctypes.c_double, P, ctypes.c_int64, P, P]
        L.or_cut_crosses.restype = ctypes.c_int
        L.or_cut_crosses.argtypes = [P, P, P]
        L.or_apply_cuts.restype = None
        L.or_apply_cuts.argtypes = [P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P]
        L.or_step.restype = None
        L.or_step.argtypes = [ctypes.POINTER(_Model), ctypes.c_int64, P, P, P, P, P, P, P]
        L.or_run.restype = None
        L.or_run.argtypes = [ctypes.POINTER(_Model), ctypes.c_int64, ctypes.c_int64, P, P, P, P]
        L.or_damage.restype = None
        L.or_damage.argtypes = [ctypes.POINTER(_Model), P, P]
        L.or_energy_density.restype = None
        L.or_energy_density.argtypes = [ctypes.POINTER(_Model), P, P, P]
        L.or_osb_weighted_volume.restype = None
        L.or_osb_weighted_volume.argtypes = [ctypes.POINTER(_Model), P]
        L.or_set_threads.restype = None
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_scale.restype = ctypes.c_double
        L.or_scale.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int64]
        L.or_run_vv.restype = None
        L.or_run_vv.argtypes = [ctypes.POINTER(_Model), ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int, P, P, P, P, P]
        L.or_stiffness_factors.restype = None
        L.or_stiffness_factors.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, P, P,
                                           ctypes.c_int, ctypes.c_double, P]
        L.or_stiffness_factors2.restype = None
        L.or_stiffness_factors2.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, P, P,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def scale(rate: float, ramp_steps: int, k: int) -> float:
    """Displacement scale after step k (linear, or the smooth start; see oracle.c)."""
    return lib().or_scale(rate, int(ramp_steps), int(k))


def set_threads(n: int) -> None:
    """OpenMP threads used by the oracle's loops (for CPU-baseline timing)."""
    lib().or_set_threads(int(n))


def micromodulus(K: float, delta: float) -> float:
    return lib().or_micromodulus(K, delta)


def critical_stretch_3d(G_F: float, E: float, delta: float) -> float:
    return lib().or_critical_stretch_3d(G_F, E, delta)


def critical_stretch(G_F: float, E: float, delta: float, kind: str = "3d") -> float:
    """Eq. 7 for kind "3d", "plane_stress" or "plane_strain"."""
    if kind == "3d":
        return lib().or_critical_stretch_3d(G_F, E, delta)
    if kind not in ("plane_stress", "plane_strain"):
        raise ValueError(kind)
    return lib().or_critical_stretch_2d(G_F, E, delta, int(kind == "plane_strain"))


def youngs_modulus(K: float, nu: float) -> float:
    return lib().or_youngs_modulus(K, nu)


def splitmix64(seed: int, m: int) -> int:
    return int(lib().or_splitmix64(seed, m))


def sc_bond(seed: int, lo: float, hi: float, i: int, j: int) -> float:
    return lib().or_sc_bond(seed, lo, hi, i, j)


def family(coords: np.ndarray, delta: float, rows: Optional[np.ndarray] = None,
           method: str = "cells"):
    """CSR family (Eq. 9) of ``rows`` (default all nodes): (off int64, idx int32)."""
    x = _c64(coords)
    n = x.shape[0]
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = n if r is None else r.shape[0]
    off = np.zeros(nrows + 1, dtype=np.int64)
    f = lib().or_family_bruteforce if method == "brute" else lib().or_family_cells
    total = f(x.ctypes.data, n, delta, _p(r), nrows, off.ctypes.data, None)
    idx = np.zeros(max(int(total), 1), dtype=np.int32)
    f(x.ctypes.data, n, delta, _p(r), nrows, off.ctypes.data, idx.ctypes.data)
    return off, idx[:total]


def cut_keep(coords, off, idx, cuts, rows=None):
    """uint8 mask over family entries: 0 where the bond crosses a notch rectangle."""
    x = _c64(coords)
    cuts = _c64(np.asarray(cuts, dtype=np.float64).reshape(-1, 6))
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = x.shape[0] if r is None else r.shape[0]
    keep = np.ones(idx.shape[0], dtype=np.uint8)
    if cuts.shape[0] and idx.shape[0]:
        lib().or_apply_cuts(x.ctypes.data, _p(r), nrows, off.ctypes.data, idx.ctypes.data,
                            cuts.ctypes.data, cuts.shape[0], keep.ctypes.data)
    return keep


def cut_family(coords, delta, cuts, rows=None, method="cells"):
    """Family after the initial notch removal (Section 6)."""
    off, idx = family(coords, delta, rows, method)
    keep = cut_keep(coords, off, idx, cuts, rows)
    if keep.all():
        return off, idx
    cum = np.zeros(idx.shape[0] + 1, dtype=np.int64)
    np.cumsum(keep, out=cum[1:])
    return cum[off], idx[keep.astype(bool)]


CONICAL, SURFACE, PARTIAL = 1, 2, 4


def stiffness_factors(coords, volumes, delta, off, idx, flags, v0=0.0, dx=0.0):
    """Per family entry factors multiplying c: conical micromodulus (bit 1), the
    volume surface correction 2 V0 / (V_i + V_j) (bit 2) and the linear partial
    volume with lattice spacing dx (bit 4); see oracle.c."""
    x = _c64(coords)
    vol = _c64(volumes)
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    nrows = off.shape[0] - 1
    # rows are nodes 0..nrows-1; the volume correction needs every node as a row
    assert nrows <= x.shape[0] and (not flags & SURFACE or nrows == x.shape[0])
    out = np.zeros(max(idx.shape[0], 1))
    lib().or_stiffness_factors2(x.ctypes.data, vol.ctypes.data, nrows, delta,
                                off.ctypes.data, idx.ctypes.data, int(flags), float(v0),
                                float(dx), out.ctypes.data)
    return out[: idx.shape[0]]


class Model:
    """Arguments of the oracle step, kept alive for the C side."""

    def __init__(self, coords, volumes, off, idx, *, c, sc=None, sc_hash=None,
                 c_bond=None, no_fail=None, bc_type=None, bc_disp=None, bc_force=None,
                 disp_rate=0.0, load=0.0, dt=1e-7, damping=0.0, density=1.0, rows=None,
                 ramp_steps=0, kr=0.0, state_based=None, trilinear=None):
        self.x = _c64(coords)
        n = self.x.shape[0]
        self.vol = _c64(volumes)
        self.rows = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.idx = np.ascontiguousarray(idx, dtype=np.int32)
        self.c_bond = None if c_bond is None else _c64(c_bond)
        self.no_fail = None if no_fail is None else np.ascontiguousarray(no_fail, np.uint8)
        self.bc_type = (np.zeros((n, 3), np.uint8) if bc_type is None
                        else np.ascontiguousarray(bc_type, np.uint8))
        self.bc_disp = np.zeros((n, 3)) if bc_disp is None else _c64(bc_disp)
        self.bc_force = None if bc_force is None else _c64(bc_force)
        m = _Model()
        m.n = n
        m.x = self.x.ctypes.data
        m.vol = self.vol.ctypes.data
        m.rows = _p(self.rows)
        m.nrows = n if self.rows is None else self.rows.shape[0]
        m.off = self.off.ctypes.data
        m.idx = self.idx.ctypes.data
        m.c = float(c)
        m.c_bond = _p(self.c_bond)
        if sc_hash is not None:
            m.sc_mode = 1
            m.sc_seed, m.sc_lo, m.sc_hi = int(sc_hash[0]), float(sc_hash[1]), float(sc_hash[2])
            m.sc = 0.0
        else:
            m.sc_mode = 0
            m.sc = float(sc)
        m.no_fail = _p(self.no_fail)
        m.bc_type = self.bc_type.ctypes.data
        m.bc_disp = self.bc_disp.ctypes.data
        m.bc_force = _p(self.bc_force)
        m.disp_rate, m.load = float(disp_rate), float(load)
        m.dt, m.damping, m.density = float(dt), float(damping), float(density)
        m.ramp_steps = int(ramp_steps)
        # bilinear softening (kr > 1): the largest stretch of each family entry
        self.kappa = np.zeros(max(int(self.off[-1]), 1))
        m.kr = float(kr)
        m.kappa = self.kappa.ctypes.data
        if trilinear is not None:  # (k1 = s_1 / s_0, beta = kink force / peak force)
            m.k1, m.beta = float(trilinear[0]), float(trilinear[1])
        # ordinary state-based linear solid: state_based = (K, G); all nodes are rows
        self.wvol = np.zeros(n)
        self.theta = np.zeros(n)
        m.wvol = self.wvol.ctypes.data
        m.theta = self.theta.ctypes.data
        if state_based is not None:
            assert self.rows is None
            m.model = 1
            m.K, m.G = float(state_based[0]), float(state_based[1])
        self.m = m
        if state_based is not None:
            lib().or_osb_weighted_volume(ctypes.byref(m), self.wvol.ctypes.data)
        self.nrows = m.nrows
        self.nbonds = int(self.off[-1])

    @classmethod
    def from_workload(cls, w, off, idx, c=None, rows=None, c_bond=None):
        if c is None:
            c = micromodulus(w.bulk_modulus, w.horizon)
        return cls(w.coords, w.volumes, off, idx, c=c, sc=w.sc, sc_hash=w.sc_hash,
                   c_bond=c_bond, no_fail=w.no_fail, bc_type=w.bc_type, bc_disp=w.bc_disp,
                   bc_force=w.bc_force, disp_rate=w.disp_rate, load=w.load, dt=w.dt,
                   damping=w.damping, density=w.density, rows=rows,
                   ramp_steps=getattr(w, "ramp_steps", 0), kr=getattr(w, "kr", 0.0),
                   state_based=getattr(w, "state_based", None),
                   trilinear=getattr(w, "trilinear", None))

    def step(self, step_index, u, v, mu, margin=None, want_force=False):
        """One step; returns (u_out, v_out[, F]) per row.  mu/margin updated in place."""
        u = _c64(u)
        v = _c64(v)
        uo = np.empty((self.nrows, 3))
        vo = np.empty((self.nrows, 3))
        F = np.empty((self.nrows, 3)) if want_force else None
        lib().or_step(ctypes.byref(self.m), int(step_index), u.ctypes.data, v.ctypes.data,
                      mu.ctypes.data, _p(margin), uo.ctypes.data, vo.ctypes.data, _p(F))
        return (uo, vo, F) if want_force else (uo, vo)

    def run(self, first_step, nsteps, u, v, mu, margin=None):
        """``nsteps`` steps over all nodes; u, v, mu (and margin) updated in place."""
        assert self.rows is None
        assert u.dtype == np.float64 and u.flags.c_contiguous
        assert v.dtype == np.float64 and v.flags.c_contiguous
        lib().or_run(ctypes.byref(self.m), int(first_step), int(nsteps), u.ctypes.data,
                     v.ctypes.data, mu.ctypes.data, _p(margin))

    def run_vv(self, first_step, nsteps, u, v, a, mu, init=False, margin=None):
        """Damped velocity-Verlet steps over all nodes (see oracle.c); u, v, a
        (acceleration) and mu updated in place.  init: form a^0 from (u, v) first."""
        assert self.rows is None
        for arr in (u, v, a):
            assert arr.dtype == np.float64 and arr.flags.c_contiguous
        lib().or_run_vv(ctypes.byref(self.m), int(first_step), int(nsteps), int(bool(init)),
                        u.ctypes.data, v.ctypes.data, a.ctypes.data, mu.ctypes.data, _p(margin))

    def damage(self, mu):
        phi = np.empty(self.nrows)
        lib().or_damage(ctypes.byref(self.m), mu.ctypes.data, phi.ctypes.data)
        return phi

    def energy_density(self, u, mu):
        u = _c64(u)
        W = np.empty(self.nrows)
        lib().or_energy_density(ctypes.byref(self.m), u.ctypes.data, mu.ctypes.data,
                                W.ctypes.data)
        return W

    def fresh_bonds(self):
        return np.ones(self.nbonds, dtype=np.uint8)


def _adjoint_sig():
    L = lib()
    if not getattr(L, "_adj_ready", False):
        P = ctypes.c_void_p
        L.or_adjoint.restype = None
        L.or_adjoint.argtypes = [ctypes.POINTER(_Model), ctypes.c_int64, ctypes.c_int64,
                                 P, P, P, P, P, P, P, P, P]
        L.or_adjoint_vv.restype = None
        L.or_adjoint_vv.argtypes = L.or_adjoint.argtypes
        L._adj_ready = True
    return L


def adjoint(model: "Model", first_step, nsteps, u0, v0, mu, dLdu, dLdv=None,
            integrator="ec"):
    """Reverse-mode gradient of L(u^N, v^N) with frozen bond flags mu (see oracle.c):
    of the damped Euler-Cromer run (integrator "ec") or of the damped
    velocity-Verlet run started from (u0, v0) with its acceleration formed
    afresh (integrator "vv", or_run_vv with init).

    Returns (dL/dc per family entry, dL/dload, dL/du0, dL/dv0)."""
    assert model.rows is None
    assert integrator in ("ec", "vv")
    L = _adjoint_sig()
    fn = L.or_adjoint if integrator == "ec" else L.or_adjoint_vv
    u0 = _c64(u0); v0 = _c64(v0); dLdu = _c64(dLdu)
    dLdv = None if dLdv is None else _c64(dLdv)
    mu = np.ascontiguousarray(mu, np.uint8)
    gc = np.zeros(max(model.nbonds, 1))
    gl = ctypes.c_double()
    gu = np.empty_like(u0); gv = np.empty_like(v0)
    fn(ctypes.byref(model.m), int(first_step), int(nsteps), u0.ctypes.data,
       v0.ctypes.data, mu.ctypes.data, dLdu.ctypes.data, _p(dLdv), gc.ctypes.data,
       ctypes.byref(gl), gu.ctypes.data, gv.ctypes.data)
    return gc[: model.nbonds], gl.value, gu, gv
