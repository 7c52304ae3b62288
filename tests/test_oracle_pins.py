"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints, a closed form, an invariant, brute force, or an exact-rational
recurrence.  The expected values are computed here from integer lattice
enumeration or exact fractions, never by re-calling the oracle's formula.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = v
    return out


def _offsets(r):
    """Integer lattice offsets o != 0 with |o| <= r (enumerated, no oracle)."""
    R = int(math.floor(r))
    out = []
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for c in range(-R, R + 1):
                if (a, b, c) != (0, 0, 0) and a * a + b * b + c * c <= r * r:
                    out.append((a, b, c))
    return out


# ---------------------------------------------------------------- Eq. (5)
def test_micromodulus_matches_printed_worked_value():
    g = _read_golden("micromodulus_concrete.txt")
    E, nu, delta = float(g["E_Pa"]), float(g["nu"]), float(g["delta_m"])
    K = E / (3.0 * (1.0 - 2.0 * nu))
    c = oracle.micromodulus(K, delta)
    # Printed with three significant figures; 2.326e18 truncates to 2.32e18.
    # A wrong constant, power of delta or missing pi is off by far more than 0.5 %.
    assert abs(c / float(g["c_printed"]) - 1.0) < 5e-3


def _center_energy_ratio(r_over_dx, eps=1e-4, K=1e9, dx=1e-3):
    R = int(math.floor(r_over_dx))
    m = 2 * R + 3
    x = workloads.lattice(m, m, m, dx)
    center = np.array([(m // 2 * m + m // 2) * m + m // 2], dtype=np.int64)
    delta = r_over_dx * dx
    off, idx = oracle.family(x, delta, rows=center)
    c = oracle.micromodulus(K, delta)
    mdl = oracle.Model(x, np.full(x.shape[0], dx ** 3), off, idx, c=c, sc=1.0, rows=center)
    u = eps * x
    W = mdl.energy_density(u, mdl.fresh_bonds())[0]
    return W / (4.5 * K * eps * eps), len(idx)


def test_bulk_response_lattice_quadrature_ratio():
    # Uniform dilation u = eps X: every bond has s = eps, so the interior energy
    # density is 1/4 c eps^2 dx^4 sum|o|, while the continuum identity behind
    # Eq. (5) gives 9/2 K eps^2.  Their ratio is sum|o| / (pi r^4), r = delta/dx.
    for r in (3.01, math.pi):
        offs = _offsets(r)
        expect = sum(math.sqrt(a * a + b * b + c * c) for a, b, c in offs) / (math.pi * r ** 4)
        ratio, nfam = _center_energy_ratio(r)
        assert nfam == len(offs) == 122
        assert abs(ratio / expect - 1.0) < 1e-9
    assert abs(expect - 0.93204) < 1e-4  # delta = pi dx


def test_bulk_response_tends_to_continuum():
    # For a large horizon-to-spacing ratio the lattice sum approaches the
    # integral, so the energy density tends to 9/2 K eps^2: this pins the
    # 18/pi constant of Eq. (5) independently of any lattice bookkeeping.
    ratio, _ = _center_energy_ratio(12.01)
    assert abs(ratio - 1.0) < 0.03


# ---------------------------------------------------------------- Eq. (9)
def test_family_bruteforce_equals_cell_grid():
    x = workloads.lattice(9, 7, 6, 1e-3, jitter=0.25, seed=3)
    for delta in (1.5e-3, 2.6e-3, 3.01e-3):
        o1, i1 = oracle.family(x, delta, method="brute")
        o2, i2 = oracle.family(x, delta, method="cells")
        assert np.array_equal(o1, o2) and np.array_equal(i1, i2)
        # symmetric, self-excluded, ascending
        pairs = set()
        for i in range(x.shape[0]):
            row = i1[o1[i]:o1[i + 1]]
            assert np.all(np.diff(row) > 0) and i not in row
            pairs.update((i, int(j)) for j in row)
        assert all((j, i) in pairs for i, j in pairs)


def test_family_counts_match_lattice_enumeration():
    nx, ny, nz = 40, 10, 10
    x = workloads.lattice(nx, ny, nz, 1e-3)
    off, idx = oracle.family(x, 3.01e-3)
    offs = _offsets(3.01)
    total = sum(max(0, nx - abs(a)) * max(0, ny - abs(b)) * max(0, nz - abs(c))
                for a, b, c in offs)
    assert total == 370728
    assert int(off[-1]) == total
    cnt = np.diff(off).reshape(nx, ny, nz)
    assert np.all(cnt[3:-3, 3:-3, 3:-3] == 122)
    assert cnt.max() == 122


# ---------------------------------------------------------------- Eqs. (4)-(5), (10)
def _small_model(seed=0, jitter=0.2, sc=1.0, **kw):
    x = workloads.lattice(8, 7, 6, 1e-3, jitter=jitter, seed=seed)
    delta = 3.01e-3
    off, idx = oracle.family(x, delta)
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0.5, 1.5, x.shape[0]) * 1e-9
    c = oracle.micromodulus(3e10, delta)
    return x, vol, off, idx, oracle.Model(x, vol, off, idx, c=c, sc=sc, **kw)


def test_rigid_translation_gives_zero_force():
    x, vol, off, idx, mdl = _small_model(sc=1e-12)
    u = np.tile(np.array([[3e-4, -2e-4, 1e-4]]), (x.shape[0], 1))
    mu = mdl.fresh_bonds()
    _, _, F = mdl.step(0, u, np.zeros_like(u), mu, want_force=True)
    assert np.all(F == 0.0)
    assert mu.all()  # s = 0 exactly, nothing reaches s_c


def test_rigid_rotation_gives_no_force_and_no_break():
    x, vol, off, idx, mdl = _small_model(sc=1e-9)
    th = 0.5
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    u = x @ R.T - x
    mu = mdl.fresh_bonds()
    _, _, F = mdl.step(0, u, np.zeros_like(u), mu, want_force=True)
    scale = mdl.m.c * vol.mean() * 3.01e-3  # one bond at unit stretch
    assert np.abs(F).max() < 1e-10 * scale
    assert mu.all()


def test_pairwise_forces_are_antisymmetric():
    x, vol, off, idx, mdl = _small_model()
    u, _ = workloads.random_state(x.shape[0], 5, 1e-6, 0.0)
    _, _, F = mdl.step(0, u, np.zeros_like(u), mdl.fresh_bonds(), want_force=True)
    net = (vol[:, None] * F).sum(axis=0)
    gross = (vol[:, None] * np.abs(F)).sum(axis=0)
    assert np.all(np.abs(net) < 1e-12 * gross)


def test_momentum_decays_by_damping_factor():
    x, vol, off, idx, mdl = _small_model(damping=2.5e6, density=2400.0, dt=1e-7)
    u, v = workloads.random_state(x.shape[0], 9, 1e-6, 1e-2)
    mu = mdl.fresh_bonds()
    rho = 2400.0
    P0 = (rho * vol[:, None] * v).sum(axis=0)
    mdl.run(0, 50, u, v, mu)
    P = (rho * vol[:, None] * v).sum(axis=0)
    factor = (1.0 - 1e-7 * 2.5e6 / rho) ** 50
    gross = (rho * vol[:, None] * np.abs(v)).sum(axis=0)
    assert np.all(np.abs(P - factor * P0) < 1e-11 * gross)


def test_force_is_minus_energy_gradient():
    # f = dw/deta (Eq. 2) with w = c s^2 |xi| / 2 (Eq. 4): V_i F_i = -dE/du_i,
    # E = sum_i V_i W_i.  Central differences in FP64.
    x, vol, off, idx, mdl = _small_model(seed=1)
    u, _ = workloads.random_state(x.shape[0], 2, 2e-6, 0.0)
    mu = mdl.fresh_bonds()
    _, _, F = mdl.step(0, u, np.zeros_like(u), mu.copy(), want_force=True)
    rng = np.random.default_rng(4)
    h = 1e-9
    for i in rng.choice(x.shape[0], 6, replace=False):
        for a in range(3):
            up = u.copy(); up[i, a] += h
            um = u.copy(); um[i, a] -= h
            Ep = (vol * mdl.energy_density(up, mu)).sum()
            Em = (vol * mdl.energy_density(um, mu)).sum()
            g = -(Ep - Em) / (2 * h)
            assert abs(g - vol[i] * F[i, a]) < 1e-5 * abs(vol[i]) * np.abs(F[i]).max() + 1e-30


def _two_nodes(L=1.0, **kw):
    x = np.array([[0.0, 0.0, 0.0], [L, 0.0, 0.0]])
    off = np.array([0, 1, 2], dtype=np.int64)
    idx = np.array([1, 0], dtype=np.int32)
    return x, off, idx


def test_two_node_euler_cromer_matches_exact_recurrence():
    # Node 0 is held at u = 0; node 1 starts displaced by a along the bond.
    # With s = u/L the scalar force on node 1 is -(c V / L) u, so the damped
    # Euler-Cromer reading is a linear recurrence, iterated here in exact rationals.
    L, c, V, rho, eta, dt, a = 1.0, 3.0, 2.0, 5.0, 0.7, 0.05, 1e-3
    x, off, idx = _two_nodes(L)
    bt = np.zeros((2, 3), np.uint8); bt[0, :] = 1
    mdl = oracle.Model(x, np.array([V, V]), off, idx, c=c, sc=1.0, bc_type=bt,
                       disp_rate=0.0, dt=dt, damping=eta, density=rho)
    u = np.zeros((2, 3)); u[1, 0] = a
    v = np.zeros((2, 3))
    mu = mdl.fresh_bonds()
    k = Fraction(c) * Fraction(V) / Fraction(L)
    fr, fe, fd = Fraction(rho), Fraction(eta), Fraction(dt)
    uq, vq = Fraction(a), Fraction(0)
    for n in range(200):
        u, v = mdl.step(n, u, v, mu)
        vq = vq + fd * (-k * uq - fe * vq) / fr
        uq = uq + fd * vq
        assert abs(u[1, 0] - float(uq)) <= 1e-12 * a
        assert abs(v[1, 0] - float(vq)) <= 1e-12 * a / dt
    assert np.all(u[0] == 0.0) and np.all(u[1, 1:] == 0.0)


def test_two_node_break_step_is_analytic_and_force_free():
    # Both ends prescribed at -/+ r per step: at step n the bond sees s = 2 r n / L,
    # so it breaks at the first n with s >= s_c: n* = ceil(s_c L / (2 r)).
    L, r, sc = 1.0, 1e-3, 0.0105
    x, off, idx = _two_nodes(L)
    bt = np.ones((2, 3), np.uint8)
    g = np.zeros((2, 3)); g[0, 0] = -r; g[1, 0] = r
    mdl = oracle.Model(x, np.ones(2), off, idx, c=1.0, sc=sc, bc_type=bt, bc_disp=g,
                       disp_rate=1.0, dt=1.0, damping=0.0, density=1.0)
    u = np.zeros((2, 3)); v = np.zeros((2, 3))
    mu = mdl.fresh_bonds()
    nstar = math.ceil(sc * L / (2 * r))
    for n in range(10):
        _, _, F = mdl.step(n, u, v, mu, want_force=True)
        if n < nstar:
            assert mu.all() and (F[1, 0] < 0.0 or n == 0)  # intact bond pulls node 1 back
        else:
            assert not mu.any() and np.all(F == 0.0)  # broken in the same step
        u, v = mdl.step(n, u, v, mu.copy())
        assert u[1, 0] == pytest.approx(r * (n + 1), rel=1e-15)
        assert v[1, 0] == pytest.approx(r, rel=1e-12)


def test_compressed_bond_never_breaks():
    L = 1.0
    x, off, idx = _two_nodes(L)
    bt = np.ones((2, 3), np.uint8)
    g = np.zeros((2, 3)); g[0, 0] = 0.01; g[1, 0] = -0.01
    mdl = oracle.Model(x, np.ones(2), off, idx, c=1.0, sc=1e-3, bc_type=bt, bc_disp=g,
                       disp_rate=1.0, dt=1.0, density=1.0)
    u = np.zeros((2, 3)); v = np.zeros((2, 3)); mu = mdl.fresh_bonds()
    for n in range(20):
        u, v = mdl.step(n, u, v, mu)
    assert mu.all()


# ---------------------------------------------------------------- Eq. (8)
def test_damage_next_to_full_planar_cut_equals_offset_fraction():
    m = 14
    dx = 1.0
    x = workloads.lattice(m, m, m, dx)
    delta = 3.01
    off, idx = oracle.family(x, delta)
    plane = 6.5
    cut = [(0, plane, -1.0, m + 1.0, -1.0, m + 1.0)]
    mu = 1 - (1 - oracle.cut_keep(x, off, idx, cut))  # intact = not crossing
    mdl = oracle.Model(x, np.ones(x.shape[0]), off, idx, c=1.0, sc=1.0)
    phi = mdl.damage(mu.astype(np.uint8))
    offs = _offsets(3.01)
    for ix, dist in ((6, 1), (5, 2), (4, 3), (7, 1), (8, 2)):
        i = (ix * m + 7) * m + 7
        k = dist  # crossing offsets: o_x >= k toward the plane
        cross = sum(1 for a, b, c in offs if (a >= k if ix < plane else -a >= k))
        assert phi[i] == pytest.approx(cross / 122.0, abs=1e-15)
    assert phi[(3 * m + 7) * m + 7] == 0.0


def test_damage_is_zero_at_start_bounded_and_monotone():
    w = workloads.tensile_bar(20, 6, 6, rate=2e-6, steps=120)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    mdl = oracle.Model.from_workload(w, off, idx)
    u = np.zeros((w.n, 3)); v = np.zeros((w.n, 3)); mu = mdl.fresh_bonds()
    prev = mdl.damage(mu)
    assert np.all(prev == 0.0)
    for k in range(0, w.steps, 10):
        mdl.run(k, 10, u, v, mu)
        phi = mdl.damage(mu)
        assert np.all(phi >= prev) and np.all(phi <= 1.0) and np.all(phi >= 0.0)
        prev = phi
    assert prev.max() > 0.0  # the pulled bar does crack


def test_displacement_bc_follows_ramp():
    w = workloads.tensile_bar(12, 5, 5, rate=1e-7, steps=5)
    off, idx = oracle.family(w.coords, w.horizon)
    mdl = oracle.Model.from_workload(w, off, idx)
    u = np.zeros((w.n, 3)); v = np.zeros((w.n, 3)); mu = mdl.fresh_bonds()
    mdl.run(0, 5, u, v, mu)
    ctl = w.bc_type[:, 0] == 1
    assert np.allclose(u[ctl, 0], w.bc_disp[ctl, 0] * 5, rtol=1e-15, atol=0)
    assert np.allclose(v[ctl, 0], w.bc_disp[ctl, 0] / w.dt, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- notch rule
def test_cut_crossing_predicate():
    cut = np.array([0, 0.5, 0.0, 1.0, 0.0, 2.0])

    def P(a, b):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        return oracle.lib().or_cut_crosses(a.ctypes.data, b.ctypes.data, cut.ctypes.data)
    assert P([0, 0.5, 1], [1, 0.5, 1]) == 1
    assert P([1, 0.5, 1], [0, 0.5, 1]) == 1          # symmetric
    assert P([0, 0.5, 1], [0.4, 0.5, 1]) == 0        # does not reach the plane
    assert P([0, 0.5, 2.5], [1, 0.5, 2.5]) == 0      # outside the rectangle (z)
    assert P([0, 1.5, 1], [1, 1.5, 1]) == 0          # outside the rectangle (y)
    assert P([0, 0.0, 0.0], [1, 1.0, 2.0]) == 1      # oblique, crosses at (0.5, 0.5, 1)


# ---------------------------------------------------------------- SplitMix64 draw
@pytest.mark.parametrize("kind,nu", [("3d", 0.25), ("plane_stress", 1.0 / 3.0),
                                     ("plane_strain", 0.25)])
def test_critical_stretch_equals_fracture_energy_integral(kind, nu):
    # Eq. 7 against its derivation (Silling & Askari 2005), both integrals by
    # quadrature: the micromodulus is fixed by equating the peridynamic energy
    # density under a uniform isotropic strain with the classical one (the
    # bond-based Poisson ratio: 1/4 in 3D and plane strain, 1/3 in plane
    # stress), and G_F is the energy of every bond crossing a unit fracture area
    # when each bond is stretched to s_c (micropotential c s^2 xi / 2).
    from scipy import integrate
    delta, E, G = 0.0157, 37e9, 120.0
    if kind == "3d":
        W = E / (2.0 * (1.0 - 2.0 * nu)) * 3.0           # (9/2) K with K = E / (3 (1 - 2 nu))
        shell = integrate.quad(lambda x: 0.5 * (x / 2.0) * 4.0 * math.pi * x * x, 0, delta,
                               epsabs=0, epsrel=1e-13)[0]
        c = W / shell
        I = integrate.tplquad(lambda ph, x, z: (x / 2.0) * 2.0 * math.pi * x * x * math.sin(ph),
                              0, delta, lambda z: z, lambda z: delta,
                              lambda z, x: 0.0, lambda z, x: math.acos(min(1.0, z / x)),
                              epsabs=0, epsrel=1e-11)[0]
    else:
        # thickness t enters c as 1/t and the crack area as t: work with c t
        W = E / (1.0 - nu) if kind == "plane_stress" else E / ((1.0 + nu) * (1.0 - 2.0 * nu))
        ring = integrate.quad(lambda x: 0.5 * (x / 2.0) * 2.0 * math.pi * x, 0, delta,
                              epsabs=0, epsrel=1e-13)[0]
        c = W / ring
        I = integrate.tplquad(lambda ph, x, z: (x / 2.0) * x,
                              0, delta, lambda z: z, lambda z: delta,
                              lambda z, x: -math.acos(min(1.0, z / x)),
                              lambda z, x: math.acos(min(1.0, z / x)),
                              epsabs=0, epsrel=1e-11)[0]
    expect = math.sqrt(G / (c * I))
    got = oracle.critical_stretch(G, E, delta, kind)
    assert abs(got - expect) <= 1e-8 * expect, (got, expect)


def test_youngs_modulus_from_lame_parameters():
    # E = 3 K (1 - 2 nu) against E, K and nu written from the Lame parameters
    for lam, mu in [(1.0e9, 2.0e9), (3.0e10, 1.2e10), (5.0, 5.0)]:
        K = lam + 2.0 * mu / 3.0
        nu = lam / (2.0 * (lam + mu))
        E = mu * (3.0 * lam + 2.0 * mu) / (lam + mu)
        assert abs(oracle.youngs_modulus(K, nu) - E) <= 1e-12 * E


def test_splitmix64_reference_outputs():
    lines = [l.split() for l in open(os.path.join(GOLD, "splitmix64_seed1234567.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    for m, val in lines[1:]:
        assert oracle.splitmix64(seed, int(m)) == int(val)


def test_per_bond_critical_stretch_draw():
    lo, hi = 9e-5, 1.1e-4
    rng = np.random.default_rng(0)
    pairs = rng.integers(0, 1 << 30, size=(4000, 2))
    vals = np.array([oracle.sc_bond(7, lo, hi, int(a), int(b)) for a, b in pairs])
    sym = np.array([oracle.sc_bond(7, lo, hi, int(b), int(a)) for a, b in pairs])
    assert np.array_equal(vals, sym)
    assert vals.min() >= lo and vals.max() < hi
    # uniform on [lo, hi): mean and variance within 5 standard errors
    w = hi - lo
    assert abs(vals.mean() - (lo + hi) / 2) < 5 * w / math.sqrt(12 * len(vals))
    assert abs(vals.var() / (w * w / 12) - 1) < 0.1


def test_break_threshold_is_inclusive():
    # Eq. (6): mu = 1 only for s < s_c, so a bond breaks when s reaches s_c.
    # With L = 1 and ends at -/+ 0.125 n the stretch 0.25 n is exact in binary.
    L = 1.0
    x, off, idx = _two_nodes(L)
    bt = np.ones((2, 3), np.uint8)
    g = np.zeros((2, 3)); g[0, 0] = -0.125; g[1, 0] = 0.125
    mdl = oracle.Model(x, np.ones(2), off, idx, c=1.0, sc=0.5, bc_type=bt, bc_disp=g,
                       disp_rate=1.0, dt=1.0, density=1.0)
    u = np.zeros((2, 3)); v = np.zeros((2, 3)); mu = mdl.fresh_bonds()
    u, v = mdl.step(0, u, v, mu)
    u, v = mdl.step(1, u, v, mu)
    assert mu.all()                     # s = 0.25 at step 1
    mdl.step(2, u, v, mu)               # s = 0.5 == s_c at step 2
    assert not mu.any()


def test_family_boundary_is_inclusive():
    # Eq. (9) uses |x_i - x_j| <= delta: with integer coordinates and delta = 2
    # the offsets of length exactly 2 belong to the family (32 offsets, not 26).
    x = workloads.lattice(9, 9, 9, 1.0)
    center = np.array([(4 * 9 + 4) * 9 + 4], dtype=np.int64)
    for method in ("brute", "cells"):
        off, idx = oracle.family(x, 2.0, rows=center, method=method)
        assert len(idx) == len(_offsets(2.0)) == 32


# ------------------------------------------- Eq. (8) with unequal volumes
def test_damage_weights_neighbours_by_their_volume():
    # A star: node 0 bonded to nodes 1..4 (and each of them to node 0 only),
    # with unequal volumes.  Eq. (8) weights each bond of the family by the
    # neighbour's volume V_j, so with bonds 0-2 and 0-4 broken
    #   phi_0 = 1 - (V_1 + V_3) / (V_1 + V_2 + V_3 + V_4),
    # while node 2 (its only bond broken) has phi = 1 and node 1 has phi = 0.
    # An unweighted count (1 - 2/4) or the owner's volume in place of V_j
    # gives 0.5 for node 0 instead.
    V = [Fraction(5, 4), Fraction(1, 2), Fraction(2), Fraction(3), Fraction(7)]
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0],
                  [0.0, 0.0, 1.0], [-1.0, 0.0, 0.0]])
    off = np.array([0, 4, 5, 6, 7, 8], dtype=np.int64)
    idx = np.array([1, 2, 3, 4, 0, 0, 0, 0], dtype=np.int32)
    mdl = oracle.Model(x, np.array([float(a) for a in V]), off, idx, c=1.0, sc=1.0)
    mu = np.array([1, 0, 1, 0, 1, 0, 1, 0], dtype=np.uint8)  # both directions of 0-2, 0-4
    phi = mdl.damage(mu)
    expect0 = 1 - (V[1] + V[3]) / (V[1] + V[2] + V[3] + V[4])
    assert expect0 == Fraction(18, 25)
    assert phi[0] == pytest.approx(float(expect0), abs=1e-15)
    assert phi[1] == 0.0 and phi[3] == 0.0
    assert phi[2] == 1.0 and phi[4] == 1.0
    # a partly broken family of a node whose neighbours differ only in volume:
    # node 0 keeps the bond to the heaviest neighbour only
    mu2 = np.array([0, 0, 0, 1, 1, 1, 1, 1], dtype=np.uint8)
    phi2 = mdl.damage(mu2)
    assert phi2[0] == pytest.approx(float(1 - V[4] / (V[1] + V[2] + V[3] + V[4])), abs=1e-15)


# ------------------------------------------------- no-fail nodes (Section 6)
@pytest.mark.parametrize("flagged", [0, 1])
def test_no_fail_flag_on_either_end_keeps_bond(flagged):
    # A bond with one end in a no-fail zone never breaks, whichever end carries
    # the flag: both directions of the pair stay intact past s_c, and the bond
    # keeps pulling the ends together with c s V_j (as in the two-node
    # recurrence).  Without the flag the same motion breaks it at
    # n* = ceil(s_c L / (2 r)).
    L, r, sc = 1.0, 1e-3, 0.0105
    x, off, idx = _two_nodes(L)
    bt = np.ones((2, 3), np.uint8)
    g = np.zeros((2, 3)); g[0, 0] = -r; g[1, 0] = r
    nf = np.zeros(2, np.uint8); nf[flagged] = 1
    nstar = math.ceil(sc * L / (2 * r))
    for flags in (nf, None):
        mdl = oracle.Model(x, np.array([2.0, 3.0]), off, idx, c=1.5, sc=sc, bc_type=bt,
                           bc_disp=g, disp_rate=1.0, dt=1.0, damping=0.0, density=1.0,
                           no_fail=flags)
        u = np.zeros((2, 3)); v = np.zeros((2, 3)); mu = mdl.fresh_bonds()
        for n in range(nstar + 5):
            _, _, F = mdl.step(n, u, v, mu, want_force=True)
            u = np.array([[-r * n, 0, 0], [r * n, 0, 0]], dtype=float)
            s = 2 * r * n / L
            if flags is not None or n < nstar:
                assert mu[0] == 1 and mu[1] == 1
                # force density on node 0 (+x toward node 1) and node 1 (-x)
                assert F[0, 0] == pytest.approx(1.5 * s * 3.0, rel=1e-12, abs=1e-300)
                assert F[1, 0] == pytest.approx(-1.5 * s * 2.0, rel=1e-12, abs=1e-300)
            else:
                assert mu[0] == 0 and mu[1] == 0
                assert np.all(F == 0.0)
            u, v = mdl.step(n, u, v, mu.copy())


# ------------------------------------- body force in Eqs. (10)-(11)
@pytest.mark.parametrize("state_based", [None, (2.0, 1.0)])
def test_body_force_drives_free_node_by_exact_recurrence(state_based):
    # A node with no bonds feels only the body force load * b_i (Eq. 11: the
    # force density it adds to the internal force of Eq. 10).  Under the damped
    # Euler-Cromer reading its velocity and displacement follow
    #   v <- v + dt (load b - eta v) / rho,   u <- u + dt v,
    # iterated here in exact rationals per component.  A flipped sign, a
    # missing load factor or a force divided by the volume fails this.
    b = [Fraction(3, 2), Fraction(-5, 4), Fraction(1, 8)]
    load, rho, eta, dt, V = Fraction(7, 2), Fraction(5), Fraction(3, 4), Fraction(1, 16), 2.5
    x = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0]])
    off = np.array([0, 0, 0], dtype=np.int64)
    idx = np.zeros(0, dtype=np.int32)
    bf = np.zeros((2, 3)); bf[0] = [float(t) for t in b]
    mdl = oracle.Model(x, np.array([V, V]), off, idx, c=1.0, sc=1.0, bc_force=bf,
                       load=float(load), dt=float(dt), damping=float(eta),
                       density=float(rho), state_based=state_based)
    u = np.zeros((2, 3)); v = np.zeros((2, 3)); mu = np.ones(1, np.uint8)
    uq = [Fraction(0)] * 3
    vq = [Fraction(0)] * 3
    for n in range(240):
        _, _, F = mdl.step(n, u, v, mu, want_force=True)
        for a in range(3):
            assert F[0, a] == float(load * b[a])
        u, v = mdl.step(n, u, v, mu)
        for a in range(3):
            vq[a] = vq[a] + dt * (load * b[a] - eta * vq[a]) / rho
            uq[a] = uq[a] + dt * vq[a]
            assert u[0, a] == pytest.approx(float(uq[a]), rel=1e-13, abs=1e-300)
            assert v[0, a] == pytest.approx(float(vq[a]), rel=1e-13, abs=1e-300)
        assert np.all(u[1] == 0.0) and np.all(v[1] == 0.0)
    # approaching the steady velocity the damping admits, load b / eta
    # (15 time units = 2.25 relaxation times rho / eta)
    for a in range(3):
        assert float(vq[a]) == pytest.approx(float(load * b[a] / eta), rel=0.2)
