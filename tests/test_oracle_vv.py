"""Pins of the oracle's damped velocity-Verlet integrator and smooth loading
ramp (Section 3.6 "Time integration"; Sections 5-6 loading), CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_smooth_ramp_closed_form_and_continuation():
    r, T = 2.5e-8, 40
    # P(1/2) = 1/16 - 3/160 = 7/160
    assert oracle.scale(r, T, T // 2) == pytest.approx(r * T * 7 / 160, rel=1e-14)
    assert oracle.scale(r, T, 0) == 0.0
    for k in (T, T + 1, 3 * T):
        assert oracle.scale(r, T, k) == pytest.approx(r * (k - 0.6 * T), rel=1e-14)
    s = np.array([oracle.scale(r, T, k) for k in range(2 * T)])
    vel, acc = np.diff(s), np.diff(s, 2)
    # starts at rest with zero acceleration, ends on the steady rate r with zero acceleration
    # (discrete: the first increments are O(r / T^2), the second difference
    # across the junction O(r / T^2) against r / T in mid-ramp)
    assert vel[0] < r / T ** 2 and acc[0] < r / T ** 2
    assert abs(vel[T] - r) < 1e-12 * r and abs(acc[T - 1]) < 0.1 * r / T
    assert acc[T // 2] > 0.5 * r / T
    assert oracle.scale(r, 0, 7) == 7 * r


def _two_nodes(L=1.0):
    x = np.array([[0.0, 0.0, 0.0], [L, 0.0, 0.0]])
    return x, np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32)


def test_two_node_velocity_verlet_matches_exact_recurrence():
    # node 0 held; the bond force on node 1 is -(c V / L) u: a linear oscillator,
    # the damped velocity-Verlet recurrence iterated in exact rationals
    L, c, V, rho, eta, dt, a0 = 1.0, 3.0, 2.0, 5.0, 0.75, 0.0625, 1e-3
    x, off, idx = _two_nodes(L)
    bt = np.zeros((2, 3), np.uint8); bt[0, :] = 1
    mdl = oracle.Model(x, np.array([V, V]), off, idx, c=c, sc=1.0, bc_type=bt, dt=dt,
                       damping=eta, density=rho)
    u = np.zeros((2, 3)); u[1, 0] = a0
    v = np.zeros((2, 3)); acc = np.zeros((2, 3))
    mu = mdl.fresh_bonds()
    k = Fraction(c) * Fraction(V) / Fraction(L)
    fr, fe, fd = Fraction(rho), Fraction(eta), Fraction(dt)
    uq, vq = Fraction(a0), Fraction(0)
    aq = (-k * uq - fe * vq) / fr
    for n in range(150):
        mdl.run_vv(n, 1, u, v, acc, mu, init=(n == 0))
        uq = uq + fd * vq + fd * fd / 2 * aq
        vt = vq + fd / 2 * aq
        an = (-k * uq - fe * vt) / fr
        vq = vq + fd / 2 * (aq + an)
        aq = an
        assert abs(u[1, 0] - float(uq)) <= 1e-12 * a0
        assert abs(v[1, 0] - float(vq)) <= 1e-12 * a0 / dt
        assert abs(acc[1, 0] - float(aq)) <= 1e-12 * a0 / dt ** 2
    assert np.all(u[0] == 0.0) and np.all(u[1, 1:] == 0.0)


def _free_body(seed=3):
    x = workloads.lattice(7, 6, 5, 1e-3, jitter=0.2, seed=seed)
    off, idx = oracle.family(x, 3.01e-3)
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0.8e-9, 1.2e-9, x.shape[0])
    c = oracle.micromodulus(5e9, 3.01e-3)
    return x, vol, off, idx, c, rng


def test_undamped_velocity_verlet_is_time_reversible():
    x, vol, off, idx, c, rng = _free_body()
    mdl = oracle.Model(x, vol, off, idx, c=c, sc=1.0, dt=1e-7, damping=0.0, density=2400.0)
    u0 = rng.uniform(-1e-7, 1e-7, x.shape)
    v0 = rng.uniform(-1e-2, 1e-2, x.shape)
    u, v, a = u0.copy(), v0.copy(), np.zeros_like(u0)
    mu = mdl.fresh_bonds()
    mdl.run_vv(0, 300, u, v, a, mu, init=True)
    assert np.abs(u - u0).max() > 1e-8          # it moved
    v = -v
    mdl.run_vv(300, 300, u, v, a, mu)
    assert np.abs(u - u0).max() <= 1e-9 * np.abs(u0).max()
    assert np.abs(v + v0).max() <= 1e-8 * np.abs(v0).max()


def test_damped_total_momentum_follows_the_scalar_recurrence():
    # internal forces cancel in sum_i V_i F_i, so M = sum V v and A = sum V a obey
    # A' = -(eta/rho) (M + dt/2 A),  M' = M + dt/2 (A + A')  (damping on the half-step velocity)
    x, vol, off, idx, c, rng = _free_body(4)
    rho, eta, dt = 2400.0, 2.5e6, 1e-7
    mdl = oracle.Model(x, vol, off, idx, c=c, sc=1.0, dt=dt, damping=eta, density=rho)
    u = rng.uniform(-1e-7, 1e-7, x.shape)
    v = rng.uniform(-1e-2, 1e-2, x.shape) + np.array([0.3, -0.2, 0.1])
    a = np.zeros_like(u)
    mu = mdl.fresh_bonds()
    mdl.run_vv(0, 0, u, v, a, mu, init=True)
    M = (vol[:, None] * v).sum(0)
    A = (vol[:, None] * a).sum(0)
    assert np.allclose(A, -(eta / rho) * M, rtol=1e-9, atol=0)
    for n in range(100):
        mdl.run_vv(n, 1, u, v, a, mu)
        An = -(eta / rho) * (M + dt / 2 * A)
        M = M + dt / 2 * (A + An)
        A = An
        assert np.allclose((vol[:, None] * v).sum(0), M, rtol=1e-9, atol=0)


def test_displacement_bc_follows_the_smooth_ramp():
    x, off, idx = _two_nodes(1.0)
    bt = np.zeros((2, 3), np.uint8); bt[1, 0] = 1
    g = np.zeros((2, 3)); g[1, 0] = 1.0
    r, T = 1e-4, 20
    mdl = oracle.Model(x, np.ones(2), off, idx, c=1.0, sc=1.0, bc_type=bt, bc_disp=g,
                       disp_rate=r, dt=0.5, density=1.0, ramp_steps=T)
    u = np.zeros((2, 3)); v = np.zeros((2, 3)); a = np.zeros((2, 3)); mu = mdl.fresh_bonds()
    for n in range(2 * T):
        mdl.run_vv(n, 1, u, v, a, mu, init=(n == 0))
        assert u[1, 0] == oracle.scale(r, T, n + 1)
        assert v[1, 0] == pytest.approx((oracle.scale(r, T, n + 1) - oracle.scale(r, T, n)) / 0.5)
    # the Euler-Cromer step uses the same scale
    u = np.zeros((2, 3)); v = np.zeros((2, 3))
    for n in range(T + 3):
        u, v = mdl.step(n, u, v, mu)
        assert u[1, 0] == oracle.scale(r, T, n + 1)
