"""Pins of the oracle's ordinary state-based model (linear peridynamic solid,
omega = 1), CPU only.

Uniform dilation gives theta = 3 eps at every node, so W = (9/2) K eps^2
exactly (not only in the bulk); simple shear gives G gamma^2 / 2 times a lattice
quadrature ratio computed here from the stencil offsets (-> 1 for large
horizons); the force density is minus the gradient of the total energy.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _model(x, delta, K=3e9, G=1.7e9, vol=None, **kw):
    off, idx = oracle.family(x, delta)
    vol = np.full(x.shape[0], 1e-9) if vol is None else vol
    return oracle.Model(x, vol, off, idx, c=1.0, sc=1.0, state_based=(K, G), **kw), off, idx


def test_uniform_dilation_gives_nine_halves_K_eps_squared_everywhere():
    x = workloads.lattice(9, 8, 7, 1e-3, jitter=0.2, seed=2)
    K, eps = 3e9, 1e-4
    m, _, _ = _model(x, 3.01e-3, K=K)
    W = m.energy_density(eps * x, m.fresh_bonds())
    assert np.allclose(m.theta, 3 * eps, rtol=1e-9, atol=0)
    assert np.allclose(W, 4.5 * K * eps * eps, rtol=1e-8, atol=0)


def _offsets(r):
    R = int(math.floor(r))
    return [(a, b, c) for a in range(-R, R + 1) for b in range(-R, R + 1) for c in range(-R, R + 1)
            if (a, b, c) != (0, 0, 0) and a * a + b * b + c * c <= r * r]


def _shear_ratio(r, gamma=1e-6, G=1.7e9):
    R = int(math.floor(r))
    n = 2 * R + 3
    x = workloads.lattice(n, n, n, 1.0)
    m, off, idx = _model(x, r, G=G, vol=np.ones(x.shape[0]))
    u = np.zeros_like(x)
    u[:, 0] = gamma * x[:, 1]
    W = m.energy_density(u, m.fresh_bonds())
    c = (n // 2 * n + n // 2) * n + n // 2
    return W[c] / (G * gamma * gamma / 2)


def test_simple_shear_lattice_ratio_and_continuum_limit():
    offs = _offsets(3.01)
    expect = 15 * sum((a * a * b * b) / (a * a + b * b + c * c) for a, b, c in offs) / \
        sum(a * a + b * b + c * c for a, b, c in offs)
    assert _shear_ratio(3.01) == pytest.approx(expect, rel=1e-4)
    assert abs(_shear_ratio(9.01) - 1.0) < 0.03


def test_force_is_minus_energy_gradient():
    x = workloads.lattice(5, 5, 4, 1e-3, jitter=0.2, seed=4)
    rng = np.random.default_rng(5)
    vol = rng.uniform(0.8e-9, 1.2e-9, x.shape[0])
    m, _, _ = _model(x, 2.2e-3, vol=vol)
    u = rng.uniform(-2e-6, 2e-6, x.shape)
    mu = m.fresh_bonds()
    _, _, F = m.step(0, u, np.zeros_like(u), mu, want_force=True)
    h = 1e-10
    for i in rng.choice(x.shape[0], 6, replace=False):
        for a in range(3):
            up = u.copy(); up[i, a] += h
            um = u.copy(); um[i, a] -= h
            Ep = (vol * m.energy_density(up, mu)).sum()
            Em = (vol * m.energy_density(um, mu)).sum()
            g = -(Ep - Em) / (2 * h)
            assert abs(g - vol[i] * F[i, a]) <= 1e-5 * vol[i] * np.abs(F).max()


def test_rigid_motion_is_force_free_and_momentum_is_conserved():
    x = workloads.lattice(6, 5, 5, 1e-3, jitter=0.2, seed=6)
    rng = np.random.default_rng(7)
    vol = rng.uniform(0.8e-9, 1.2e-9, x.shape[0])
    m, _, _ = _model(x, 2.6e-3, vol=vol)
    mu = m.fresh_bonds()
    th = 0.3
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    for u in (np.tile([1e-3, -2e-3, 5e-4], (x.shape[0], 1)), x @ R.T - x):
        _, _, F = m.step(0, u, np.zeros_like(u), mu, want_force=True)
        # zero up to rounding: against the force scale K / delta of a unit strain
        assert np.abs(F).max() <= 1e-12 * 3e9 / 2.6e-3
    u = rng.uniform(-2e-6, 2e-6, x.shape)
    _, _, F = m.step(0, u, np.zeros_like(u), mu, want_force=True)
    assert np.abs((vol[:, None] * F).sum(0)).max() <= 1e-12 * np.abs(vol[:, None] * F).sum()


def test_velocity_verlet_conserves_the_state_based_energy():
    # undamped, unloaded, nothing breaks: the velocity-Verlet run of the linear
    # solid keeps kinetic + strain energy to O(dt^2) (it is symplectic), which it
    # does only if the integrator applies this model's forces (minus the gradient
    # of the same energy); the Euler-Cromer run of the same state agrees to O(dt)
    x = workloads.lattice(8, 6, 6, 1e-3, jitter=0.15, seed=4)
    vol = np.full(x.shape[0], 1e-9)
    off, idx = oracle.family(x, 3.01e-3)
    K, G, rho = 3e9, 1.4e9, 2400.0
    mk = lambda dt: oracle.Model(x, vol, off, idx, c=1.0, sc=1.0, state_based=(K, G),
                                 dt=dt, damping=0.0, density=rho)
    rng = np.random.default_rng(9)
    u0 = rng.normal(0.0, 2e-8, x.shape)
    v0 = rng.normal(0.0, 1e-3, x.shape)

    def energy(m, u, v, mu):
        return float((vol * (0.5 * rho * (v * v).sum(axis=1) + m.energy_density(u, mu))).sum())

    dt, n = 2e-8, 400
    m = mk(dt)
    u, v, a, mu = u0.copy(), v0.copy(), np.zeros_like(x), m.fresh_bonds()
    E0 = energy(m, u, v, mu)
    m.run_vv(0, 1, u, v, a, mu, init=True)
    drift = 0.0
    for k in range(1, n):
        m.run_vv(k, 1, u, v, a, mu)
        drift = max(drift, abs(energy(m, u, v, mu) - E0) / E0)
    assert mu.all() and drift < 2e-4, drift
    # a wrong force (here: half of it) is not conservative with this energy
    m2 = oracle.Model(x, vol, off, idx, c=1.0, sc=1.0, state_based=(K, G), dt=dt, damping=0.0,
                      density=2.0 * rho)
    u2, v2, a2, mu2 = u0.copy(), v0.copy(), np.zeros_like(x), m2.fresh_bonds()
    m2.run_vv(0, n, u2, v2, a2, mu2, init=True)
    assert abs(energy(m, u2, v2, mu2) - E0) / E0 > 20 * drift
    # Euler-Cromer agrees to first order in dt
    errs = []
    for h in (dt, dt / 2):
        steps = int(round(n * dt / h))
        mv, me = mk(h), mk(h)
        uv, vv_, av, bv = u0.copy(), v0.copy(), np.zeros_like(x), mv.fresh_bonds()
        mv.run_vv(0, steps, uv, vv_, av, bv, init=True)
        ue, ve, be = u0.copy(), v0.copy(), me.fresh_bonds()
        me.run(0, steps, ue, ve, be)
        errs.append(np.abs(ue - uv).max())
    assert 1.6 < errs[0] / errs[1] < 2.5, errs
