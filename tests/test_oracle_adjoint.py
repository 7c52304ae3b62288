"""Pins of the oracle's reverse-mode gradient against central finite differences
of the oracle's forward run (FP64), with the bond flags frozen.

The loss is L = <g_u, u^N> + <g_v, v^N> for random g.  Directions: per-bond
stiffness (not symmetric: every directed entry is its own parameter), the
body-force load, and the initial state.  The case has force-loaded edges and
displacement-controlled nodes, so the zeroing of controlled components in the
reverse sweep is exercised.
"""
import numpy as np
import pytest

import oracle
import workloads


def symmetric(off, idx, vals):
    """Average of the two directed entries of every bond (c_ij = c_ji)."""
    rows = np.repeat(np.arange(len(off) - 1), np.diff(off))
    key = {(int(i), int(j)): q for q, (i, j) in enumerate(zip(rows, idx))}
    rev = np.array([key[(int(j), int(i))] for i, j in zip(rows, idx)])
    return 0.5 * (vals + vals[rev])


def _case(seed=0):
    w = workloads.cracked_plate_force(9, 7, 3, load=3e11, steps=25)
    # a few displacement-controlled components as well
    w.bc_type[:3, 0] = 1
    w.bc_disp[:3, 0] = 1e-9
    w.disp_rate = 1.0
    w.sc = 1.0  # far above any stretch: the flags stay frozen
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    rng = np.random.default_rng(seed)
    c0 = oracle.micromodulus(w.bulk_modulus, w.horizon)
    # the forward's stiffness is symmetric (Newton's third law); perturbation
    # directions below need not be
    cb = symmetric(off, idx, c0 * (1.0 + 0.1 * rng.standard_normal(len(idx))))
    u0, v0 = workloads.random_state(w.n, seed + 1, 1e-7, 1e-3)
    u0[w.bc_type == 1] = 0.0
    v0[w.bc_type == 1] = 0.0
    gu = rng.standard_normal((w.n, 3))
    gv = rng.standard_normal((w.n, 3)) * 1e-7
    return w, off, idx, c0, cb, u0, v0, gu, gv, rng


def _loss(w, off, idx, c0, cb, u0, v0, gu, gv, load=None, steps=None):
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    if load is not None:
        m.m.load = load
    u = u0.copy(); v = v0.copy(); mu = m.fresh_bonds()
    m.run(0, steps or w.steps, u, v, mu)
    assert mu.all()
    return float((gu * u).sum() + (gv * v).sum())


def test_oracle_adjoint_matches_central_differences():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case()
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc, gl, gu0, gv0 = oracle.adjoint(m, 0, w.steps, u0, v0, m.fresh_bonds(), gu, gv)

    def fd(f, h):
        return (f(h) - f(-h)) / (2 * h)

    # per-bond stiffness, two random directions
    for k in range(2):
        dc = rng.standard_normal(len(idx)) * c0
        h = 1e-6
        num = fd(lambda t: _loss(w, off, idx, c0, cb + t * dc, u0, v0, gu, gv), h)
        ana = float(gc @ dc)
        assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)
    # load
    h = 1e-6 * w.load
    num = fd(lambda t: _loss(w, off, idx, c0, cb, u0, v0, gu, gv, load=w.load + t), h)
    assert abs(num - gl) <= 1e-6 * abs(gl), (num, gl)
    # initial displacement and velocity
    du = rng.standard_normal(u0.shape) * 1e-7
    du[w.bc_type == 1] = 0.0
    num = fd(lambda t: _loss(w, off, idx, c0, cb, u0 + t * du, v0, gu, gv), 1e-3)
    ana = float((gu0 * du).sum())
    assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)
    dv = rng.standard_normal(v0.shape) * 1e-3
    dv[w.bc_type == 1] = 0.0
    num = fd(lambda t: _loss(w, off, idx, c0, cb, u0, v0 + t * dv, gu, gv), 1e-3)
    ana = float((gv0 * dv).sum())
    assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)


def test_oracle_adjoint_controlled_velocity_carries_no_sensitivity():
    # a controlled component's initial velocity is overwritten before it is used;
    # its initial displacement still enters the first force evaluation
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(3)
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    _, _, gu0, gv0 = oracle.adjoint(m, 0, w.steps, u0, v0, m.fresh_bonds(), gu, gv)
    ctl = w.bc_type == 1
    assert np.all(gv0[ctl] == 0.0) and np.any(gu0[ctl] != 0.0)


def test_oracle_adjoint_zero_steps_is_identity():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(5)
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc, gl, gu0, gv0 = oracle.adjoint(m, 0, 0, u0, v0, m.fresh_bonds(), gu, gv)
    assert np.all(gc == 0.0) and gl == 0.0
    assert np.array_equal(gu0, gu) and np.array_equal(gv0, gv)


# ---------------------------------------------------------------- velocity-Verlet
def _loss_vv(w, off, idx, c0, cb, u0, v0, gu, gv, load=None):
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    if load is not None:
        m.m.load = load
    u = u0.copy(); v = v0.copy(); a = np.zeros_like(u0); mu = m.fresh_bonds()
    m.run_vv(0, w.steps, u, v, a, mu, init=True)
    assert mu.all()
    return float((gu * u).sum() + (gv * v).sum())


def test_oracle_vv_adjoint_matches_central_differences():
    # the reverse sweep of the damped velocity-Verlet run (acceleration formed
    # from the initial state) against central differences of that run
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(7)
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc, gl, gu0, gv0 = oracle.adjoint(m, 0, w.steps, u0, v0, m.fresh_bonds(), gu, gv,
                                      integrator="vv")

    def fd(f, h):
        return (f(h) - f(-h)) / (2 * h)

    for k in range(2):
        dc = rng.standard_normal(len(idx)) * c0
        num = fd(lambda t: _loss_vv(w, off, idx, c0, cb + t * dc, u0, v0, gu, gv), 1e-6)
        ana = float(gc @ dc)
        assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)
    h = 1e-6 * w.load
    num = fd(lambda t: _loss_vv(w, off, idx, c0, cb, u0, v0, gu, gv, load=w.load + t), h)
    assert abs(num - gl) <= 1e-6 * abs(gl), (num, gl)
    du = rng.standard_normal(u0.shape) * 1e-7
    num = fd(lambda t: _loss_vv(w, off, idx, c0, cb, u0 + t * du, v0, gu, gv), 1e-3)
    ana = float((gu0 * du).sum())
    assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)
    dv = rng.standard_normal(v0.shape) * 1e-3
    num = fd(lambda t: _loss_vv(w, off, idx, c0, cb, u0, v0 + t * dv, gu, gv), 1e-3)
    ana = float((gv0 * dv).sum())
    assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)
    ctl = w.bc_type == 1
    assert np.all(gv0[ctl] == 0.0) and np.any(gu0[ctl] != 0.0)


def test_oracle_vv_adjoint_zero_steps_is_identity():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(9)
    m = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc, gl, gu0, gv0 = oracle.adjoint(m, 0, 0, u0, v0, m.fresh_bonds(), gu, gv,
                                      integrator="vv")
    assert np.all(gc == 0.0) and gl == 0.0
    assert np.array_equal(gu0, gu) and np.array_equal(gv0, gv)


def test_bond_jacobian_dot_product():
    # <J v, w> = <v, J^T w> for J = dF/du of the pairwise force density: J v by
    # central differences of the oracle's force, J^T w from one reverse step
    # (L = <w, v^1> with v^1 = v^0 + dt (F(u^0) - eta v^0) / rho, so
    # dL/du^0 = (dt / rho) J^T w); no controlled components
    w = workloads.cracked_plate_force(9, 7, 3, load=3e11, steps=1)
    w.bc_type[:] = 0
    w.sc = 1.0
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    c0 = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = oracle.Model.from_workload(w, off, idx, c=c0)
    rng = np.random.default_rng(21)
    u0, v0 = workloads.random_state(w.n, 22, 1e-7, 1e-3)
    vdir = rng.standard_normal((w.n, 3)) * 1e-7
    wvec = rng.standard_normal((w.n, 3))

    def force(u):
        _, _, F = m.step(0, u.copy(), v0.copy(), m.fresh_bonds(), want_force=True)
        return F

    h = 1e-3
    Jv = (force(u0 + h * vdir) - force(u0 - h * vdir)) / (2 * h)
    _, _, gu0, _ = oracle.adjoint(m, 0, 1, u0, v0, m.fresh_bonds(), np.zeros_like(u0), wvec)
    JTw = gu0 * w.density / w.dt
    lhs, rhs = float((Jv * wvec).sum()), float((vdir * JTw).sum())
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)
