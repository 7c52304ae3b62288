"""Pins of the oracle's bilinear softening bond law (Section 6, Example 3: the
damage model with linear elastic limit s_0 and k_r = s_c / s_0), CPU only."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _bar_models(kr):
    w = workloads.tensile_bar(20, 6, 6, steps=700)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    a = oracle.Model.from_workload(w, off, idx)
    w.kr = kr
    b = oracle.Model.from_workload(w, off, idx)
    return w, a, b


def test_kr_one_is_the_pmb_law_bit_for_bit():
    w, pmb, soft = _bar_models(1.0)
    ua, va, ma = np.zeros((w.n, 3)), np.zeros((w.n, 3)), pmb.fresh_bonds()
    ub, vb, mb = np.zeros((w.n, 3)), np.zeros((w.n, 3)), soft.fresh_bonds()
    pmb.run(0, w.steps, ua, va, ma)
    soft.run(0, w.steps, ub, vb, mb)
    assert (ma == 0).sum() > 0
    assert np.array_equal(ua, ub) and np.array_equal(va, vb) and np.array_equal(ma, mb)
    assert np.array_equal(pmb.damage(ma), soft.damage(mb))


def test_two_node_bond_follows_envelope_secant_unloading_and_breaks():
    L, c, V, sc, kr = 1.0, 2.0, 3.0, 0.01, 4.0
    s0 = sc / kr
    x = np.array([[0.0, 0.0, 0.0], [L, 0.0, 0.0]])
    off, idx = np.array([0, 1, 2]), np.array([1, 0], dtype=np.int32)
    bt = np.ones((2, 3), np.uint8)
    m = oracle.Model(x, np.array([V, V]), off, idx, c=c, sc=sc, bc_type=bt, dt=1.0,
                     density=1.0, kr=kr)
    mu = m.fresh_bonds()
    v = np.zeros((2, 3))

    def envelope(s):
        return c * s if s <= s0 else c * s0 * (sc - s) / (sc - s0)

    kmax = 0.0
    path = list(np.linspace(0, 0.006, 13)) + list(np.linspace(0.006, 0.002, 9)) + \
        list(np.linspace(0.002, 0.0095, 16)) + [0.0101, 0.004, 0.0]
    for n, s in enumerate(path):
        u = np.zeros((2, 3)); u[1, 0] = s * L
        _, _, F = m.step(n, u, v, mu, want_force=True)
        kmax = max(kmax, s)
        if kmax >= sc:
            assert not mu.any() and np.all(F == 0.0)
            continue
        mu_k = 1.0 if kmax <= s0 else s0 * (sc - kmax) / (kmax * (sc - s0))
        expect = c * s * mu_k * V          # pulls node 0 towards node 1 (+x)
        assert F[0, 0] == pytest.approx(expect, rel=1e-12, abs=1e-15)
        if s == kmax:                      # on the loading envelope
            assert F[0, 0] == pytest.approx(envelope(s) * V, rel=1e-12, abs=1e-15)
        assert m.kappa[0] == pytest.approx(kmax, rel=1e-12) and m.kappa[1] == m.kappa[0]
        # one-bond family: damage (Eq. 8 with the bond's integrity) is 1 - mu(kappa)
        assert m.damage(mu)[0] == pytest.approx(1.0 - mu_k, rel=1e-9, abs=1e-12)


def test_history_and_damage_are_monotone():
    w, _, soft = _bar_models(3.0)
    u, v, mu = np.zeros((w.n, 3)), np.zeros((w.n, 3)), soft.fresh_bonds()
    prev_k = soft.kappa.copy()
    prev_phi = soft.damage(mu)
    assert np.all(prev_phi == 0.0)
    for k in range(0, w.steps, 100):
        soft.run(k, 100, u, v, mu)
        phi = soft.damage(mu)
        assert np.all(soft.kappa >= prev_k)
        assert np.all(phi >= prev_phi - 1e-15) and np.all((phi >= 0) & (phi <= 1))
        prev_k, prev_phi = soft.kappa.copy(), phi
    assert prev_phi.max() > 0.0


def test_trilinear_envelope_kink_and_bilinear_limit():
    L, c, V, sc, kr, k1, beta = 1.0, 2.0, 3.0, 0.012, 6.0, 2.5, 0.25
    s0 = sc / kr
    s1 = k1 * s0
    x = np.array([[0.0, 0.0, 0.0], [L, 0.0, 0.0]])
    off, idx = np.array([0, 1, 2]), np.array([1, 0], dtype=np.int32)
    bt = np.ones((2, 3), np.uint8)

    def envelope(s):
        if s <= s0:
            return c * s
        if s <= s1:
            return c * s0 * ((1 - beta) * (s1 - s) / (s1 - s0) + beta)
        return c * s0 * beta * (sc - s) / (sc - s1)

    m = oracle.Model(x, np.array([V, V]), off, idx, c=c, sc=sc, bc_type=bt, dt=1.0,
                     density=1.0, kr=kr, trilinear=(k1, beta))
    mu = m.fresh_bonds()
    v = np.zeros((2, 3))
    kmax = 0.0
    path = list(np.linspace(0, 0.0095, 40)) + [0.003, 0.0, 0.011]
    for n, s in enumerate(path):
        u = np.zeros((2, 3)); u[1, 0] = s * L
        _, _, F = m.step(n, u, v, mu, want_force=True)
        kmax = max(kmax, s)
        expect = envelope(s) * V if s >= kmax else c * s * envelope(kmax) / (c * kmax) * V
        assert F[0, 0] == pytest.approx(expect, rel=1e-10, abs=1e-14)
    # continuity at the kink and the bilinear law at k1 = 1, beta = 1
    assert envelope(s1 * (1 - 1e-12)) == pytest.approx(envelope(s1 * (1 + 1e-12)), rel=1e-9)
    a = oracle.Model(x, np.array([V, V]), off, idx, c=c, sc=sc, bc_type=bt, dt=1.0,
                     density=1.0, kr=kr, trilinear=(1.0, 1.0))
    b = oracle.Model(x, np.array([V, V]), off, idx, c=c, sc=sc, bc_type=bt, dt=1.0,
                     density=1.0, kr=kr)
    for n, s in enumerate((0.001, 0.004, 0.008, 0.006)):
        u = np.zeros((2, 3)); u[1, 0] = s * L
        _, _, Fa = a.step(n, u, v, a.fresh_bonds(), want_force=True)
        _, _, Fb = b.step(n, u, v, b.fresh_bonds(), want_force=True)
        assert np.array_equal(Fa, Fb)
