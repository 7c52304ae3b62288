"""Pins of the oracle's stiffness corrections (micromodulus functions of Section
2.2 and the "Surface correction factors" volume method), CPU only.

Conical micromodulus c(|xi|) = c1 (1 - |xi|/delta): the strain-energy identity
behind Eq. (5) fixes c1 = 90 K / (pi delta^4); on a lattice the interior energy
density under uniform dilation is (9/2) K eps^2 times the quadrature ratio
5 sum_o (1 - |o|/r) |o| / (pi r^4), which tends to 1 as r = delta/dx grows.
Volume correction lambda_ij = 2 V0 / (V_i + V_j), V_i = family volume.
"""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import oracle  # noqa: E402
import workloads  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _offsets(r):
    R = int(math.floor(r))
    return [(a, b, c) for a in range(-R, R + 1) for b in range(-R, R + 1) for c in range(-R, R + 1)
            if (a, b, c) != (0, 0, 0) and a * a + b * b + c * c <= r * r]


def _conical_center_ratio(r, eps=1e-4, K=1e9, dx=1e-3):
    R = int(math.floor(r))
    m = 2 * R + 3
    x = workloads.lattice(m, m, m, dx)
    ci = (m // 2 * m + m // 2) * m + m // 2
    center = np.array([ci], dtype=np.int64)
    delta = r * dx
    off, idx = oracle.family(x, delta, rows=center)
    # one-row model for the factors: the centre is node 0, neighbours shifted by 1
    x1 = np.vstack([x[ci:ci + 1], x])
    fac = oracle.stiffness_factors(x1, np.full(x1.shape[0], dx ** 3), delta,
                                   np.array([0, len(idx)]), idx + 1, oracle.CONICAL)
    c = oracle.micromodulus(K, delta)
    mdl = oracle.Model(x, np.full(x.shape[0], dx ** 3), off, idx, c=c, c_bond=c * fac, sc=1.0,
                       rows=center)
    W = mdl.energy_density(eps * x, mdl.fresh_bonds())[0]
    return W / (4.5 * K * eps * eps), fac


def test_conical_lattice_quadrature_ratio():
    for r in (3.01, math.pi):
        offs = _offsets(r)
        expect = 5.0 * sum((1.0 - math.sqrt(a * a + b * b + c * c) / r) * math.sqrt(a * a + b * b + c * c)
                           for a, b, c in offs) / (math.pi * r ** 4)
        ratio, fac = _conical_center_ratio(r)
        assert len(fac) == len(offs)
        assert abs(ratio / expect - 1.0) < 1e-9


def test_conical_tends_to_continuum():
    # pins c1 = 5 c (a factor 4 or 6 would be off by 20 %)
    ratio, _ = _conical_center_ratio(12.01)
    assert abs(ratio - 1.0) < 0.03


def test_conical_factor_vanishes_at_the_horizon_and_is_5_at_zero_length():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    off = np.array([0, 2, 3, 4])
    idx = np.array([1, 2, 0, 0], dtype=np.int32)
    f = oracle.stiffness_factors(x, np.ones(3), 2.0, off, idx, oracle.CONICAL)
    assert np.allclose(f, [2.5, 0.0, 2.5, 0.0], atol=1e-15)


def _lattice_family(m, r):
    x = workloads.lattice(m, m, m, 1.0)
    off, idx = oracle.family(x, r)
    return x, off, idx


def test_volume_correction_bulk_face_and_symmetry():
    m, r = 12, 3.01
    x, off, idx = _lattice_family(m, r)
    n = x.shape[0]
    offs = _offsets(r)
    v_bulk = float(len(offs))                               # unit volumes
    v_face = float(sum(1 for a, b, c in offs if c >= 0))    # node on the z = 0 face
    f = oracle.stiffness_factors(x, np.ones(n), r, off, idx, oracle.SURFACE, v0=v_bulk)
    rows = np.repeat(np.arange(n), np.diff(off))
    rev = workloads.reverse_bond(n, off, idx)
    assert np.array_equal(f, f[rev])
    gi = np.rint(x).astype(int)

    def node(a, b, c):
        return (a * m + b) * m + c

    # both ends at least r from every face: full families
    i, j = node(5, 5, 5), node(6, 5, 5)
    k = off[i] + np.searchsorted(idx[off[i]:off[i + 1]], j)
    assert f[k] == 1.0
    # face node (z = 0) to a bulk node (z = 3)
    i, j = node(5, 5, 0), node(5, 5, 3)
    k = off[i] + np.searchsorted(idx[off[i]:off[i + 1]], j)
    assert idx[k] == j
    assert abs(f[k] - 2 * v_bulk / (v_face + v_bulk)) < 1e-15
    # face to face
    i, j = node(5, 5, 0), node(6, 5, 0)
    k = off[i] + np.searchsorted(idx[off[i]:off[i + 1]], j)
    assert abs(f[k] - v_bulk / v_face) < 1e-15
    # every bond whose two ends have full families
    full = np.all((gi >= 3) & (gi <= m - 4), axis=1)
    both = full[rows] & full[idx]
    assert both.sum() > 1000 and np.all(f[both] == 1.0)


def test_factors_multiply():
    x, off, idx = _lattice_family(8, 3.01)
    n = x.shape[0]
    a = oracle.stiffness_factors(x, np.ones(n), 3.01, off, idx, oracle.CONICAL)
    b = oracle.stiffness_factors(x, np.ones(n), 3.01, off, idx, oracle.SURFACE, v0=122.0)
    both = oracle.stiffness_factors(x, np.ones(n), 3.01, off, idx, oracle.CONICAL | oracle.SURFACE,
                                    v0=122.0)
    assert np.allclose(both, a * b, rtol=1e-15, atol=0)


def test_partial_volume_rule_values_and_quadrature():
    # a bond of length L gets (delta + dx/2 - L) / dx clipped to [0, 1]
    x = np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0], [0.0, 3.1, 0.0], [0.0, 0.0, 3.4]])
    off = np.array([0, 3, 4, 5, 6])
    idx = np.array([1, 2, 3, 0, 0, 0], dtype=np.int32)
    f = oracle.stiffness_factors(x, np.ones(4), 3.01, off, idx, oracle.PARTIAL, dx=1.0)
    assert np.allclose(f, [1.0, 0.41, 0.11, 1.0, 0.41, 0.11], atol=1e-12)
    # on a lattice, the partial volumes of the horizon (family built with
    # delta + dx/2) approximate the sphere volume 4/3 pi delta^3 better than counts
    r = 3.01
    m = 11
    xl = workloads.lattice(m, m, m, 1.0)
    c = (m // 2 * m + m // 2) * m + m // 2
    off2, idx2 = oracle.family(xl, r + 0.5, rows=np.array([c]))
    x1 = np.vstack([xl[c:c + 1], xl])
    pv = oracle.stiffness_factors(x1, np.ones(x1.shape[0]), r, np.array([0, len(idx2)]),
                                  idx2 + 1, oracle.PARTIAL, dx=1.0)
    sphere = 4.0 / 3.0 * np.pi * r ** 3
    full = len(_offsets(r))
    assert abs(pv.sum() - sphere) < abs(full - sphere)
