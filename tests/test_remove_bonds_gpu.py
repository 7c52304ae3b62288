"""pd_remove_bonds: a notch cut into a built model (the initial-notch rule of Section 6).

The notched beam is built WITHOUT its notch, the bonds the notch plane crosses
are removed through the C ABI, and the run is compared with the FP64 oracle
stepping the same un-notched family whose flags start broken on exactly those
bonds.  Bars as in the parity tests: FP64 and PD_PREC_DW u within 1e-10 and v
within 1e-9 relative, broken sets identical except bonds the oracle saw within
1e-9 of s_c; FP32 u within 1e-4 over the first 250 steps, < 0.1 % of bonds
differing.  The damage counts the removed bonds (they stay in the family).
"""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu

F32, F64, DW = pdgb.PD_PREC_F32, pdgb.PD_PREC_F64, pdgb.PD_PREC_DW
BAND = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()
    oracle.build()


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def rows_of(off):
    return np.repeat(np.arange(len(off) - 1), np.diff(off))


@pytest.fixture(scope="module")
def notch():
    """(beam without notch, its family, mask of the bonds the notch crosses, pairs i<j)."""
    w = workloads.notched_beam(48, 10, 12, length=0.08, rate=1e-7, steps=400)
    plain = dataclasses.replace(w, cuts=[])
    off0, idx0 = oracle.cut_family(w.coords, w.horizon, plain.cuts_array())
    off1, idx1 = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    r0, r1 = rows_of(off0), rows_of(off1)
    key0 = r0.astype(np.int64) * w.n + idx0
    key1 = r1.astype(np.int64) * w.n + idx1
    crossed = ~np.isin(key0, key1)
    sel = crossed & (r0 < idx0)
    pairs = np.stack([r0[sel], idx0[sel]], axis=1).astype(np.int64)
    assert crossed.sum() == 2 * len(pairs) > 100
    return w, plain, off0, idx0, crossed, pairs


def oracle_run(plain, off, idx, crossed, steps):
    m = oracle.Model.from_workload(plain, off, idx)
    u = np.zeros((plain.n, 3))
    v = np.zeros((plain.n, 3))
    mu = m.fresh_bonds()
    mu[crossed] = 0
    phi0 = m.damage(mu)
    margin = np.full(m.nbonds, np.inf)
    m.run(0, steps, u, v, mu, margin)
    return dict(u=u, v=v, mu=mu, margin=margin, phi=m.damage(mu), phi0=phi0)


def gpu_run(plain, pairs, crossed, steps, precision, **kw):
    c = oracle.micromodulus(plain.bulk_modulus, plain.horizon)
    m = pdgb.Model.from_workload(plain, precision=precision, c=c, **kw)
    m.remove_bonds(pairs)
    mu0 = m.bonds()
    assert not mu0[crossed].any() and mu0[~crossed].all()
    phi0 = m.damage()
    m.step(steps)
    m.sync()
    u, v = m.state()
    out = dict(u=u, v=v, mu=m.bonds(), phi=m.damage(), phi0=phi0, fam=m.family())
    m.close()
    return out


@pytest.mark.parametrize("prec", [F64, DW])
def test_removed_notch_matches_oracle(notch, prec):
    w, plain, off, idx, crossed, pairs = notch
    o = oracle_run(plain, off, idx, crossed, w.steps)
    g = gpu_run(plain, pairs, crossed, w.steps, prec, graph_steps=50)
    assert np.array_equal(g["fam"][0], off) and np.array_equal(g["fam"][1], idx)
    assert np.abs(g["phi0"] - o["phi0"]).max() <= 1e-12 and g["phi0"].max() > 0.1
    assert rel(g["u"], o["u"]) <= 1e-10, rel(g["u"], o["u"])
    assert rel(g["v"], o["v"]) <= 1e-9, rel(g["v"], o["v"])
    diff = g["mu"] != o["mu"]
    assert np.all(o["margin"][diff] < BAND), int(diff.sum())
    assert (o["mu"] == 0).sum() > crossed.sum()  # the run breaks bonds beyond the notch
    assert np.abs(g["phi"] - o["phi"]).max() <= 1e-12 + 2.0 * diff.sum() / len(diff)


def test_removed_notch_fp32_matches_oracle(notch):
    w, plain, off, idx, crossed, pairs = notch
    o = oracle_run(plain, off, idx, crossed, 250)
    g = gpu_run(plain, pairs, crossed, 250, F32, graph_steps=25)
    assert rel(g["u"], o["u"]) <= 1e-4, rel(g["u"], o["u"])
    assert (g["mu"] != o["mu"]).mean() < 1e-3


def test_removed_notch_moves_nodes_like_the_initial_cut(notch):
    # the forces of a model whose notch bonds were removed are those of the model
    # built with the notch: only the damage denominators differ
    w, plain, off, idx, crossed, pairs = notch
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    a = pdgb.Model.from_workload(w, precision=F64, c=c)
    b = pdgb.Model.from_workload(plain, precision=F64, c=c)
    b.remove_bonds(pairs)
    a.step(200)
    b.step(200)
    ua, va = a.state()
    ub, vb = b.state()
    assert rel(ub, ua) <= 1e-10 and rel(vb, va) <= 1e-9
    a.close()
    b.close()


def test_remove_bonds_zeroes_the_softening_integrity(notch):
    w, plain, off, idx, crossed, pairs = notch
    soft = dataclasses.replace(plain, kr=4.0)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    for prec in (F32, F64, DW):
        m = pdgb.Model.from_workload(soft, precision=prec, c=c)
        m.remove_bonds(pairs)
        mu = pdgb.pd_get_bond_integrity(m.h)
        assert np.all(mu[crossed] == 0.0) and np.all(mu[~crossed] == 1.0)
        m.step(50)
        m.sync()
        assert not m.bonds()[crossed].any()
        m.close()


def test_remove_bonds_rejects_bad_pairs_and_changes_nothing(notch):
    w, plain, off, idx, crossed, pairs = notch
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(plain, precision=F64, c=c)
    far = np.array([[0, w.n - 1]], np.int64)  # two ends of the beam: not a bond
    bad = [np.concatenate([pairs[:5], far]), [[0, 0]], [[-1, 3]], [[0, w.n]]]
    for p in bad:
        with pytest.raises(pdgb.PdError):
            m.remove_bonds(p)
        assert m.bonds().all()
    m.remove_bonds(np.zeros((0, 2), np.int64))
    assert m.bonds().all()
    m.remove_bonds(np.concatenate([pairs[:3], pairs[:3, ::-1]]))  # repeats, either order
    mu = m.bonds()
    assert (mu == 0).sum() == 6
    m.close()
