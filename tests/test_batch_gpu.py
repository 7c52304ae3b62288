"""Batched multi-instance form and the launch-shape autotuner, through the C ABI.

A batch advances independent models in one launch per step; each instance must
behave as the same model created alone: in FP64 bitwise (state, bond flags,
damage); in FP32 within the FP32 tolerances (the batch keeps FP32 positions in
one length unit, the largest horizon, so instances with a smaller horizon round
differently than alone).  The oracle agrees with one instance at the
single-model tolerances.
"""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu
F64, F32, DW = pdgb.PD_PREC_F64, pdgb.PD_PREC_F32, pdgb.PD_PREC_DW


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()
    oracle.build()


def _instances():
    ws = []
    ws.append(workloads.tensile_bar(16, 5, 5, rate=2e-6, steps=80, K=5e9, sc=3e-3))
    b = workloads.notched_beam(30, 6, 8, length=0.05, rate=3e-7, steps=80)
    ws.append(b)  # per-bond s_c draw (instance-local ids)
    ws.append(workloads.tensile_bar(11, 4, 3, rate=3e-6, slab=2, steps=80, K=2e10, sc=2e-3))
    ws.append(workloads.tensile_bar(1, 1, 1, steps=80))          # single node, no family
    p = workloads.cracked_plate_force(14, 10, 3, load=4e11, steps=80)
    ws.append(p)  # body force, pre-crack
    ws.append(workloads.tensile_bar(20, 3, 3, rate=4e-6, steps=80, K=8e9, sc=1.5e-3))
    return ws


def _alone(w, prec, steps):
    c = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=prec, c=c)
    m.step(steps)
    u, v = m.state()
    out = dict(u=u, v=v, mu=m.bonds(), phi=m.damage(), fam=m.family())
    m.close()
    return out


@pytest.mark.parametrize("prec", [F64, F32, DW])
def test_batch_instances_equal_models_alone(prec):
    ws = _instances()
    # all instances share dt, damping, density; loads/rates must agree across the batch
    for w in ws:
        # shared by the whole batch: the plate has no displacement-controlled node and
        # the bars no body force, so a common disp_rate and load change nothing else
        w.dt, w.damping, w.density = 1e-7, 2.5e6, 2400.0
        w.disp_rate, w.load = 1.0, 4e11
    steps = 80
    bm = pdgb.Model.batch(ws, precision=prec, graph_steps=16)
    off = bm.offsets()
    assert off[-1] == sum(w.n for w in ws) and len(off) == len(ws) + 1
    bm.step(steps)
    u, v = bm.state()
    mu = bm.bonds()
    phi = bm.damage()
    boff, bidx = bm.family()
    bm.close()
    broke = 0
    for k, w in enumerate(ws):
        a = _alone(w, prec, steps)
        s = slice(off[k], off[k + 1])
        fo, fi = a["fam"]
        assert np.array_equal(boff[off[k]:off[k + 1] + 1] - boff[off[k]], fo)
        assert np.array_equal(bidx[boff[off[k]]:boff[off[k + 1]]] - off[k], fi)
        mk = mu[boff[off[k]]:boff[off[k + 1]]]
        broke += int((mk == 0).sum())
        if prec == F64:
            assert np.array_equal(mk, a["mu"])
            assert np.array_equal(u[s], a["u"]) and np.array_equal(v[s], a["v"])
            assert np.array_equal(phi[s], a["phi"])
        elif prec == DW:
            # a batch takes the per-node-weight variant of the double-word step
            # (alone: one weight per model), which rounds differently
            den = max(np.abs(a["u"]).max(), 1e-300)
            assert np.abs(u[s] - a["u"]).max() <= 1e-12 * den
            assert np.array_equal(mk, a["mu"])
            assert np.abs(phi[s] - a["phi"]).max() <= 1e-12
        else:
            assert (mk != a["mu"]).mean() < 1e-3 if len(mk) else True
            den = max(np.abs(a["u"]).max(), 1e-300)
            assert np.abs(u[s] - a["u"]).max() <= 1e-4 * den
            assert np.abs(phi[s] - a["phi"]).max() <= 1e-3
    assert broke > 0


@pytest.mark.parametrize("prec", [F64, F32, DW])
def test_batch_with_softening_equals_models_alone(prec):
    ws = [workloads.tensile_bar(16, 5, 5, rate=1e-7, steps=300, K=5e9, sc=3e-3),
          workloads.tensile_bar(20, 4, 4, rate=1e-7, steps=300, K=8e9, sc=2e-3),
          workloads.notched_beam(30, 6, 8, length=0.05, rate=2e-7, steps=300)]
    for w in ws:
        w.dt, w.damping, w.density = 1e-7, 2.5e6, 2400.0
        w.disp_rate, w.load = 1.0, 0.0
        w.kr = 2.5
    steps = 300
    bm = pdgb.Model.batch(ws, precision=prec, graph_steps=10)
    off = bm.offsets()
    bm.step(steps)
    u, _ = bm.state()
    mu = bm.bonds()
    integ = pdgb.pd_get_bond_integrity(bm.h)
    boff, _ = bm.family()
    bm.close()
    softened = 0
    for k, w in enumerate(ws):
        c = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
        m = pdgb.Model.from_workload(w, precision=prec, c=c)
        m.step(steps)
        ua, _ = m.state()
        ma, ia = m.bonds(), pdgb.pd_get_bond_integrity(m.h)
        m.close()
        s = slice(off[k], off[k + 1])
        sb = slice(boff[off[k]], boff[off[k + 1]])
        softened += int(((ia > 0) & (ia < 1)).sum())
        den = np.abs(ua).max()
        if prec == F64:
            assert np.array_equal(u[s], ua) and np.array_equal(mu[sb], ma)
            assert np.array_equal(integ[sb], ia)
        elif prec == DW:
            # per-node-weight variant in the batch, one weight alone: ~1e-13 rounding
            # differences, which the softening response amplifies (1.7e-11 measured)
            assert np.abs(u[s] - ua).max() <= 1e-9 * den and np.array_equal(mu[sb], ma)
            assert np.abs(integ[sb] - ia).max() <= 1e-7
        else:
            assert np.abs(u[s] - ua).max() <= 1e-4 * den
            assert (mu[sb] != ma).mean() < 1e-3
    assert softened > 0


@pytest.mark.parametrize("prec", [F64, F32, DW])
def test_batch_of_state_based_models_equals_models_alone(prec):
    # the ordinary state-based solid in a batch: one (K, G) for the batch, each
    # instance its own size and s_c (one a per-bond draw keyed by local ids)
    K = 5e9
    ws = [workloads.tensile_bar(16, 5, 5, rate=4e-6, steps=100, K=K, sc=3e-3),
          workloads.tensile_bar(11, 4, 3, rate=5e-6, slab=2, steps=100, K=K, sc=2e-3),
          workloads.tensile_bar(20, 3, 3, rate=4e-6, steps=100, K=K, sc=2.5e-3)]
    ws[2].sc_hash = (2105041507, 2e-3, 3e-3)
    for w in ws:
        w.state_based = (K, 0.6 * K)  # nu = 1/4
    steps = 100
    bm = pdgb.Model.batch(ws, precision=prec, graph_steps=20)
    off = bm.offsets()
    bm.step(steps)
    u, v = bm.state()
    mu = bm.bonds()
    phi = bm.damage()
    boff, _ = bm.family()
    bm.close()
    broke = 0
    for k, w in enumerate(ws):
        a = _alone(w, prec, steps)
        s = slice(off[k], off[k + 1])
        mk = mu[boff[off[k]]:boff[off[k + 1]]]
        broke += int((a["mu"] == 0).sum())
        den = np.abs(a["u"]).max()
        if prec == F64:
            assert np.array_equal(u[s], a["u"]) and np.array_equal(v[s], a["v"])
            assert np.array_equal(mk, a["mu"]) and np.array_equal(phi[s], a["phi"])
        elif prec == DW:
            # per-node weights in the batch, one weight alone: rounding only
            assert np.abs(u[s] - a["u"]).max() <= 1e-10 * den
            assert (mk != a["mu"]).mean() <= 1e-3
        else:
            assert np.abs(u[s] - a["u"]).max() <= 1e-4 * den
            assert (mk != a["mu"]).mean() < 1e-3
    assert broke > 0


def test_batch_rejects_mixed_state_based_parameters():
    ws = [workloads.tensile_bar(6, 3, 3, steps=5), workloads.tensile_bar(5, 3, 3, steps=5)]
    ws[0].state_based = (5e9, 3e9)
    with pytest.raises(pdgb.PdError) as e:  # one bond-based, one state-based
        pdgb.Model.batch(ws, precision=F64)
    assert e.value.name == "PD_ERR_ARG"
    ws[1].state_based = (5e9, 2e9)
    with pytest.raises(pdgb.PdError):        # different shear moduli
        pdgb.Model.batch(ws, precision=F64)


@pytest.mark.parametrize("prec", [F64, DW])
def test_batch_instance_matches_oracle(prec):
    ws = _instances()[:3]
    for w in ws:
        w.dt, w.damping, w.density = 1e-7, 2.5e6, 2400.0
    bm = pdgb.Model.batch(ws, precision=prec)
    bm.step(80)
    u, _ = bm.state()
    off = bm.offsets()
    bm.close()
    w = ws[1]
    fo, fi = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, fo, fi, c=oracle.micromodulus(w.bulk_modulus, w.horizon))
    uo = np.zeros((w.n, 3)); vo = np.zeros((w.n, 3)); mo = om.fresh_bonds()
    om.run(0, 80, uo, vo, mo)
    ub = u[off[1]:off[2]]
    assert np.abs(ub - uo).max() <= 1e-10 * np.abs(uo).max()


def test_batch_rejects_set_params_and_mismatched_loads():
    ws = _instances()[:2]
    for w in ws:
        w.dt, w.damping, w.density = 1e-7, 2.5e6, 2400.0
    bm = pdgb.Model.batch(ws)
    with pytest.raises(pdgb.PdError) as e:
        bm.set_params(1.0, 1e-3, 0.0, 1.0)
    assert e.value.name == "PD_ERR_STATE"
    bm.close()
    ws[1].disp_rate = 2.0
    with pytest.raises(pdgb.PdError) as e:
        pdgb.Model.batch(ws)
    assert e.value.name == "PD_ERR_ARG"


@pytest.mark.parametrize("prec", [F64, F32])
def test_autotune_keeps_state_and_results(prec):
    w = workloads.notched_beam(40, 8, 10, length=0.06, rate=4e-7, steps=60)
    c = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
    a = pdgb.Model.from_workload(w, precision=prec, c=c, graph_steps=10)
    b = pdgb.Model.from_workload(w, precision=prec, c=c, graph_steps=10)
    a.step(30)
    b.step(30)
    ub0, vb0 = b.state()
    mub0 = b.bonds()
    block, bps = b.autotune(5)
    assert block in (128, 256) and bps >= 1
    ub1, vb1 = b.state()
    assert np.array_equal(ub0, ub1) and np.array_equal(vb0, vb1)
    assert np.array_equal(mub0, b.bonds()) and b.info()["step"] == 30
    a.step(30)
    b.step(30)
    ua, va = a.state()
    ub, vb = b.state()
    # the launch shape does not change any node's arithmetic
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    assert np.array_equal(a.bonds(), b.bonds())
    a.close()
    b.close()
