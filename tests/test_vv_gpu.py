"""Damped velocity-Verlet and the smooth loading ramp on the GPU, through the C
ABI, against the oracle (Section 3.6 "Time integration"; Sections 5-6 loading)."""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu
F64, F32 = pdgb.PD_PREC_F64, pdgb.PD_PREC_F32
VV, EC = pdgb.PD_INTEGRATOR_VV, pdgb.PD_INTEGRATOR_EC
BAND = 1e-9  # bonds whose oracle stretch came within this of s_c may differ


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()
    oracle.build()


def _bar(steps=1000, ramp=0):
    w = workloads.tensile_bar(steps=steps)
    w.ramp_steps = ramp
    return w


def _oracle(w, integrator, steps):
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    u, v, a = np.zeros((w.n, 3)), np.zeros((w.n, 3)), np.zeros((w.n, 3))
    mu = om.fresh_bonds()
    margin = np.full(len(mu), np.inf)
    if integrator == VV:
        om.run_vv(0, steps, u, v, a, mu, init=True, margin=margin)
    else:
        om.run(0, steps, u, v, mu, margin)
    return u, v, mu, margin


def _gpu(w, precision, integrator, steps, **kw):
    m = pdgb.Model.from_workload(w, precision=precision, integrator=integrator, **kw)
    m.step(steps)
    u, v = m.state()
    b = m.bonds()
    m.close()
    return u, v, b


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("ramp", [0, 300])
def test_velocity_verlet_fp64_matches_oracle(ramp):
    w = _bar(ramp=ramp)
    uo, vo, mo, margin = _oracle(w, VV, w.steps)
    u, v, b = _gpu(w, F64, VV, w.steps, graph_steps=16)
    assert (mo == 0).sum() > 0
    assert rel(u, uo) <= 1e-10 and rel(v, vo) <= 1e-9
    diff = b != mo
    assert np.all(margin[diff] < BAND), int(diff.sum())


def test_velocity_verlet_fp32_matches_oracle():
    w = _bar()
    uo, vo, mo, _ = _oracle(w, VV, w.steps)
    u, v, b = _gpu(w, F32, VV, w.steps, graph_steps=16)
    assert rel(u, uo) <= 1e-4
    assert (b != mo).sum() <= 1e-3 * len(mo)


@pytest.mark.parametrize("precision", [F64, F32])
def test_smooth_ramp_euler_cromer_matches_oracle(precision):
    w = _bar(ramp=250)
    uo, vo, mo, margin = _oracle(w, EC, w.steps)
    u, v, b = _gpu(w, precision, EC, w.steps)
    tol = 1e-10 if precision == F64 else 1e-4
    assert rel(u, uo) <= tol
    diff = b != mo
    if precision == F64:
        assert np.all(margin[diff] < BAND), int(diff.sum())
    else:
        assert diff.sum() <= 1e-3 * len(mo)


@pytest.mark.parametrize("precision", [F64, F32])
def test_full_step_velocity_read_changes_nothing(precision):
    # pd_get_state on a velocity-Verlet handle evaluates the forces once more to
    # form v^n; the run must not notice, with or without graphs
    w = _bar(steps=300)
    ref_u, ref_v, ref_b = _gpu(w, precision, VV, 300, graph_steps=0)
    for G in (0, 25):
        m = pdgb.Model.from_workload(w, precision=precision, integrator=VV, graph_steps=G)
        for k in range(6):
            m.step(50)
            m.state()
            m.state()
        u, v = m.state()
        b = m.bonds()
        m.close()
        assert np.array_equal(u, ref_u) and np.array_equal(v, ref_v) and np.array_equal(b, ref_b)


def test_set_state_starts_a_new_history():
    # restarting from (u^n, v^n) forms a^n from them, as the oracle's init step does
    w = _bar(steps=400)
    m = pdgb.Model.from_workload(w, precision=F64, integrator=VV)
    m.step(200)
    u, v = m.state()
    m.set_state(u, v, step=200)
    m.step(200)
    ug, vg = m.state()
    m.close()
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    uo, vo, ao = np.zeros((w.n, 3)), np.zeros((w.n, 3)), np.zeros((w.n, 3))
    mu = om.fresh_bonds()
    om.run_vv(0, 200, uo, vo, ao, mu, init=True)
    uo, vo = u.copy(), v.copy()
    om.run_vv(200, 200, uo, vo, ao, mu, init=True)
    assert rel(ug, uo) <= 1e-10 and rel(vg, vo) <= 1e-9


def test_velocity_verlet_batch_instance_equals_alone():
    ws = [workloads.tensile_bar(12, 5, 5, steps=300), workloads.tensile_bar(16, 6, 5, steps=300)]
    for w in ws:
        w.ramp_steps = 100
    bm = pdgb.Model.batch(ws, precision=F64, integrator=VV)
    bm.step(300)
    ub, vb = bm.state()
    offs = bm.offsets()
    bm.close()
    for k, w in enumerate(ws):
        u, v, _ = _gpu(w, F64, VV, 300)
        assert np.array_equal(ub[offs[k]:offs[k + 1]], u)
        assert np.array_equal(vb[offs[k]:offs[k + 1]], v)


def test_adjoint_rejects_velocity_verlet_with_softening_or_fp32():
    # the velocity-Verlet adjoint (tests/test_adjoint_gpu.py) covers FP64-grade
    # PMB handles without softening, as for Euler-Cromer
    w = _bar(steps=5)
    for kw in (dict(precision=F32), dict(precision=F64, kr=3.0)):
        ws = w
        if "kr" in kw:
            ws = _bar(steps=5)
            ws.kr = kw.pop("kr")
        m = pdgb.Model.from_workload(ws, integrator=VV, **kw)
        with pytest.raises(pdgb.PdError) as e:
            pdgb.pd_adjoint_forward(m.h, 5)
        assert e.value.name == "PD_ERR_STATE"
        m.close()


def test_velocity_verlet_with_softening_matches_oracle():
    # the read-only force pass also lowers integrities at u^n (idempotently)
    w = _bar(steps=700)
    w.kr = 3.0
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    u, v, a = np.zeros((w.n, 3)), np.zeros((w.n, 3)), np.zeros((w.n, 3))
    mu = om.fresh_bonds()
    margin = np.full(len(mu), np.inf)
    om.run_vv(0, w.steps, u, v, a, mu, init=True, margin=margin)
    m = pdgb.Model.from_workload(w, precision=F64, integrator=VV, graph_steps=10)
    for _ in range(7):
        m.step(100)
        m.state()
    ug, vg = m.state()
    b = m.bonds()
    m.close()
    assert rel(ug, u) <= 1e-10 and rel(vg, v) <= 1e-9
    assert np.all(margin[b != mu] < BAND)
