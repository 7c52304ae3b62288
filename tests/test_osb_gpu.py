"""Ordinary state-based linear solid on the GPU (FP64), through the C ABI,
against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu
F64, F32, DW = pdgb.PD_PREC_F64, pdgb.PD_PREC_F32, pdgb.PD_PREC_DW
BAND = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()
    oracle.build()


def _moduli(K, nu):
    return K, 3 * K * (1 - 2 * nu) / (2 * (1 + nu))


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _compare(w, steps, precision=F64):
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    u, v, mu = np.zeros((w.n, 3)), np.zeros((w.n, 3)), om.fresh_bonds()
    margin = np.full(len(mu), np.inf)
    om.run(0, steps, u, v, mu, margin)
    m = pdgb.Model.from_workload(w, precision=precision, graph_steps=16)
    m.step(steps)
    ug, vg = m.state()
    b, phi = m.bonds(), m.damage()
    m.close()
    assert rel(ug, u) <= 1e-10 and rel(vg, v) <= 1e-9, (rel(ug, u), rel(vg, v))
    diff = b != mu
    assert np.all(margin[diff] < BAND), int(diff.sum())
    assert np.abs(phi - om.damage(mu)).max() <= 1e-12 + 2.0 * diff.sum() / len(diff)
    return mu


@pytest.mark.parametrize("precision", [F64, DW])
@pytest.mark.parametrize("nu", [0.25, 0.35])
def test_state_based_tensile_bar_matches_oracle(nu, precision):
    # FP64 and the FP64-grade double-word step are held to the same bar
    w = workloads.tensile_bar(steps=1000)
    w.state_based = _moduli(w.bulk_modulus, nu)
    mu = _compare(w, w.steps, precision)
    assert (mu == 0).sum() > 0


@pytest.mark.parametrize("precision", [F64, DW])
def test_state_based_notched_beam_per_bond_sc(precision):
    w = workloads.notched_beam(48, 10, 12, length=48 / 600, rate=1e-7, steps=300)
    w.state_based = _moduli(w.bulk_modulus, 0.2)
    _compare(w, w.steps, precision)


@pytest.mark.parametrize("precision", [F64, DW])
def test_state_based_restrictions(precision):
    w = workloads.tensile_bar(8, 4, 4, steps=5)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    m = pdgb.Model.from_workload(w, precision=precision)
    off, idx = m.family()
    with pytest.raises(pdgb.PdError) as e:
        m.set_params(1.0, w.sc, 0.0, w.disp_rate, np.ones(len(idx)))
    assert e.value.name == "PD_ERR_STATE"
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_adjoint_forward(m.h, 3)
    assert e.value.name == "PD_ERR_STATE"
    m.close()


def test_state_based_fp32_matches_oracle():
    # u compared before the first breaks (R13: FP32 rounding moves break steps
    # once fracture runs), the broken set at the end
    w = workloads.tensile_bar(steps=1000)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    u, v, mu = np.zeros((w.n, 3)), np.zeros((w.n, 3)), om.fresh_bonds()
    om.run(0, 400, u, v, mu)
    assert (mu == 0).sum() == 0
    m = pdgb.Model.from_workload(w, precision=F32, graph_steps=16)
    m.step(400)
    ug, _ = m.state()
    assert rel(ug, u) <= 1e-4
    om.run(400, 600, u, v, mu)
    m.step(600)
    b = m.bonds()
    m.close()
    assert (mu == 0).sum() > 0 and (b != mu).sum() <= 1e-3 * len(mu)


@pytest.mark.parametrize("precision", [F64, DW])
def test_state_based_with_smooth_ramp_matches_oracle(precision):
    w = workloads.tensile_bar(steps=600)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    w.ramp_steps = 300
    _compare(w, w.steps, precision)


@pytest.mark.parametrize("precision", [F64, DW, F32])
def test_state_based_velocity_verlet_matches_oracle(precision):
    w = workloads.tensile_bar(steps=700)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    steps = w.steps if precision != F32 else 400  # FP32: before the first breaks (R13)
    u, v, acc = np.zeros((w.n, 3)), np.zeros((w.n, 3)), np.zeros((w.n, 3))
    mu = om.fresh_bonds()
    margin = np.full(len(mu), np.inf)
    om.run_vv(0, steps, u, v, acc, mu, init=True, margin=margin)
    m = pdgb.Model.from_workload(w, precision=precision, graph_steps=16,
                                 integrator=pdgb.PD_INTEGRATOR_VV)
    m.step(steps)
    ug, vg = m.state()
    b = m.bonds()
    m.close()
    if precision == F32:
        assert (mu == 0).sum() == 0 and rel(ug, u) <= 1e-4
        return
    assert (mu == 0).sum() > 0
    assert rel(ug, u) <= 1e-10 and rel(vg, v) <= 1e-9, (rel(ug, u), rel(vg, v))
    diff = b != mu
    assert np.all(margin[diff] < BAND), int(diff.sum())


@pytest.mark.parametrize("precision", [F64, DW, F32])
def test_state_based_full_step_velocity_read_changes_nothing(precision):
    w = workloads.tensile_bar(steps=300)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    vv = pdgb.PD_INTEGRATOR_VV
    ref = pdgb.Model.from_workload(w, precision=precision, integrator=vv)
    ref.step(300)
    ur, vr = ref.state()
    br = ref.bonds()
    ref.close()
    m = pdgb.Model.from_workload(w, precision=precision, integrator=vv, graph_steps=25)
    for _ in range(6):
        m.step(50)
        m.state()
        m.bonds()
    u, v = m.state()
    b = m.bonds()
    m.close()
    assert np.array_equal(u, ur) and np.array_equal(v, vr) and np.array_equal(b, br)
