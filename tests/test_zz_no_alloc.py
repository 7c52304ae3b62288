"""pd_adjoint_backward_static (no device allocation, static scratch) against
pd_adjoint_backward, through the C ABI on the GPU.

Collected last on purpose: it must give the same gradients whether it runs
alone in a fresh process or after every other test has used the device.
"""
import numpy as np
import pytest

import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu
F64 = pdgb.PD_PREC_F64
TOL = 1e-9  # relative, as the adjoint's parity tests


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()


def _model(nx, ny, nz, steps, seed, precision=F64, integrator=pdgb.PD_INTEGRATOR_EC):
    w = workloads.cracked_plate_force(nx, ny, nz, load=3e11, steps=steps)
    w.bc_type[:4, 0] = 1
    w.bc_disp[:4, 0] = 1e-9
    w.disp_rate = 1.0
    w.sc = 1.0
    c0 = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=precision, c=c0, integrator=integrator)
    off, idx = m.family()
    rows = np.repeat(np.arange(w.n), np.diff(off))
    om, ph = workloads.grf_params(2105041507 + seed, 5 * w.dx)
    g = workloads.grf_eval(0.5 * (w.coords[rows] + w.coords[idx]), om, ph)  # symmetric in i, j
    m.set_params(c0, w.sc, w.load, w.disp_rate, c0 * (1.0 + 0.1 * g))
    u0, v0 = workloads.random_state(w.n, seed, 1e-7, 1e-3)
    u0[w.bc_type == 1] = 0.0
    v0[w.bc_type == 1] = 0.0
    m.set_state(u0, v0, step=0)
    rng = np.random.default_rng(seed)
    return w, m, rng.standard_normal((w.n, 3)), rng.standard_normal((w.n, 3)) * 1e-7


def _close(a, b):
    return np.abs(a - b).max() <= TOL * max(np.abs(b).max(), 1e-300)


def _same(got, ref):
    assert _close(got[0], ref[0]), "dL/dc"
    assert abs(got[1] - ref[1]) <= TOL * abs(ref[1]), "dL/dload"
    assert _close(got[2], ref[2]) and _close(got[3], ref[3]), "dL/du0, dL/dv0"


def test_static_backward_matches_allocating_backward_twice():
    w, m, gu, gv = _model(16, 10, 3, 45, 11)
    pdgb.pd_adjoint_forward(m.h, w.steps, 7)
    uN, vN = m.state()
    ref = pdgb.pd_adjoint_backward(m.h, gu, gv)
    for _ in range(2):  # the second call finds the first call's data in the shared array
        got = pdgb.pd_adjoint_backward_static(m.h, gu, gv)
        _same(got, ref)
        u, v = m.state()
        assert np.array_equal(u, uN) and np.array_equal(v, vN) and m.info()["step"] == w.steps
    m.close()


@pytest.mark.parametrize("precision", [F64, pdgb.PD_PREC_DW])
@pytest.mark.parametrize("integrator", [pdgb.PD_INTEGRATOR_EC, pdgb.PD_INTEGRATOR_VV])
def test_static_backward_on_every_accepted_handle(precision, integrator):
    # double-word handles (the static sweep is the FP64 one; the allocating
    # sweep is in double-word arithmetic, equal to ~1e-10) and velocity-Verlet
    # handles (half kicks at both ends of the run), each called twice in a row
    w, m, gu, gv = _model(14, 9, 3, 30, 21 + precision + integrator, precision, integrator)
    pdgb.pd_adjoint_forward(m.h, w.steps, 6)
    uN, vN = m.state()
    for dv in (gv, None):
        ref = pdgb.pd_adjoint_backward(m.h, gu, dv)
        for _ in range(2):
            _same(pdgb.pd_adjoint_backward_static(m.h, gu, dv), ref)
            u, v = m.state()
            assert np.array_equal(u, uN) and np.array_equal(v, vN)
    m.close()


def test_static_backward_writes_device_outputs():
    # every input and output a device pointer: dL/dc is then written in place by
    # the scatter to canonical order, without the host staging copy
    import ctypes
    import torch
    w, m, gu, gv = _model(15, 9, 3, 25, 31)
    pdgb.pd_adjoint_forward(m.h, w.steps, 5)
    ref = pdgb.pd_adjoint_backward(m.h, gu, gv)
    info = m.info()
    n, nb = info["n"], info["n_bonds"]
    dev = torch.device("cuda", 0)
    du = torch.from_numpy(np.ascontiguousarray(gu)).to(dev)
    dv = torch.from_numpy(np.ascontiguousarray(gv)).to(dev)
    for _ in range(2):
        gc = torch.full((nb,), float("nan"), dtype=torch.float64, device=dev)
        g0 = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        g1 = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        gl = ctypes.c_double()
        torch.cuda.synchronize()
        st = pdgb.lib().pd_adjoint_backward_static(m.h, du.data_ptr(), dv.data_ptr(),
                                                   gc.data_ptr(), ctypes.byref(gl),
                                                   g0.data_ptr(), g1.data_ptr())
        assert st == 0, pdgb.lib().pd_last_error()
        torch.cuda.synchronize()
        _same((gc.cpu().numpy(), gl.value, g0.cpu().numpy(), g1.cpu().numpy()), ref)
    m.close()


def test_static_backward_after_a_larger_model_used_the_array():
    wa, a, gua, gva = _model(12, 8, 3, 20, 12)
    wb, b, gub, gvb = _model(20, 12, 3, 20, 13)
    for w, m in ((wa, a), (wb, b)):
        pdgb.pd_adjoint_forward(m.h, w.steps, 0)
    ref_a = pdgb.pd_adjoint_backward(a.h, gua, gva)
    ref_b = pdgb.pd_adjoint_backward(b.h, gub, gvb)
    _same(pdgb.pd_adjoint_backward_static(b.h, gub, gvb), ref_b)
    _same(pdgb.pd_adjoint_backward_static(a.h, gua, gva), ref_a)
    _same(pdgb.pd_adjoint_backward_static(a.h, gua, None), pdgb.pd_adjoint_backward(a.h, gua))
    a.close()
    b.close()


def test_static_backward_rejects_models_above_the_maximum():
    w = workloads.tensile_bar(120, 30, 30)
    m = pdgb.Model.from_workload(w, precision=F64)
    pdgb.pd_adjoint_forward(m.h, 1, 0)
    gu = np.zeros((w.n, 3))
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_adjoint_backward_static(m.h, gu)
    assert e.value.name == "PD_ERR_ARG" and "static maximum" in str(e.value)
    m.close()
    m = pdgb.Model.from_workload(workloads.tensile_bar(8, 4, 4), precision=F64)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_adjoint_backward_static(m.h, np.zeros((m.info()["n"], 3)))
    assert e.value.name == "PD_ERR_STATE"
    m.close()
