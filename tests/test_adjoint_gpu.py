"""The hand-written adjoint (pd_adjoint_forward/backward) on the GPU, through the C ABI.

Checked against the oracle's FP64 reverse mode (1e-6 relative, the stated bar;
in practice the two agree to rounding) and against central differences of the
GPU's own forward run in random directions, with checkpoint intervals 1, 7 and
the default; the handle's state after the sweep is the forward's final state.
"""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu
F64, F32 = pdgb.PD_PREC_F64, pdgb.PD_PREC_F32


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()
    oracle.build()


def symmetric(off, idx, vals):
    rows = np.repeat(np.arange(len(off) - 1), np.diff(off))
    key = {(int(i), int(j)): q for q, (i, j) in enumerate(zip(rows, idx))}
    rev = np.array([key[(int(j), int(i))] for i, j in zip(rows, idx)])
    return 0.5 * (vals + vals[rev])


def _case(seed=0, nx=16, ny=10, nz=3, steps=60):
    w = workloads.cracked_plate_force(nx, ny, nz, load=3e11, steps=steps)
    w.bc_type[:4, 0] = 1
    w.bc_disp[:4, 0] = 1e-9
    w.disp_rate = 1.0
    w.sc = 1.0
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    rng = np.random.default_rng(seed)
    c0 = oracle.micromodulus(w.bulk_modulus, w.horizon)
    om, ph = workloads.grf_params(2105041505 + seed, 5 * w.dx)
    rows = np.repeat(np.arange(w.n), np.diff(off))
    cb = symmetric(off, idx, c0 * (1.0 + 0.1 * workloads.grf_eval(
        0.5 * (w.coords[rows] + w.coords[idx]), om, ph)))
    u0, v0 = workloads.random_state(w.n, seed + 1, 1e-7, 1e-3)
    u0[w.bc_type == 1] = 0.0
    v0[w.bc_type == 1] = 0.0
    gu = rng.standard_normal((w.n, 3))
    gv = rng.standard_normal((w.n, 3)) * 1e-7
    return w, off, idx, c0, cb, u0, v0, gu, gv, rng


def _gpu_model(w, c0, cb, u0, v0, **kw):
    m = pdgb.Model.from_workload(w, precision=F64, c=c0, **kw)
    m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
    m.set_state(u0, v0, step=0)
    return m


def _gpu_grad(w, c0, cb, u0, v0, gu, gv, C=0, **kw):
    m = _gpu_model(w, c0, cb, u0, v0, **kw)
    pdgb.pd_adjoint_forward(m.h, w.steps, C)
    uN, vN = m.state()
    out = pdgb.pd_adjoint_backward(m.h, gu, gv)
    uA, vA = m.state()
    assert np.array_equal(uN, uA) and np.array_equal(vN, vA) and m.info()["step"] == w.steps
    m.close()
    return out, uN, vN


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_adjoint_matches_oracle_reverse_mode():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case()
    om = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc_o, gl_o, gu_o, gv_o = oracle.adjoint(om, 0, w.steps, u0, v0, om.fresh_bonds(), gu, gv)
    (gc, gl, gu0, gv0), uN, _ = _gpu_grad(w, c0, cb, u0, v0, gu, gv)
    uo = u0.copy(); vo = v0.copy(); mu = om.fresh_bonds()
    om.run(0, w.steps, uo, vo, mu)
    assert rel(uN, uo) <= 1e-12
    assert rel(gc, gc_o) <= 1e-9
    assert abs(gl - gl_o) <= 1e-9 * abs(gl_o)
    assert rel(gu0, gu_o) <= 1e-9 and rel(gv0, gv_o) <= 1e-9


def test_adjoint_independent_of_checkpoint_interval():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(2, steps=50)
    ref, _, _ = _gpu_grad(w, c0, cb, u0, v0, gu, gv, C=1)
    for C in (7, 0, 50):
        got, _, _ = _gpu_grad(w, c0, cb, u0, v0, gu, gv, C=C, graph_steps=5)
        for a, b in zip(got[:1] + got[2:], ref[:1] + ref[2:]):
            assert np.array_equal(a, b)
        assert got[1] == ref[1]


def test_adjoint_matches_central_differences_of_gpu_forward():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(4, steps=40)
    (gc, gl, gu0, gv0), _, _ = _gpu_grad(w, c0, cb, u0, v0, gu, gv)

    def loss(cbv, load, uu, vv):
        m = _gpu_model(w, c0, cbv, uu, vv)
        m.set_params(c0, w.sc, load, w.disp_rate, cbv)
        m.step(w.steps)
        u, v = m.state()
        m.close()
        return float((gu * u).sum() + (gv * v).sum())

    for k in range(3):
        dc = symmetric(off, idx, rng.standard_normal(len(idx))) * c0 * 1e-6
        num = (loss(cb + dc, w.load, u0, v0) - loss(cb - dc, w.load, u0, v0)) / 2
        ana = float(gc @ dc)
        assert abs(num - ana) <= 1e-6 * abs(ana), (num, ana)
    h = 1e-6 * w.load
    num = (loss(cb, w.load + h, u0, v0) - loss(cb, w.load - h, u0, v0)) / (2 * h)
    assert abs(num - gl) <= 1e-6 * abs(gl), (num, gl)


def test_adjoint_error_paths():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(5, steps=5)
    m = pdgb.Model.from_workload(w, precision=F64, c=c0)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_adjoint_backward(m.h, gu)
    assert e.value.name == "PD_ERR_STATE"
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_adjoint_forward(m.h, 0)
    assert e.value.name == "PD_ERR_ARG"
    m.close()
    m = pdgb.Model.from_workload(w, precision=F32, c=c0)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_adjoint_forward(m.h, 5)
    assert e.value.name == "PD_ERR_STATE"
    m.close()


def test_autograd_function_returns_adjoint_gradients():
    import torch
    from paper_2105_04150_gb300 import autograd as pdag
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(6, steps=30)
    m = pdgb.Model.from_workload(w, precision=F64, c=c0)
    pdag.prepare(m, c0, w.sc, w.disp_rate)
    c_t = torch.tensor(cb, requires_grad=True)
    l_t = torch.tensor(w.load, dtype=torch.float64, requires_grad=True)
    u_t = torch.tensor(u0, requires_grad=True)
    v_t = torch.tensor(v0, requires_grad=True)
    uN = pdag.PeridynamicRun.apply(c_t, l_t, u_t, v_t, m, w.steps, 0)
    loss = (torch.tensor(gu) * uN).sum()
    loss.backward()
    (gc, gl, gu0, gv0), _, _ = _gpu_grad(w, c0, cb, u0, v0, gu, np.zeros_like(gv))
    assert np.array_equal(c_t.grad.numpy(), gc)
    assert float(l_t.grad) == gl
    assert np.array_equal(u_t.grad.numpy(), gu0) and np.array_equal(v_t.grad.numpy(), gv0)
    m.close()


def test_sensitivity_plate_full_size():
    """The 100k-node pre-cracked plate with the 10 % stiffness field: nothing
    breaks even at half the critical stretch; the gradient equals the oracle's
    reverse mode over 100 steps (checkpoints every 45: a ragged last segment)
    and central differences of the full 2000-step run on random directions."""
    w = workloads.sensitivity_plate()
    c0 = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=F64, c=c0, graph_steps=50)
    off, idx = m.family()
    cb = workloads.bond_stiffness_grf(w, off, idx, c0)
    rev = workloads.reverse_bond(w.n, off, idx)
    above, below = workloads.mouth_nodes(w)
    zero = np.zeros((w.n, 3))

    def cmod2(u):
        cm = u[above, 1].mean() - u[below, 1].mean()
        g = np.zeros_like(u)
        g[above, 1] = 2 * cm / len(above)
        g[below, 1] = -2 * cm / len(below)
        return cm * cm, g

    def loss(c_bond, load, steps):
        m.set_params(c0, w.sc, load, w.disp_rate, c_bond)
        m.set_state(zero, zero, step=0)
        m.step(steps)
        return cmod2(m.state()[0])[0]

    def grad(steps):
        m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
        m.set_state(zero, zero, step=0)
        pdgb.pd_adjoint_forward(m.h, steps, 45)
        L, g = cmod2(m.state()[0])
        gc, gl, _, _ = pdgb.pd_adjoint_backward(m.h, g)
        return g, gc, gl

    m.set_params(c0, 0.5 * w.sc, w.load, w.disp_rate, cb)
    m.set_state(zero, zero, step=0)
    m.step(w.steps)
    assert m.bonds().all()

    S = 100
    g, gc, gl = grad(S)
    om = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc_o, gl_o, _, _ = oracle.adjoint(om, 0, S, zero, zero, om.fresh_bonds(), g, None)
    assert rel(gc, gc_o) <= 1e-6 and abs(gl - gl_o) <= 1e-6 * abs(gl_o)

    _, gc, gl = grad(w.steps)
    rng = np.random.default_rng(2105041506)
    h = 1e-3
    for _ in range(4):
        r = rng.standard_normal(len(idx))
        dc = 0.5 * (r + r[rev]) * 0.1 * c0
        dl = rng.standard_normal() * 0.1 * w.load
        fd = (loss(cb + h * dc, w.load + h * dl, w.steps)
              - loss(cb - h * dc, w.load - h * dl, w.steps)) / (2 * h)
        ana = float(gc @ dc) + gl * dl
        assert abs(fd - ana) <= 1e-6 * abs(ana), (fd, ana)
    m.close()


# ---------------------------------------------------------------- velocity-Verlet
VV = pdgb.PD_INTEGRATOR_VV


@pytest.mark.parametrize("prec", [F64, pdgb.PD_PREC_DW])
def test_velocity_verlet_adjoint_matches_oracle_reverse_mode(prec):
    # the damped velocity-Verlet run from a set state (acceleration formed
    # afresh), loss on u^N and the full-step v^N, checkpoints every 7 steps;
    # both reverse sweeps (pd_adjoint_backward, and the FP64 one of
    # pd_adjoint_backward_static) against the oracle's
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(11, steps=60)
    om = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc_o, gl_o, gu_o, gv_o = oracle.adjoint(om, 0, w.steps, u0, v0, om.fresh_bonds(), gu, gv,
                                            integrator="vv")
    uo, vo, ao, mu = u0.copy(), v0.copy(), np.zeros_like(u0), om.fresh_bonds()
    om.run_vv(0, w.steps, uo, vo, ao, mu, init=True)
    m = pdgb.Model.from_workload(w, precision=prec, c=c0, integrator=VV)
    m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
    m.set_state(u0, v0, step=0)
    pdgb.pd_adjoint_forward(m.h, w.steps, 7)
    uN, vN = m.state()
    assert rel(uN, uo) <= 1e-10 and rel(vN, vo) <= 1e-9
    for backward in (pdgb.pd_adjoint_backward, pdgb.pd_adjoint_backward_static):
        gc, gl, gu0, gv0 = backward(m.h, gu, gv)
        uA, vA = m.state()
        assert np.array_equal(uN, uA) and np.array_equal(vN, vA)
        assert rel(gc, gc_o) <= 1e-9, rel(gc, gc_o)
        assert abs(gl - gl_o) <= 1e-9 * abs(gl_o)
        assert rel(gu0, gu_o) <= 1e-9 and rel(gv0, gv_o) <= 1e-9
    # without dL/dv^N the closing half kick drops out
    gc_o, gl_o, gu_o, gv_o = oracle.adjoint(om, 0, w.steps, u0, v0, om.fresh_bonds(), gu, None,
                                            integrator="vv")
    gc, gl, gu0, gv0 = pdgb.pd_adjoint_backward(m.h, gu)
    assert rel(gc, gc_o) <= 1e-9 and rel(gu0, gu_o) <= 1e-9 and rel(gv0, gv_o) <= 1e-9
    m.close()


def test_velocity_verlet_adjoint_starts_from_a_set_state():
    w, off, idx, c0, cb, u0, v0, gu, gv, rng = _case(12, steps=10)
    m = pdgb.Model.from_workload(w, precision=F64, c=c0, integrator=VV)
    pdgb.pd_adjoint_forward(m.h, 5)          # from creation: allowed
    with pytest.raises(pdgb.PdError) as e:   # mid-run: the history is not fresh
        pdgb.pd_adjoint_forward(m.h, 5)
    assert e.value.name == "PD_ERR_STATE"
    m.set_state(u0, v0)
    pdgb.pd_adjoint_forward(m.h, 5)
    m.close()
