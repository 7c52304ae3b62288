"""GPU parity of the double-word step (PD_PREC_DW) against the FP64 oracle.

PD_PREC_DW keeps the node state and the integration in FP64 and computes every
bond in double-word FP32 arithmetic (~48-bit significand), so it is held to the
FP64 bar: u within 1e-10 and v within 1e-9 relative (max node error / max node
value), the broken-bond set identical except bonds the oracle saw within 1e-9
(absolute stretch) of s_c, damage within 1e-12 plus the share of such bonds.
"""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

pytestmark = pytest.mark.gpu

DW, F64 = pdgb.PD_PREC_DW, pdgb.PD_PREC_F64
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


def oracle_run(w, steps, u0=None, v0=None):
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    m = oracle.Model.from_workload(w, off, idx)
    u = np.zeros((w.n, 3)) if u0 is None else u0.copy()
    v = np.zeros((w.n, 3)) if v0 is None else v0.copy()
    mu = m.fresh_bonds()
    margin = np.full(m.nbonds, np.inf)
    m.run(0, steps, u, v, mu, margin)
    return dict(u=u, v=v, mu=mu, margin=margin, phi=m.damage(mu), off=off, idx=idx)


def gpu_run(w, steps, precision=DW, u0=None, v0=None, **kw):
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=precision, c=c, **kw)
    if u0 is not None or v0 is not None:
        m.set_state(u0, v0)
    m.step(steps)
    m.sync()
    u, v = m.state()
    out = dict(u=u, v=v, mu=m.bonds(), phi=m.damage(), fam=m.family(), info=m.info())
    m.close()
    return out


def check(g, o, tol=1e-10):
    assert np.array_equal(g["fam"][0], o["off"]) and np.array_equal(g["fam"][1], o["idx"])
    assert rel(g["u"], o["u"]) <= tol, rel(g["u"], o["u"])
    assert rel(g["v"], o["v"]) <= tol * 10, rel(g["v"], o["v"])
    diff = g["mu"] != o["mu"]
    assert np.all(o["margin"][diff] < BAND), int(diff.sum())
    assert np.abs(g["phi"] - o["phi"]).max() <= 1e-12 + 2.0 * diff.sum() / max(len(diff), 1)


def test_tensile_bar_matches_oracle():
    w = workloads.tensile_bar()
    o = oracle_run(w, w.steps)
    assert (o["mu"] == 0).sum() > 0
    g = gpu_run(w, w.steps, graph_steps=50)
    assert g["info"]["precision"] == DW and g["info"]["step"] == w.steps
    check(g, o)


def test_notched_beam_hashed_sc_matches_oracle():
    w = workloads.notched_beam(48, 10, 12, length=0.08, rate=1e-7, steps=400)
    o = oracle_run(w, w.steps)
    assert (o["mu"] == 0).sum() > 0
    check(gpu_run(w, w.steps), o)


def test_jittered_lattice_non_uniform_volumes_and_wide_family():
    w = workloads.tensile_bar(14, 9, 8, rate=5e-7, steps=150)
    w.coords = workloads.lattice(14, 9, 8, w.dx, jitter=0.25, seed=11)
    w.horizon = 3.9 * w.dx  # families up to 255 members
    rng = np.random.default_rng(2)
    w.volumes = w.volumes * rng.uniform(0.7, 1.3, w.n)
    u0, v0 = workloads.random_state(w.n, 4, 1e-7, 1e-2)
    o = oracle_run(w, w.steps, u0=u0, v0=v0)
    g = gpu_run(w, w.steps, u0=u0, v0=v0)
    assert g["info"]["ell_width"] == 256
    check(g, o)


def test_ragged_sizes_and_degenerate_bodies():
    for shape in ((1, 1, 1), (2, 1, 1), (11, 3, 1), (37, 11, 9)):
        w = workloads.tensile_bar(*shape, rate=1e-6, slab=1, steps=30)
        u0, v0 = workloads.random_state(w.n, 1, 1e-6, 1e-1)
        o = oracle_run(w, w.steps, u0=u0, v0=v0)
        check(gpu_run(w, w.steps, u0=u0, v0=v0), o)


def test_no_fail_nodes_keep_their_bonds():
    w = workloads.tensile_bar(20, 6, 6, rate=4e-6, steps=100)
    nf = np.zeros(w.n, np.uint8)
    nf[w.bc_type[:, 0] == 1] = 1
    w.no_fail = nf
    o = oracle_run(w, w.steps)
    rows = np.repeat(np.arange(w.n), np.diff(o["off"]))
    touching = (nf[rows] == 1) | (nf[o["idx"]] == 1)
    assert o["mu"][touching].all() and (o["mu"] == 0).any()
    g = gpu_run(w, w.steps)
    assert g["mu"][touching].all()
    check(g, o)


def test_graph_direct_chunks_and_repeat_are_bitwise_equal():
    w = workloads.notched_beam(40, 8, 10, length=0.06, rate=4e-7, steps=100)
    ref = gpu_run(w, 100, graph_steps=0)
    for kw in (dict(graph_steps=16), dict(graph_steps=0)):
        g = gpu_run(w, 100, **kw)
        assert np.array_equal(g["u"], ref["u"]) and np.array_equal(g["v"], ref["v"])
        assert np.array_equal(g["mu"], ref["mu"]) and np.array_equal(g["phi"], ref["phi"])
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=DW, c=c, graph_steps=7)
    for k in (1, 13, 29, 57):
        m.step(k)
    u, v = m.state()
    m.close()
    assert np.array_equal(u, ref["u"]) and np.array_equal(v, ref["v"])


def test_restart_from_intermediate_state_is_bitwise_continuous():
    # pd_set_state rebuilds the double-word records from the FP64 state with the
    # same rounding the step kernel uses, so a restart changes nothing
    w = workloads.notched_beam(40, 8, 10, length=0.06, rate=4e-7, steps=120)
    ref = gpu_run(w, 120)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=DW, c=c)
    m.step(70)
    u, v = m.state()
    m.set_state(u, v, step=70)
    m.step(50)
    u2, v2 = m.state()
    b2 = m.bonds()
    m.close()
    assert np.array_equal(u2, ref["u"]) and np.array_equal(v2, ref["v"])
    assert np.array_equal(b2, ref["mu"])


def test_set_params_equals_fresh_handle():
    w = workloads.tensile_bar(16, 6, 6, rate=2e-6, steps=120)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    a = pdgb.Model.from_workload(w, precision=DW, c=1.3 * c)
    a.step(120)
    ua, _ = a.state()
    a.close()
    b = pdgb.Model.from_workload(w, precision=DW, c=c)
    b.set_params(1.3 * c, w.sc, w.load, w.disp_rate)
    b.step(120)
    ub, _ = b.state()
    b.close()
    assert np.array_equal(ua, ub)


def test_agrees_with_the_fp64_path():
    w = workloads.notched_beam(40, 8, 10, length=0.06, rate=4e-7, steps=200)
    g = gpu_run(w, 200)
    f = gpu_run(w, 200, precision=F64)
    assert rel(g["u"], f["u"]) <= 1e-11, rel(g["u"], f["u"])
    assert (g["mu"] == 0).sum() > 0


@pytest.mark.parametrize("ramp", [0, 300])
def test_velocity_verlet_matches_oracle(ramp):
    w = workloads.tensile_bar()
    w.ramp_steps = ramp
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx)
    u, v, acc = np.zeros((w.n, 3)), np.zeros((w.n, 3)), np.zeros((w.n, 3))
    mu = om.fresh_bonds()
    margin = np.full(len(mu), np.inf)
    om.run_vv(0, w.steps, u, v, acc, mu, init=True, margin=margin)
    assert (mu == 0).sum() > 0
    g = gpu_run(w, w.steps, graph_steps=16, integrator=pdgb.PD_INTEGRATOR_VV)
    assert rel(g["u"], u) <= 1e-10 and rel(g["v"], v) <= 1e-9
    diff = g["mu"] != mu
    assert np.all(margin[diff] < BAND), int(diff.sum())


def test_velocity_verlet_full_step_velocity_read_changes_nothing():
    w = workloads.tensile_bar(steps=300)
    ref = gpu_run(w, 300, integrator=pdgb.PD_INTEGRATOR_VV)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=DW, c=c, graph_steps=25,
                                 integrator=pdgb.PD_INTEGRATOR_VV)
    for _ in range(6):
        m.step(50)
        m.state()
        m.bonds()
    u, v = m.state()
    b = m.bonds()
    m.close()
    assert np.array_equal(u, ref["u"]) and np.array_equal(v, ref["v"])
    assert np.array_equal(b, ref["mu"])


def _grf_stiffness(w, off, idx, c0, seed=2105041505):
    om, ph = workloads.grf_params(seed, 5 * w.dx)
    rows = np.repeat(np.arange(w.n), np.diff(off))
    return c0 * (1.0 + 0.1 * workloads.grf_eval(0.5 * (w.coords[rows] + w.coords[idx]), om, ph))


def test_per_bond_stiffness_matches_oracle():
    w = workloads.cracked_plate_force(30, 16, 4, load=2e11, steps=120)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    c0 = oracle.micromodulus(w.bulk_modulus, w.horizon)
    cb = _grf_stiffness(w, off, idx, c0)
    om = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    u = np.zeros((w.n, 3)); v = np.zeros((w.n, 3)); mu = om.fresh_bonds()
    om.run(0, w.steps, u, v, mu)
    m = pdgb.Model.from_workload(w, precision=DW, c=c0, graph_steps=10)
    m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
    m.step(w.steps)
    ug, vg = m.state()
    m.close()
    assert np.abs(u).max() > 0
    assert rel(ug, u) <= 1e-10 and rel(vg, v) <= 1e-9


def test_adjoint_on_a_double_word_handle_matches_oracle_reverse_mode():
    # the adjoint's recorded and recomputed forward runs use the double-word
    # step; the reverse sweep is the FP64 one
    w = workloads.cracked_plate_force(16, 10, 3, load=3e11, steps=60)
    w.sc = 1.0
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    c0 = oracle.micromodulus(w.bulk_modulus, w.horizon)
    cb = _grf_stiffness(w, off, idx, c0, seed=2105041506)
    rows = np.repeat(np.arange(w.n), np.diff(off))
    key = {(int(i), int(j)): q for q, (i, j) in enumerate(zip(rows, idx))}
    cb = 0.5 * (cb + cb[[key[(int(j), int(i))] for i, j in zip(rows, idx)]])
    u0, v0 = workloads.random_state(w.n, 3, 1e-7, 1e-3)
    rng = np.random.default_rng(1)
    gu = rng.standard_normal((w.n, 3))
    gv = rng.standard_normal((w.n, 3)) * 1e-7
    om = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
    gc_o, gl_o, gu_o, gv_o = oracle.adjoint(om, 0, w.steps, u0, v0, om.fresh_bonds(), gu, gv)
    m = pdgb.Model.from_workload(w, precision=DW, c=c0)
    m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
    m.set_state(u0, v0, step=0)
    pdgb.pd_adjoint_forward(m.h, w.steps, 7)
    uN, vN = m.state()
    gc, gl, gu0, gv0 = pdgb.pd_adjoint_backward(m.h, gu, gv)
    uA, vA = m.state()
    m.close()
    assert np.array_equal(uN, uA) and np.array_equal(vN, vA)
    assert rel(gc, gc_o) <= 1e-9
    assert abs(gl - gl_o) <= 1e-9 * abs(gl_o)
    assert rel(gu0, gu_o) <= 1e-9 and rel(gv0, gv_o) <= 1e-9


def test_adjoint_gradient_of_small_stretches_equals_fp64_handle():
    # from rest under a force load the stretches stay small for many steps: the
    # double-word reverse step must keep s accurate in absolute terms (a form
    # like |y| / L - 1 loses it to the positions' rounding)
    w = workloads.cracked_plate_force(40, 16, 4, load=8e6, steps=300)
    c0 = oracle.micromodulus(w.bulk_modulus, w.horizon)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    cb = workloads.bond_stiffness_grf(w, off, idx, c0)
    above, below = workloads.mouth_nodes(w)
    out = {}
    for prec in (F64, DW):
        m = pdgb.Model.from_workload(w, precision=prec, c=c0)
        m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
        pdgb.pd_adjoint_forward(m.h, w.steps, 17)
        u, _ = m.state()
        gu = np.zeros((w.n, 3))
        cmod = u[above, 1].mean() - u[below, 1].mean()
        gu[above, 1] = 2 * cmod / len(above)
        gu[below, 1] = -2 * cmod / len(below)
        out[prec] = pdgb.pd_adjoint_backward(m.h, gu)
        m.close()
    (gc64, gl64, gu64, _), (gcdw, gldw, gudw, _) = out[F64], out[DW]
    assert np.abs(gc64).max() > 0
    assert rel(gcdw, gc64) <= 1e-8, rel(gcdw, gc64)
    assert abs(gldw - gl64) <= 1e-8 * abs(gl64)
    assert rel(gudw, gu64) <= 1e-8


def test_full_size_notched_beam_sampled_one_step():
    """1,009,200-node beam in the benchmark's launch configuration: one step from
    a common state with broken bonds against the oracle's step of 2000 sampled
    nodes computed one by one."""
    w = workloads.notched_beam()
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=DW, c=c, graph_steps=20)
    info = m.info()
    assert info["n"] == 1009200 and info["ell_width"] == 128 and info["precision"] == DW
    rng = np.random.default_rng(7)
    u0 = 1.0e-4 * (w.coords - w.coords.mean(axis=0)) * np.array([1.0, 0.3, 0.5])
    u0 += rng.normal(0.0, 2e-8, size=u0.shape)
    v0 = rng.normal(0.0, 1e-3, size=u0.shape)
    m.set_state(u0, v0, step=40)
    m.step(3)
    m.sync()
    u_s, v_s = m.state()
    mu_all = m.bonds()
    m.step(1)
    u_g, v_g = m.state()
    mu_g = m.bonds()
    off_g, idx_g = m.family()
    m.close()

    rows = np.sort(rng.choice(w.n, 2000, replace=False))
    rows = np.unique(np.concatenate([rows, np.nonzero(w.bc_type.any(axis=1))[0][:50],
                                     np.arange(149 * 58 * 58, 149 * 58 * 58 + 40)]))
    off_r, idx_r = oracle.cut_family(w.coords, w.horizon, w.cuts_array(), rows=rows)
    sel = np.concatenate([np.arange(off_g[i], off_g[i + 1]) for i in rows])
    assert np.array_equal(idx_g[sel], idx_r)
    mu = mu_all[sel].copy()
    assert (mu == 0).any()
    om = oracle.Model.from_workload(w, off_r, idx_r, c=c, rows=rows)
    margin = np.full(len(mu), np.inf)
    uo, vo = om.step(43, u_s, v_s, mu, margin)
    diff = mu != mu_g[sel]
    assert rel(u_g[rows], uo) <= 1e-12
    assert rel(u_g[rows] - u_s[rows], uo - u_s[rows]) <= 1e-9
    assert rel(v_g[rows], vo) <= 1e-9
    assert np.all(margin[diff] < BAND)
