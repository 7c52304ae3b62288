"""The regular-lattice stencil kernel (FP32 Euler-Cromer PMB models whose nodes
fill a cubic lattice box with delta in [3 dx, sqrt(10) dx)) through the C ABI.

Which models take it, and that it matches the FP64 oracle (at the FP32 bar of
the parity tests: u within 1e-4 relative, v within 1e-3, broken sets within
0.1 %, damage equal to Eq. 8 of the GPU's own flags) and the general sliced-ELL
kernel on the same model: short lattice axes where a warp's offsets wrap
around lattice lines, ragged last slices, a notch, per-bond critical stretch
and no-fail nodes, per-bond stiffness; bond flags read, written and cut in
stencil order.  Lattice models keep u in FP64 and publish it rounded to FP32
for the bulk bond arithmetic (the FP32-bulk reading).
"""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

from test_parity_gpu import check_f32, gpu_run, oracle_run, rel

pytestmark = pytest.mark.gpu

F32, F64 = pdgb.PD_PREC_F32, pdgb.PD_PREC_F64
LAT, SELL = pdgb.PD_LAYOUT_LATTICE, pdgb.PD_LAYOUT_SELL


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pdgb.build()
    oracle.build()


def _layout(w, precision=F32, **kw):
    m = pdgb.Model.from_workload(w, precision=precision, **kw)
    lay = m.info()["layout"]
    m.close()
    return lay


def test_which_models_take_the_lattice_kernel():
    w = workloads.tensile_bar(20, 7, 6, rate=1e-6, steps=10)
    assert _layout(w) == LAT
    assert _layout(w, precision=F64) == SELL
    assert _layout(w, precision=pdgb.PD_PREC_DW) == SELL
    assert _layout(w, reorder=1) == SELL
    assert _layout(w, integrator=pdgb.PD_INTEGRATOR_VV) == SELL
    b = workloads.notched_beam(30, 8, 9, length=0.05, rate=1e-7, steps=10)
    assert _layout(b) == LAT                       # a notch removes bonds: still a lattice
    j = workloads.tensile_bar(12, 6, 6, rate=1e-6, steps=10)
    j.coords = workloads.lattice(12, 6, 6, j.dx, jitter=0.2, seed=3)
    assert _layout(j) == SELL                      # not on a lattice
    s = workloads.tensile_bar(12, 6, 6, rate=1e-6, steps=10)
    s.horizon = 2.01 * s.dx
    assert _layout(s) == SELL                      # a smaller stencil
    s.horizon = 3.3 * s.dx
    assert _layout(s) == SELL                      # a larger one
    v = workloads.tensile_bar(12, 6, 6, rate=1e-6, steps=10)
    v.volumes = v.volumes * np.linspace(0.9, 1.1, v.n)
    assert _layout(v) == SELL                      # non-uniform volumes
    p = workloads.tensile_bar(12, 6, 6, rate=1e-6, steps=10)
    perm = np.random.default_rng(1).permutation(p.n)
    p.coords = p.coords[perm]                      # any node order: the lattice order is internal
    assert _layout(p) == LAT


@pytest.mark.parametrize("shape", [(13, 5, 6), (9, 4, 3), (25, 11, 2), (17, 9, 8), (25, 11, 3),
                                   (7, 3, 3)])
def test_short_axes_and_ragged_slices_match_oracle(shape):
    # Nz < 7: offsets of a warp wrap across several lattice lines; n not a
    # multiple of 32 (and odd for the last two shapes: 825 and 63 nodes); a
    # random start state so that every component moves
    w = workloads.tensile_bar(*shape, rate=3e-7, slab=1, steps=80)
    u0, v0 = workloads.random_state(w.n, 7, 1e-7, 1e-2)
    o = oracle_run(w, w.steps, u0=u0, v0=v0)
    g = gpu_run(w, w.steps, F32, u0=u0, v0=v0, graph_steps=8)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)


def test_node_order_of_the_caller_is_kept():
    # nodes handed over in a shuffled order: results come back in that order
    w = workloads.tensile_bar(18, 7, 6, rate=4e-7, slab=2, steps=120)
    perm = np.random.default_rng(5).permutation(w.n)
    for name in ("coords", "volumes", "bc_type", "bc_disp"):
        setattr(w, name, np.ascontiguousarray(getattr(w, name)[perm]))
    o = oracle_run(w, w.steps)
    g = gpu_run(w, w.steps, F32)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)


def test_notched_beam_hashed_sc_no_fail_matches_oracle():
    # per-bond s_c drawn from the pair of caller ids, a notch, and a no-fail strip
    # under the load: the near-s_c decisions run through the stencil's resolver.
    # As the FP32 fracture-run reading has it, u and v are compared up to the
    # first step at which the oracle decides a bond within BAND of its s_c (a
    # decision the FP32 bulk arithmetic may move by one step, after which the
    # crack dynamics amplify the difference); the broken set and the damage of
    # the GPU's own flags are compared at the end
    from test_parity_gpu import BAND
    w = workloads.notched_beam(40, 9, 10, length=0.07, rate=2e-7, steps=220)
    nf = np.zeros(w.n, np.uint8)
    top = w.coords[:, 2] > w.coords[:, 2].max() - 1.5 * w.dx
    nf[top] = 1
    w.no_fail = nf
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    om = oracle.Model.from_workload(w, off, idx, c=c)
    u, v, mu = np.zeros((w.n, 3)), np.zeros((w.n, 3)), om.fresh_bonds()
    close = None  # oracle state before the first step with a decision within BAND
    for k in range(w.steps):
        before = dict(u=u.copy(), v=v.copy(), mu=mu.copy(), off=off, idx=idx, model=om)
        step_margin = np.full(om.nbonds, np.inf)
        om.run(k, 1, u, v, mu, step_margin)
        if close is None and step_margin.min() < BAND:
            close = (k, before)
    assert (mu == 0).sum() > 100                         # the run breaks bonds
    k, o_k = close if close is not None else (w.steps, dict(u=u, v=v, mu=mu, off=off, idx=idx,
                                                             model=om))
    assert (o_k["mu"] == 0).sum() > 100, k               # ... before the compared state
    g = gpu_run(w, k, F32, graph_steps=20)
    assert g["info"]["layout"] == LAT
    check_f32(g, o_k)
    g = gpu_run(w, w.steps, F32, graph_steps=20)
    assert (g["mu"] != mu).mean() < 1e-3
    phi_own = om.damage(np.ascontiguousarray(g["mu"], dtype=np.uint8))
    assert np.abs(g["phi"] - phi_own).max() <= 1e-5


def test_lattice_kernel_agrees_with_general_kernel():
    # the same model through both FP32 kernels (reorder = 1 takes the general
    # one): both within the FP32 bar of the oracle, and of each other
    w = workloads.notched_beam(36, 8, 9, length=0.06, rate=2e-7, steps=150)
    o = oracle_run(w, w.steps)
    a = gpu_run(w, w.steps, F32)
    b = gpu_run(w, w.steps, F32, reorder=1)
    assert a["info"]["layout"] == LAT and b["info"]["layout"] == SELL
    check_f32(a, o)
    check_f32(b, o)
    assert rel(a["u"], b["u"]) <= 1e-4, rel(a["u"], b["u"])
    assert (a["mu"] != b["mu"]).mean() < 1e-3


@pytest.mark.parametrize("state_based", [False, True])
@pytest.mark.parametrize("strain, no_fail, half",
                         [(-0.01, False, False), (0.01, True, False), (-2e-3, False, False),
                          (-0.01, False, True)])
def test_large_strains_take_the_exact_coefficient(strain, no_fail, half, state_based):
    # the walk forms num / D from its series in x = num / |xi|^2 up to |x| = 3e-3;
    # bonds past it (uniform 1 % compression, 1 % tension of a bar whose nodes are
    # all no-fail so that nothing breaks) are candidates corrected to the exact
    # coefficient, 0.2 % compression (|x| about 4e-3 and 1e-3 for the stencil's
    # offsets) mixes both: one step from that state, the force through v, against
    # the oracle.  The state-based dilation loop forms |xi| e~ from the same kind
    # of series and corrects the same candidates; its force loop takes the series
    # of |xi| / |y| and e~ / |y| on slices of nodes without a candidate, the exact
    # form on the others ("half": only the nodes past mid-length strained, so that
    # both kinds of slice meet).
    w = workloads.tensile_bar(16, 6, 7, rate=0.0, steps=1)
    if state_based:
        w.state_based = _moduli(w.bulk_modulus, 0.25)
    if no_fail:
        w.no_fail = np.ones(w.n, np.uint8)
    u0 = strain * (w.coords - w.coords.mean(axis=0))
    if half:
        u0 *= (w.coords[:, 0] > np.median(w.coords[:, 0]))[:, None]
    v0 = np.zeros_like(u0)
    o = oracle_run(w, 1, u0=u0, v0=v0)
    assert np.abs(o["v"]).max() > 0
    for variant in ((0,) if state_based else (0, 2)):
        g = gpu_run(w, 1, F32, u0=u0, v0=v0, lat_variant=variant)
        assert g["info"]["layout"] == LAT
        assert rel(g["v"], o["v"]) <= 2e-5, rel(g["v"], o["v"])
        assert np.array_equal(g["mu"], o["mu"])


def _tile_case(case):
    """(w, steps, u0, v0, c_bond) for the tile-step comparisons."""
    u0 = v0 = cb = None
    if case == "beam":       # notch, per-bond s_c, no-fail strip: breaks resolved per node
        w = workloads.notched_beam(40, 9, 10, length=0.07, rate=2e-7, steps=220)
        nf = np.zeros(w.n, np.uint8)
        nf[w.coords[:, 2] > w.coords[:, 2].max() - 1.5 * w.dx] = 1
        w.no_fail = nf
    elif case == "pbc":      # per-bond stiffness
        w = workloads.tensile_bar(16, 6, 7, rate=5e-7, steps=100)
        off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
        rows = np.repeat(np.arange(w.n), np.diff(off))
        mid = 0.5 * (w.coords[rows] + w.coords[idx])
        c = oracle.micromodulus(w.bulk_modulus, w.horizon)
        cb = c * (1.0 + 0.1 * np.sin(mid[:, 0] / w.dx) * np.cos(mid[:, 1] / w.dx))
    else:                    # short axes, ragged boxes, odd n, random start
        shape = {"odd": (25, 11, 3), "short": (13, 5, 6), "tiny": (5, 3, 2),
                 "fit": (32, 8, 16)}[case]  # fit: boxes of 16x2x8 and 8x4x8 tile it exactly
        w = workloads.tensile_bar(*shape, rate=3e-7, slab=1, steps=80)
        u0, v0 = workloads.random_state(w.n, 7, 1e-7, 1e-2)
    return w, w.steps, u0, v0, cb


def _run_variant(w, steps, u0, v0, cb, variant, restart=False, tune=False):
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=F32, c=c, lat_variant=variant, graph_steps=8)
    info = m.info()
    assert info["layout"] == LAT and info["lat_variant"] == variant
    if cb is not None:
        m.set_params(c, w.sc, w.load, w.disp_rate, cb)
    if u0 is not None:
        m.set_state(u0, v0)
    if tune:
        m.autotune(3)
    if restart:
        m.step(steps // 2)
        u, v = m.state()
        m.set_state(u, v)
        m.step(steps - steps // 2)
    else:
        m.step(steps)
    u, v = m.state()
    out = (u, v, m.bonds(), m.damage(), m.info())
    m.close()
    return out


@pytest.mark.parametrize("variant", [2, 3, 4])
@pytest.mark.parametrize("case", ["odd", "short", "tiny", "fit", "beam", "pbc", "restart"])
def test_tile_step_equals_l1_step_bitwise(case, variant):
    # records staged in shared memory by one TMA copy per block (lat_variant
    # 2..4) against the same step reading them through L1 (variant 0): the same
    # operations per node, so the same bits
    w, steps, u0, v0, cb = _tile_case("beam" if case == "restart" else case)
    a = _run_variant(w, steps, u0, v0, cb, 0, restart=case == "restart")
    b = _run_variant(w, steps, u0, v0, cb, variant, restart=case == "restart")
    assert np.abs(a[0]).max() > 0
    if case == "beam":
        assert (a[2] == 0).sum() > 100
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)


def test_autotune_over_stencil_variants_keeps_results():
    w, steps, u0, v0, cb = _tile_case("odd")
    a = _run_variant(w, steps, u0, v0, cb, 0)
    b = _run_variant(w, steps, u0, v0, cb, 0, tune=True)
    assert 0 <= b[4]["lat_variant"] <= 4
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)


def test_tile_step_bounded_wait_reports_timeout_and_recovers():
    # the test hook makes every block's barrier wait for bytes no copy delivers:
    # the wait runs out, the next synchronising call reports PD_ERR_TIMEOUT, and
    # after a state reset the handle steps as a fresh one
    w, steps, u0, v0, _ = _tile_case("tiny")
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=F32, c=c, lat_variant=2)
    m.set_state(u0, v0)
    pdgb.pd_test_tile_wait_extra(m.h, 16)
    m.step(1)
    with pytest.raises(pdgb.PdError) as e:
        m.sync()
    assert e.value.name == "PD_ERR_TIMEOUT"
    pdgb.pd_test_tile_wait_extra(m.h, 0)
    m.set_state(u0, v0, step=0)
    m.step(steps)
    u, v = m.state()
    ref = _run_variant(w, steps, u0, v0, None, 0)
    assert np.array_equal(u, ref[0]) and np.array_equal(v, ref[1])
    m.close()


def test_stencil_variants_only_on_bond_based_lattice_handles():
    # lat_variant != 0 on a model that does not run the bond-based stencil step
    # (the general layout, FP64, the state-based model) is refused
    w = workloads.tensile_bar(12, 6, 6, rate=1e-6, steps=10)
    for variant in (1, 2):
        for kw in ({"precision": F32, "reorder": 1}, {"precision": F64}):
            with pytest.raises(pdgb.PdError) as e:
                pdgb.Model.from_workload(w, lat_variant=variant, **kw)
            assert e.value.name == "PD_ERR_ARG"
    s = workloads.tensile_bar(12, 6, 6, rate=1e-6, steps=10)
    s.state_based = _moduli(s.bulk_modulus, 0.25)
    with pytest.raises(pdgb.PdError):
        pdgb.Model.from_workload(s, precision=F32, lat_variant=2)
    m = pdgb.Model.from_workload(w, precision=F32, lat_variant=3)
    assert m.info()["lat_variant"] == 3
    m.close()


def test_per_bond_stiffness_on_a_lattice_handle():
    # per-bond c read per stencil slot by the lattice kernel
    w = workloads.tensile_bar(16, 6, 7, rate=5e-7, steps=100)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    rows = np.repeat(np.arange(w.n), np.diff(off))
    mid = 0.5 * (w.coords[rows] + w.coords[idx])
    cb = c * (1.0 + 0.1 * np.sin(mid[:, 0] / w.dx) * np.cos(mid[:, 1] / w.dx))
    o = oracle_run(w, w.steps, c=c, c_bond=cb, off_idx=(off, idx))
    g = gpu_run(w, w.steps, F32, c=c, c_bond=cb)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)


def test_bond_flags_round_trip_and_cut_in_stencil_order():
    w = workloads.tensile_bar(14, 6, 6, rate=2e-6, steps=60)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    m = pdgb.Model.from_workload(w, precision=F32, c=c)
    assert m.info()["layout"] == LAT
    off, idx = m.family()
    rng = np.random.default_rng(9)
    mu = (rng.random(len(idx)) > 0.2).astype(np.uint8)
    rows = np.repeat(np.arange(w.n), np.diff(off))
    key = np.minimum(rows, idx) * w.n + np.maximum(rows, idx)
    _, inv = np.unique(key, return_inverse=True)
    mu = mu[np.unique(key, return_index=True)[1]][inv]   # symmetric flags
    m.set_bonds(mu)
    assert np.array_equal(m.bonds(), mu)
    # cut a few intact pairs: exactly those directions become 0
    pairs = np.stack([rows, idx], 1)[(mu == 1) & (rows < idx)][:25]
    m.remove_bonds(pairs)
    expect = mu.copy()
    for i, j in pairs:
        expect[(rows == i) & (idx == j)] = 0
        expect[(rows == j) & (idx == i)] = 0
    assert np.array_equal(m.bonds(), expect)
    # and a run from those flags equals the oracle's from the same flags
    om = oracle.Model.from_workload(w, off, idx, c=c)
    u = np.zeros((w.n, 3)); v = np.zeros((w.n, 3)); omu = expect.copy()
    om.run(0, w.steps, u, v, omu)
    m.step(w.steps)
    ug, vg = m.state()
    assert rel(ug, u) <= 1e-4 and (m.bonds() != omu).mean() < 1e-3
    m.close()


# ------------------------------------------------------------------ batches of lattices
def _lattice_instances():
    ws = [workloads.tensile_bar(16, 5, 5, rate=2e-6, steps=80, K=5e9, sc=3e-3),
          workloads.notched_beam(30, 6, 8, length=0.05, rate=3e-7, steps=80),   # delta = pi dx
          workloads.tensile_bar(11, 4, 3, rate=3e-6, slab=2, steps=80, K=2e10, sc=2e-3),
          workloads.cracked_plate_force(14, 10, 3, load=4e11, steps=80),       # body force
          workloads.tensile_bar(20, 3, 3, rate=4e-6, steps=80, K=8e9, sc=1.5e-3)]
    for w in ws:
        w.dt, w.damping, w.density = 1e-7, 2.5e6, 2400.0
        w.disp_rate, w.load = 1.0, 4e11
    return ws


def test_lattice_batch_matches_oracle_per_instance():
    # instances of different shapes, spacings and horizons (3.01 dx and pi dx),
    # per-bond s_c in one of them, a body force in another, concatenated so that
    # 32-node slices straddle instances: each instance against its own oracle run
    ws = _lattice_instances()
    bm = pdgb.Model.batch(ws, precision=F32, graph_steps=16)
    assert bm.info()["layout"] == LAT
    off = bm.offsets()
    bm.step(80)
    u, v = bm.state()
    mu = bm.bonds()
    phi = bm.damage()
    boff, _ = bm.family()
    bm.close()
    broke = 0
    for k, w in enumerate(ws):
        o = oracle_run(w, 80)
        s = slice(off[k], off[k + 1])
        mk = mu[boff[off[k]]:boff[off[k + 1]]]
        broke += int((o["mu"] == 0).sum())
        assert rel(u[s], o["u"]) <= 1e-4, (k, rel(u[s], o["u"]))
        assert rel(v[s], o["v"]) <= 1e-3, (k, rel(v[s], o["v"]))
        assert (mk != o["mu"]).mean() < 1e-3
        phi_own = o["model"].damage(np.ascontiguousarray(mk, dtype=np.uint8))
        assert np.abs(phi[s] - phi_own).max() <= 1e-5
    assert broke > 0


def test_lattice_batch_only_when_every_instance_is_a_lattice():
    ws = _lattice_instances()
    bm = pdgb.Model.batch(ws, precision=F32)
    assert bm.info()["layout"] == LAT
    bm.close()
    j = workloads.tensile_bar(10, 5, 5, rate=1e-6, steps=10)
    j.coords = workloads.lattice(10, 5, 5, j.dx, jitter=0.2, seed=1)
    j.dt, j.damping, j.density, j.disp_rate, j.load = 1e-7, 2.5e6, 2400.0, 1.0, 4e11
    bm = pdgb.Model.batch(ws + [j], precision=F32)
    assert bm.info()["layout"] == SELL
    bm.close()
    bm = pdgb.Model.batch(ws, precision=F64)
    assert bm.info()["layout"] == SELL
    bm.close()


def test_lattice_batch_bond_flags_and_cuts():
    # flags read and written in canonical order, and a cut into one instance
    ws = _lattice_instances()[:3]
    bm = pdgb.Model.batch(ws, precision=F32)
    off = bm.offsets()
    boff, bidx = bm.family()
    rows = np.repeat(np.arange(int(off[-1])), np.diff(boff))
    mu = bm.bonds()
    assert mu.all()
    k = 1  # the beam: cut the first 20 pairs of its row of node off[1] + 500
    i = int(off[k]) + 500
    js = bidx[boff[i]:boff[i + 1]][:20]
    bm.remove_bonds(np.stack([np.full(len(js), i), js], 1))
    mu2 = bm.bonds()
    gone = ((rows == i) & np.isin(bidx, js)) | (np.isin(rows, js) & (bidx == i))
    assert np.array_equal(mu2 == 0, gone)
    bm.set_bonds(mu)
    assert np.array_equal(bm.bonds(), mu)
    bm.close()


# ------------------------------------------------------------------ state-based on a lattice
def _moduli(K, nu):
    return (K, 3.0 * K * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu)))


@pytest.mark.parametrize("nu", [0.25, 0.33])
def test_state_based_lattice_matches_oracle_and_general_kernel(nu):
    # the two stencil loops (dilation, force) against the oracle's two loops, and
    # the general state-based kernels (general = 1) on the same model.  As for
    # every FP32 fracture run (R13), u is compared early in the fracture (50
    # steps: 11k-15k bonds broken) and the broken set later: on this beam with
    # nu = 0.33 both FP32 kernels separate from the oracle once fracture runs
    # (lattice from about step 100, general from 125), through breaks that move
    # by a step; nu = 0.25 (no dilation term: 3K = 5G) stays at ~1e-7 to step 150.
    w = workloads.notched_beam(36, 8, 9, length=0.06, rate=2e-7, steps=50)
    w.state_based = _moduli(w.bulk_modulus, nu)
    o = oracle_run(w, w.steps)
    assert (o["mu"] == 0).sum() > 5000
    g = gpu_run(w, w.steps, F32, graph_steps=10)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)
    b = gpu_run(w, w.steps, F32, general=True)
    assert b["info"]["layout"] == SELL
    check_f32(b, o)
    o = oracle_run(w, 150)
    for kw in ({}, {"general": True}):
        g = gpu_run(w, 150, F32, **kw)
        assert (g["mu"] != o["mu"]).mean() < 1e-3
        if nu == 0.25:
            check_f32(g, o)


def test_state_based_lattice_tensile_bar():
    # u before the first breaks (400 steps), the broken set after 1000 (R13)
    w = workloads.tensile_bar(steps=1000)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    o = oracle_run(w, 400)
    assert (o["mu"] == 0).sum() == 0
    g = gpu_run(w, 400, F32, graph_steps=16)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)
    o = oracle_run(w, 1000)
    g = gpu_run(w, 1000, F32, graph_steps=16)
    assert (o["mu"] == 0).sum() > 0 and (g["mu"] != o["mu"]).mean() < 1e-3


def test_state_based_lattice_short_axes_random_state():
    w = workloads.tensile_bar(13, 5, 4, rate=3e-7, slab=1, steps=60)
    w.state_based = _moduli(w.bulk_modulus, 0.3)
    u0, v0 = workloads.random_state(w.n, 3, 1e-7, 1e-2)
    o = oracle_run(w, w.steps, u0=u0, v0=v0)
    g = gpu_run(w, w.steps, F32, u0=u0, v0=v0)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)
