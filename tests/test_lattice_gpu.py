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
    # under the load: the near-s_c decisions run through the stencil's resolver
    w = workloads.notched_beam(40, 9, 10, length=0.07, rate=2e-7, steps=220)
    nf = np.zeros(w.n, np.uint8)
    top = w.coords[:, 2] > w.coords[:, 2].max() - 1.5 * w.dx
    nf[top] = 1
    w.no_fail = nf
    o = oracle_run(w, w.steps)
    assert (o["mu"] == 0).sum() > 100                   # the run breaks bonds
    g = gpu_run(w, w.steps, F32, graph_steps=20)
    assert g["info"]["layout"] == LAT
    check_f32(g, o)


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
