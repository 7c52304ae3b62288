"""CPU checks of the C-ABI library: it builds, loads, exports every declared
symbol, and its host-side validation rejects bad input with status codes.
No test here launches GPU work."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pdgb.build()
    return pdgb.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "pd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(L):
    names = _declared()
    assert "pd_create" in names and "pd_step" in names and "pd_damage" in names
    out = subprocess.run(["nm", "-D", "--defined-only", pdgb._build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pd_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)


def test_micromodulus_matches_oracle(L):
    for K, d in ((5e9, 3.01e-3), (3e10, np.pi / 600), (37e9 / 1.5, 0.0157)):
        assert pdgb.pd_micromodulus(K, d) == oracle.micromodulus(K, d)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_micromodulus(-1.0, 1.0)
    assert e.value.name == "PD_ERR_ARG"



def test_critical_stretch_matches_oracle(L):
    kinds = {pdgb.PD_DIM_3D: "3d", pdgb.PD_PLANE_STRESS: "plane_stress",
             pdgb.PD_PLANE_STRAIN: "plane_strain"}
    for G_F, E, d in [(120.0, 37e9, 0.0157), (6.9e4, 190e9, 4.7e-3), (1.0, 1.0, 1.0)]:
        for dim, kind in kinds.items():
            got = pdgb.pd_critical_stretch(G_F, E, d, dim)
            want = oracle.critical_stretch(G_F, E, d, kind)
            assert abs(got - want) <= 1e-15 * want
    for bad in [(-1.0, 1.0, 1.0, 3), (1.0, 0.0, 1.0, 3), (1.0, 1.0, float("inf"), 3),
                (1.0, 1.0, 1.0, 0), (1.0, 1.0, 1.0, 4)]:
        with pytest.raises(pdgb.PdError):
            pdgb.pd_critical_stretch(*bad)

def _args(w, **over):
    kw = dict(coords=w.coords, volumes=w.volumes, horizon=w.horizon, c=1e20, sc=1e-3,
              bc_type=w.bc_type, bc_disp=w.bc_disp, dt=1e-7, damping=0.0, density=2400.0)
    kw.update(over)
    return kw


@pytest.mark.parametrize("over, status", [
    (dict(horizon=-1.0), "PD_ERR_ARG"),
    (dict(c=0.0), "PD_ERR_ARG"),
    (dict(sc=-1.0), "PD_ERR_ARG"),
    (dict(dt=0.0), "PD_ERR_ARG"),
    (dict(density=float("nan")), "PD_ERR_ARG"),
    (dict(precision=16), "PD_ERR_ARG"),
    (dict(graph_steps=-2), "PD_ERR_ARG"),
    (dict(block_threads=48), "PD_ERR_ARG"),
    (dict(sc_hash=(1, 2e-4, 1e-4)), "PD_ERR_ARG"),
    # integrators, loading ramp, softening laws, state-based model
    (dict(integrator=2), "PD_ERR_ARG"),
    (dict(ramp_steps=-1), "PD_ERR_ARG"),
    (dict(kr=0.5), "PD_ERR_ARG"),
    (dict(kr=float("inf")), "PD_ERR_ARG"),
    (dict(kr=4.0, trilinear=(5.0, 0.25)), "PD_ERR_ARG"),      # kink past s_c
    (dict(kr=4.0, trilinear=(2.0, 1.5)), "PD_ERR_ARG"),       # kink force above the peak
    (dict(trilinear=(2.0, 0.25)), "PD_ERR_ARG"),              # kink without softening
    (dict(state_based=(0.0, 1e9)), "PD_ERR_ARG"),
    (dict(state_based=(1e9, -1.0)), "PD_ERR_ARG"),
    (dict(state_based=(1e9, 1e9), kr=2.0), "PD_ERR_ARG"),
])
def test_create_rejects_bad_arguments(L, over, status):
    w = workloads.tensile_bar(6, 4, 4)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_create(**_args(w, **over))
    assert e.value.name == status


def test_create_rejects_an_empty_body(L):
    w = workloads.tensile_bar(6, 4, 4)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_create(**_args(w, coords=np.zeros((0, 3)), volumes=np.zeros(0),
                               bc_type=np.zeros((0, 3), np.uint8), bc_disp=np.zeros((0, 3))))
    assert e.value.name == "PD_ERR_ARG" and "n must be" in str(e.value)


def test_batch_rejects_differing_softening_laws(L):
    # the softening law is handle-wide: every instance must agree with instance 0
    # (checked before any device work)
    ws = [workloads.tensile_bar(6, 4, 4), workloads.tensile_bar(7, 4, 4)]
    for (kr0, t0), (kr1, t1) in (((2.0, None), (3.0, None)), ((0.0, None), (2.0, None)),
                                 ((4.0, (2.0, 0.25)), (4.0, (2.0, 0.5)))):
        ws[0].kr, ws[0].trilinear, ws[1].kr, ws[1].trilinear = kr0, t0, kr1, t1
        with pytest.raises(pdgb.PdError) as e:
            pdgb.Model.batch(ws, precision=pdgb.PD_PREC_DW)
        assert e.value.name == "PD_ERR_ARG" and "instance 1" in str(e.value)


def test_create_rejects_bad_geometry_and_family(L):
    w = workloads.tensile_bar(6, 4, 4)
    x = w.coords.copy()
    x[3, 1] = np.inf
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_create(**_args(w, coords=x))
    assert e.value.name == "PD_ERR_ARG"
    vol = w.volumes.copy()
    vol[0] = 0.0
    with pytest.raises(pdgb.PdError):
        pdgb.pd_create(**_args(w, volumes=vol))
    off, idx = oracle.family(w.coords, w.horizon)
    bad = idx.copy()
    bad[0] = 0  # self bond of node 0
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_create(**_args(w, fam_off=off, fam_idx=bad))
    assert "self" in str(e.value)
    # asymmetric family: drop one direction
    with pytest.raises(pdgb.PdError) as e:
        o2 = off.copy()
        o2[1:] -= 1
        pdgb.pd_create(**_args(w, fam_off=o2, fam_idx=idx[1:].copy()))
    assert e.value.name == "PD_ERR_ARG"


def test_create_rejects_too_many_bc_classes(L):
    w = workloads.tensile_bar(8, 6, 6)
    bt = np.ones((w.n, 3), np.uint8)
    g = np.arange(3 * w.n, dtype=np.float64).reshape(-1, 3)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_create(**_args(w, bc_type=bt, bc_disp=g))
    assert "256" in str(e.value)


def test_create_rejects_unstable_dt(L):
    w = workloads.tensile_bar(8, 4, 4)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_create(**_args(w, c=c, dt=1e-5, check_dt=True))
    assert e.value.name == "PD_ERR_UNSTABLE_DT"


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(pdgb, "_lib", None)
    monkeypatch.setattr(pdgb._build, "LIB", "/nonexistent/_libpd.so")
    with pytest.raises(ImportError):
        pdgb.lib()


def test_batch_create_rejects_bad_instances(L):
    w = workloads.tensile_bar(6, 4, 4)
    inst = pdgb.instance_from_workload(w, c=1e20)
    bad = dict(inst, horizon=-1.0)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_batch_create([inst, bad], dt=1e-7, damping=0.0, density=2400.0)
    assert e.value.name == "PD_ERR_ARG" and "instance 1" in str(e.value)
    other = dict(inst, load=5.0)
    with pytest.raises(pdgb.PdError) as e:
        pdgb.pd_batch_create([inst, other], dt=1e-7, damping=0.0, density=2400.0)
    assert "disp_rate, load and ramp_steps" in str(e.value)
    with pytest.raises(pdgb.PdError):
        pdgb.pd_batch_create([inst], dt=0.0, damping=0.0, density=2400.0)
