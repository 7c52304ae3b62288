"""Stiffness corrections (conical micromodulus, volume surface correction):
the library's per-bond factors against the oracle's (CPU), and the GPU step
with the corrected per-bond stiffness against the oracle (GPU)."""
import numpy as np
import pytest

import oracle
import paper_2105_04150_gb300 as pdgb
import workloads

CON, SUR, PAR = pdgb.PD_STIFF_CONICAL, pdgb.PD_STIFF_SURFACE, pdgb.PD_STIFF_PARTIAL


@pytest.fixture(scope="module")
def libs():
    oracle.build()
    try:
        pdgb.lib()
    except ImportError:
        pdgb.build()
    return True


def _jittered():
    x = workloads.lattice(11, 8, 7, 1e-3, jitter=0.25, seed=5)
    rng = np.random.default_rng(6)
    vol = rng.uniform(0.6e-9, 1.4e-9, x.shape[0])
    cuts = np.array([[0, 5.5e-3, -1.0, 4.2e-3, -1.0, 1.0]])
    off, idx = oracle.cut_family(x, 3.01e-3, cuts)
    return x, vol, off, idx


@pytest.mark.parametrize("flags", [CON, SUR, CON | SUR, PAR, CON | SUR | PAR])
def test_library_factors_equal_oracle(libs, flags):
    x, vol, off, idx = _jittered()
    v0 = 122 * 1e-9
    got = pdgb.pd_stiffness_factors(x, vol, 3.01e-3, off, idx, flags, v0, dx=1e-3)
    ref = oracle.stiffness_factors(x, vol, 3.01e-3, off, idx, flags, v0, dx=1e-3)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


def test_library_factors_reject_bad_arguments(libs):
    x, vol, off, idx = _jittered()
    for flags, v0 in ((0, 1.0), (8, 1.0), (SUR, 0.0), (SUR, float("nan")), (PAR, 1.0)):
        with pytest.raises(pdgb.PdError) as e:
            pdgb.pd_stiffness_factors(x, vol, 3.01e-3, off, idx, flags, v0)
        assert e.value.name == "PD_ERR_ARG"
    bad = idx.copy()
    bad[0] = x.shape[0] + 5
    with pytest.raises(pdgb.PdError):
        pdgb.pd_stiffness_factors(x, vol, 3.01e-3, off, bad, CON)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [pdgb.PD_PREC_F64, pdgb.PD_PREC_F32])
def test_corrected_stiffness_step_matches_oracle(libs, precision):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = workloads.tensile_bar(24, 8, 8, steps=1000)
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
    fac = pdgb.pd_stiffness_factors(w.coords, w.volumes, w.horizon, off, idx, CON | SUR | PAR,
                                    122 * w.dx ** 3, dx=w.dx)
    m = pdgb.Model.from_workload(w, precision=precision, c=c)
    m.set_params(c, w.sc, w.load, w.disp_rate, c * fac)
    m.step(w.steps)
    u, v = m.state()
    b = m.bonds()
    m.close()
    om = oracle.Model.from_workload(w, off, idx, c=c, c_bond=c * fac)
    uo, vo = np.zeros((w.n, 3)), np.zeros((w.n, 3))
    mu = om.fresh_bonds()
    om.run(0, w.steps, uo, vo, mu)
    rel = np.abs(u - uo).max() / np.abs(uo).max()
    if precision == pdgb.PD_PREC_F64:
        assert rel <= 1e-10
        assert np.array_equal(b, mu)
    else:
        assert rel <= 1e-4
        assert (b != mu).sum() <= 1e-3 * len(mu)
    assert (mu == 0).sum() > 0  # the run breaks bonds
