"""GB300-native bond-based peridynamic time stepper (arXiv 2105.04150).

Thin ctypes binding over the C ABI of ``include/pd.h``: the functions keep the
C names (``pd_create``, ``pd_step``, ...) and only marshal arguments.  Every
step of the computation runs in the CUDA library ``_libpd.so`` built for
sm_103a; there is no CPU fallback, and importing the binding raises when the
library has not been built.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they must
be C-contiguous with the documented dtype.  PyTorch is only used by callers
for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any, Optional, Sequence

import numpy as np

from . import _build

__all__ = [
    "PdError", "build", "lib", "pd_micromodulus", "pd_critical_stretch", "pd_create", "pd_destroy", "pd_last_error",
    "pd_get_info", "pd_get_family", "pd_step", "pd_sync", "pd_get_state", "pd_set_state",
    "pd_get_bonds", "pd_set_bonds", "pd_remove_bonds", "pd_damage", "pd_set_params", "pd_batch_create",
    "pd_batch_offsets", "pd_autotune", "pd_test_tile_wait_extra", "pd_adjoint_forward",
    "pd_adjoint_backward",
    "pd_adjoint_backward_static", "pd_stiffness_factors", "pd_get_bond_integrity", "PD_STIFF_CONICAL",
    "PD_STIFF_SURFACE", "PD_STIFF_PARTIAL", "PD_INTEGRATOR_EC", "PD_INTEGRATOR_VV",
    "PD_LAYOUT_SELL", "PD_LAYOUT_LATTICE",
    "instance_from_workload", "Model",
    "PD_PREC_F32", "PD_PREC_F64", "PD_PREC_DW", "PD_DIM_3D", "PD_PLANE_STRESS", "PD_PLANE_STRAIN",
]

PD_PREC_F64 = 64
PD_PREC_F32 = 32
PD_PREC_DW = 48  # FP64-grade bonds in double-word FP32 arithmetic, FP64 node state
PD_STIFF_CONICAL = 1
PD_STIFF_SURFACE = 2
PD_STIFF_PARTIAL = 4
PD_PLANE_STRESS = 1  # pd_critical_stretch body kinds (Eq. 7)
PD_PLANE_STRAIN = 2
PD_DIM_3D = 3
PD_LAYOUT_SELL = 0      # pd_get_info()["layout"]: sliced ELL, the general step kernel
PD_LAYOUT_LATTICE = 1   # regular lattice: the stencil kernel (no neighbour ids read)
PD_INTEGRATOR_EC = 0
PD_INTEGRATOR_VV = 1
_STATUS = {0: "PD_OK", 1: "PD_ERR_ARG", 2: "PD_ERR_CUDA", 3: "PD_ERR_OOM",
           4: "PD_ERR_NONFINITE", 5: "PD_ERR_UNSTABLE_DT", 6: "PD_ERR_FAMILY_TOO_LARGE",
           7: "PD_ERR_TIMEOUT", 8: "PD_ERR_STATE"}


class PdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = _STATUS.get(status, str(status))


class _Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("dt", ctypes.c_double), ("damping", ctypes.c_double),
                ("density", ctypes.c_double), ("check_dt", ctypes.c_int32),
                ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("reorder", ctypes.c_int32), ("integrator", ctypes.c_int32),
                ("general", ctypes.c_int32), ("lat_variant", ctypes.c_int32)]


class _Material(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("sc", ctypes.c_double), ("sc_mode", ctypes.c_int32),
                ("model", ctypes.c_int32), ("sc_seed", ctypes.c_uint64),
                ("sc_lo", ctypes.c_double), ("sc_hi", ctypes.c_double),
                ("kr", ctypes.c_double), ("bulk_modulus", ctypes.c_double),
                ("shear_modulus", ctypes.c_double), ("kink_ratio", ctypes.c_double),
                ("kink_force", ctypes.c_double)]


class _Bc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_void_p), ("disp", ctypes.c_void_p),
                ("force", ctypes.c_void_p), ("no_fail", ctypes.c_void_p),
                ("disp_rate", ctypes.c_double), ("load", ctypes.c_double),
                ("ramp_steps", ctypes.c_int64)]


class _Instance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("coords", ctypes.c_void_p), ("volumes", ctypes.c_void_p),
                ("horizon", ctypes.c_double), ("cuts", ctypes.c_void_p), ("n_cuts", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("mat", _Material), ("bc", _Bc)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_bonds", ctypes.c_int64), ("step", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("ell_width", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("layout", ctypes.c_int32),
                ("step_registers", ctypes.c_int32), ("lat_variant", ctypes.c_int32)]


_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (sm_103a)."""
    return _build.build(force=force)


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(
                f"CUDA library {_build.LIB} is missing: run paper_2105_04150_gb300.build()")
        L = ctypes.CDLL(_build.LIB)
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        sig = {
            "pd_micromodulus": [D, D, P],
            "pd_critical_stretch": [D, D, D, I32, P],
            "pd_create": [I64, P, P, D, P, P, P, I32, P, P, P, P],
            "pd_get_info": [P, P],
            "pd_get_family": [P, P, P],
            "pd_step": [P, I64],
            "pd_sync": [P],
            "pd_get_state": [P, P, P, P],
            "pd_set_state": [P, P, P, I64],
            "pd_get_bonds": [P, P],
            "pd_set_bonds": [P, P],
            "pd_remove_bonds": [P, P, I64],
            "pd_damage": [P, P],
            "pd_set_params": [P, D, D, D, D, P],
            "pd_batch_create": [I32, P, P, P],
            "pd_batch_offsets": [P, P, P],
            "pd_autotune": [P, I32, P, P],
            "pd_test_tile_wait_extra": [P, I32],
            "pd_adjoint_forward": [P, I64, I64],
            "pd_adjoint_backward": [P, P, P, P, P, P, P],
            "pd_adjoint_backward_static": [P, P, P, P, P, P, P],
            "pd_stiffness_factors": [I64, P, P, D, P, P, I32, D, D, P],
            "pd_get_bond_integrity": [P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.pd_destroy.argtypes = [P]
        L.pd_destroy.restype = None
        L.pd_last_error.argtypes = []
        L.pd_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def pd_last_error() -> str:
    return lib().pd_last_error().decode()


def _check(st: int):
    if st != 0:
        raise PdError(st, pd_last_error())


def _ptr(a: Any, dtype, count: Optional[int] = None, writable: bool = False):
    """(address, keep-alive) of a numpy array or torch tensor; None -> (None, None)."""
    if a is None:
        return None, None
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32,
               np.uint8: torch.uint8, np.float32: torch.float32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {tdt}")
        if count is not None and a.numel() != count:
            raise ValueError(f"expected {count} elements, got {a.numel()}")
        return a.data_ptr(), a
    arr = np.asarray(a)
    if writable:
        if arr.dtype != dtype or not arr.flags.c_contiguous or not arr.flags.writeable:
            raise TypeError(f"output array must be writable C-contiguous {np.dtype(dtype)}")
    else:
        arr = np.ascontiguousarray(arr, dtype=dtype)
    if count is not None and arr.size != count:
        raise ValueError(f"expected {count} elements, got {arr.size}")
    return arr.ctypes.data, arr


def pd_micromodulus(K: float, delta: float) -> float:
    c = ctypes.c_double()
    _check(lib().pd_micromodulus(float(K), float(delta), ctypes.byref(c)))
    return c.value


def pd_critical_stretch(G_F: float, E: float, delta: float, dim: int = PD_DIM_3D) -> float:
    """s_c of Eq. 7 from the fracture energy G_F, Young's modulus E and the horizon."""
    s = ctypes.c_double()
    _check(lib().pd_critical_stretch(float(G_F), float(E), float(delta), int(dim), ctypes.byref(s)))
    return s.value


def pd_create(coords, volumes, horizon: float, *, c: float, sc: float = 0.0,
              sc_hash=None, fam_off=None, fam_idx=None, cuts=None, bc_type=None, bc_disp=None,
              bc_force=None, no_fail=None, disp_rate: float = 0.0, load: float = 0.0,
              dt: float, damping: float, density: float, precision: int = PD_PREC_F64,
              graph_steps: int = 0, check_dt: bool = False, device: int = 0, stream=None,
              block_threads: int = 0, blocks_per_sm: int = 0, reorder: int = 0,
              integrator: int = 0, ramp_steps: int = 0, kr: float = 0.0,
              state_based=None, trilinear=None, general: bool = False,
              lat_variant: int = 0) -> int:
    """Create a model; returns an opaque handle (int).  See pd.h for the semantics."""
    x, kx = _ptr(coords, np.float64)
    n = (kx.numel() if hasattr(kx, "numel") else kx.size) // 3
    vol, kv = _ptr(volumes, np.float64, n)
    fo, kfo = _ptr(fam_off, np.int64, n + 1 if fam_off is not None else None)
    fi, kfi = _ptr(fam_idx, np.int32)
    if cuts is not None and len(cuts):
        cuts_arr = np.ascontiguousarray(np.asarray(cuts, dtype=np.float64).reshape(-1, 6))
    else:
        cuts_arr = None
    cp, kc = _ptr(cuts_arr, np.float64)
    ncut = 0 if cuts_arr is None else cuts_arr.shape[0]
    if bc_type is None:
        bc_type = np.zeros((n, 3), np.uint8)
    bt, kbt = _ptr(bc_type, np.uint8, 3 * n)
    bd, kbd = _ptr(bc_disp, np.float64, 3 * n if bc_disp is not None else None)
    bf, kbf = _ptr(bc_force, np.float64, 3 * n if bc_force is not None else None)
    nf, knf = _ptr(no_fail, np.uint8, n if no_fail is not None else None)
    mat = _Material(c=float(c), sc=float(sc), sc_mode=0, kr=float(kr))
    if trilinear is not None:  # (s_1 / s_0, kink force / peak force)
        mat.kink_ratio, mat.kink_force = float(trilinear[0]), float(trilinear[1])
    if state_based is not None:  # (K, G): ordinary state-based linear solid
        mat.model = 1
        mat.bulk_modulus, mat.shear_modulus = float(state_based[0]), float(state_based[1])
    if sc_hash is not None:
        mat.sc_mode = 1
        mat.sc_seed, mat.sc_lo, mat.sc_hi = int(sc_hash[0]), float(sc_hash[1]), float(sc_hash[2])
    bc = _Bc(type=bt, disp=bd, force=bf, no_fail=nf, disp_rate=float(disp_rate),
             load=float(load), ramp_steps=int(ramp_steps))
    cfg = _config(precision, graph_steps, dt, damping, density, check_dt, device, stream,
                  block_threads, blocks_per_sm, reorder, integrator, general, lat_variant)
    h = ctypes.c_void_p()
    _check(lib().pd_create(n, x, vol, float(horizon), fo, fi, cp, ncut, ctypes.byref(mat),
                           ctypes.byref(bc), ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def pd_destroy(h: int) -> None:
    if h:
        lib().pd_destroy(h)


def pd_get_info(h: int) -> dict:
    info = _Info()
    _check(lib().pd_get_info(h, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in _Info._fields_}


def pd_get_family(h: int):
    info = pd_get_info(h)
    off = np.empty(info["n"] + 1, np.int64)
    idx = np.empty(max(info["n_bonds"], 1), np.int32)
    _check(lib().pd_get_family(h, off.ctypes.data, idx.ctypes.data))
    return off, idx[: info["n_bonds"]]


def pd_step(h: int, n_steps: int) -> None:
    _check(lib().pd_step(h, int(n_steps)))


def pd_sync(h: int) -> None:
    _check(lib().pd_sync(h))


def pd_get_state(h: int, u=None, v=None) -> int:
    """Fill u and/or v (n*3 float64, host or device); returns the step counter."""
    n = pd_get_info(h)["n"]
    up, ku = _ptr(u, np.float64, 3 * n, writable=True)
    vp, kv = _ptr(v, np.float64, 3 * n, writable=True)
    step = ctypes.c_int64()
    _check(lib().pd_get_state(h, up, vp, ctypes.byref(step)))
    return step.value


def pd_set_state(h: int, u=None, v=None, step: int = -1) -> None:
    n = pd_get_info(h)["n"]
    up, ku = _ptr(u, np.float64, 3 * n)
    vp, kv = _ptr(v, np.float64, 3 * n)
    _check(lib().pd_set_state(h, up, vp, int(step)))


def pd_get_bonds(h: int) -> np.ndarray:
    nb = pd_get_info(h)["n_bonds"]
    mu = np.empty(max(nb, 1), np.uint8)
    _check(lib().pd_get_bonds(h, mu.ctypes.data))
    return mu[:nb]


def pd_get_bond_integrity(h: int) -> np.ndarray:
    """Integrity mu in [0, 1] of every directed bond, canonical order."""
    out = np.zeros(max(pd_get_info(h)["n_bonds"], 1))
    _check(lib().pd_get_bond_integrity(h, out.ctypes.data))
    return out[: pd_get_info(h)["n_bonds"]]


def pd_set_bonds(h: int, mu) -> None:
    nb = pd_get_info(h)["n_bonds"]
    p, k = _ptr(mu, np.uint8, nb)
    if nb == 0:
        return
    _check(lib().pd_set_bonds(h, p))


def pd_remove_bonds(h: int, pairs) -> None:
    """Break the bonds (i, j) and (j, i) of every row of pairs (m x 2 node ids)."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
    _check(lib().pd_remove_bonds(h, pr.ctypes.data if pr.size else None, pr.shape[0]))


def pd_damage(h: int, phi=None):
    """Damage per node (Eq. 8) into phi (n float64, host or device) or a new numpy array."""
    n = pd_get_info(h)["n"]
    if phi is None:
        phi = np.empty(n, np.float64)
    p, k = _ptr(phi, np.float64, n, writable=True)
    _check(lib().pd_damage(h, p))
    return phi


def pd_set_params(h: int, c: float, sc: float, load: float, disp_rate: float,
                  c_bond=None) -> None:
    nb = pd_get_info(h)["n_bonds"]
    p, k = _ptr(c_bond, np.float64, nb if c_bond is not None else None)
    _check(lib().pd_set_params(h, float(c), float(sc), float(load), float(disp_rate), p))


def _config(precision, graph_steps, dt, damping, density, check_dt, device, stream,
            block_threads, blocks_per_sm, reorder, integrator=0, general=0, lat_variant=0):
    return _Config(precision=int(precision), graph_steps=int(graph_steps), dt=float(dt),
                   damping=float(damping), density=float(density), check_dt=int(bool(check_dt)),
                   device=int(device), stream=stream, block_threads=int(block_threads),
                   blocks_per_sm=int(blocks_per_sm), reorder=int(reorder),
                   integrator=int(integrator), general=int(bool(general)),
                   lat_variant=int(lat_variant))


def pd_batch_create(instances, *, dt: float, damping: float, density: float,
                    precision: int = PD_PREC_F64, graph_steps: int = 0, check_dt: bool = False,
                    device: int = 0, stream=None, block_threads: int = 0,
                    blocks_per_sm: int = 0, reorder: int = 0, integrator: int = 0,
                    lat_variant: int = 0) -> int:
    """Create a batch handle from a list of dicts with the keys of ``pd_create``'s
    body arguments: coords, volumes, horizon, c, sc / sc_hash, cuts, bc_type,
    bc_disp, bc_force, no_fail, disp_rate, load, ramp_steps, kr, trilinear,
    state_based.  lat_variant (batches of bond-based FP32 lattice models): the
    stencil kernel's register budget, 0 (64 registers) or 1 (80); pd_autotune
    chooses between them."""
    keep = []
    arr = (_Instance * len(instances))()
    for k, I in enumerate(instances):
        x, kx = _ptr(I["coords"], np.float64)
        n = kx.size // 3
        vol, kv = _ptr(I["volumes"], np.float64, n)
        cuts = I.get("cuts")
        ca = (np.ascontiguousarray(np.asarray(cuts, np.float64).reshape(-1, 6))
              if cuts is not None and len(cuts) else None)
        cp, kc = _ptr(ca, np.float64)
        bt, kbt = _ptr(I["bc_type"], np.uint8, 3 * n)
        bd, kbd = _ptr(I.get("bc_disp"), np.float64, 3 * n if I.get("bc_disp") is not None else None)
        bf, kbf = _ptr(I.get("bc_force"), np.float64, 3 * n if I.get("bc_force") is not None else None)
        nf, knf = _ptr(I.get("no_fail"), np.uint8, n if I.get("no_fail") is not None else None)
        keep += [kx, kv, kc, kbt, kbd, kbf, knf]
        mat = _Material(c=float(I["c"]), sc=float(I.get("sc", 0.0)), sc_mode=0,
                        kr=float(I.get("kr", 0.0)))
        if I.get("trilinear") is not None:  # (s_1 / s_0, kink force / peak force)
            mat.kink_ratio, mat.kink_force = float(I["trilinear"][0]), float(I["trilinear"][1])
        if I.get("state_based") is not None:  # (K, G): ordinary state-based linear solid
            mat.model = 1
            mat.bulk_modulus = float(I["state_based"][0])
            mat.shear_modulus = float(I["state_based"][1])
        if I.get("sc_hash") is not None:
            s = I["sc_hash"]
            mat.sc_mode, mat.sc_seed, mat.sc_lo, mat.sc_hi = 1, int(s[0]), float(s[1]), float(s[2])
        arr[k] = _Instance(n=n, coords=x, volumes=vol, horizon=float(I["horizon"]), cuts=cp,
                           n_cuts=0 if ca is None else ca.shape[0], mat=mat,
                           bc=_Bc(type=bt, disp=bd, force=bf, no_fail=nf,
                                  disp_rate=float(I.get("disp_rate", 0.0)),
                                  load=float(I.get("load", 0.0)),
                                  ramp_steps=int(I.get("ramp_steps", 0))))
    cfg = _config(precision, graph_steps, dt, damping, density, check_dt, device, stream,
                  block_threads, blocks_per_sm, reorder, integrator, lat_variant=lat_variant)
    h = ctypes.c_void_p()
    _check(lib().pd_batch_create(len(instances), arr, ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def pd_batch_offsets(h: int) -> np.ndarray:
    k = ctypes.c_int32()
    _check(lib().pd_batch_offsets(h, ctypes.byref(k), None))
    off = np.empty(k.value + 1, np.int64)
    _check(lib().pd_batch_offsets(h, ctypes.byref(k), off.ctypes.data))
    return off


def pd_test_tile_wait_extra(h: int, nbytes: int):
    """Test hook of the tile step's bounded wait (see pd.h)."""
    _check(lib().pd_test_tile_wait_extra(h, int(nbytes)))


def pd_autotune(h: int, trial_steps: int = 20):
    """Pick the fastest (threads per block, blocks per SM and, on lattice models,
    the stencil step's variant); the state is unchanged."""
    b, s = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().pd_autotune(h, int(trial_steps), ctypes.byref(b), ctypes.byref(s)))
    return b.value, s.value


def pd_adjoint_forward(h: int, n_steps: int, checkpoint_every: int = 0) -> None:
    """Advance n_steps with frozen bond flags, recording checkpoints for the adjoint."""
    _check(lib().pd_adjoint_forward(h, int(n_steps), int(checkpoint_every)))


def pd_adjoint_backward(h: int, dLdu, dLdv=None, want_c: bool = True):
    """Reverse sweep of the last pd_adjoint_forward.

    Returns (dL/dc per directed bond in canonical order or None, dL/dload,
    dL/du0, dL/dv0) as numpy arrays (n x 3 for the state gradients)."""
    info = pd_get_info(h)
    n, nb = info["n"], info["n_bonds"]
    up, ku = _ptr(dLdu, np.float64, 3 * n)
    vp, kv = _ptr(dLdv, np.float64, 3 * n if dLdv is not None else None)
    gc = np.zeros(max(nb, 1)) if want_c else None
    gl = ctypes.c_double()
    gu = np.empty((n, 3))
    gv = np.empty((n, 3))
    _check(lib().pd_adjoint_backward(h, up, vp, None if gc is None else gc.ctypes.data,
                                     ctypes.byref(gl), gu.ctypes.data, gv.ctypes.data))
    return (None if gc is None else gc[:nb]), gl.value, gu, gv


def pd_adjoint_backward_static(h: int, dLdu, dLdv=None, want_c: bool = True):
    """pd_adjoint_backward through the entry point that allocates no device memory
    (its working memory is a fixed static device array shared by all calls on a
    device; models above PD_STATIC_SCRATCH_BYTES of scratch raise PD_ERR_ARG).
    Same returns as pd_adjoint_backward."""
    info = pd_get_info(h)
    n, nb = info["n"], info["n_bonds"]
    up, ku = _ptr(dLdu, np.float64, 3 * n)
    vp, kv = _ptr(dLdv, np.float64, 3 * n if dLdv is not None else None)
    gc = np.zeros(max(nb, 1)) if want_c else None
    gl = ctypes.c_double()
    gu = np.empty((n, 3))
    gv = np.empty((n, 3))
    _check(lib().pd_adjoint_backward_static(h, up, vp, None if gc is None else gc.ctypes.data,
                                            ctypes.byref(gl), gu.ctypes.data, gv.ctypes.data))
    return (None if gc is None else gc[:nb]), gl.value, gu, gv


def pd_stiffness_factors(coords, volumes, horizon, off, idx, flags, v0=0.0, dx=0.0):
    """Per directed bond stiffness factors (canonical order) for the conical
    micromodulus, the volume surface correction and/or the partial volume;
    c_bond = c * factor."""
    x = np.ascontiguousarray(coords, dtype=np.float64)
    vol = np.ascontiguousarray(volumes, dtype=np.float64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = x.shape[0]
    out = np.zeros(max(idx.shape[0], 1))
    _check(lib().pd_stiffness_factors(n, x.ctypes.data, vol.ctypes.data, float(horizon),
                                      off.ctypes.data, idx.ctypes.data, int(flags), float(v0),
                                      float(dx), out.ctypes.data))
    return out[: idx.shape[0]]


def instance_from_workload(w, c=None) -> dict:
    """pd_batch_create instance dict of a workloads.Workload."""
    if c is None:
        c = pd_micromodulus(w.bulk_modulus, w.horizon)
    return dict(coords=w.coords, volumes=w.volumes, horizon=w.horizon, c=c, sc=w.sc,
                sc_hash=w.sc_hash, cuts=w.cuts_array(), bc_type=w.bc_type, bc_disp=w.bc_disp,
                bc_force=w.bc_force, no_fail=w.no_fail, disp_rate=w.disp_rate, load=w.load,
                ramp_steps=getattr(w, "ramp_steps", 0), kr=getattr(w, "kr", 0.0),
                trilinear=getattr(w, "trilinear", None),
                state_based=getattr(w, "state_based", None))


class Model:
    """Owning wrapper of one handle (calls the pd_* functions above)."""

    def __init__(self, handle=None, **kw):
        self.h = handle if handle is not None else pd_create(**kw)

    @classmethod
    def batch(cls, workload_list, precision=PD_PREC_F64, c_list=None, **kw):
        """One handle advancing every workload of the list together."""
        insts = [instance_from_workload(w, None if c_list is None else c_list[k])
                 for k, w in enumerate(workload_list)]
        w0 = workload_list[0]
        return cls(handle=pd_batch_create(insts, dt=w0.dt, damping=w0.damping,
                                          density=w0.density, precision=precision, **kw))

    def offsets(self):
        return pd_batch_offsets(self.h)

    def autotune(self, trial_steps=20):
        return pd_autotune(self.h, trial_steps)

    @classmethod
    def from_workload(cls, w, precision=PD_PREC_F64, c=None, **kw):
        if c is None:
            c = pd_micromodulus(w.bulk_modulus, w.horizon)
        return cls(coords=w.coords, volumes=w.volumes, horizon=w.horizon, c=c, sc=w.sc,
                   sc_hash=w.sc_hash, cuts=w.cuts_array(), bc_type=w.bc_type, bc_disp=w.bc_disp,
                   bc_force=w.bc_force, no_fail=w.no_fail, disp_rate=w.disp_rate, load=w.load,
                   dt=w.dt, damping=w.damping, density=w.density, precision=precision,
                   ramp_steps=getattr(w, "ramp_steps", 0), kr=getattr(w, "kr", 0.0),
                   state_based=getattr(w, "state_based", None),
                   trilinear=getattr(w, "trilinear", None), **kw)

    def close(self):
        if self.h:
            pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return pd_get_info(self.h)

    def step(self, n):
        pd_step(self.h, n)

    def sync(self):
        pd_sync(self.h)

    def state(self):
        n = self.info()["n"]
        u = np.empty((n, 3))
        v = np.empty((n, 3))
        pd_get_state(self.h, u, v)
        return u, v

    def set_state(self, u=None, v=None, step=-1):
        pd_set_state(self.h, u, v, step)

    def bonds(self):
        return pd_get_bonds(self.h)

    def set_bonds(self, mu):
        pd_set_bonds(self.h, mu)

    def remove_bonds(self, pairs):
        pd_remove_bonds(self.h, pairs)

    def damage(self, phi=None):
        return pd_damage(self.h, phi)

    def family(self):
        return pd_get_family(self.h)

    def set_params(self, c, sc, load, disp_rate, c_bond=None):
        pd_set_params(self.h, c, sc, load, disp_rate, c_bond)
