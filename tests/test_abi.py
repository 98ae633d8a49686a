"""C-ABI boundary checks that need no GPU: the library builds and loads, it
exports every function include/vbc.h declares, and argument validation
rejects bad configurations before any CUDA call is made."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2609_07842_b300 import build as vbuild
from paper_2609_07842_b300 import vbc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    vbuild.build()
    return vbc.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "vbc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vbc_[a-z_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert sorted(vbc.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {vbc.LIB_PATH}").read()
    for name in _declared():
        assert re.search(rf"\bT {name}\b", out), name


def test_library_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(vbuild.NVCC_FLAGS)


def test_every_source_triggers_a_rebuild():
    """A change to any source or header of the library makes build() recompile it,
    so a stale libvbc.so cannot pass for the current sources."""
    csrc = os.path.join(ROOT, "paper_2609_07842_b300", "csrc")
    srcs = {os.path.join(csrc, f) for f in os.listdir(csrc)} | {os.path.join(ROOT, "include", "vbc.h")}
    assert srcs <= set(vbuild.DEPS)


def _cfg(n=100, box=(12.0, 12.0, 12.0), prec=vbc.VBC_FP32_SPLIT, skin=0.4, **prm):
    pos = np.zeros((max(n, 1), 3))
    c = vbc._Config(n=n, box=(ctypes.c_double * 3)(*box), pos=ctypes.c_void_p(pos.ctypes.data), vel=None,
                    params=vbc.params(**prm), skin=skin, seed=1, precision=prec, nlist_cap=0,
                    stream=None, inputs_on_device=0)
    return c, pos


@pytest.mark.parametrize("kw,needle", [
    (dict(n=0), "n must be"),
    (dict(box=(12.0, 12.0, -1.0)), "box edges"),
    (dict(box=(12.0, 12.0, 13.0)), "cubic"),
    (dict(box=(6.0, 6.0, 6.0)), "fewer than 3 cells"),
    (dict(skin=0.0), "skin"),
    (dict(prec=7), "precision"),
    (dict(r_a=0.5), "pair parameters"),
    (dict(r_l=2.0, r_h=1.0), "pair parameters"),
    (dict(E_a=-1.0), "pair parameters"),
    (dict(f=float("nan")), "pair parameters"),
])
def test_create_rejects_bad_arguments(lib, kw, needle):
    c, _keep = _cfg(**kw)
    h = ctypes.c_void_p()
    rc = lib.vbc_create_system(ctypes.byref(c), ctypes.byref(h))
    assert rc == vbc.VBC_ERR_INVALID_ARG
    assert needle in lib.vbc_last_error().decode()
    assert not h.value


def test_null_arguments(lib):
    assert lib.vbc_create_system(None, None) == vbc.VBC_ERR_INVALID_ARG
    assert lib.vbc_build_neighbors(None) == vbc.VBC_ERR_INVALID_ARG
    assert lib.vbc_step_langevin(None, 1, 0.01, 1.0, 1.0) == vbc.VBC_ERR_INVALID_ARG
    assert lib.vbc_compute_forces(None, None, None, None, None, 0) == vbc.VBC_ERR_INVALID_ARG
    lib.vbc_destroy(None)  # accepted


def test_orthorhombic_box_allowed_in_fp64_until_device_needed(lib):
    """A non-cubic box passes validation in FP64 mode; without a GPU the call then
    fails with a CUDA error (not a crash, not a CPU fallback)."""
    import torch
    c, _keep = _cfg(box=(12.0, 13.0, 14.0), prec=vbc.VBC_FP64)
    h = ctypes.c_void_p()
    rc = lib.vbc_create_system(ctypes.byref(c), ctypes.byref(h))
    if torch.cuda.is_available():
        assert rc == vbc.VBC_OK
        lib.vbc_destroy(h)
    else:
        assert rc in (vbc.VBC_ERR_CUDA, vbc.VBC_ERR_OOM)
        assert not h.value


# ----------------------------------------------------------------- multi-type creation (host checks)
def _typed(n=100, T=2, types=None, pair=None, mask=None, bonds=None, k_bond=100.0, r0=1.0,
           prec=vbc.VBC_FP64):
    c, keep = _cfg(n=n, prec=prec)
    t = np.ascontiguousarray(np.zeros(n) if types is None else types, dtype=np.int32)
    P = pair if pair is not None else [[vbc.params(E_a=0.0), vbc.params(E_a=0.0)],
                                       [vbc.params(E_a=0.0), vbc.params(E_a=10.0, f=1.0)]][:T]
    tab = (vbc.PairParams * (T * T))(*[P[a][b] for a in range(T) for b in range(T)])
    m = np.ascontiguousarray(np.asarray([[0, 0], [0, 1]] if mask is None else mask, dtype=np.int32).reshape(-1))
    bd = np.ascontiguousarray(np.zeros((0, 2)) if bonds is None else bonds, dtype=np.int64).reshape(-1, 2)
    ty = vbc._Types(ntypes=T, type=ctypes.c_void_p(t.ctypes.data), pair=ctypes.cast(tab, ctypes.c_void_p),
                    count_mask=ctypes.c_void_p(m.ctypes.data), nbonds=bd.shape[0],
                    bonds=ctypes.c_void_p(bd.ctypes.data) if bd.shape[0] else None, k_bond=k_bond, r0_bond=r0)
    return c, ty, (keep, t, tab, m, bd)


@pytest.mark.parametrize("kw,needle", [
    (dict(prec=7), "precision"),
    (dict(T=0), "ntypes"),
    (dict(types=np.full(100, 2)), "type of particle"),
    (dict(types=np.full(100, -1)), "type of particle"),
    (dict(mask=[[0, 0], [0, 3]]), "0 or 1"),
    (dict(pair=[[vbc.params(E_a=0.0), vbc.params(E_a=1.0)], [vbc.params(E_a=0.0), vbc.params()]]), "symmetric"),
    (dict(pair=[[vbc.params(r_a=0.5), vbc.params()], [vbc.params(), vbc.params()]]), "pair parameters"),
    (dict(bonds=[[0, 100]]), "bond 0"),
    (dict(bonds=[[0, 1], [5, 5]]), "bond 1"),
    (dict(k_bond=-1.0), "k_bond"),
    (dict(r0=float("inf")), "k_bond"),
])
def test_typed_create_rejects_bad_arguments(lib, kw, needle):
    if kw.get("T") == 0:
        c, ty, _keep = _typed()
        ty.ntypes = 0
    else:
        c, ty, _keep = _typed(**kw)
    h = ctypes.c_void_p()
    rc = lib.vbc_create_typed_system(ctypes.byref(c), ctypes.byref(ty), ctypes.byref(h))
    assert rc == vbc.VBC_ERR_INVALID_ARG
    assert needle in lib.vbc_last_error().decode()
    assert not h.value


def test_typed_create_valid_until_device_needed(lib):
    """A valid two-type description with bonds passes every host check; without a
    GPU the call then fails with a CUDA error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("covered by the GPU tests")
    c, ty, _keep = _typed(types=np.arange(100) % 2, bonds=[[k, k + 1] for k in range(99)])
    h = ctypes.c_void_p()
    rc = lib.vbc_create_typed_system(ctypes.byref(c), ctypes.byref(ty), ctypes.byref(h))
    assert rc in (vbc.VBC_ERR_CUDA, vbc.VBC_ERR_OOM)
    assert not h.value
    assert lib.vbc_create_typed_system(None, None, None) == vbc.VBC_ERR_INVALID_ARG


# ----------------------------------------------------------------- serving admission estimate
def test_device_bytes_estimate_scales_with_n(lib):
    """vbc_estimate_device_bytes touches no device: it sizes the arrays of a
    system from n, the box and the list radius.  Per particle it must cover at
    least the resident state (unwrapped positions and velocities, both FP64
    copies, positions, force slots, close lists), and grow linearly with n at a
    fixed density."""
    prm = vbc.params(E_a=8.0, f=2.0)
    b1 = vbc.estimate_device_bytes(100_000, (100_000 / 0.5) ** (1 / 3), prm)
    b2 = vbc.estimate_device_bytes(800_000, (800_000 / 0.5) ** (1 / 3), prm)
    assert b1 >= 100_000 * (4 * 24 + 4 * 16 + 48 + 16)
    assert 7.0 < b2 / b1 < 9.0
    assert vbc.estimate_device_bytes(100_000, (100_000 / 0.5) ** (1 / 3), prm, precision=vbc.VBC_FP64) > b1


@pytest.mark.parametrize("kw,needle", [
    (dict(n=0), "n must be"),
    (dict(box=(6.0, 6.0, 6.0)), "fewer than 3 cells"),
    (dict(skin=0.0), "skin"),
])
def test_device_bytes_estimate_rejects_bad_configs(lib, kw, needle):
    c, _pos = _cfg(**kw)
    out = ctypes.c_int64(0)
    rc = lib.vbc_estimate_device_bytes(ctypes.byref(c), ctypes.byref(out))
    assert rc == vbc.VBC_ERR_INVALID_ARG
    assert needle in lib.vbc_last_error().decode()
