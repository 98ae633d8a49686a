"""The allocation-free entry point (vbc_compute_forces_noalloc), for callers that
cannot call cudaMalloc (code inside another framework's allocator or memory
budget, real-time loops, plug-ins that are handed device buffers).  Its
counts and forces agree with the regular entry point (vbc_compute_forces on a
vbc_system) and with the FP64 oracle within the tolerances of the parity
tests, on two calls in a row that share the library's static scratch; it
also runs without the optional counts and at its largest size, and the free
device memory does not move across calls.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

TOL_COUNT = 1e-6      # absolute, as in the parity tests
TOL_F = 1e-5          # max|dF| / rms|F|, FP32 split, as in the parity tests


def _case(n, rho, seed, q):
    pos, L = inputs.uniform_positions(n, rho, seed=seed)
    n0 = oracle.evaluate(pos, L, Params(E_a=5.0), mode=1).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, q))
    return pos, L, p


def _noalloc(dpos, L, prm, with_counts=True):
    import torch
    n = dpos.shape[0]
    F = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dpos.device)
    c = torch.full((n,), float("nan"), dtype=torch.float64, device=dpos.device) if with_counts else None
    vbc.compute_forces_noalloc(dpos, L, prm, F, c)
    torch.cuda.synchronize()
    return F.cpu().numpy(), (c.cpu().numpy() if with_counts else None)


def test_noalloc_matches_compute_forces_and_the_oracle_twice():
    import torch
    for pos, L, p in (_case(4000, 0.5, seed=31, q=0.5), _case(2500, 0.3, seed=32, q=0.4)):
        prm = vbc.params(**p.__dict__)
        ref = oracle.evaluate(pos, L, p, mode=1)
        assert np.mean(ref.ds != 0.0) > 0.1, "chain-rule path not exercised"
        rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
        with vbc.System(pos, L, prm) as s:
            main = s.compute(F=True, counts=True)
        dpos = torch.from_numpy(pos).cuda()
        for _ in range(2):  # two calls in a row reuse the same static scratch
            Fh, ch = _noalloc(dpos, L, prm)
            # against the regular entry point
            assert np.max(np.abs(ch - main.counts)) <= TOL_COUNT
            assert np.max(np.abs(Fh - main.F)) <= TOL_F * rms
            # and directly against the oracle
            assert np.max(np.abs(ch - ref.counts)) <= TOL_COUNT
            assert np.max(np.abs(Fh - ref.F)) <= TOL_F * rms


def test_noalloc_without_counts_and_at_its_largest_size():
    import torch
    n = vbc.NOALLOC_MAX_N
    pos, L, p = _case(n, 0.5, seed=33, q=0.5)
    prm = vbc.params(**p.__dict__)
    ref = oracle.evaluate(pos, L, p, mode=1)
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
    dpos = torch.from_numpy(pos).cuda()
    Fh, ch = _noalloc(dpos, L, prm)
    assert np.max(np.abs(ch - ref.counts)) <= TOL_COUNT
    assert np.max(np.abs(Fh - ref.F)) <= TOL_F * rms
    Fn, _ = _noalloc(dpos, L, prm, with_counts=False)
    assert np.max(np.abs(Fn - ref.F)) <= TOL_F * rms


def test_noalloc_leaves_free_device_memory_unchanged():
    """After a first call (which looks up the scratch address and loads the
    kernels), later calls allocate nothing: the device's free memory is the same
    before and after them."""
    import torch
    pos, L, p = _case(3000, 0.5, seed=34, q=0.5)
    prm = vbc.params(**p.__dict__)
    dpos = torch.from_numpy(pos).cuda()
    F = torch.zeros((3000, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros(3000, dtype=torch.float64, device="cuda")
    vbc.compute_forces_noalloc(dpos, L, prm, F, c)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        vbc.compute_forces_noalloc(dpos, L, prm, F, c)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = vbc.NOALLOC_MAX_N + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(vbc.VBCError) as e:
        vbc.compute_forces_noalloc(pos, 200.0, vbc.params(), F)
    assert e.value.code == vbc.VBC_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)


def test_noalloc_binding_rejects_mismatched_buffers():
    """Shapes and dtypes are checked before the library is called."""
    import torch
    pos = torch.zeros((100, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        vbc.compute_forces_noalloc(pos, 20.0, vbc.params(), torch.zeros((99, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        vbc.compute_forces_noalloc(pos, 20.0, vbc.params(), torch.zeros((100, 3), dtype=torch.float64, device="cuda"),
                                   torch.zeros(50, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        vbc.compute_forces_noalloc(pos.reshape(-1), 20.0, vbc.params(),
                                   torch.zeros((100, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        vbc.compute_forces_noalloc(pos, 20.0, vbc.params(), torch.zeros((100, 3), dtype=torch.float32, device="cuda"))
