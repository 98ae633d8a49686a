"""The allocation-free entry point (vbc_compute_forces_noalloc), for callers that
cannot call cudaMalloc: its counts and forces agree with the regular entry point
(vbc_compute_forces on a vbc_system) within the tolerances of the parity tests,
on two calls in a row that share the library's static scratch.

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
    return pos, L, vbc.params(**p.__dict__)


def test_noalloc_matches_compute_forces_twice():
    import torch
    cases = [_case(4000, 0.5, seed=31, q=0.5), _case(2500, 0.3, seed=32, q=0.4)]
    for pos, L, prm in cases:
        with vbc.System(pos, L, prm) as s:
            ref = s.compute(F=True, counts=True)
        rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
        dpos = torch.from_numpy(pos).cuda()
        for _ in range(2):  # two calls in a row reuse the same static scratch
            F = torch.full((len(pos), 3), float("nan"), dtype=torch.float64, device="cuda")
            c = torch.full((len(pos),), float("nan"), dtype=torch.float64, device="cuda")
            vbc.compute_forces_noalloc(dpos, L, prm, F, c)
            torch.cuda.synchronize()
            Fh, ch = F.cpu().numpy(), c.cpu().numpy()
            assert np.max(np.abs(ch - ref.counts)) <= TOL_COUNT
            assert np.max(np.abs(Fh - ref.F)) <= TOL_F * rms


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = vbc.NOALLOC_MAX_N + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(vbc.VBCError) as e:
        vbc.compute_forces_noalloc(pos, 200.0, vbc.params(), F)
    assert e.value.code == vbc.VBC_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
