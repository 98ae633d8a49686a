"""The device reductions of vbc_compute_thermo (U, W, KE, mean count, in-window
and pair counts, FP64 fixed-order sums) against the FP64 oracle at the
state the library holds, and the claim that logging them between chunks of
steps leaves the trajectory bitwise unchanged.

Tolerances: U <= 1e-9 relative (both precisions: the reduction recomputes the
counts and switches in FP64); W <= 1e-6 relative (FP32 split, positions on the
32-bit word grid) and 1e-9 (FP64); mean count <= 1e-6 absolute (the count
tolerance); KE <= 1e-12 relative of the velocities read back; the in-window
count exactly in FP64 and within one particle in the FP32 split (its counts
come from the 32-bit words, so a particle within ~1e-7 of a window edge may
fall either side); pairs within r_c exactly in FP64."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

F32, F64 = vbc.VBC_FP32_SPLIT, vbc.VBC_FP64
TOL_W = {F32: 1e-6, F64: 1e-9}
DT, KT, GAMMA = 0.005, 1.0, 1.0


def _params(pos, L, q=0.5):
    n0 = oracle.evaluate(pos, L, Params(E_a=5.0), mode=1).counts
    return Params(E_a=5.0, f=inputs.quantile_valency(n0, q))


def _check(th, x, v, L, p, prec):
    ref = oracle.evaluate(x, L, p, mode=1)
    assert abs(th.U - ref.U) <= 1e-9 * abs(ref.U)
    assert abs(th.W - ref.W) <= TOL_W[prec] * abs(ref.W)
    assert abs(th.mean_n - ref.counts.mean()) <= 1e-6
    ke = 0.5 * np.sum(v * v)
    assert abs(th.KE - ke) <= 1e-12 * ke
    win = int(np.sum(ref.ds != 0.0))
    assert win > 0.1 * len(x), "in-window fraction too small to test"
    assert abs(th.in_window - win) <= (0 if prec == F64 else 1)
    if prec == F64:
        assert th.pairs_within_rc == len(oracle.pairs_within(x, L, 2.0))


@pytest.mark.parametrize("prec", [F32, F64])
def test_thermo_matches_the_oracle_after_steps(prec):
    pos, L = inputs.uniform_positions(6000, 0.5, seed=81)
    vel = inputs.maxwell_velocities(6000, KT, seed=82)
    p = _params(pos, L)
    with vbc.System(pos, L, vbc.params(**p.__dict__), vel=vel, precision=prec) as s:
        th = s.thermo()
        x, v, st = s.get_state()
        assert th.step == st == 0
        _check(th, x, v, L, p, prec)
        s.step(37, DT, KT, GAMMA)
        th = s.thermo()
        x, v, st = s.get_state()
        assert th.step == st == 37
        _check(th, x, v, L, p, prec)


@pytest.mark.parametrize("prec", [F32, F64])
def test_thermo_between_chunks_leaves_the_trajectory_unchanged(prec):
    pos, L = inputs.uniform_positions(4000, 0.5, seed=83)
    vel = inputs.maxwell_velocities(4000, KT, seed=84)
    p = _params(pos, L, q=0.4)
    outs = []
    for log in (False, True):
        with vbc.System(pos, L, vbc.params(**p.__dict__), vel=vel, seed=5, precision=prec) as s:
            for _ in range(8):
                s.step(9, DT, KT, GAMMA)
                if log:
                    s.thermo()
            outs.append(s.get_state())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("prec", [F64, F32])
def test_thermo_of_a_multi_type_system(prec):
    """Sticker chains with bonds (counts over stickers only): U, W, KE and the
    mean masked count against the oracle's typed evaluation."""
    pos, L, t, bonds = inputs.sticker_chains(300, 16, 0.3, seed=85)
    vel = inputs.maxwell_velocities(pos.shape[0], KT, seed=86)
    spacer, mixed, sticker = Params(E_a=0.0, f=2.0), Params(E_a=0.0), Params(E_a=10.0, f=1.0)
    P = [[spacer, mixed], [mixed, sticker]]
    mask = [[0, 0], [0, 1]]
    VP = [[vbc.params(**q.__dict__) for q in row] for row in P]
    with vbc.System.typed(pos, L, t, VP, mask, bonds=bonds, k_bond=100.0, r0_bond=1.0, vel=vel, precision=prec) as s:
        s.step(20, DT, KT, GAMMA)
        th = s.thermo()
        x, v, _ = s.get_state()
    ref = oracle.evaluate_typed(x, L, t, P, mask, bonds=bonds, k_b=100.0, r_0=1.0, mode=1)
    assert abs(th.U - ref.U) <= 1e-9 * abs(ref.U)
    assert abs(th.W - ref.W) <= TOL_W[prec] * abs(ref.W)
    assert abs(th.mean_n - ref.counts.mean()) <= 1e-6
    assert abs(th.in_window - int(np.sum(ref.ds != 0.0))) <= (0 if prec == F64 else 1)
    assert abs(th.KE - 0.5 * np.sum(v * v)) <= 1e-12 * 0.5 * np.sum(v * v)
