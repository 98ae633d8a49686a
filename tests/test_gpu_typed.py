"""GPU parity of multi-type systems with a count mask and harmonic bonds (the
counter restricted to chosen neighbour types, Sec. 2; the sticker chains of
Sec. 4) against the oracle's typed evaluation, element by element, in both
precisions, with the tolerances of the single-type parity tests:
  counts  <= 1e-6 absolute (both)
  s, s'   <= 1e-12 (FP64), 1e-6 and 4e-6 (FP32 split)
  A_i     <= 1e-10 max|A| (FP64), 1e-5 max|A| (FP32 split)
  forces  <= 1e-10 rms|F| (FP64), 1e-5 rms|F| (FP32 split)
  U       <= 1e-9 relative (both; FP64 energies in both)
  W       <= 1e-9 relative (FP64), 1e-6 (FP32 split: positions on the 32-bit word grid)"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu


def _vp(p: Params) -> vbc.PairParams:
    return vbc.params(**p.__dict__)


def _sticker_model(f_sticker=1.0, E_ss=10.0):
    """Spacers (type 0) and stickers (type 1): stickers attract stickers only, and
    count stickers only; every pair keeps the soft core."""
    spacer, mixed, sticker = Params(E_a=0.0, f=2.0), Params(E_a=0.0), Params(E_a=E_ss, f=f_sticker)
    return [[spacer, mixed], [mixed, sticker]], [[0, 0], [0, 1]]


def _mixed(n_chains=300, beads=12, rho=0.45, seed=31):
    """Three types with different wells, radii and valencies, an asymmetric count
    mask and bonded chains; each type's valency at the median of its counts."""
    pos, L, _, bonds = inputs.sticker_chains(n_chains, beads, rho, seed=seed)
    pos = np.mod(pos + np.random.default_rng(3).normal(0.0, 0.05, pos.shape), L)
    t = (np.arange(pos.shape[0]) % 3).astype(np.int32)
    a = Params(E_a=4.0, f=1.2)
    b = Params(E_a=6.0, r_l=1.3, r_h=1.8, f=0.7, delta=0.2)
    c = Params(E_a=0.0, f=3.0)
    ab = Params(E_a=3.0, r_a=1.4, r_l=1.4, r_h=1.9)
    P = [[a, ab, Params(E_a=2.0)], [ab, b, Params(E_a=0.0)], [Params(E_a=2.0), Params(E_a=0.0), c]]
    mask = [[1, 1, 0], [0, 1, 1], [1, 0, 0]]
    n0 = oracle.evaluate_typed(pos, L, t, P, mask, mode=1).counts
    for k in range(3):
        d = P[k][k]
        P[k][k] = Params(**{**d.__dict__, "f": inputs.quantile_valency(n0[t == k], 0.5) + d.delta})
    return pos, L, t, P, mask, bonds


F32, F64 = vbc.VBC_FP32_SPLIT, vbc.VBC_FP64
TOL = {F64: dict(s=1e-12, A=1e-10, F=1e-10, W=1e-9), F32: dict(s=1e-6, A=1e-5, F=1e-5, W=1e-6)}


def _create(pos, L, t, P, mask, bonds, k_b, r_0, vel=None, seed=1, prec=F64):
    VP = [[_vp(x) for x in row] for row in P]
    return vbc.System.typed(pos, L, t, VP, mask, bonds=bonds, k_bond=k_b, r0_bond=r_0, vel=vel, seed=seed,
                            precision=prec)


def _check(s, pos, L, t, P, mask, bonds, k_b, r_0, min_window=0, prec=F64):
    tol = TOL[prec]
    ref = oracle.evaluate_typed(pos, L, t, P, mask, bonds=bonds, k_b=k_b, r_0=r_0, mode=1)
    r = s.compute(F=True, counts=True, energy=True, virial=True)
    sw, dsw, A = s.switch()
    assert np.max(np.abs(r.counts - ref.counts)) <= 1e-6
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
    assert np.max(np.abs(r.F - ref.F)) <= tol["F"] * rms
    assert np.max(np.abs(sw - ref.s)) <= tol["s"]
    assert np.max(np.abs(dsw - ref.ds)) <= 4 * tol["s"]
    assert np.max(np.abs(A - ref.A)) <= tol["A"] * max(np.max(np.abs(ref.A)), 1e-12)
    assert abs(r.energy - ref.U) <= 1e-9 * abs(ref.U)
    assert abs(r.virial - ref.W) <= tol["W"] * abs(ref.W)
    assert np.sum(ref.ds != 0.0) >= min_window
    return ref


@pytest.mark.parametrize("prec", [F64, F32])
def test_sticker_chains_against_oracle(prec):
    """Chains of 16 beads at bead density 0.3 with stickers every fourth bead."""
    pos, L, t, bonds = inputs.sticker_chains(1500, 16, 0.3, seed=5)
    P, mask = _sticker_model(f_sticker=1.0)
    with _create(pos, L, t, P, mask, bonds, 100.0, 1.0, prec=prec) as s:
        ref = _check(s, pos, L, t, P, mask, bonds, 100.0, 1.0, prec=prec)
    # spacers count nothing, so they all sit at s = 1
    assert np.all(ref.counts[t == 0] == 0.0)


@pytest.mark.parametrize("prec", [F64, F32])
def test_three_types_asymmetric_mask_against_oracle(prec):
    pos, L, t, P, mask, bonds = _mixed()
    with _create(pos, L, t, P, mask, bonds, 100.0, 1.0, prec=prec) as s:
        _check(s, pos, L, t, P, mask, bonds, 100.0, 1.0, min_window=200, prec=prec)


@pytest.mark.parametrize("prec", [F64, F32])
def test_after_steps_and_rebuilds(prec):
    """After Langevin steps with list rebuilds (the sorted order, the type map and
    the bond partners' sorted indices all change), forces at the new state still
    match the oracle at those positions."""
    pos, L, t, P, mask, bonds = _mixed(seed=32)
    vel = inputs.maxwell_velocities(pos.shape[0], 1.0, seed=9)
    with _create(pos, L, t, P, mask, bonds, 100.0, 1.0, vel=vel, prec=prec) as s:
        r0 = s.stats().rebuilds
        s.step(300, 0.005, 1.0, 1.0)
        assert s.stats().rebuilds > r0 + 1
        x, _, _ = s.get_state()
        _check(s, x, L, t, P, mask, bonds, 100.0, 1.0, prec=prec)


def test_fp32_split_sticker_trajectory_stays_near_fp64():
    """The FP32-split typed path and the FP64 one, from the same state and noise,
    stay within a small distance over 50 steps (the one-step maps differ by
    rounding only)."""
    pos, L, t, bonds = inputs.sticker_chains(400, 16, 0.3, seed=7)
    vel = inputs.maxwell_velocities(pos.shape[0], 1.0, seed=8)
    P, mask = _sticker_model(f_sticker=1.0)
    out = []
    for prec in (F64, F32):
        with _create(pos, L, t, P, mask, bonds, 100.0, 1.0, vel=vel, seed=3, prec=prec) as s:
            s.step(50, 0.005, 1.0, 1.0)
            out.append(s.get_state()[0])
    assert np.max(np.abs(out[0] - out[1])) < 1e-4


def test_one_type_matches_single_type_system():
    """One type with a full mask and no bonds is the single-type FP64 system, to
    rounding (the two walks add the terms in different orders)."""
    pos, L = inputs.uniform_positions(20000, 0.5, seed=12)
    n0 = oracle.evaluate(pos, L, Params(E_a=5.0), 1).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, 0.5))
    with _create(pos, L, np.zeros(20000), [[p]], [[1]], None, 0.0, 1.0) as s:
        a = s.compute(F=True, counts=True, energy=True)
    with vbc.System(pos, L, _vp(p), precision=vbc.VBC_FP64) as s:
        b = s.compute(F=True, counts=True, energy=True)
    assert np.max(np.abs(a.counts - b.counts)) <= 1e-12
    rms = np.sqrt(np.mean(np.sum(b.F ** 2, axis=1)))
    assert np.max(np.abs(a.F - b.F)) <= 1e-11 * rms
    assert abs(a.energy - b.energy) <= 1e-11 * abs(b.energy)


def test_bad_typed_arguments_rejected():
    pos, L, t, bonds = inputs.sticker_chains(20, 8, 0.3, seed=6)
    P, mask = _sticker_model()
    VP = [[_vp(x) for x in row] for row in P]
    with pytest.raises(vbc.VBCError, match="type of particle"):
        vbc.System.typed(pos, L, np.full(len(t), 2), VP, mask)
    with pytest.raises(vbc.VBCError, match="0 or 1"):
        vbc.System.typed(pos, L, t, VP, [[0, 0], [0, 2]])
    asym = [[VP[0][0], _vp(Params(E_a=1.0))], [VP[1][0], VP[1][1]]]
    with pytest.raises(vbc.VBCError, match="symmetric"):
        vbc.System.typed(pos, L, t, asym, mask)
    with pytest.raises(vbc.VBCError, match="bond"):
        vbc.System.typed(pos, L, t, VP, mask, bonds=[[0, len(t)]])
    with pytest.raises(vbc.VBCError, match="bond"):
        vbc.System.typed(pos, L, t, VP, mask, bonds=[[3, 3]])
    with vbc.System.typed(pos, L, t, VP, mask, bonds=bonds, k_bond=100.0) as s:
        with pytest.raises(vbc.VBCError, match="multi-type"):
            s.set_params(vbc.params())
