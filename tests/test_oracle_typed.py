"""Pins of the oracle's multi-type evaluation with harmonic bonds: counts
restricted to selected neighbour types (Sec. 2) and the bead-spring sticker
chains of Sec. 4.  The pins are the reduction to the single-type evaluation
(itself pinned in test_oracle_pins.py), closed forms of small configurations,
-grad U by central differences with every term switched on, and the
invariances of a sum of central pair and bond terms."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs

STD = Params()


def _line(xs, box=100.0):
    pos = np.zeros((len(xs), 3))
    pos[:, 0] = xs
    return pos, box


def _sticker_model(f_sticker=1.0, E_ss=10.0, f_spacer=2.0, delta=0.0):
    """Two types: 0 spacer, 1 sticker.  Stickers attract stickers only (E_a = E_ss);
    every pair keeps the soft core.  Stickers count stickers only."""
    spacer = Params(E_a=0.0, f=f_spacer)
    mixed = Params(E_a=0.0)
    sticker = Params(E_a=E_ss, f=f_sticker, delta=delta)
    P = [[spacer, mixed], [mixed, sticker]]
    cmask = [[0, 0], [0, 1]]
    return P, cmask


def _compare(a, b, rel=1e-12):
    for name in ("counts", "s", "ds", "A", "e"):
        x, y = getattr(a, name), getattr(b, name)
        assert np.allclose(x, y, rtol=rel, atol=rel), name
    rms = max(np.sqrt(np.mean(np.sum(b.F ** 2, axis=1))), 1e-300)
    assert np.max(np.abs(a.F - b.F)) <= rel * rms
    assert math.isclose(a.U, b.U, rel_tol=rel, abs_tol=1e-300)
    assert math.isclose(a.W, b.W, rel_tol=rel, abs_tol=1e-300)


def test_one_type_is_the_single_type_evaluation():
    pos, L = inputs.uniform_positions(80, 0.4, seed=21)
    n0 = oracle.evaluate(pos, L, Params(E_a=5.0)).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, 0.5))
    ref = oracle.evaluate(pos, L, p)
    got = oracle.evaluate_typed(pos, L, np.zeros(80), [[p]], [[1]])
    assert np.mean(ref.ds != 0.0) > 0.1
    _compare(got, ref)


def test_identical_types_are_one_type():
    """Three labels with the same parameters everywhere and a full count mask."""
    pos, L = inputs.uniform_positions(90, 0.4, seed=22)
    n0 = oracle.evaluate(pos, L, Params(E_a=5.0)).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, 0.4))
    t = np.random.default_rng(5).integers(0, 3, 90)
    got = oracle.evaluate_typed(pos, L, t, [[p] * 3] * 3, np.ones((3, 3)), mode=1 if L >= 6.0 else 0)
    _compare(got, oracle.evaluate(pos, L, p))


def test_count_mask_closed_form():
    """Sticker A at 0, sticker B at 1.2, spacer C at -1.2: r_AB = r_AC = 1.2 <= r_l
    (weight 1), r_BC = 2.4 >= r_h.  Stickers count stickers only, so n = (1, 1, 0);
    with f = 1 the stickers sit at the top of the window (t = 0: s = 1, s' = 0) and
    the energy is V_r-free (r > r_r) with one sticker well: U = V_a(1.2)."""
    P, cm = _sticker_model(f_sticker=1.0)
    pos, box = _line([0.0, 1.2, -1.2])
    r = oracle.evaluate_typed(pos, box, [1, 1, 0], P, cm)
    assert list(r.counts) == [1.0, 1.0, 0.0]
    assert list(r.s) == [1.0, 1.0, 1.0] and list(r.ds) == [0.0, 0.0, 0.0]
    assert math.isclose(r.U, oracle.Va(1.2, P[1][1]), rel_tol=1e-15)
    # with f = 0.5 the stickers are half-way up the window: t = 0.5, s = (3/4)^2
    P, cm = _sticker_model(f_sticker=0.5)
    r = oracle.evaluate_typed(pos, box, [1, 1, 0], P, cm)
    assert list(r.s[:2]) == [0.5625, 0.5625]
    assert math.isclose(r.U, 0.5625 ** 2 * oracle.Va(1.2, P[1][1]), rel_tol=1e-15)
    # a spacer between them changes no sticker count, whatever its distance
    pos2, _ = _line([0.0, 1.2, 0.6])
    r2 = oracle.evaluate_typed(pos2, box, [1, 1, 0], P, cm)
    assert list(r2.counts) == [1.0, 1.0, 0.0]


def test_bond_closed_form():
    """Two spacers bonded at r = 1.3 with nothing else acting (r > r_r, no wells):
    U = k/2 (r - r0)^2, F_0 = -k (r - r0) along +x, W = -k (r - r0) r."""
    P, cm = _sticker_model()
    pos, box = _line([0.0, 1.3])
    r = oracle.evaluate_typed(pos, box, [0, 0], P, cm, bonds=[[0, 1]], k_b=100.0, r_0=1.0)
    g = 100.0 * 0.3
    assert math.isclose(r.U, 0.5 * 100.0 * 0.3 ** 2, rel_tol=1e-14)
    assert math.isclose(r.F[0, 0], g, rel_tol=1e-14) and math.isclose(r.F[1, 0], -g, rel_tol=1e-14)
    assert np.all(r.F[:, 1:] == 0.0)
    assert math.isclose(r.W, -g * 1.3, rel_tol=1e-14)
    # a bond inside the soft core adds to V_r: r = 0.8
    pos, _ = _line([0.0, 0.8])
    r = oracle.evaluate_typed(pos, box, [0, 0], P, cm, bonds=[[0, 1]], k_b=100.0, r_0=1.0)
    assert math.isclose(r.U, oracle.Vr(0.8, P[0][0]) + 50.0 * 0.04, rel_tol=1e-14)
    assert math.isclose(r.F[0, 0], -(-oracle.dVr(0.8, P[0][0]) + 100.0 * 0.2), rel_tol=1e-14)


def _fd_forces(pos, box, args, kw, h=1e-6):
    F = np.zeros_like(pos)
    for i in range(pos.shape[0]):
        for a in range(3):
            xp = pos.copy(); xp[i, a] += h
            xm = pos.copy(); xm[i, a] -= h
            F[i, a] = -(oracle.evaluate_typed(xp, box, *args, **kw).U -
                        oracle.evaluate_typed(xm, box, *args, **kw).U) / (2 * h)
    return F


def _mixed_system():
    """36 beads in 6 chains of 6 in a small box (dense enough that counts sit in
    the windows), three types with different wells, radii and valencies, and an
    asymmetric count mask, so that every term of g_ij is exercised."""
    pos, L, _, bonds = inputs.sticker_chains(6, 6, 0.45, seed=31)
    # bonds of exactly r_0 = r_r would sit on the kink of V_r'' (and of V_a''), where a
    # central difference is off by O(h): move every bead a little off the chain's lattice
    pos = np.mod(pos + np.random.default_rng(3).normal(0.0, 0.05, pos.shape), L)
    t = np.arange(36) % 3
    a = Params(E_a=4.0, f=1.2)
    b = Params(E_a=6.0, r_l=1.3, r_h=1.8, f=0.7, delta=0.2)
    c = Params(E_a=0.0, f=3.0)
    ab = Params(E_a=3.0, r_a=1.4, r_l=1.4, r_h=1.9)
    ac = Params(E_a=2.0)
    bc = Params(E_a=0.0)
    P = [[a, ab, ac], [ab, b, bc], [ac, bc, c]]
    cmask = [[1, 1, 0], [0, 1, 1], [1, 0, 0]]
    # each type's valency at the median of its own counts, so that half of them sit in the window
    n0 = oracle.evaluate_typed(pos, L, t, P, cmask).counts
    for k in range(3):
        d = P[k][k]
        P[k][k] = Params(**{**d.__dict__, "f": inputs.quantile_valency(n0[t == k], 0.5) + d.delta})
    return pos, L, t, P, cmask, bonds


def test_forces_match_finite_differences():
    pos, L, t, P, cmask, bonds = _mixed_system()
    kw = dict(bonds=bonds, k_b=100.0, r_0=1.0)
    r = oracle.evaluate_typed(pos, L, t, P, cmask, **kw)
    assert np.sum(r.A != 0.0) >= 5, "chain-rule path not exercised"
    Ffd = _fd_forces(pos, L, (t, P, cmask), kw)
    rms = np.sqrt(np.mean(np.sum(r.F ** 2, axis=1)))
    assert np.max(np.abs(r.F - Ffd)) <= 1e-7 * rms
    # the mask must sit on the right index in the chain-rule term: its transpose gives other forces
    rt = oracle.evaluate_typed(pos, L, t, P, np.asarray(cmask).T, **kw)
    assert np.max(np.abs(rt.F - r.F)) > 1e-3 * rms


def test_invariances():
    pos, L, t, P, cmask, bonds = _mixed_system()
    kw = dict(k_b=100.0, r_0=1.0)
    r = oracle.evaluate_typed(pos, L, t, P, cmask, bonds=bonds, **kw)
    # central pair and bond terms: no net force
    assert np.max(np.abs(r.F.sum(axis=0))) <= 1e-11 * np.abs(r.F).max()
    # permuting the beads (types and bond indices with them) permutes every output
    perm = np.random.default_rng(7).permutation(36)
    inv = np.argsort(perm)
    rp = oracle.evaluate_typed(pos[perm], L, t[perm], P, cmask, bonds=inv[bonds], **kw)
    for name in ("counts", "s", "A", "e"):
        assert np.allclose(getattr(rp, name), getattr(r, name)[perm], rtol=1e-12, atol=1e-13)
    assert np.allclose(rp.F, r.F[perm], rtol=1e-11, atol=1e-11)
    # relabelling the types (with the tables permuted to match) changes nothing
    sig = [2, 0, 1]
    Ps = [[None] * 3 for _ in range(3)]
    cs = np.zeros((3, 3), dtype=int)
    for a_ in range(3):
        for b_ in range(3):
            Ps[sig[a_]][sig[b_]] = P[a_][b_]
            cs[sig[a_], sig[b_]] = cmask[a_][b_]
    rs = oracle.evaluate_typed(pos, L, np.asarray(sig)[t], Ps, cs, bonds=bonds, **kw)
    assert np.allclose(rs.F, r.F, rtol=1e-13, atol=1e-13) and math.isclose(rs.U, r.U, rel_tol=1e-13)
    # bonds listed in either direction give the same result
    rb = oracle.evaluate_typed(pos, L, t, P, cmask, bonds=bonds[:, ::-1], **kw)
    assert np.allclose(rb.F, r.F, rtol=1e-13, atol=1e-13)


def test_cell_mode_equals_all_pairs():
    pos, L, t, b = inputs.sticker_chains(40, 16, 0.3, seed=41)
    P, cm = _sticker_model(f_sticker=1.0)
    r0 = oracle.evaluate_typed(pos, L, t, P, cm, bonds=b, k_b=100.0, r_0=1.0, mode=0)
    r1 = oracle.evaluate_typed(pos, L, t, P, cm, bonds=b, k_b=100.0, r_0=1.0, mode=1)
    _compare(r1, r0, rel=1e-11)


def test_bad_indices_rejected():
    P, cm = _sticker_model()
    pos, box = _line([0.0, 1.3])
    with pytest.raises(ValueError):
        oracle.evaluate_typed(pos, box, [0, 2], P, cm)
    with pytest.raises(ValueError):
        oracle.evaluate_typed(pos, box, [0, 1], P, cm, bonds=[[0, 2]])


def test_sticker_chain_inputs():
    pos, L, t, b = inputs.sticker_chains(5, 64, 0.3, seed=1)
    assert pos.shape == (320, 3) and t.shape == (320,) and b.shape == (315, 2)
    assert math.isclose(L, (320 / 0.3) ** (1 / 3))
    assert np.all((pos >= 0) & (pos < L))
    assert np.sum(t) == 5 * 16 and t[0] == 1 and t[4] == 1 and t[1] == 0
    d = pos[b[:, 0]] - pos[b[:, 1]]
    d -= L * np.round(d / L)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-9)
    assert not np.any(b[:, 0] % 64 == 63)
