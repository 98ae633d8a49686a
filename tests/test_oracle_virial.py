"""Pins of the oracle's pair virial W = sum_{i<j} -g_ij r_ij (g_ij = dU/dr_ij,
every term of the pair force including the chain rule through the counts).

The virial is the response of U to a uniform dilation: scaling every
position and the box by lambda scales every separation, so
dU/dlambda at lambda = 1 is sum_{i<j} r_ij dU/dr_ij = -W.  That identity ties
W to U, which test_oracle_pins.py pins by closed forms and by finite
differences of the forces.  A dimer pins the sign and the factor by hand:
for one pair W = -r V'(r), with V' taken by central differences of U."""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs


def _dimer(r, box=50.0):
    pos = np.zeros((2, 3))
    pos[1, 0] = r
    return pos, box


def _dilation_virial(energy, pos, box, h=1e-6):
    """-dU/dlambda at lambda = 1 for x -> lambda x, L -> lambda L (central difference)."""
    return -(energy(pos * (1 + h), box * (1 + h)) - energy(pos * (1 - h), box * (1 - h))) / (2 * h)


def test_dimer_virial_in_core_and_well():
    """One pair of the bare potential (f = 1000, so s = 1 and s' = 0): W = -r dU/dr.
    In the core (r = 0.7) the pair repels and W > 0; inside the well's inner
    half (r = 1.15, V_a rising towards the core) it also pushes apart, W > 0;
    in its outer half (r = 1.45) it attracts and W < 0.  The core value is also the
    closed form -r V_r'(r) with V_r'(r) = -4 E_r r (1 - r^2) for r_r = 1:
    W(0.7) = 0.7 * 4 * 20 * 0.7 * 0.51 = 19.992."""
    p = Params(E_a=5.0, f=1000.0)
    for r, sign in ((0.7, 1.0), (1.15, 1.0), (1.45, -1.0)):
        pos, box = _dimer(r)
        res = oracle.evaluate(pos, box, p)
        h = 1e-6
        dU = (oracle.evaluate(_dimer(r + h)[0], box, p).U - oracle.evaluate(_dimer(r - h)[0], box, p).U) / (2 * h)
        assert math.isclose(res.W, -r * dU, rel_tol=1e-8)
        assert math.copysign(1.0, res.W) == sign
    res = oracle.evaluate(_dimer(0.7)[0], 50.0, p)
    assert math.isclose(res.W, 0.7 * 4.0 * 20.0 * 0.7 * (1.0 - 0.49), rel_tol=1e-13)


def test_dimer_virial_with_counts_in_the_window():
    """A dimer at r = 1.7 inside the counting window (n = omega(1.7; 1.5, 2) for
    both) and below the valency threshold: the pair has no well term (r > r_a)
    but each particle's switch depends on r through its count, so the virial
    carries the chain-rule term.  Here V_a(1.7) = 0 and hence A = 0: W = 0
    exactly.  At r = 1.4 (inside the well and r < r_l, n = 1) with f = 0.5 the
    switch is s = 9/16 at fixed n, so W = -r (V_r' + (9/16)^2 V_a')(r)."""
    p = Params(E_a=5.0, f=0.5)
    res = oracle.evaluate(_dimer(1.7)[0], 50.0, p)
    assert res.W == 0.0
    r, h = 1.4, 1e-6
    res = oracle.evaluate(_dimer(r)[0], 50.0, p)
    dU = (oracle.evaluate(_dimer(r + h)[0], 50.0, p).U - oracle.evaluate(_dimer(r - h)[0], 50.0, p).U) / (2 * h)
    assert math.isclose(res.W, -r * dU, rel_tol=1e-8)
    assert math.isclose(res.U, (9.0 / 16.0) ** 2 * oracle.Va(r, p), rel_tol=1e-13)


def test_virial_is_minus_the_dilation_derivative():
    """W = -dU/dlambda on random configurations with counts in the switching
    window (f at the median count), for the standard, shifted and optimised
    presets: every term of g_ij, the chain-rule one included, enters W."""
    for base, q, seed in ((Params(E_a=5.0), 0.5, 61), (Params(E_a=5.0, delta=0.3), 0.3, 62),
                          (Params(r_l=1.29, r_h=1.50, delta=0.30, E_a=5.0), 0.5, 63)):
        pos, L = inputs.uniform_positions(80, 0.35, seed=seed)
        n0 = oracle.evaluate(pos, L, base).counts
        p = Params(**{**base.__dict__, "f": inputs.quantile_valency(n0, q) + base.delta})
        r = oracle.evaluate(pos, L, p)
        assert np.mean(r.ds != 0.0) > 0.1, "chain-rule path not exercised"
        Wfd = _dilation_virial(lambda x, b: oracle.evaluate(x, b, p).U, pos, L)
        assert math.isclose(r.W, Wfd, rel_tol=1e-7, abs_tol=1e-7 * np.abs(r.e).sum())
        # the chain-rule part of W is not negligible here: the bare-pair virial differs
        bare = oracle.evaluate(pos, L, Params(**{**p.__dict__, "f": 1000.0}))
        assert abs(bare.W - r.W) > 1e-3 * abs(r.W)
    # the cell-list mode gives the same virial
    pos, L = inputs.uniform_positions(3000, 0.5, seed=64)
    p = Params(E_a=8.0, f=6.0)
    assert math.isclose(oracle.evaluate(pos, L, p, mode=1).W, oracle.evaluate(pos, L, p, mode=0).W,
                        rel_tol=1e-11)


def test_typed_virial_is_minus_the_dilation_derivative():
    """The same identity for the multi-type evaluation with harmonic bonds and
    an asymmetric count mask (three types, counts in their windows)."""
    pos, L, _, bonds = inputs.sticker_chains(6, 6, 0.45, seed=31)
    pos = np.mod(pos + np.random.default_rng(3).normal(0.0, 0.05, pos.shape), L)
    t = np.arange(36) % 3
    a = Params(E_a=4.0, f=1.2)
    b = Params(E_a=6.0, r_l=1.3, r_h=1.8, f=0.7, delta=0.2)
    c = Params(E_a=0.0, f=3.0)
    ab = Params(E_a=3.0, r_a=1.4, r_l=1.4, r_h=1.9)
    P = [[a, ab, Params(E_a=2.0)], [ab, b, Params(E_a=0.0)], [Params(E_a=2.0), Params(E_a=0.0), c]]
    cmask = [[1, 1, 0], [0, 1, 1], [1, 0, 0]]
    n0 = oracle.evaluate_typed(pos, L, t, P, cmask).counts
    for k in range(3):
        d = P[k][k]
        P[k][k] = Params(**{**d.__dict__, "f": inputs.quantile_valency(n0[t == k], 0.5) + d.delta})
    kw = dict(bonds=bonds, k_b=100.0, r_0=1.0)
    r = oracle.evaluate_typed(pos, L, t, P, cmask, **kw)
    assert np.sum(r.A != 0.0) >= 5
    Wfd = _dilation_virial(lambda x, bx: oracle.evaluate_typed(x, bx, t, P, cmask, **kw).U, pos, L)
    assert math.isclose(r.W, Wfd, rel_tol=1e-7)
