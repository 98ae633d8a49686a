"""GPU Langevin integration (BAOAB, Philox noise) against the FP64 oracle.

Tolerances:
  one step, FP64 mode:   |dx| <= 1e-12, |dv| <= 1e-10   (same FP64 noise as the oracle)
  one step, FP32 split:  |dx| <= 1e-8,  |dv| <= 5e-6    (FP32 forces, FP32 Box-Muller)
  100 steps with rebuilds, FP64 mode: |dx| <= 1e-8
Multi-step FP32 trajectories are compared statistically (chaos amplifies the
FP32 force error), and for bitwise equality between identical runs.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

F32, F64 = vbc.VBC_FP32_SPLIT, vbc.VBC_FP64


def _system(n, rho, seed, E_a=5.0, q=0.5, clustered=False):
    if clustered:
        pos, L = inputs.clustered_positions(n, rho, seed=seed, cluster_size=3, spread=0.9)
    else:
        pos, L = inputs.uniform_positions(n, rho, seed=seed)
    vel = inputs.maxwell_velocities(n, 1.0, seed=seed + 100)
    n0 = oracle.evaluate(pos, L, Params(E_a=E_a), 1 if n > 3000 else 0).counts
    p = Params(E_a=E_a, f=inputs.quantile_valency(n0, q))
    return pos, vel, L, p


def _vp(p):
    return vbc.params(**p.__dict__)


@pytest.mark.parametrize("prec,tx,tv", [(F64, 1e-12, 1e-10), (F32, 1e-8, 5e-6)])
def test_one_step_map(prec, tx, tv):
    pos, vel, L, p = _system(2000, 0.5, seed=1)
    dt, kT, gamma, seed = 0.005, 1.0, 1.0, 77
    with vbc.System(pos, L, _vp(p), vel=vel, seed=seed, precision=prec) as s:
        s.set_state(pos, vel, step=5)
        s.step(1, dt, kT, gamma)
        x, v, st = s.get_state()
    xo, vo, so = oracle.baoab(pos, vel, L, p, 1, dt, kT, gamma, seed=seed, step=5)
    assert st == so == 6
    assert np.max(np.abs(x - xo)) <= tx
    assert np.max(np.abs(v - vo)) <= tv


def test_fp64_trajectory_with_rebuilds():
    """100 steps in FP64 mode cross several automatic rebuilds (Morton re-sorts of
    the particles); the trajectory stays on the oracle's."""
    pos, vel, L, p = _system(1000, 0.5, seed=2)
    dt, kT, gamma, seed = 0.005, 1.0, 1.0, 5
    with vbc.System(pos, L, _vp(p), vel=vel, seed=seed, precision=F64) as s:
        r0 = s.stats().rebuilds
        s.step(100, dt, kT, gamma)
        x, v, st = s.get_state()
        stats = s.stats()
    xo, vo, _ = oracle.baoab(pos, vel, L, p, 100, dt, kT, gamma, seed=seed)
    assert stats.rebuilds - r0 >= 2, "the run did not cross two rebuilds"
    assert np.max(np.abs(x - xo)) <= 1e-8
    assert np.max(np.abs(v - vo)) <= 1e-6


def test_chunked_calls_equal_one_call():
    """Ten calls of 10 steps (and uneven calls of 1, 2 and 3 steps) give bitwise
    the same state as one call of 100, also when other calls come between them:
    reads leave the resident forces in place, a force evaluation (which
    overwrites them) makes the next call recompute its opening force the way the
    loop does, and new grid settings make it capture its graphs again."""
    pos, vel, L, p = _system(3000, 0.5, seed=3)
    outs = []
    plans = ((100,), (10,) * 10, (1, 2, 3) * 16 + (4,), (10,) * 10)
    for k, chunks in enumerate(plans):
        with vbc.System(pos, L, _vp(p), vel=vel, seed=9) as s:
            for j, c in enumerate(chunks):
                s.step(c, 0.005, 1.0, 1.0)
                if k == 3:  # other calls between the chunks
                    s.get_state()
                    s.stats()
                    if j % 3 == 0:
                        s.compute(F=True, counts=True)
                    elif j % 3 == 1:
                        s.set_tuning(rows_blocks_per_sm=1 + j % 4, count_blocks_per_sm=j % 3)
                    else:
                        s.observables()
            outs.append(s.get_state())
    for o in outs[1:]:
        assert o[2] == 100
        # chunk boundaries reuse the closing forces as the opening ones: bitwise equal
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])


def test_deterministic_runs_bitwise():
    pos, vel, L, p = _system(20000, 0.5, seed=4)
    outs = []
    for _ in range(2):
        with vbc.System(pos, L, _vp(p), vel=vel, seed=3) as s:
            s.step(200, 0.005, 1.0, 1.0)
            outs.append(s.get_state())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_overflow_during_steps_is_transparent():
    """Starting with a 6-entry list forces overflows at rebuilds inside the run; the
    library grows the list and resumes, giving bitwise the same trajectory."""
    pos, vel, L, p = _system(4000, 0.5, seed=5)
    outs = []
    for cap in (0, 6):
        with vbc.System(pos, L, _vp(p), vel=vel, seed=11, nlist_cap=cap) as s:
            s.step(60, 0.005, 1.0, 1.0)
            outs.append(s.get_state())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_checkpoint_restart_fp64():
    pos, vel, L, p = _system(1500, 0.5, seed=6)
    with vbc.System(pos, L, _vp(p), vel=vel, seed=21, precision=F64) as s:
        s.step(40, 0.005, 1.0, 1.0)
        ck = s.get_state()
        s.step(40, 0.005, 1.0, 1.0)
        x1, v1, st1 = s.get_state()
    with vbc.System(pos, L, _vp(p), seed=21, precision=F64) as s:
        s.set_state(ck[0], ck[1], step=ck[2])
        s.step(40, 0.005, 1.0, 1.0)
        x2, v2, st2 = s.get_state()
    assert st1 == st2 == 80
    assert np.max(np.abs(x1 - x2)) <= 1e-10 and np.max(np.abs(v1 - v2)) <= 1e-8


def test_equipartition():
    """Langevin at kT = 1.2: <KE>/N -> 3/2 kT (FP32 split, 8000 particles of the
    throughput workload: rho = 0.5, E_a = 8, valency 2, which relaxes quickly)."""
    pos, L = inputs.uniform_positions(8000, 0.5, seed=7)
    vel = inputs.maxwell_velocities(8000, 1.2, seed=8)
    p = Params(E_a=8.0, f=2.0)
    kT = 1.2
    with vbc.System(pos, L, _vp(p), vel=vel, seed=2) as s:
        s.step(1000, 0.005, kT, 1.0)
        ke = []
        for _ in range(40):
            s.step(50, 0.005, kT, 1.0)
            _, v, _ = s.get_state()
            ke.append(0.5 * np.sum(v ** 2) / len(v))
    ke = np.array(ke)
    assert abs(ke.mean() / (1.5 * kT) - 1.0) < 0.01


@pytest.mark.parametrize("prec", [F32, F64])
def test_nve_energy_conservation(prec):
    """gamma = 0: total energy is conserved (no drift beyond O(dt^2) noise)."""
    pos, vel, L, p = _system(3000, 0.3, seed=8, E_a=4.0, clustered=True)
    with vbc.System(pos, L, _vp(p), vel=vel, seed=1, precision=prec) as s:
        s.step(300, 0.002, 1.0, 5.0)  # relax the random start
        e0 = None
        es = []
        for _ in range(10):
            r = s.compute(energy=True)
            _, v, _ = s.get_state()
            e = r.energy + 0.5 * np.sum(v ** 2)
            e0 = e if e0 is None else e0
            es.append(e)
            s.step(100, 0.002, 1.0, 0.0)
    es = np.array(es)
    assert np.max(np.abs(es - e0)) / (abs(e0) + len(pos)) < 2e-4


def test_kernel_launch_accounting():
    pos, vel, L, p = _system(2000, 0.5, seed=9)
    with vbc.System(pos, L, _vp(p), vel=vel) as s:
        # direct launches (per-kernel timing on): one iteration counter reset, then per
        # iteration a gate, 7 rebuild kernels (returning at once when no rebuild is due),
        # the two count kernels, chain, force rows and the update
        s.profile(True)
        before = s.kernel_launches()
        s.step(10, 0.005, 1.0, 1.0)
        assert s.kernel_launches() - before == 1 + 11 * 13
        s.profile(False)
        # graphs: the previous call left the forces of the current state in place, so
        # iteration 0 is the iteration counter and the update alone; iterations 1..8 run
        # as four two-step graphs of 12 kernels (a system this small takes no eight-step
        # graphs and counts after the conditional), 9 and 10 as one-iteration graphs of 6
        # (gate, the two counts, chain, force rows, update), plus 7 kernels for every
        # rebuild the graphs' conditionals executed
        before = s.kernel_launches()
        s.step(10, 0.005, 1.0, 1.0)
        d = s.kernel_launches() - before
        base = 2 + 8 * 6 + 2 * 6
        assert d >= base and (d - base) % 7 == 0


@pytest.mark.parametrize("prec", [F32, F64])
def test_graph_and_direct_launches_agree_bitwise(prec):
    """The two-step CUDA graphs (conditional rebuild body) and plain launches run the
    same kernels on the same data: trajectories are bitwise equal, rebuilds included."""
    pos, vel, L, p = _system(3000, 0.5, seed=10)
    outs = []
    for direct in (False, True):
        with vbc.System(pos, L, _vp(p), vel=vel, seed=4, precision=prec) as s:
            if direct:
                s.profile(True, 1 << 14)
            r0 = s.stats().rebuilds
            s.step(61, 0.005, 1.0, 1.0)
            outs.append(s.get_state())
            st = s.stats()
    assert st.rebuilds - r0 >= 3
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_eight_step_graphs_agree_with_direct_launches():
    """Large systems run their middle iterations as eight-step graphs, with the close
    count beside the rebuild conditional; 300 000 particles (the throughput
    workload's rho = 0.5, E_a = 8, valency 2) over 40 steps, rebuilds included, end
    bitwise where plain launches end, and where uneven calls with reads between them
    end (the work-list counters restart at every call and step)."""
    n = 300_000
    pos, L = inputs.uniform_positions(n, 0.5, seed=12)
    vel = inputs.maxwell_velocities(n, 1.0, seed=13)
    p = Params(E_a=8.0, f=2.0)
    outs = []
    for mode in ("graphs", "direct", "chunks"):
        with vbc.System(pos, L, _vp(p), vel=vel, seed=6) as s:
            if mode == "direct":
                s.profile(True, 1 << 14)
            r0 = s.stats().rebuilds
            for c in ((40,) if mode != "chunks" else (7, 1, 13, 19)):
                s.step(c, 0.005, 1.0, 1.0)
                st = s.stats()
                assert 0 < st.unsaturated < n // 16  # the last iteration's count, kept for the statistics
            outs.append(s.get_state())
        assert st.rebuilds - r0 >= 1
    for o in outs[1:]:
        assert o[2] == 40
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])


@pytest.mark.parametrize("prec", [F32, F64])
def test_set_state_keeps_a_valid_list(prec):
    """Loading a system's own state back keeps its neighbour list (no particle
    moved): in FP64 the run then continues bit for bit as if it had not been
    interrupted; in the FP32 split the double positions of the interface
    round the 2^-52 L fixed point by up to one unit, so the run continues to
    within 1e-9 (30 steps).  A load that moves a particle farther than
    skin / 2 from its position at the last build has the next pass rebuild
    the list, and one that moves none does not."""
    pos, vel, L, p = _system(3000, 0.5, seed=9)
    outs = []
    for interrupt in (False, True):
        with vbc.System(pos, L, _vp(p), vel=vel, seed=4, precision=prec) as s:
            s.step(30, 0.005, 1.0, 1.0)
            if interrupt:
                x, v, st = s.get_state()
                s.set_state(x, v, step=st)
            s.step(30, 0.005, 1.0, 1.0)
            outs.append(s.get_state())
    assert outs[0][2] == outs[1][2] == 60
    if prec == F64:
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    else:
        assert np.max(np.abs(outs[0][0] - outs[1][0])) <= 1e-9
        assert np.max(np.abs(outs[0][1] - outs[1][1])) <= 1e-7
    skin = 0.4  # the default
    with vbc.System(pos, L, _vp(p), vel=vel, seed=4, precision=prec) as s:
        s.step(10, 0.005, 1.0, 1.0)
        x, v, st = s.get_state()
        r0 = s.stats().rebuilds
        s.set_state(x, v, step=st)
        s.compute(F=True)
        assert s.stats().rebuilds == r0
        x2 = x.copy()
        x2[17, 0] += 0.6 * skin
        s.set_state(x2, v, step=st)
        s.compute(F=True)
        assert s.stats().rebuilds == r0 + 1
