"""Batched stepping (vbc_batch_*): systems of uneven size, valency and
temperature advanced together, either by one cooperative launch per iteration
for all systems (the fused mode, the default) or by their two-step graphs
captured side by side into one CUDA graph.  Every system must end bitwise
where it ends when stepped alone, over runs long enough to rebuild the
neighbour lists, for odd and even step counts.  A grid-wide wait that gives
up (a wait limit of zero spins) must come back as VBC_ERR_TIMEOUT with the
GPU context usable and every system halted until its state is loaded again."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

# (n, rho, valency f, kT, seed)
SYS = [(3000, 0.5, 2.0, 1.0, 21), (12000, 0.3, 4.0, 1.2, 22), (25000, 0.6, 1.0, 0.9, 23), (7000, 0.5, 6.0, 1.1, 24)]


def _make(n, rho, f, kT, seed, prec):
    pos, L = inputs.uniform_positions(n, rho, seed=seed)
    vel = inputs.maxwell_velocities(n, kT, seed=seed + 1)
    return vbc.System(pos, L, vbc.params(E_a=8.0, f=f), vel=vel, seed=seed, precision=prec)


@pytest.mark.parametrize("mode", [vbc.VBC_BATCH_FUSED, vbc.VBC_BATCH_GRAPHS])
@pytest.mark.parametrize("prec", [vbc.VBC_FP32_SPLIT, vbc.VBC_FP64])
def test_batch_equals_each_system_alone(prec, mode):
    kts = [c[3] for c in SYS]
    alone = []
    for c in SYS:
        with _make(*c, prec) as s:
            s.step(151, 0.005, c[3], 1.0)
            s.step(40, 0.005, c[3], 1.0)
            alone.append(s.get_state()[:2])
    systems = [_make(*c, prec) for c in SYS]
    try:
        with vbc.Batch(systems) as b:
            b.set_mode(mode)
            b.step(151, 0.005, kts, 1.0)
            b.step(40, 0.005, kts, 1.0)
            assert b.fused_launches() == (191 if mode == vbc.VBC_BATCH_FUSED else 0)
        for s, (pos, vel) in zip(systems, alone):
            p2, v2, step = s.get_state()
            assert step == 191
            np.testing.assert_array_equal(p2, pos)
            np.testing.assert_array_equal(v2, vel)
            assert s.stats().rebuilds > 1
    finally:
        for s in systems:
            s.close()


def test_fused_wait_that_gives_up_is_reported_and_recoverable():
    """With a wait limit of zero every grid-wide wait gives up at once: the step
    returns VBC_ERR_TIMEOUT, the systems refuse to step until a state is loaded,
    and after loading one they step bitwise like a fresh system from that state."""
    kts = [c[3] for c in SYS[:3]]
    systems = [_make(*c, vbc.VBC_FP32_SPLIT) for c in SYS[:3]]
    try:
        states = [s.get_state() for s in systems]
        with vbc.Batch(systems) as b:
            b.set_mode(vbc.VBC_BATCH_FUSED, wait_limit=0)
            with pytest.raises(vbc.VBCError) as e:
                b.step(10, 0.005, kts, 1.0)
            assert e.value.code == vbc.VBC_ERR_TIMEOUT
            with pytest.raises(vbc.VBCError) as e:
                systems[0].step(2, 0.005, kts[0], 1.0)
            assert e.value.code == vbc.VBC_ERR_TIMEOUT
            with pytest.raises(vbc.VBCError) as e:
                b.step(4, 0.005, kts, 1.0)
            assert e.value.code == vbc.VBC_ERR_TIMEOUT
            # load the states again: the default limit, and the batch steps as the systems do alone
            for s, (x, v, st) in zip(systems, states):
                s.set_state(x, v, step=st)
            b.set_mode(vbc.VBC_BATCH_FUSED)
            b.step(30, 0.005, kts, 1.0)
        for s, c, (x, v, st) in zip(systems, SYS[:3], states):
            with _make(*c, vbc.VBC_FP32_SPLIT) as ref:
                ref.set_state(x, v, step=st)
                ref.step(30, 0.005, c[3], 1.0)
                xr, vr, sr = ref.get_state()
            xb, vb, sb = s.get_state()
            assert sb == sr
            np.testing.assert_array_equal(xb, xr)
            np.testing.assert_array_equal(vb, vr)
    finally:
        for s in systems:
            s.close()


def test_batches_the_fused_launch_does_not_take_use_the_graphs():
    """A system on another row-walk block shape keeps the batch on the graphs;
    the result is still each system's own."""
    kts = [c[3] for c in SYS[:2]]
    alone = []
    for c in SYS[:2]:
        with _make(*c, vbc.VBC_FP32_SPLIT) as s:
            s.set_tuning(rows_threads_per_block=256)
            s.step(25, 0.005, c[3], 1.0)
            alone.append(s.get_state()[:2])
    systems = [_make(*c, vbc.VBC_FP32_SPLIT) for c in SYS[:2]]
    try:
        for s in systems:
            s.set_tuning(rows_threads_per_block=256)
        with vbc.Batch(systems) as b:
            b.step(25, 0.005, kts, 1.0)
            assert b.fused_launches() == 0
        for s, (pos, vel) in zip(systems, alone):
            p2, v2, _ = s.get_state()
            np.testing.assert_array_equal(p2, pos)
            np.testing.assert_array_equal(v2, vel)
    finally:
        for s in systems:
            s.close()


def test_batch_rejects_bad_arguments():
    a = _make(*SYS[0], vbc.VBC_FP32_SPLIT)
    try:
        with pytest.raises(vbc.VBCError) as e:
            vbc.Batch([a, a])
        assert e.value.code == vbc.VBC_ERR_INVALID_ARG
        with vbc.Batch([a]) as b:
            with pytest.raises(vbc.VBCError) as e:
                b.step(10, -0.1, 1.0, 1.0)
            assert e.value.code == vbc.VBC_ERR_INVALID_ARG
            b.step(0, 0.005, 1.0, 1.0)
    finally:
        a.close()


# ----------------------------------------------------------------- autotuning
@pytest.mark.parametrize("prec", [vbc.VBC_FP32_SPLIT, vbc.VBC_FP64])
def test_grid_settings_change_no_result(prec):
    """The tunable grids (blocks per SM of the close count and of the row walks)
    decide only which block takes which cell group or row: a system on the
    smallest grids ends bitwise where its twin on the default grids ends."""
    c = SYS[2]
    a, b = _make(*c, prec), _make(*c, prec)
    try:
        b.set_tuning(rows_blocks_per_sm=1, count_blocks_per_sm=1)
        for s in (a, b):
            s.step(120, 0.005, c[3], 1.0)
        pa, va, _ = a.get_state()
        pb, vb, _ = b.get_state()
        np.testing.assert_array_equal(pa, pb)
        np.testing.assert_array_equal(va, vb)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", [vbc.VBC_FP32_SPLIT, vbc.VBC_FP64])
def test_block_shape_and_threads_per_row_keep_parity(prec):
    """The row walks' block shape (128, 256, 512 threads) and the cap on threads
    per row only re-split the dense walks between threads: the FP32-split
    counts (integer sums) are the same under every setting, the FP64 ones agree
    to rounding, and forces stay within the parity tolerances of the oracle
    (1e-5 rms|F| in the FP32 split, 1e-10 in FP64)."""
    import oracle
    pos, L = inputs.uniform_positions(30000, 0.5, seed=91)
    n0 = oracle.evaluate(pos, L, oracle.Params(E_a=8.0), mode=1).counts
    p = oracle.Params(E_a=8.0, f=inputs.quantile_valency(n0, 0.5))
    ref = oracle.evaluate(pos, L, p, mode=1)
    assert np.mean(ref.ds != 0.0) > 0.1
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
    tol = 1e-5 if prec == vbc.VBC_FP32_SPLIT else 1e-10
    counts = []
    with vbc.System(pos, L, vbc.params(E_a=8.0, f=p.f), precision=prec) as s:
        for tpb, tmax in ((128, 32), (256, 32), (512, 32), (256, 1), (512, 4), (128, 2)):
            s.set_tuning(rows_threads_per_block=tpb, threads_per_row_max=tmax)
            r = s.compute(F=True, counts=True)
            counts.append(r.counts)
            assert np.max(np.abs(r.counts - ref.counts)) <= 1e-6
            assert np.max(np.abs(r.F - ref.F)) <= tol * rms
        with pytest.raises(vbc.VBCError):
            s.set_tuning(rows_threads_per_block=200)
        with pytest.raises(vbc.VBCError):
            s.set_tuning(threads_per_row_max=3)
    for c in counts[1:]:
        if prec == vbc.VBC_FP32_SPLIT:
            np.testing.assert_array_equal(c, counts[0])
        else:
            assert np.max(np.abs(c - counts[0])) <= 1e-12


def test_autotune_picks_a_setting_and_keeps_stepping():
    c = SYS[1]
    with _make(*c, vbc.VBC_FP32_SPLIT) as s:
        t = s.autotune(trial_steps=8, kT=c[3])
        assert t.rows_blocks_per_sm in (0, 1, 2, 4, 8) and t.count_blocks_per_sm in (0, 1, 2, 4, 8)
        assert t.rows_threads_per_block in (128, 256, 512) and t.threads_per_row_max in (2, 4, 8, 32)
        assert 0.0 < t.ms_per_step < 100.0
        s.step(20, 0.005, c[3], 1.0)
        assert s.get_state()[2] > 20
