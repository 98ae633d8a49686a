"""Failure detection, made on the host: a state with a non-finite velocity, a
collapsed state with more particles in one cell than the cell tables hold,
and a long create/destroy loop.  Each error comes back as a status code with
the system still usable; nothing here faults the GPU (the bad values are
caught where they are loaded, and the crowded cell where the cells are
counted, before any kernel indexes with them)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

DT, KT, GAMMA = 0.005, 1.0, 1.0


@pytest.mark.parametrize("prec", [vbc.VBC_FP32_SPLIT, vbc.VBC_FP64])
def test_non_finite_velocity_is_reported_and_the_handle_stays_usable(prec):
    pos, L = inputs.uniform_positions(3000, 0.5, seed=71)
    vel = inputs.maxwell_velocities(3000, KT, seed=72)
    with vbc.System(pos, L, vbc.params(E_a=5.0), vel=vel, precision=prec) as s:
        s.step(10, DT, KT, GAMMA)
        good_x, good_v, st = s.get_state()
        bad = good_v.copy()
        bad[1234, 1] = np.nan
        with pytest.raises(vbc.VBCError) as e:
            s.set_state(good_x, bad, step=st)
            s.step(1, DT, KT, GAMMA)
        assert e.value.code == vbc.VBC_ERR_UNSTABLE
        # every later call reports the same until a good state is loaded
        with pytest.raises(vbc.VBCError) as e2:
            s.step(1, DT, KT, GAMMA)
        assert e2.value.code == vbc.VBC_ERR_UNSTABLE
        # a good state makes the handle usable again, and it steps as before
        s.set_state(good_x, good_v, step=st)
        s.step(5, DT, KT, GAMMA)
        x, v, st2 = s.get_state()
        assert st2 == st + 5 and np.all(np.isfinite(x)) and np.all(np.isfinite(v))


def test_out_of_range_velocity_is_reported_in_the_fixed_point_mode():
    """The FP32-split state holds |v| < 2^22 in its 2^-40 fixed point."""
    pos, L = inputs.uniform_positions(2000, 0.5, seed=73)
    vel = np.zeros_like(pos)
    vel[7, 0] = 1e7
    with pytest.raises(vbc.VBCError) as e:
        vbc.System(pos, L, vbc.params(), vel=vel)
    assert e.value.code == vbc.VBC_ERR_UNSTABLE and "fixed-point range" in str(e.value)


@pytest.mark.parametrize("prec", [vbc.VBC_FP32_SPLIT, vbc.VBC_FP64])
def test_crowded_cell_is_reported(prec):
    """600 coincident particles (more than the 512 one cell may hold) in a fluid of
    2000: creation fails with VBC_ERR_UNSTABLE naming the crowded cell."""
    pos, L = inputs.uniform_positions(2000, 0.5, seed=74)
    pos[:600] = pos[0]
    with pytest.raises(vbc.VBCError) as e:
        vbc.System(pos, L, vbc.params(), precision=prec)
    assert e.value.code == vbc.VBC_ERR_UNSTABLE and "one cell" in str(e.value)
    # a system created afterwards works
    pos2, L2 = inputs.uniform_positions(2000, 0.5, seed=75)
    with vbc.System(pos2, L2, vbc.params(), precision=prec) as s:
        s.step(3, DT, KT, GAMMA)


def test_create_destroy_loop_returns_device_memory():
    """200 systems created, stepped (which captures their CUDA graphs) and
    destroyed leave the device's free memory where it was after the first one."""
    import torch
    pos, L = inputs.uniform_positions(2000, 0.5, seed=76)
    for prec in (vbc.VBC_FP32_SPLIT, vbc.VBC_FP64):  # lazy module loads, first graphs
        with vbc.System(pos, L, vbc.params(), precision=prec) as s:
            s.step(4, DT, KT, GAMMA)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(200):
        with vbc.System(pos, L, vbc.params(), seed=k, precision=vbc.VBC_FP64 if k % 5 == 0 else vbc.VBC_FP32_SPLIT) as s:
            s.step(4, DT, KT, GAMMA)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
