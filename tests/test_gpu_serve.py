"""Serving loop (vbc_server_*) on the GPU.

Requests are independent Langevin simulations of different sizes, valencies
and temperatures.  A server admits them in arrival order as slots and device
memory free up and advances each in chunks on its own stream.  Each result must
be bitwise the same whether the request ran alone or in a mix with others;
admission must respect the memory budget; errors come back as codes.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

# (n, rho, valency f, kT, seed): uneven sizes, densities and parameters
REQS = [(3000, 0.5, 2.0, 1.0, 11), (20000, 0.3, 4.0, 1.2, 12), (8000, 0.6, 1.0, 0.9, 13),
        (50000, 0.5, 6.0, 1.1, 14)]


def _submit(srv, n, rho, f, kT, seed, nsteps, precision=vbc.VBC_FP32_SPLIT):
    pos, L = inputs.uniform_positions(n, rho, seed=seed)
    return srv.submit(pos, L, vbc.params(E_a=8.0, f=f), nsteps=nsteps, kT=kT, seed=seed, precision=precision)


@pytest.mark.parametrize("precision", [vbc.VBC_FP32_SPLIT, vbc.VBC_FP64])
def test_results_alone_equal_results_in_the_mix(precision):
    nsteps = 300
    alone = {}
    with vbc.Server(slots=1, chunk_steps=100) as srv:
        for r in REQS:
            rid = _submit(srv, *r, nsteps, precision=precision)
            assert srv.wait(rid).status == vbc.VBC_OK
            alone[r] = srv.result(rid)
    with vbc.Server(slots=4, chunk_steps=100) as srv:
        ids = {r: _submit(srv, *r, nsteps, precision=precision) for r in REQS}
        srv.wait()
        spans = []
        for r, rid in ids.items():
            pos, vel, info = srv.result(rid)
            assert info.status == vbc.VBC_OK and info.steps_done == nsteps and info.n == r[0]
            assert info.t_submit <= info.t_admit <= info.t_done
            np.testing.assert_array_equal(pos, alone[r][0])
            np.testing.assert_array_equal(vel, alone[r][1])
            spans.append((info.t_admit, info.t_done))
    # with four slots every request was admitted before the first one finished
    assert max(a for a, _ in spans) < min(d for _, d in spans)


def test_budget_admits_one_system_at_a_time():
    n, rho = 20000, 0.5
    pos, L = inputs.uniform_positions(n, rho, seed=5)
    prm = vbc.params(E_a=8.0, f=2.0)
    est = vbc.estimate_device_bytes(n, L, prm)
    with vbc.Server(hbm_budget=int(1.2 * est), slots=4, chunk_steps=50) as srv:
        ids = [srv.submit(pos, L, prm, nsteps=200, seed=s) for s in range(3)]
        srv.wait()
        infos = sorted((srv.result(i)[2] for i in ids), key=lambda x: x.t_admit)
    for a, b in zip(infos, infos[1:]):
        assert b.t_admit >= a.t_done
    assert all(0 < x.device_bytes <= est for x in infos)


def test_errors_are_codes():
    pos, L = inputs.uniform_positions(2000, 0.5, seed=1)
    with vbc.Server(hbm_budget=1 << 19, slots=2, chunk_steps=1000) as srv:
        with pytest.raises(vbc.VBCError) as e:
            srv.submit(pos, L, nsteps=10)            # needs about 1 MB, above the 512 KiB budget
        assert e.value.code == vbc.VBC_ERR_OOM
    with vbc.Server(slots=1, chunk_steps=1000) as srv:
        with pytest.raises(vbc.VBCError) as e:
            srv.submit(pos, L, nsteps=10, dt=-1.0)
        assert e.value.code == vbc.VBC_ERR_INVALID_ARG
        with pytest.raises(vbc.VBCError) as e:
            srv.info(12345)
        assert e.value.code == vbc.VBC_ERR_INVALID_ARG
        rid = srv.submit(pos, L, nsteps=200_000)
        with pytest.raises(vbc.VBCError) as e:
            srv.wait(rid, timeout=0.0)
        assert e.value.code == vbc.VBC_ERR_TIMEOUT
        with pytest.raises(vbc.VBCError) as e:
            srv.result(rid)                          # not finished
        assert e.value.code == vbc.VBC_ERR_INVALID_ARG
    # closing stopped the long request after its current chunk


def test_systems_created_side_by_side_equal_systems_alone():
    """Sixteen systems of different sizes created and stepped from sixteen host
    threads at once, each on its own stream, while others release their memory:
    every state ends bitwise where the same system created and stepped alone ends.
    (Each system's tables reach the device in copies ordered on its own stream, so
    its first kernels never read an allocation's previous contents.)"""
    import threading

    cases = [(1000 + 2500 * k, 0.5, 1.0 + k % 6, 100 + k) for k in range(16)]

    def run(n, rho, f, seed):
        pos, L = inputs.uniform_positions(n, rho, seed=seed)
        with vbc.System(pos, L, vbc.params(E_a=8.0, f=f), seed=seed) as s:
            s.step(60, 0.005, 1.0, 1.0)
            return s.get_state()

    alone = [run(*c) for c in cases]
    mixed = [None] * len(cases)
    errors = []

    def worker(k):
        try:
            for _ in range(2):  # create, step, release twice: later creations reuse released memory
                mixed[k] = run(*cases[k])
        except Exception as e:  # reported below, in the test's own thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for a, m in zip(alone, mixed):
        assert m[2] == a[2] == 60
        assert np.array_equal(a[0], m[0]) and np.array_equal(a[1], m[1])
