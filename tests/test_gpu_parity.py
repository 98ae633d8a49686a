"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs, element by element.

Tolerances (written here, used by every test of this file):
  counts n_i        <= 1e-6 absolute                    (both precisions)
  forces F_i        max|dF| <= 1e-5 rms|F| (FP32 split),  1e-10 rms|F| (FP64)
  energy U          <= 1e-9 relative                     (FP64 accumulation in both)
  virial W          <= 1e-6 relative (FP32 split),       1e-9 (FP64)
  switch s, s'      <= 1e-6 absolute (FP32 split),       1e-12 (FP64)
  chain term A_i    <= 1e-5 max|A| (FP32 split),         1e-10 max|A| (FP64)
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs, vbc

pytestmark = pytest.mark.gpu

F32, F64 = vbc.VBC_FP32_SPLIT, vbc.VBC_FP64
TOL = {
    F32: dict(F=1e-5, W=1e-6, s=1e-6, A=1e-5),
    F64: dict(F=1e-10, W=1e-9, s=1e-12, A=1e-10),
}
TOL_COUNT = 1e-6
TOL_U = 1e-9


def to_vbc(p: Params) -> vbc.PairParams:
    return vbc.params(**p.__dict__)


def with_quantile_valency(pos, L, p: Params, q: float, mode=0) -> Params:
    n0 = oracle.evaluate(pos, L, p, mode).counts
    return Params(**{**p.__dict__, "f": inputs.quantile_valency(n0, q) + p.delta})


def compare(pos, L, p: Params, prec, mode=0, min_window=0.0, ref=None, nlist_cap=0):
    ref = ref if ref is not None else oracle.evaluate(pos, L, p, mode)
    tol = TOL[prec]
    with vbc.System(pos, L, to_vbc(p), precision=prec, nlist_cap=nlist_cap) as s:
        r = s.compute(F=True, counts=True, energy=True, virial=True)
        sw, dsw, A = s.switch()
        st = s.stats()
    n = len(pos)
    assert np.max(np.abs(r.counts - ref.counts)) <= TOL_COUNT
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1))) if n else 0.0
    assert np.max(np.abs(r.F - ref.F)) <= tol["F"] * max(rms, 1e-12)
    assert abs(r.energy - ref.U) <= TOL_U * max(abs(ref.U), 1e-12)
    assert abs(r.virial - ref.W) <= tol["W"] * max(abs(ref.W), 1e-12)
    assert np.max(np.abs(sw - ref.s)) <= tol["s"]
    assert np.max(np.abs(dsw - ref.ds)) <= 4 * tol["s"]
    amax = max(np.max(np.abs(ref.A)), 1e-12)
    assert np.max(np.abs(A - ref.A)) <= tol["A"] * amax
    frac = np.mean(ref.ds != 0.0)
    assert frac >= min_window, f"in-window fraction {frac:.3f} too small to exercise the chain rule"
    assert st.in_window == int(np.sum(dsw != 0.0))
    return r, ref, st


# ----------------------------------------------------------------- uniform fluids
@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("q", [0.25, 0.5, 0.75])
def test_uniform_rho05_quantile_valency(prec, q):
    pos, L = inputs.uniform_positions(1000, 0.5, seed=1)
    p = with_quantile_valency(pos, L, Params(E_a=5.0), q)
    # counts spread with a standard deviation near 3, so a unit window holds ~10%
    compare(pos, L, p, prec, min_window=0.05)


@pytest.mark.parametrize("prec", [F32, F64])
def test_ragged_tail_shifted_window(prec):
    """4099 particles (not a multiple of the block size), delta = 0.3, E_a = 8."""
    pos, L = inputs.uniform_positions(4099, 0.5, seed=2)
    p = with_quantile_valency(pos, L, Params(E_a=8.0, delta=0.3), 0.5, mode=1)
    compare(pos, L, p, prec, mode=1, min_window=0.1)


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("f", [1.0, 2.0])
def test_paper_shape_low_density_clusters(prec, f):
    """Standard VBC at rho = 0.05 (the paper's benchmark density), clustered start."""
    pos, L = inputs.clustered_positions(2000, 0.05, seed=3, cluster_size=3, spread=0.9)
    compare(pos, L, Params(E_a=2.0, f=f), prec, min_window=0.05)


@pytest.mark.parametrize("prec", [F32, F64])
def test_dense_rows_longer_than_a_chunk_window(prec):
    """Tight clusters of 160: rows of about 140 list entries, 83% of them longer than 128
    (the dense count's 32 chunks of 4), so that rows continue across lane windows and across
    the warps of a group; counts, switch and forces against the oracle."""
    pos, L = inputs.clustered_positions(3200, 0.05, seed=21, cluster_size=160, spread=1.2)
    p = with_quantile_valency(pos, L, Params(E_a=5.0), 0.5, mode=1)
    compare(pos, L, p, prec, mode=1)


@pytest.mark.parametrize("prec", [F32, F64])
def test_optimised_vbc(prec):
    """VBC(1.29, 1.50, 0.30) of Sec. 4."""
    pos, L = inputs.clustered_positions(1500, 0.1, seed=4, cluster_size=4, spread=0.8)
    p = with_quantile_valency(pos, L, Params(r_l=1.29, r_h=1.50, delta=0.30, E_a=2.0), 0.5)
    compare(pos, L, p, prec, min_window=0.1)


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("name,kw", [
    ("standard", dict(r_l=1.5, r_h=2.0, f=12.0)),
    ("partial", dict(r_l=0.75, r_h=1.25, f=0.5)),
    ("blind", dict(r_l=0.5, r_h=1.0, f=0.001)),
    ("no_vbc", dict(f=1000.0)),
])
def test_four_counter_configurations(prec, name, kw):
    """The four counter configurations of Sec. 5 (N = 1000, rho = 0.05, E_a = 5),
    on a collapsed-cluster start so that the counters see many neighbours."""
    pos, L = inputs.clustered_positions(1000, 0.05, seed=5, cluster_size=8, spread=0.7)
    compare(pos, L, Params(E_a=5.0, **kw), prec)


# ----------------------------------------------------------------- edge cases
@pytest.mark.parametrize("prec", [F32, F64])
def test_single_particle(prec):
    pos = np.array([[1.0, 2.0, 3.0]])
    with vbc.System(pos, 10.0, vbc.params(), precision=prec) as s:
        r = s.compute(F=True, counts=True, energy=True, virial=True)
    assert r.counts[0] == 0.0 and np.all(r.F == 0.0) and r.energy == 0.0 and r.virial == 0.0


@pytest.mark.parametrize("prec", [F32, F64])
def test_dimer_closed_form(prec):
    """Dimer at the well centre with f = 0.5: n = 1, s = 9/16, U = -E_a (9/16)^2."""
    pos = np.array([[5.0, 5.0, 5.0], [6.25, 5.0, 5.0]])
    with vbc.System(pos, 10.0, vbc.params(f=0.5), precision=prec) as s:
        r = s.compute(F=True, counts=True, energy=True)
    assert np.all(np.abs(r.counts - 1.0) <= TOL_COUNT)
    assert abs(r.energy + 2.0 * 81.0 / 256.0) <= 1e-9
    assert np.max(np.abs(r.F)) <= 1e-5


@pytest.mark.parametrize("prec", [F32, F64])
def test_coincident_particles(prec):
    """Fully overlapping soft cores (r = 0) give finite energy and zero pair force."""
    pos, L = inputs.uniform_positions(300, 0.3, seed=6)
    pos[1] = pos[0]
    pos[2] = pos[0]
    p = with_quantile_valency(pos, L, Params(E_a=4.0), 0.5)
    r, ref, _ = compare(pos, L, p, prec)
    assert np.all(np.isfinite(r.F))


@pytest.mark.parametrize("prec", [F32, F64])
def test_positions_outside_the_box(prec):
    """Any periodic image is accepted: shifting particles by box vectors changes nothing."""
    pos, L = inputs.uniform_positions(800, 0.5, seed=7)
    p = with_quantile_valency(pos, L, Params(E_a=5.0), 0.5)
    shifted = pos.copy()
    shifted[::2] += L * np.array([3.0, -1.0, 7.0])
    ref = oracle.evaluate(pos, L, p)
    compare(shifted, L, p, prec, ref=ref)


@pytest.mark.parametrize("prec", [F32, F64])
def test_list_overflow_grows_and_matches(prec):
    """A tiny initial capacity overflows; the library grows the list and the result
    is the oracle's."""
    pos, L = inputs.uniform_positions(1000, 0.5, seed=8)
    p = with_quantile_valency(pos, L, Params(E_a=5.0), 0.5)
    _, _, st = compare(pos, L, p, prec, nlist_cap=4)
    assert st.nlist_cap >= st.nlist_max


def test_orthorhombic_box_fp64():
    rng = np.random.Generator(np.random.PCG64(9))
    box = np.array([11.0, 13.5, 9.0])
    pos = rng.uniform(0, 1, (650, 3)) * box
    p = with_quantile_valency(pos, box, Params(E_a=5.0), 0.5)
    compare(pos, box, p, F64, min_window=0.1)


# ----------------------------------------------------------------- neighbour list
@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("n,rho", [(3000, 0.5), (30000, 0.5), (20000, 0.25)])
def test_neighbour_list_is_exact(prec, n, rho):
    """The list holds every pair closer than r_c + skin and none beyond.  3000
    particles give 7 cells per edge (the build on fixed-point words); the larger
    systems have 8 or more (the build on block-relative floats, which skips
    whole neighbour cells beyond the list radius)."""
    pos, L = inputs.uniform_positions(n, rho, seed=10)
    rlist = 2.0 + 0.4
    with vbc.System(pos, L, vbc.params(), precision=prec, skin=0.4) as s:
        nnb, nbr = s.neighbors(cap=256)
    assert nnb.max() < 256
    got = set()
    for i in range(len(pos)):
        row = nbr[i, : nnb[i]]
        assert len(set(row.tolist())) == nnb[i]
        got.update((i, int(j)) for j in row)
    pairs = oracle.pairs_within(pos, L, rlist)
    d = pos[pairs[:, 0]] - pos[pairs[:, 1]]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(1))
    sure = pairs[r < rlist - 1e-6]
    for i, j in sure:
        assert (i, j) in got and (j, i) in got
    # nothing beyond the radius: up to the fixed-point resolution, and for the block-relative
    # float build up to its relative margin of 1e-5 (a few extra entries, never a missing one)
    gi = np.array([a for a, _ in got])
    gj = np.array([b for _, b in got])
    dd = pos[gi] - pos[gj]
    dd -= L * np.round(dd / L)
    assert np.sqrt((dd * dd).sum(1)).max() < rlist * (1.0 + 1.1e-5) + 1e-6
    assert len(got) >= 2 * len(sure)


# ----------------------------------------------------------------- determinism, API forms
def test_deterministic_bitwise():
    pos, L = inputs.uniform_positions(5000, 0.5, seed=11)
    p = with_quantile_valency(pos, L, Params(E_a=5.0), 0.5, mode=1)
    outs = []
    for _ in range(2):
        with vbc.System(pos, L, to_vbc(p)) as s:
            r = s.compute(F=True, counts=True, energy=True)
            outs.append((r.F.copy(), r.counts.copy(), r.energy))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_device_pointers_match_host_path():
    import torch
    pos, L = inputs.uniform_positions(2000, 0.5, seed=12)
    p = with_quantile_valency(pos, L, Params(E_a=5.0), 0.5)
    with vbc.System(pos, L, to_vbc(p)) as s:
        rh = s.compute(F=True, counts=True, energy=True, virial=True)
    dpos = torch.from_numpy(pos).cuda()
    F = torch.zeros((2000, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros(2000, dtype=torch.float64, device="cuda")
    with vbc.System(dpos, L, to_vbc(p)) as s:
        rd = s.compute(F=F, counts=c, energy=True, virial=True)
    torch.cuda.synchronize()
    assert np.array_equal(F.cpu().numpy(), rh.F) and np.array_equal(c.cpu().numpy(), rh.counts)
    assert rd.energy == rh.energy and rd.virial == rh.virial


def test_set_params_recomputes():
    pos, L = inputs.uniform_positions(1000, 0.5, seed=13)
    p1 = with_quantile_valency(pos, L, Params(E_a=5.0), 0.3)
    p2 = with_quantile_valency(pos, L, Params(E_a=3.0, delta=0.2), 0.6)
    ref = oracle.evaluate(pos, L, p2)
    with vbc.System(pos, L, to_vbc(p1)) as s:
        s.compute(F=True)
        s.set_params(to_vbc(p2))
        r = s.compute(F=True, counts=True, energy=True)
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
    assert np.max(np.abs(r.F - ref.F)) <= 1e-5 * rms
    assert abs(r.energy - ref.U) <= TOL_U * abs(ref.U)


def test_bad_step_arguments_rejected():
    pos, L = inputs.uniform_positions(500, 0.5, seed=14)
    with vbc.System(pos, L, vbc.params()) as s:
        for args in ((1, -0.01, 1.0, 1.0), (1, 0.01, -1.0, 1.0), (-1, 0.01, 1.0, 1.0)):
            with pytest.raises(vbc.VBCError) as e:
                s.step(*args)
            assert e.value.code == vbc.VBC_ERR_INVALID_ARG


# ----------------------------------------------------------------- row-walk modes
def _window_valency(n0: np.ndarray, lo: float, hi: float) -> float:
    """A valency f (delta = 0) whose window (f, f + 1) holds a fraction of the
    particles between lo and hi, taken from the oracle's counts."""
    for q in (0.01, 0.005, 0.02, 0.002, 0.04):
        f = float(np.quantile(n0, q))
        frac = np.mean((n0 > f) & (n0 < f + 1.0))
        if lo <= frac <= hi:
            return f
    raise AssertionError("no valency gives the wanted window fraction")


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("case", ["saturated", "few_in_window", "many_in_window"])
def test_forces_only_row_walk_modes(prec, case):
    """A force evaluation without counts takes the saturation split: the close
    lists settle saturated particles, and the row walks pick their sparse or dense
    mode from their list lengths (threshold n/16).  Three valencies on a 30k
    uniform fluid cover sparse counts and forces with nearly every particle
    saturated, a sparse chain pass that clears whole-force tags, and the dense
    passes."""
    n = 30_000
    pos, L = inputs.uniform_positions(n, 0.5, seed=11)
    base = Params(E_a=8.0)
    n0 = oracle.evaluate(pos, L, base, 1).counts
    if case == "saturated":
        f = 2.0
    elif case == "few_in_window":
        f = _window_valency(n0, 0.005, 0.05)
    else:
        f = inputs.quantile_valency(n0, 0.5)
    p = Params(**{**base.__dict__, "f": f})
    ref = oracle.evaluate(pos, L, p, 1)
    tol = TOL[prec]
    with vbc.System(pos, L, to_vbc(p), precision=prec) as s:
        r = s.compute(F=True)
        sw, dsw, A = s.switch()
        st = s.stats()
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
    assert np.max(np.abs(r.F - ref.F)) <= tol["F"] * rms
    assert np.max(np.abs(sw - ref.s)) <= tol["s"]
    assert np.max(np.abs(dsw - ref.ds)) <= 4 * tol["s"]
    assert np.max(np.abs(A - ref.A)) <= tol["A"] * max(np.max(np.abs(ref.A)), 1e-12)
    assert st.in_window == int(np.sum(dsw != 0.0))
    if case == "saturated":
        assert st.in_window <= n // 16 and st.unsaturated <= n // 16
    elif case == "few_in_window":
        assert 0 < st.in_window <= n // 16
    else:
        assert st.in_window > n // 16 and st.unsaturated > n // 16


# ----------------------------------------------------------------- valency observables
def _borderline(pos, L, i, r_a, eps=1e-6):
    """Particle i has a pair within eps of r_a, where the two sides' position
    representations (FP64 here, fixed point on the device) may decide r < r_a
    differently."""
    d = pos - pos[i]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(1))
    return bool(np.any(np.abs(r - r_a) < eps))


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("rho,n", [(0.05, 20000), (0.5, 30000)])
def test_valency_observables(prec, rho, n):
    """z_i, <z>, P_err and the z histogram (Sec. 3) against the oracle, element by
    element (integers: equal except for particles with a pair within 1e-6 of r_a),
    on a fresh state and after 50 Langevin steps with rebuilds."""
    pos, L = inputs.uniform_positions(n, rho, seed=17)
    p = Params(E_a=8.0, f=2.0)
    with vbc.System(pos, L, to_vbc(p), precision=prec) as s:
        for nsteps in (0, 50):
            if nsteps:
                s.step(nsteps, 0.005, 1.0, 1.0)
            cur, _, _ = s.get_state()
            ob, z = s.observables(z=True)
            ref = oracle.observables(cur, L, p)
            bad = np.nonzero(z != ref.z)[0]
            assert len(bad) <= 4
            assert all(_borderline(cur, L, i, p.r_a) for i in bad)
            assert ob.mean_z == pytest.approx(z.mean(), abs=1e-12)
            assert ob.p_err == pytest.approx(np.mean(z > p.f), abs=1e-12)
            assert list(ob.z_hist) == np.bincount(np.minimum(z, vbc.ZHIST - 1), minlength=vbc.ZHIST).tolist()
            assert abs(ob.mean_z - ref.mean_z) <= 2.0 * len(bad) / n


# ----------------------------------------------------------------- full sizes
@pytest.mark.parametrize("n", [100_000, 1_000_000])
def test_full_size_uniform_rho05(n):
    """The single-system workloads at full size (100k: the valency-sweep system;
    1M: the throughput workload), FP32 split, against the oracle's cell-list mode
    over every particle."""
    pos, L = inputs.uniform_positions(n, 0.5, seed=3)
    p = with_quantile_valency(pos, L, Params(E_a=8.0), 0.5, mode=1)
    compare(pos, L, p, F32, mode=1, min_window=0.1)


@pytest.mark.parametrize("n", [20_000, 1_000_000])
def test_counts_finer_than_the_position_words(n):
    """FP32 split: window pairs of the counts (Sec. 2, Eq. n_i) are measured
    with the residual bits of the 64-bit state below the 32-bit position words,
    so n_i carries only the 2^-32 rounding of each window term -- far below the
    ~5e-7 (at N = 1M, L = 126) that the L / 2^32 grid alone would leave."""
    pos, L = inputs.uniform_positions(n, 0.5, seed=3)
    p = Params(E_a=8.0, f=8.0)
    ref = oracle.evaluate(pos, L, p, 1)
    with vbc.System(pos, L, to_vbc(p), precision=F32) as s:
        r = s.compute(counts=True)
    assert np.max(np.abs(r.counts - ref.counts)) <= 1e-8


@pytest.mark.parametrize("valency", [2.0, 8.0])
def test_full_size_forces_only_as_benchmarked(valency):
    """The throughput workload as the benchmark runs it: N = 1M, density 0.5,
    E_a = 8, forces without counts, so that the close lists settle the saturated
    particles and the row walks run sparse (valency 2: under 1% unsettled) or dense
    (valency 8: most particles unsettled or beside a window particle).  Forces,
    s, s' and A of every particle against the oracle's cell-list mode."""
    n = 1_000_000
    pos, L = inputs.uniform_positions(n, 0.5, seed=3)
    p = Params(E_a=8.0, f=valency)
    ref = oracle.evaluate(pos, L, p, 1)
    tol = TOL[F32]
    with vbc.System(pos, L, to_vbc(p), precision=F32) as s:
        r = s.compute(F=True)
        sw, dsw, A = s.switch()
        st = s.stats()
    rms = np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1)))
    assert np.max(np.abs(r.F - ref.F)) <= tol["F"] * rms
    assert np.max(np.abs(sw - ref.s)) <= tol["s"]
    assert np.max(np.abs(dsw - ref.ds)) <= 4 * tol["s"]
    assert np.max(np.abs(A - ref.A)) <= tol["A"] * max(np.max(np.abs(ref.A)), 1e-12)
    if valency == 2.0:
        assert st.unsaturated <= n // 16
    else:
        assert st.unsaturated > n // 16
