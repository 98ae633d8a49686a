"""Pins for the FP64 oracle: each test checks it against something the paper or
the mathematics fixes independently of the oracle's own code (closed forms,
hand-derived worked examples, finite differences of the energy, conservation
laws, the Fisher-Ruelle bound of Eq. Hstable, the paper's shell-occupancy
estimate, published Philox test vectors)."""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2609_07842_b300 import inputs

STD = Params()  # standard VBC(1.5, 2.0, 0), E_r = 20, E_a = 2


# ------------------------------------------------------------ Philox (SC'11)
def test_philox_known_answers(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox4x32_10(r[0:4], r[4:6]) == tuple(r[6:10])


def test_normals_distribution():
    """The Langevin noise: zero mean, unit variance, no correlation between the
    three components, and each word maps through Box-Muller."""
    z = np.array([oracle.normals(7, s, i) for s in range(40) for i in range(1000)])
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.015
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(3))) < 0.02
    # fourth moment of a Gaussian is 3
    assert abs((z ** 4).mean() - 3.0) < 0.08
    # Box-Muller radius: z0^2 + z1^2 = -2 ln u0 with u0 from the first Philox word
    x = oracle.philox4x32_10([5, 0, 3, 0], [11, 0])
    u0 = ((x[0] >> 9) + 0.5) / 2.0 ** 23
    zz = oracle.normals(11, 5, 3)
    assert math.isclose(zz[0] ** 2 + zz[1] ** 2, -2.0 * math.log(u0), rel_tol=1e-13)


# ------------------------------------------------------------ Eq. omega
def test_omega_closed_forms():
    assert oracle.omega(0.3, 1.0, 2.0) == 1.0
    assert oracle.omega(1.0, 1.0, 2.0) == 1.0
    assert oracle.omega(2.0, 1.0, 2.0) == 0.0
    assert oracle.omega(7.0, 1.0, 2.0) == 0.0
    # t = 1/2 -> (3/4)^2; t = 1/4 -> (15/16)^2; t = 3/4 -> (7/16)^2
    assert oracle.omega(1.5, 1.0, 2.0) == 9.0 / 16.0
    assert oracle.omega(1.25, 1.0, 2.0) == 225.0 / 256.0
    assert oracle.omega(3.5, 2.0, 4.0) == 49.0 / 256.0
    # derivative -4 t (1 - t^2) / w: t = 1/2, w = 2 -> -3/4
    assert math.isclose(oracle.domega(3.0, 2.0, 4.0), -0.75, rel_tol=1e-15)


def test_omega_is_c1():
    """Continuously differentiable: the derivative matches central differences
    everywhere and vanishes at both ends of the window."""
    h = 1e-6
    for x in np.linspace(0.5, 2.5, 401):
        fd = (oracle.omega(x + h, 1.0, 2.0) - oracle.omega(x - h, 1.0, 2.0)) / (2 * h)
        # a central difference straddling a jump of omega'' (8/w^2 at the ends)
        # is off by at most h * 8 / 2
        assert abs(fd - oracle.domega(x, 1.0, 2.0)) < 5e-6
    assert oracle.domega(1.0, 1.0, 2.0) == 0.0 and oracle.domega(2.0, 1.0, 2.0) == 0.0


# ------------------------------------------------------------ Eq. softcore
def test_softcore_closed_forms():
    p = STD
    assert oracle.Vr(0.0, p) == 20.0
    assert oracle.Vr(1.0, p) == 0.0
    assert math.isclose(oracle.Vr(math.sqrt(0.5), p), 5.0, rel_tol=1e-14)
    assert oracle.Vr(0.5, p) == 11.25
    # the well reaches -E_a at its centre (r_a + r_r)/2 and vanishes at both ends
    assert oracle.Va(1.25, p) == -2.0
    assert oracle.Va(1.0, p) == 0.0 and oracle.Va(1.5, p) == 0.0
    assert oracle.Va(0.3, p) == 0.0 and oracle.Va(1.8, p) == 0.0
    # u = 1/2 -> -E_a (3/4)^2
    assert math.isclose(oracle.Va(1.375, p), -2.0 * 0.5625, rel_tol=1e-15)
    assert oracle.dVa(1.25, p) == 0.0
    h = 1e-6
    for r in np.linspace(0.05, 1.7, 167):
        fd = (oracle.Vr(r + h, p) - oracle.Vr(r - h, p)) / (2 * h)
        assert abs(fd - oracle.dVr(r, p)) < 1e-6
        fd = (oracle.Va(r + h, p) - oracle.Va(r - h, p)) / (2 * h)
        assert abs(fd - oracle.dVa(r, p)) < 1e-6


# ------------------------------------------------------------ worked examples
def _line(xs, box=100.0):
    pos = np.zeros((len(xs), 3))
    pos[:, 0] = np.asarray(xs) + 50.0
    pos[:, 1:] = 50.0
    return pos, box


def test_dimer_closed_forms():
    # dimer inside the well, valency 0.5: n = 1 each, s = omega(1; 0.5, 1.5) = 9/16
    p = Params(f=0.5)
    pos, box = _line([0.0, 1.25])
    r = oracle.evaluate(pos, box, p)
    assert np.all(r.counts == 1.0)
    assert np.all(r.s == 9.0 / 16.0)
    assert r.U == -2.0 * (81.0 / 256.0)
    # dimer in the counting window only: n = 9/16, no energy
    r = oracle.evaluate(*_line([0.0, 1.75]), Params(f=2.0))
    assert np.all(r.counts == 9.0 / 16.0) and r.U == 0.0
    # overlapping cores: V_r(0.5) whatever the valency
    for f in (0.001, 1.0, 1000.0):
        r = oracle.evaluate(*_line([0.0, 0.5]), Params(f=f))
        assert r.U == 11.25
    # fully overlapping pair: finite energy E_r, zero force
    r = oracle.evaluate(*_line([0.0, 0.0]), STD)
    assert r.U == 20.0 and np.all(r.F == 0.0)


def test_trimer_worked_example(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "trimer_collinear.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = Fraction(v)
    r = oracle.evaluate(*_line([0.0, 1.25, 1.75]), Params(f=1.2))
    assert r.counts[0] == float(vals["n0"]) and r.counts[1] == float(vals["n1"])
    assert r.counts[2] == float(vals["n2"])
    assert math.isclose(r.s[0], float(vals["s0"]), rel_tol=1e-15)
    assert math.isclose(r.s[1], float(vals["s1"]), rel_tol=1e-14)
    assert math.isclose(r.U, float(vals["U"]), rel_tol=1e-15)


# ------------------------------------------------------------ limits of Psi
def _pair_sum(pos, box, fn):
    n = pos.shape[0]
    tot = 0.0
    for i in range(n):
        d = pos[i] - pos[i + 1:]
        d -= box * np.round(d / box)
        for r in np.sqrt((d * d).sum(1)):
            tot += fn(r)
    return tot


def test_bare_limit_large_valency():
    """f = 1000 (the 'no VBC' configuration of Sec. 5): the cap is never reached
    and U is the bare soft-core sum."""
    pos, L = inputs.uniform_positions(120, 0.5, seed=3)
    p = Params(E_a=5.0, f=1000.0)
    bare = _pair_sum(pos, L, lambda r: oracle.Vr(r, p) + oracle.Va(r, p))
    r = oracle.evaluate(pos, L, p)
    assert np.all(r.s == 1.0) and np.all(r.A == 0.0)
    assert math.isclose(r.U, bare, rel_tol=1e-12)


def test_full_suppression():
    """Every count above f - delta + 1: Psi = 0, only the repulsive core remains."""
    pos, L = inputs.uniform_positions(150, 0.5, seed=4)
    p = Params(E_a=8.0, f=0.5)
    r = oracle.evaluate(pos, L, p)
    assert r.counts.min() > 1.5
    assert np.all(r.s == 0.0) and np.all(r.A == 0.0)
    assert math.isclose(r.U, _pair_sum(pos, L, lambda x: oracle.Vr(x, p)), rel_tol=1e-12)


# ------------------------------------------------------------ forces = -grad U
def _fd_forces(pos, box, p, h=1e-6):
    F = np.zeros_like(pos)
    for i in range(pos.shape[0]):
        for a in range(3):
            xp = pos.copy(); xp[i, a] += h
            xm = pos.copy(); xm[i, a] -= h
            F[i, a] = -(oracle.energy(xp, box, p) - oracle.energy(xm, box, p)) / (2 * h)
    return F


@pytest.mark.parametrize("preset", ["standard_q50", "shifted_q30", "optimised", "partial"])
def test_forces_match_finite_differences(preset):
    pos, L = inputs.uniform_positions(60, 0.35, seed=11)
    base = {"standard_q50": Params(E_a=5.0),
            "shifted_q30": Params(E_a=5.0, delta=0.3),
            "optimised": Params(r_l=1.29, r_h=1.50, delta=0.30, E_a=5.0),
            "partial": Params(r_l=0.75, r_h=1.25, E_a=5.0)}[preset]
    q = {"standard_q50": 0.5, "shifted_q30": 0.3, "optimised": 0.5, "partial": 0.5}[preset]
    n0 = oracle.evaluate(pos, L, base).counts
    p = Params(**{**base.__dict__, "f": inputs.quantile_valency(n0, q) + base.delta})
    r = oracle.evaluate(pos, L, p)
    assert np.mean(r.ds != 0.0) > 0.1, "chain-rule path not exercised"
    Ffd = _fd_forces(pos, L, p)
    rms = np.sqrt(np.mean(np.sum(r.F ** 2, axis=1)))
    assert np.max(np.abs(r.F - Ffd)) <= 1e-7 * rms


def test_chain_rule_term_matters():
    """The chain-rule coefficient A_i = s'_i sum_j s_j V_a(r_ij) = dU/dn_i equals a
    direct sum over the pinned pair functions, and is large enough on this
    configuration that the finite-difference tests above would fail without
    the (A_i + A_j) omega' force term."""
    pos, L = inputs.uniform_positions(60, 0.35, seed=12)
    p0 = Params(E_a=5.0)
    n0 = oracle.evaluate(pos, L, p0).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, 0.5))
    r = oracle.evaluate(pos, L, p)
    # A_i = s'_i sum_j s_j V_a(r_ij): check against a direct sum with the pinned pair functions
    for i in np.nonzero(r.ds)[0][:10]:
        d = pos[i] - pos
        d -= L * np.round(d / L)
        rr = np.sqrt((d * d).sum(1))
        tot = sum(r.s[j] * oracle.Va(rr[j], p) for j in range(len(rr)) if j != i)
        assert math.isclose(r.A[i], r.ds[i] * tot, rel_tol=1e-12, abs_tol=1e-14)
    assert np.max(np.abs(r.A)) > 0.1


# ------------------------------------------------------------ invariants
def _cluster(n, seed, radius=2.2):
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    while len(pts) < n:
        x = rng.uniform(-radius, radius, 3)
        if np.dot(x, x) <= radius * radius:
            pts.append(x)
    return np.array(pts) + 50.0, 100.0


def test_momentum_and_torque_conservation():
    pos, box = _cluster(40, 5)
    n0 = oracle.evaluate(pos, box, Params(E_a=5.0)).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, 0.5))
    r = oracle.evaluate(pos, box, p)
    scale = np.abs(r.F).max()
    assert np.all(np.abs(r.F.sum(0)) < 1e-12 * scale * len(pos))
    torque = np.cross(pos - pos.mean(0), r.F).sum(0)
    assert np.all(np.abs(torque) < 1e-11 * scale * len(pos))


def test_translation_permutation_periodic_shift():
    pos, L = inputs.uniform_positions(100, 0.5, seed=6)
    n0 = oracle.evaluate(pos, L, Params(E_a=5.0)).counts
    p = Params(E_a=5.0, f=inputs.quantile_valency(n0, 0.5))
    r = oracle.evaluate(pos, L, p)
    r2 = oracle.evaluate(pos + np.array([0.37, -1.9, 5.2]), L, p)
    assert np.allclose(r2.F, r.F, rtol=0, atol=1e-11) and math.isclose(r2.U, r.U, rel_tol=1e-12)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(len(pos))
    r3 = oracle.evaluate(pos[perm], L, p)
    assert np.allclose(r3.F, r.F[perm], rtol=0, atol=1e-11)
    assert np.allclose(r3.counts, r.counts[perm], rtol=0, atol=1e-13)
    shifted = pos.copy()
    shifted[::3] += L * np.array([1, -2, 3])
    r4 = oracle.evaluate(shifted, L, p)
    assert np.allclose(r4.F, r.F, rtol=0, atol=1e-10) and math.isclose(r4.U, r.U, rel_tol=1e-12)


def test_fisher_ruelle_bound():
    """Eq. (Hstable): with r_l >= r_a (omega_min = 1), U_a >= -N (f + 1) E_a / 2."""
    for f in (1.0, 2.0, 3.5):
        for seed in range(3):
            for pos, box in (_cluster(30, seed, radius=1.0), _cluster(60, seed, radius=2.0),
                             inputs.uniform_positions(200, 0.6, seed)):
                p = Params(E_r=0.0, E_a=7.0, f=f)
                Ua = oracle.evaluate(pos, box, p).U
                assert Ua >= -len(pos) * (f + 1) * 7.0 / 2 - 1e-9
    # an isolated bonded dimer at f = 1 sits at U_a = -E_a = -N E_a / 2, above -N E_a
    pos, box = _line([0.0, 1.25])
    assert oracle.evaluate(pos, box, Params(E_r=0.0, E_a=7.0, f=1.0)).U == -7.0


# ------------------------------------------------------------ statistics of the counts
def test_paper_shell_occupancy(golden_dir):
    """Sec. 3: at rho = 0.05 about 0.5 particles occupy the shell r_r < r < r_a and
    about 9% of particles have two or more.  Counting radii set to a near-step
    at r_a and at r_r give the shell population per particle."""
    vals = {}
    with open(os.path.join(golden_dir, "paper_shell_occupancy.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                t = line.split()
                vals[t[0]] = [float(x) for x in t[1:]]
    rho = vals["rho"][0]
    pos, L = inputs.uniform_positions(40000, rho, seed=21)
    eps = 1e-9
    within_a = oracle.evaluate(pos, L, Params(r_l=1.5 - eps, r_h=1.5, f=1e9), mode=1).counts
    within_r = oracle.evaluate(pos, L, Params(r_l=1.0 - eps, r_h=1.0, f=1e9), mode=1).counts
    shell = np.rint(within_a - within_r)
    mean, tol = vals["mean_shell_occupants"]
    assert abs(shell.mean() - mean) < tol + 0.01  # paper rounds to 0.5; sampling error ~0.004
    p2, tol2 = vals["p_two_or_more"]
    assert abs(np.mean(shell >= 2) - p2) < tol2 + 0.005


def test_uniform_fluid_mean_count():
    """The mean smoothed count of an ideal (uniform) fluid is rho times the
    integral of omega(r) over space; for the standard radii that is
    rho (4 pi/3 r_l^3 + 4 pi int_{r_l}^{r_h} omega r^2 dr)."""
    from scipy.integrate import quad
    rho = 0.5
    w = quad(lambda r: 4 * np.pi * r * r * (1 - ((r - 1.5) / 0.5) ** 2) ** 2, 1.5, 2.0)[0]
    expect = rho * (4 * np.pi / 3 * 1.5 ** 3 + w)
    pos, L = inputs.uniform_positions(20000, rho, seed=8)
    n = oracle.evaluate(pos, L, STD, mode=1).counts
    assert abs(n.mean() - expect) < 0.06


def test_cell_mode_equals_all_pairs():
    pos, L = inputs.uniform_positions(3000, 0.5, seed=9)
    n0 = oracle.evaluate(pos, L, Params(E_a=8.0), mode=1).counts
    p = Params(E_a=8.0, f=inputs.quantile_valency(n0, 0.5), delta=0.2)
    a = oracle.evaluate(pos, L, p, mode=0)
    b = oracle.evaluate(pos, L, p, mode=1)
    assert np.max(np.abs(a.counts - b.counts)) < 1e-12
    assert np.max(np.abs(a.A - b.A)) < 1e-11
    assert np.max(np.abs(a.F - b.F)) < 1e-10
    assert math.isclose(a.U, b.U, rel_tol=1e-13) and math.isclose(a.W, b.W, rel_tol=1e-13)


def test_pairs_within_brute_force():
    pos, L = inputs.uniform_positions(300, 0.5, seed=10)
    pairs = oracle.pairs_within(pos, L, 2.4)
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    iu = np.triu_indices(len(pos), 1)
    expect = set(zip(iu[0][r[iu] < 2.4].tolist(), iu[1][r[iu] < 2.4].tolist()))
    assert set(map(tuple, pairs.tolist())) == expect


# ------------------------------------------------------------ valency observables (Sec. 3)
def test_observables_line_by_hand():
    """Four particles on a line at x = 0, 1.2, 2.5, 10 (r_a = 1.5): neighbours are
    the pairs closer than r_a, so z = (1, 2, 1, 0), <z> = 1 and, at f = 1, only the
    middle particle is over-coordinated."""
    pos = np.array([[0.0, 0, 0], [1.2, 0, 0], [2.5, 0, 0], [10.0, 0, 0]]) + 5.0
    ob = oracle.observables(pos, 40.0, Params(f=1.0), nbins=4)
    assert ob.z.tolist() == [1, 2, 1, 0]
    assert ob.mean_z == 1.0 and ob.p_err == 0.25
    assert ob.z_hist.tolist() == [1, 2, 1, 0]


def test_observables_strict_at_r_a():
    """The criterion is strict: a pair exactly r_a apart is not a neighbour."""
    pos = np.array([[5.0, 5.0, 5.0], [6.5, 5.0, 5.0]])
    assert oracle.observables(pos, 20.0, Params()).z.tolist() == [0, 0]
    pos[1, 0] = np.nextafter(6.5, 0.0)
    assert oracle.observables(pos, 20.0, Params()).z.tolist() == [1, 1]


def test_observables_paper_shell_occupancy(golden_dir):
    """Sec. 3 at rho = 0.05: about 0.5 shell occupants (r_r < r < r_a) per
    particle and about 9% of particles with two or more, as the difference of
    the neighbour numbers at r_a and at r_r; the full neighbour number of an
    ideal fluid has mean rho 4 pi r_a^3 / 3."""
    vals = {}
    with open(os.path.join(golden_dir, "paper_shell_occupancy.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                t = line.split()
                vals[t[0]] = [float(x) for x in t[1:]]
    rho = vals["rho"][0]
    pos, L = inputs.uniform_positions(20000, rho, seed=22)
    za = oracle.observables(pos, L, Params(r_a=1.5)).z
    zr = oracle.observables(pos, L, Params(r_a=1.0)).z
    shell = za - zr
    mean, tol = vals["mean_shell_occupants"]
    assert abs(shell.mean() - mean) < tol + 0.015
    p2, tol2 = vals["p_two_or_more"]
    assert abs(np.mean(shell >= 2) - p2) < tol2 + 0.008
    assert abs(za.mean() - rho * 4.0 * np.pi / 3.0 * 1.5 ** 3) < 0.035


# ------------------------------------------------------------ BAOAB Langevin
def test_free_flight_is_exact():
    """No forces, no friction: x advances by dt v, v is unchanged."""
    pos, L = inputs.uniform_positions(50, 0.1, seed=2)
    vel = inputs.maxwell_velocities(50, 1.0, seed=3)
    p = Params(E_r=0.0, E_a=0.0)
    x, v, st = oracle.baoab(pos, vel, L, p, 3, 0.01, 1.0, 0.0, seed=5)
    assert st == 3 and np.array_equal(v, vel)
    assert np.allclose(x, pos + 0.03 * vel, rtol=0, atol=1e-14)


def test_ornstein_uhlenbeck_step():
    """No forces: v1 = c1 v0 + sqrt((1 - c1^2) kT) xi, x1 = x0 + dt/2 (v0 + v1)."""
    pos, L = inputs.uniform_positions(20, 0.1, seed=2)
    vel = inputs.maxwell_velocities(20, 1.0, seed=3)
    p = Params(E_r=0.0, E_a=0.0)
    dt, kT, g = 0.01, 1.3, 2.0
    x, v, _ = oracle.baoab(pos, vel, L, p, 1, dt, kT, g, seed=9, step=41)
    c1 = math.exp(-g * dt)
    for i in range(20):
        xi = oracle.normals(9, 41, i)
        v1 = c1 * vel[i] + math.sqrt((1 - c1 * c1) * kT) * xi
        assert np.allclose(v[i], v1, rtol=0, atol=1e-14)
        assert np.allclose(x[i], pos[i] + 0.5 * dt * (vel[i] + v1), rtol=0, atol=1e-13)


def test_step_counter_and_restart():
    pos, L = inputs.uniform_positions(64, 0.3, seed=4)
    vel = inputs.maxwell_velocities(64, 1.0, seed=5)
    p = Params(E_a=4.0, f=2.0)
    xa, va, sa = oracle.baoab(pos, vel, L, p, 2, 0.005, 1.0, 1.0, seed=1, step=10)
    x1, v1, s1 = oracle.baoab(pos, vel, L, p, 1, 0.005, 1.0, 1.0, seed=1, step=10)
    xb, vb, sb = oracle.baoab(x1, v1, L, p, 1, 0.005, 1.0, 1.0, seed=1, step=s1)
    assert sa == sb == 12 and np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.slow
def test_nve_energy_drift():
    """gamma = 0: BAOAB reduces to velocity Verlet; total energy is conserved up to
    O(dt^2) fluctuations without drift."""
    pos, L = inputs.clustered_positions(64, 0.2, seed=7)
    vel = inputs.maxwell_velocities(64, 1.0, seed=8)
    n0 = oracle.evaluate(pos, L, Params(E_a=4.0)).counts
    p = Params(E_a=4.0, f=inputs.quantile_valency(n0, 0.5))
    # relax overlapping cores first so that the test starts from a smooth state
    pos, vel, _ = oracle.baoab(pos, vel, L, p, 200, 0.002, 1.0, 5.0, seed=3)
    E0 = oracle.energy(pos, L, p) + 0.5 * np.sum(vel ** 2)
    x, v = pos, vel
    Es = []
    for _ in range(10):
        x, v, _ = oracle.baoab(x, v, L, p, 100, 0.002, 1.0, 0.0, seed=3)
        Es.append(oracle.energy(x, L, p) + 0.5 * np.sum(v ** 2))
    assert max(abs(e - E0) for e in Es) < 2e-3 * (abs(E0) + 64)


@pytest.mark.slow
def test_equipartition():
    """Langevin at kT: <KE>/N -> 3/2 kT."""
    pos, L = inputs.uniform_positions(125, 0.3, seed=12)
    vel = np.zeros((125, 3))
    p = Params(E_a=3.0, f=2.0)
    x, v, st = oracle.baoab(pos, vel, L, p, 300, 0.005, 1.0, 2.0, seed=4)
    ke = []
    for _ in range(40):
        x, v, st = oracle.baoab(x, v, L, p, 25, 0.005, 1.0, 2.0, seed=4, step=st)
        ke.append(0.5 * np.sum(v ** 2) / 125)
    ke = np.array(ke)
    # samples 25 steps apart at gamma dt = 0.01 are correlated over ~4 samples
    err = 4 * ke.std() / math.sqrt(len(ke) / 4)
    assert abs(ke.mean() - 1.5) < err + 0.02
