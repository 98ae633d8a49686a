"""FP64 CPU oracle for the valency-bounding correction (VBC).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (the CUDA library and its binding) never does, and the
oracle imports nothing from the product.

The arithmetic lives in ``vbc_oracle.c`` (plain C, FP64, OpenMP over
particles).  This module compiles it with gcc on first use and exposes numpy
wrappers.  Each wrapper names the equation of the paper it follows; the C file
holds the derivation of the forces (chain rule through the counts), which the
paper defers to its supplement.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("r_r", "r_a", "r_l", "r_h", "E_r", "E_a", "f", "delta")]


@dataclass(frozen=True)
class Params:
    """VBC(r_l, r_h, delta) on the polynomial soft core (Sec. 2, Eqs. softcore, Psidelta).

    Defaults are the standard VBC: r_l = r_a = 1.5 r_r, r_h = 2 r_r, E_r = 20,
    E_a = 2, delta = 0."""

    r_r: float = 1.0
    r_a: float = 1.5
    r_l: float = 1.5
    r_h: float = 2.0
    E_r: float = 20.0
    E_a: float = 2.0
    f: float = 2.0
    delta: float = 0.0

    def c(self) -> _Params:
        return _Params(self.r_r, self.r_a, self.r_l, self.r_h, self.E_r, self.E_a, self.f, self.delta)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_omega.restype = ctypes.c_double
        L.orc_omega.argtypes = [ctypes.c_double] * 3
        L.orc_domega.restype = ctypes.c_double
        L.orc_domega.argtypes = [ctypes.c_double] * 3
        for name in ("orc_Vr", "orc_dVr", "orc_Va", "orc_dVa"):
            fn = getattr(L, name)
            fn.restype = ctypes.c_double
            fn.argtypes = [ctypes.c_double, ctypes.POINTER(_Params)]
        L.orc_eval.restype = ctypes.c_int
        L.orc_eval.argtypes = [ctypes.c_int64, dp, dp, ctypes.POINTER(_Params), ctypes.c_int] + [dp] * 8
        L.orc_pairs_within.restype = ctypes.c_int64
        L.orc_pairs_within.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int64]
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_normals.restype = None
        L.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, dp]
        L.orc_baoab.restype = ctypes.c_int
        L.orc_baoab.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.POINTER(_Params), ctypes.c_int,
                                ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)]
        L.orc_eval_typed.restype = ctypes.c_int
        L.orc_eval_typed.argtypes = ([ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                      ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_int), ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int] + [dp] * 8)
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _box3(box) -> np.ndarray:
    b = np.asarray(box, dtype=np.float64).reshape(-1)
    if b.size == 1:
        b = np.repeat(b, 3)
    return np.ascontiguousarray(b)


def omega(x: float, x1: float, x2: float) -> float:
    """Smooth step, Eq. (omega)."""
    return lib().orc_omega(x, x1, x2)


def domega(x: float, x1: float, x2: float) -> float:
    """Derivative of the smooth step with respect to x."""
    return lib().orc_domega(x, x1, x2)


def Vr(r: float, p: Params) -> float:
    """Repulsive soft core, Eq. (softcore)."""
    return lib().orc_Vr(r, ctypes.byref(p.c()))


def Va(r: float, p: Params) -> float:
    """Quartic attractive well, Eq. (softcore)."""
    return lib().orc_Va(r, ctypes.byref(p.c()))


def dVr(r: float, p: Params) -> float:
    return lib().orc_dVr(r, ctypes.byref(p.c()))


def dVa(r: float, p: Params) -> float:
    return lib().orc_dVa(r, ctypes.byref(p.c()))


@dataclass
class EvalResult:
    counts: np.ndarray   # n_i, Eq. (counter)
    s: np.ndarray        # omega(n_i; f - delta, f - delta + 1)
    ds: np.ndarray       # d s_i / d n_i
    A: np.ndarray        # dU/dn_i
    F: np.ndarray        # (n, 3) forces
    e: np.ndarray        # per-particle half pair energies, sum = U
    U: float
    W: float


def evaluate(pos: np.ndarray, box, p: Params, mode: int = 0) -> EvalResult:
    """All VBC outputs for one configuration.  mode 0 = all pairs, 1 = cell list."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    b = _box3(box)
    out = [np.zeros(n) for _ in range(4)] + [np.zeros((n, 3)), np.zeros(n)]
    U = ctypes.c_double(0.0)
    W = ctypes.c_double(0.0)
    rc = lib().orc_eval(n, _dp(b), _dp(pos), ctypes.byref(p.c()), mode,
                        *[_dp(a) for a in out], ctypes.byref(U), ctypes.byref(W))
    if rc != 0:
        raise ValueError("oracle: cell-list mode needs at least 3 cells per axis")
    return EvalResult(*out, U=U.value, W=W.value)


def evaluate_typed(pos: np.ndarray, box, types, P, cmask, bonds=None, k_b: float = 0.0, r_0: float = 1.0,
                   mode: int = 0) -> EvalResult:
    """Multi-type VBC with harmonic bonds (Sec. 2: counts restricted to selected
    neighbour types; Sec. 4: bead-spring sticker chains).  types [n] in
    [0, T); P a T x T nested list of Params (symmetric; a type's valency and
    shift from its diagonal entry); cmask T x T of 0/1 (cmask[a][b]: a
    particle of type a counts neighbours of type b); bonds [m, 2] particle
    indices, each bond once, with energy k_b/2 (r - r_0)^2.  mode 0 = all
    pairs, 1 = cell list."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    b = _box3(box)
    t = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    T = len(P)
    Pc = (_Params * (T * T))(*[P[a][c].c() for a in range(T) for c in range(T)])
    m = np.ascontiguousarray(np.asarray(cmask, dtype=np.int32).reshape(T * T))
    bd = np.ascontiguousarray(np.zeros((0, 2)) if bonds is None else bonds, dtype=np.int64).reshape(-1, 2)
    out = [np.zeros(n) for _ in range(4)] + [np.zeros((n, 3)), np.zeros(n)]
    U = ctypes.c_double(0.0)
    W = ctypes.c_double(0.0)
    rc = lib().orc_eval_typed(n, _dp(b), _dp(pos), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), T, Pc,
                              m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), bd.shape[0],
                              bd.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), k_b, r_0, mode,
                              *[_dp(a) for a in out], ctypes.byref(U), ctypes.byref(W))
    if rc == -1:
        raise ValueError("oracle: cell-list mode needs at least 3 cells per axis")
    if rc != 0:
        raise ValueError("oracle: a type or bond index is out of range")
    return EvalResult(*out, U=U.value, W=W.value)


def energy(pos: np.ndarray, box, p: Params) -> float:
    """U = sum_{i<j} [V_r + Psi V_a], Eq. (Vhat), all pairs."""
    return evaluate(pos, box, p, 0).U


def pairs_within(pos: np.ndarray, box, rcut: float) -> np.ndarray:
    """Unordered pairs (i < j) with minimum-image distance < rcut, shape (m, 2)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    b = _box3(box)
    cap = max(1, n * 64)
    while True:
        buf = np.zeros(2 * cap, dtype=np.int64)
        m = lib().orc_pairs_within(n, _dp(b), _dp(pos), rcut,
                                   buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
        if m <= cap:
            return buf[: 2 * m].reshape(-1, 2)
        cap = int(m)


@dataclass
class Observables:
    z: np.ndarray       # [n] neighbours within the attraction range, r_ij < r_a (strict)
    mean_z: float       # <z>
    p_err: float        # fraction of particles with z_i > f
    z_hist: np.ndarray  # [nbins] particles with z_i = k (last bin: z_i >= nbins - 1)


def observables(pos: np.ndarray, box, p: Params, nbins: int = 32) -> Observables:
    """Valency observables of Sec. 3: the neighbour number z_i = #{j != i : r_ij < r_a}
    (an instantaneous distance criterion, strict), its mean <z>, and the
    over-coordination probability P_err = fraction of particles with z_i > f.
    All pairs, minimum image, FP64."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    pr = pairs_within(pos, box, p.r_a)
    z = (np.bincount(pr[:, 0], minlength=n) + np.bincount(pr[:, 1], minlength=n)).astype(np.int64)
    hist = np.bincount(np.minimum(z, nbins - 1), minlength=nbins).astype(np.int64)
    return Observables(z=z, mean_z=float(z.mean()) if n else 0.0, p_err=float(np.mean(z > p.f)) if n else 0.0,
                       z_hist=hist)


def philox4x32_10(ctr, key) -> tuple:
    """Philox4x32 with 10 rounds (Salmon et al., SC'11)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def normals(seed: int, step: int, pid: int) -> np.ndarray:
    """The three Gaussian numbers the Langevin step draws for one particle."""
    z = np.zeros(3)
    lib().orc_normals(seed, step, pid, _dp(z))
    return z


def baoab(pos, vel, box, p: Params, nsteps: int, dt: float, kT: float, gamma: float,
          seed: int, step: int = 0, mode: int = 0):
    """nsteps BAOAB Langevin steps; returns (pos, vel, step) without touching the inputs."""
    x = np.array(pos, dtype=np.float64).reshape(-1, 3).copy()
    v = np.array(vel, dtype=np.float64).reshape(-1, 3).copy()
    b = _box3(box)
    st = ctypes.c_int64(step)
    rc = lib().orc_baoab(x.shape[0], _dp(b), _dp(x), _dp(v), ctypes.byref(p.c()), mode, nsteps,
                         dt, kT, gamma, seed, ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle: cell-list mode needs at least 3 cells per axis")
    return x, v, st.value


def num_threads() -> int:
    return lib().orc_num_threads()
