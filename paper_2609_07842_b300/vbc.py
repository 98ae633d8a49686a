"""ctypes binding of libvbc.so (C ABI in include/vbc.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be numpy arrays (host memory) or CUDA torch tensors
(device memory, passed by pointer); torch supplies device memory and the
stream, nothing else.  There is no CPU fallback: if the library cannot be
loaded, or a call fails, a VBCError is raised.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvbc.so")

VBC_OK = 0
VBC_ERR_INVALID_ARG = -1
VBC_ERR_CUDA = -2
VBC_ERR_OOM = -3
VBC_ERR_NLIST_OVERFLOW = -4
VBC_ERR_UNSTABLE = -5
VBC_ERR_TIMEOUT = -6
VBC_ERR_CANCELLED = -7
VBC_REQ_QUEUED = 1
VBC_REQ_RUNNING = 2
VBC_FP32_SPLIT = 0
VBC_FP64 = 1
VBC_BATCH_FUSED = 0
VBC_BATCH_GRAPHS = 1
K_REBUILD, K_COUNT, K_CHAIN, K_FORCE, K_ENERGY = range(5)

#: every function the header declares
EXPORTS = ("vbc_create_system", "vbc_create_typed_system", "vbc_build_neighbors", "vbc_compute_forces", "vbc_get_switch",
           "vbc_get_neighbors",
           "vbc_step_langevin", "vbc_get_state", "vbc_set_state", "vbc_set_params", "vbc_get_stats",
           "vbc_compute_thermo",
           "vbc_profile", "vbc_profile_read", "vbc_kernel_launches", "vbc_destroy", "vbc_last_error",
           "vbc_compute_forces_noalloc", "vbc_estimate_device_bytes", "vbc_get_observables",
           "vbc_batch_create", "vbc_batch_step", "vbc_batch_destroy", "vbc_batch_set_mode",
           "vbc_batch_fused_launches", "vbc_set_tuning", "vbc_autotune",
           "vbc_server_create", "vbc_server_submit", "vbc_server_wait", "vbc_server_info",
           "vbc_server_result", "vbc_server_destroy", "vbc_server_last_error")

#: largest n accepted by compute_forces_noalloc (size of its static device scratch)
NOALLOC_MAX_N = 16384


class VBCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libvbc error {code}: {msg}")
        self.code = code


class PairParams(ctypes.Structure):
    """VBC(r_l, r_h, delta) on the polynomial soft core (Sec. 2)."""
    _fields_ = [(k, ctypes.c_double) for k in ("r_r", "r_a", "r_l", "r_h", "E_r", "E_a", "f", "delta")]


class _Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("box", ctypes.c_double * 3), ("pos", ctypes.c_void_p),
                ("vel", ctypes.c_void_p), ("params", PairParams), ("skin", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32), ("nlist_cap", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("inputs_on_device", ctypes.c_int32)]


class _Types(ctypes.Structure):
    _fields_ = [("ntypes", ctypes.c_int32), ("type", ctypes.c_void_p), ("pair", ctypes.c_void_p),
                ("count_mask", ctypes.c_void_p), ("nbonds", ctypes.c_int64), ("bonds", ctypes.c_void_p),
                ("k_bond", ctypes.c_double), ("r0_bond", ctypes.c_double)]


#: largest number of particle types of a multi-type system
MAX_TYPES = 8

ZHIST = 32


class Tuning(ctypes.Structure):
    """Grid settings of the close count and the row walks (vbc_autotune)."""
    _fields_ = [("rows_blocks_per_sm", ctypes.c_int32), ("count_blocks_per_sm", ctypes.c_int32),
                ("rows_threads_per_block", ctypes.c_int32), ("threads_per_row_max", ctypes.c_int32),
                ("ms_per_step", ctypes.c_double)]


class Observables(ctypes.Structure):
    """Valency observables (Sec. 3): <z>, P_err and the histogram of z_i."""
    _fields_ = [("mean_z", ctypes.c_double), ("p_err", ctypes.c_double), ("z_hist", ctypes.c_int64 * ZHIST)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("slots", ctypes.c_int32), ("chunk_steps", ctypes.c_int64)]


class _Request(ctypes.Structure):
    _fields_ = [("system", _Config), ("nsteps", ctypes.c_int64), ("dt", ctypes.c_double),
                ("kT", ctypes.c_double), ("gamma", ctypes.c_double)]


class RequestInfo(ctypes.Structure):
    """Status and timeline of one served request (seconds on the server's clock)."""
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int64), ("steps_done", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("device_bytes", ctypes.c_int64)]


class Thermo(ctypes.Structure):
    """FP64 reductions of the current state (vbc_compute_thermo): U, the pair
    virial W, KE, the mean count, the in-window count, the pairs within r_c."""
    _fields_ = [("U", ctypes.c_double), ("W", ctypes.c_double), ("KE", ctypes.c_double),
                ("mean_n", ctypes.c_double), ("in_window", ctypes.c_int64), ("pairs_within_rc", ctypes.c_int64),
                ("step", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("step", ctypes.c_int64), ("rebuilds", ctypes.c_int64),
                ("nlist_cap", ctypes.c_int32), ("nlist_max", ctypes.c_int32), ("nlist_mean", ctypes.c_double),
                ("pairs_within_rc", ctypes.c_int64), ("in_window", ctypes.c_int64),
                ("unsaturated", ctypes.c_int64), ("stage_cap", ctypes.c_int32), ("group_cap", ctypes.c_int32),
                ("groups", ctypes.c_int32),
                ("capacity_grows", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libvbc.so from the package directory (built by build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2609_07842_b300.build` "
                          "(the VBC path has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i64, i32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int
    L.vbc_create_system.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
    L.vbc_create_typed_system.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Types), ctypes.POINTER(vp)]
    L.vbc_build_neighbors.argtypes = [vp]
    L.vbc_compute_forces.argtypes = [vp, vp, vp, vp, vp, i32]
    L.vbc_get_switch.argtypes = [vp, vp, vp, vp, i32]
    L.vbc_get_neighbors.argtypes = [vp, vp, vp, ctypes.c_int32, i32]
    L.vbc_step_langevin.argtypes = [vp, i64, dp, dp, dp]
    L.vbc_get_state.argtypes = [vp, vp, vp, ctypes.POINTER(i64), i32]
    L.vbc_set_state.argtypes = [vp, vp, vp, i64, i32]
    L.vbc_set_params.argtypes = [vp, ctypes.POINTER(PairParams)]
    L.vbc_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.vbc_compute_thermo.argtypes = [vp, ctypes.POINTER(Thermo)]
    L.vbc_compute_thermo.restype = i32
    L.vbc_profile.argtypes = [vp, i32, i64]
    L.vbc_profile_read.argtypes = [vp, i32, ctypes.POINTER(dp), ctypes.POINTER(i64)]
    L.vbc_kernel_launches.argtypes = [vp]
    L.vbc_kernel_launches.restype = i64
    L.vbc_destroy.argtypes = [vp]
    L.vbc_destroy.restype = None
    L.vbc_compute_forces_noalloc.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), vp,
                                             ctypes.POINTER(PairParams), vp, vp, vp]
    L.vbc_compute_forces_noalloc.restype = i32
    L.vbc_last_error.argtypes = []
    L.vbc_last_error.restype = ctypes.c_char_p
    L.vbc_estimate_device_bytes.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(i64)]
    L.vbc_get_observables.argtypes = [vp, ctypes.POINTER(Observables), vp, i32]
    L.vbc_get_observables.restype = i32
    L.vbc_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.POINTER(vp)]
    L.vbc_batch_create.restype = i32
    L.vbc_batch_step.argtypes = [vp, i64, dp, ctypes.POINTER(dp), dp]
    L.vbc_batch_step.restype = i32
    L.vbc_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.vbc_set_tuning.restype = i32
    L.vbc_autotune.argtypes = [vp, i64, dp, dp, dp, ctypes.POINTER(Tuning)]
    L.vbc_autotune.restype = i32
    L.vbc_batch_set_mode.argtypes = [vp, i32, i64]
    L.vbc_batch_set_mode.restype = i32
    L.vbc_batch_fused_launches.argtypes = [vp]
    L.vbc_batch_fused_launches.restype = i64
    L.vbc_batch_destroy.argtypes = [vp]
    L.vbc_batch_destroy.restype = None
    L.vbc_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(vp)]
    L.vbc_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(i64)]
    L.vbc_server_wait.argtypes = [vp, i64, dp, ctypes.POINTER(RequestInfo)]
    L.vbc_server_info.argtypes = [vp, i64, ctypes.POINTER(RequestInfo)]
    L.vbc_server_result.argtypes = [vp, i64, vp, vp, ctypes.POINTER(RequestInfo)]
    L.vbc_server_destroy.argtypes = [vp]
    L.vbc_server_destroy.restype = None
    L.vbc_server_last_error.argtypes = []
    L.vbc_server_last_error.restype = ctypes.c_char_p
    for name in ("vbc_estimate_device_bytes", "vbc_server_create", "vbc_server_submit", "vbc_server_wait",
                 "vbc_server_info", "vbc_server_result"):
        getattr(L, name).restype = i32
    for name in ("vbc_create_system", "vbc_build_neighbors", "vbc_compute_forces", "vbc_get_switch",
                 "vbc_get_neighbors", "vbc_step_langevin", "vbc_get_state", "vbc_set_state", "vbc_set_params", "vbc_get_stats",
                 "vbc_profile", "vbc_profile_read"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc: int):
    if rc != VBC_OK:
        raise VBCError(rc, load().vbc_last_error().decode())


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, on_device: bool | None = None):
    """(pointer, on_device) of a numpy array or torch tensor (float64, contiguous)."""
    if a is None:
        return None, on_device
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        dev = a.is_cuda
        return ctypes.c_void_p(a.data_ptr()), dev
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("arrays must be C-contiguous float64 numpy arrays or torch tensors")
    return ctypes.c_void_p(a.ctypes.data), False


def _same_side(items):
    sides = {d for _, d in items if d is not None}
    if len(sides) > 1:
        raise TypeError("all arrays of one call must be on the same side (host or device)")
    return int(sides.pop()) if sides else 0


def params(**kw) -> PairParams:
    """Pair parameters; defaults are the standard VBC (r_r=1, r_a=r_l=1.5, r_h=2, E_r=20, E_a=2,
    f=2, delta=0)."""
    d = dict(r_r=1.0, r_a=1.5, r_l=1.5, r_h=2.0, E_r=20.0, E_a=2.0, f=2.0, delta=0.0)
    d.update(kw)
    return PairParams(**d)


@dataclass
class Result:
    F: object = None
    counts: object = None
    energy: float | None = None
    virial: float | None = None
    extra: dict = field(default_factory=dict)


class System:
    """One particle system resident on the GPU (vbc_create_system ... vbc_destroy)."""

    def __init__(self, pos, box, prm: PairParams | None = None, vel=None, skin: float = 0.4,
                 seed: int = 1, precision: int = VBC_FP32_SPLIT, nlist_cap: int = 0, stream=None):
        L = load()
        prm = prm if prm is not None else params()
        b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
        n = int(pos.shape[0])
        pp, pdev = _ptr(pos)
        vv, vdev = _ptr(vel)
        on_dev = _same_side([(pp, pdev), (vv, vdev)])
        if stream is None and on_dev:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        cfg = _Config(n=n, box=(ctypes.c_double * 3)(*b), pos=pp, vel=vv, params=prm, skin=skin,
                      seed=seed, precision=precision, nlist_cap=nlist_cap,
                      stream=ctypes.c_void_p(stream) if stream else None, inputs_on_device=on_dev)
        h = ctypes.c_void_p()
        _check(L.vbc_create_system(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.n = n
        self.box = b.copy()
        self.precision = precision

    @classmethod
    def typed(cls, pos, box, types, pair, count_mask, bonds=None, k_bond: float = 0.0, r0_bond: float = 1.0,
              vel=None, skin: float = 0.4, seed: int = 1, nlist_cap: int = 0, precision: int = VBC_FP64):
        """A multi-type system (vbc_create_typed_system; FP64 or FP32 split): types [n] in [0, T),
        pair a T x T nested list of PairParams (symmetric; a type's f and delta from
        its diagonal entry), count_mask T x T of 0/1 (row type counts column type),
        bonds [m, 2] particle indices with energy k_bond/2 (r - r0_bond)^2.  Host
        arrays; pos and vel as for System."""
        L = load()
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        n = int(pos.shape[0])
        vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        t = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
        T = len(pair)
        tab = (PairParams * (T * T))(*[pair[a][b] for a in range(T) for b in range(T)])
        m = np.ascontiguousarray(np.asarray(count_mask, dtype=np.int32).reshape(T * T))
        bd = np.ascontiguousarray(np.zeros((0, 2)) if bonds is None else bonds, dtype=np.int64).reshape(-1, 2)
        b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
        cfg = _Config(n=n, box=(ctypes.c_double * 3)(*b), pos=ctypes.c_void_p(pos.ctypes.data),
                      vel=ctypes.c_void_p(vel.ctypes.data) if vel is not None else None, params=params(),
                      skin=skin, seed=seed, precision=precision, nlist_cap=nlist_cap, stream=None,
                      inputs_on_device=0)
        ty = _Types(ntypes=T, type=ctypes.c_void_p(t.ctypes.data), pair=ctypes.cast(tab, ctypes.c_void_p),
                    count_mask=ctypes.c_void_p(m.ctypes.data), nbonds=bd.shape[0],
                    bonds=ctypes.c_void_p(bd.ctypes.data) if bd.shape[0] else None, k_bond=k_bond,
                    r0_bond=r0_bond)
        h = ctypes.c_void_p()
        _check(L.vbc_create_typed_system(ctypes.byref(cfg), ctypes.byref(ty), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        self.n = n
        self.box = b.copy()
        self.precision = precision
        return self

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().vbc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def build_neighbors(self):
        _check(load().vbc_build_neighbors(self._h))

    def compute(self, F=None, counts=None, energy: bool = False, virial: bool = False) -> Result:
        """One force/energy evaluation (vbc_compute_forces).  F [n,3] and counts [n] are caller
        buffers: numpy (host) or CUDA tensors (device); pass True to get new numpy arrays."""
        if F is True:
            F = np.zeros((self.n, 3))
        if counts is True:
            counts = np.zeros(self.n)
        fp, fd = _ptr(F)
        cp, cd = _ptr(counts)
        dev = _same_side([(fp, fd), (cp, cd)])
        buf = None
        if dev and (energy or virial):
            import torch
            buf = torch.zeros(2, dtype=torch.float64, device="cuda")
            ep = ctypes.c_void_p(buf.data_ptr()) if energy else None
            wp = ctypes.c_void_p(buf.data_ptr() + 8) if virial else None
        else:
            e, w = ctypes.c_double(0.0), ctypes.c_double(0.0)
            ep = ctypes.byref(e) if energy else None
            wp = ctypes.byref(w) if virial else None
        _check(load().vbc_compute_forces(self._h, fp, cp, ep, wp, dev))
        if buf is not None:
            vals = buf.cpu().numpy()
            ev, wv = float(vals[0]), float(vals[1])
        else:
            ev, wv = e.value, w.value
        return Result(F=F, counts=counts, energy=ev if energy else None, virial=wv if virial else None)

    def switch(self):
        """(s, ds/dn, A) per particle from the last evaluation, as numpy arrays."""
        s, ds, A = np.zeros(self.n), np.zeros(self.n), np.zeros(self.n)
        _check(load().vbc_get_switch(self._h, _ptr(s)[0], _ptr(ds)[0], _ptr(A)[0], 0))
        return s, ds, A

    def neighbors(self, cap: int = 256):
        """(nnb [n], nbr [n, cap]) of the last build in caller indices; unused slots are -1."""
        nnb = np.zeros(self.n, dtype=np.int32)
        nbr = np.full((self.n, cap), -1, dtype=np.int32)
        _check(load().vbc_get_neighbors(self._h, ctypes.c_void_p(nnb.ctypes.data),
                                        ctypes.c_void_p(nbr.ctypes.data), cap, 0))
        return nnb, nbr

    def step(self, nsteps: int, dt: float, kT: float, gamma: float):
        _check(load().vbc_step_langevin(self._h, int(nsteps), dt, kT, gamma))

    def get_state(self, pos=None, vel=None):
        if pos is None:
            pos = np.zeros((self.n, 3))
        if vel is None:
            vel = np.zeros((self.n, 3))
        pp, pd = _ptr(pos)
        vv, vd = _ptr(vel)
        dev = _same_side([(pp, pd), (vv, vd)])
        st = ctypes.c_int64(0)
        _check(load().vbc_get_state(self._h, pp, vv, ctypes.byref(st), dev))
        return pos, vel, st.value

    def set_state(self, pos, vel=None, step: int = 0):
        pp, pd = _ptr(pos)
        vv, vd = _ptr(vel)
        dev = _same_side([(pp, pd), (vv, vd)])
        _check(load().vbc_set_state(self._h, pp, vv, int(step), dev))

    def set_params(self, prm: PairParams):
        _check(load().vbc_set_params(self._h, ctypes.byref(prm)))

    def autotune(self, trial_steps: int = 50, dt: float = 0.005, kT: float = 1.0, gamma: float = 1.0) -> Tuning:
        """Pick the fastest grid settings by timed trials (vbc_autotune); advances the system."""
        t = Tuning()
        _check(load().vbc_autotune(self._h, int(trial_steps), dt, kT, gamma, ctypes.byref(t)))
        return t

    def set_tuning(self, rows_blocks_per_sm: int = 0, count_blocks_per_sm: int = 0, rows_threads_per_block: int = 0,
                   threads_per_row_max: int = 0):
        t = Tuning(rows_blocks_per_sm=rows_blocks_per_sm, count_blocks_per_sm=count_blocks_per_sm,
                   rows_threads_per_block=rows_threads_per_block, threads_per_row_max=threads_per_row_max)
        _check(load().vbc_set_tuning(self._h, ctypes.byref(t)))

    def observables(self, z: bool = False):
        """(Observables, z_i per particle [n] int32 or None) of the current state."""
        out = Observables()
        zz = np.zeros(self.n, dtype=np.int32) if z else None
        _check(load().vbc_get_observables(self._h, ctypes.byref(out),
                                          ctypes.c_void_p(zz.ctypes.data) if z else None, 0))
        return out, zz

    def thermo(self) -> Thermo:
        """U, W, KE, mean count, in-window and pair counts of the current state
        (vbc_compute_thermo; leaves the trajectory unchanged)."""
        t = Thermo()
        _check(load().vbc_compute_thermo(self._h, ctypes.byref(t)))
        return t

    def stats(self) -> Stats:
        s = Stats()
        _check(load().vbc_get_stats(self._h, ctypes.byref(s)))
        return s

    def profile(self, enable: bool, max_launches: int = 1 << 16):
        _check(load().vbc_profile(self._h, int(enable), int(max_launches)))

    def profile_read(self, which: int):
        ms = ctypes.c_double(0.0)
        cnt = ctypes.c_int64(0)
        _check(load().vbc_profile_read(self._h, which, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    def kernel_launches(self) -> int:
        return int(load().vbc_kernel_launches(self._h))


def compute_forces_noalloc(pos, box: float, prm: PairParams, F, counts=None, stream=None):
    """Counts and forces of one small system without any device allocation
    (vbc_compute_forces_noalloc).  pos [n,3], F [n,3] and counts [n] are CUDA
    float64 tensors on one device; the library's static scratch holds at most
    NOALLOC_MAX_N particles.  Meant for callers that cannot allocate device
    memory.  Shapes and devices are checked here, before the library is
    called, so that a wrong buffer never reaches a kernel."""
    import torch
    tensors = [("pos", pos), ("F", F)] + ([("counts", counts)] if counts is not None else [])
    for name, t in tensors:
        if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError(f"pos must have shape (n, 3), not {tuple(pos.shape)}")
    n = int(pos.shape[0])
    if tuple(F.shape) != (n, 3):
        raise ValueError(f"F must have shape ({n}, 3), not {tuple(F.shape)}")
    if counts is not None and tuple(counts.shape) != (n,):
        raise ValueError(f"counts must have shape ({n},), not {tuple(counts.shape)}")
    dev = pos.device
    for name, t in tensors:
        if t.device != dev:
            raise ValueError(f"{name} is on {t.device}, pos on {dev}: all tensors must share one device")
    b = (ctypes.c_double * 3)(*np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        _check(load().vbc_compute_forces_noalloc(n, b, ctypes.c_void_p(pos.data_ptr()), ctypes.byref(prm),
                                                 ctypes.c_void_p(F.data_ptr()),
                                                 ctypes.c_void_p(counts.data_ptr()) if counts is not None else None,
                                                 ctypes.c_void_p(stream) if stream else None))


def _host_config(pos, box, prm: PairParams | None, vel, skin: float, seed: int, precision: int,
                 nlist_cap: int = 0):
    """A vbc_config over host float64 arrays (kept alive by the caller)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    if vel is not None:
        vel = np.ascontiguousarray(vel, dtype=np.float64)
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    cfg = _Config(n=n, box=(ctypes.c_double * 3)(*b), pos=ctypes.c_void_p(pos.ctypes.data),
                  vel=ctypes.c_void_p(vel.ctypes.data) if vel is not None else None,
                  params=prm if prm is not None else params(), skin=skin, seed=seed, precision=precision,
                  nlist_cap=nlist_cap, stream=None, inputs_on_device=0)
    return cfg, pos, vel


def estimate_device_bytes(n: int, box, prm: PairParams | None = None, skin: float = 0.4,
                          precision: int = VBC_FP32_SPLIT) -> int:
    """Device bytes vbc_create_system would allocate for n particles in this box
    (vbc_estimate_device_bytes; touches no device)."""
    pos = np.zeros((max(int(n), 1), 3))
    cfg, _, _ = _host_config(pos, box, prm, None, skin, 0, precision)
    cfg.n = int(n)
    out = ctypes.c_int64(0)
    _check(load().vbc_estimate_device_bytes(ctypes.byref(cfg), ctypes.byref(out)))
    return int(out.value)


def _check_server(rc: int):
    if rc != VBC_OK:
        raise VBCError(rc, load().vbc_server_last_error().decode())


class Server:
    """Serving loop (vbc_server_*): requests admitted in arrival order by free
    slots and a device-memory budget, advanced in chunks on their own streams,
    state resident on the device until a request finishes."""

    def __init__(self, hbm_budget: float = 150e9, slots: int = 8, chunk_steps: int = 1000):
        L = load()
        h = ctypes.c_void_p()
        cfg = _ServerConfig(hbm_budget=int(hbm_budget), slots=int(slots), chunk_steps=int(chunk_steps))
        _check_server(L.vbc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, pos, box, prm: PairParams | None = None, nsteps: int = 1000, dt: float = 0.005,
               kT: float = 1.0, gamma: float = 1.0, vel=None, skin: float = 0.4, seed: int = 0,
               precision: int = VBC_FP32_SPLIT) -> int:
        """Queue one simulation; returns its request id.  The inputs are copied."""
        cfg, _p, _v = _host_config(pos, box, prm, vel, skin, seed, precision)
        req = _Request(system=cfg, nsteps=int(nsteps), dt=dt, kT=kT, gamma=gamma)
        rid = ctypes.c_int64(0)
        _check_server(load().vbc_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)))
        return int(rid.value)

    def wait(self, rid: int = -1, timeout: float = -1.0) -> RequestInfo | None:
        """Wait for one request (or, rid = -1, for all); raises VBCError(VBC_ERR_TIMEOUT) on timeout."""
        info = RequestInfo()
        _check_server(load().vbc_server_wait(self._h, int(rid), float(timeout),
                                             ctypes.byref(info) if rid != -1 else None))
        return info if rid != -1 else None

    def info(self, rid: int) -> RequestInfo:
        info = RequestInfo()
        _check_server(load().vbc_server_info(self._h, int(rid), ctypes.byref(info)))
        return info

    def result(self, rid: int):
        """(positions [n,3] unwrapped, velocities [n,3], RequestInfo) of a finished request."""
        info = self.info(rid)
        pos = np.zeros((info.n, 3))
        vel = np.zeros((info.n, 3))
        _check_server(load().vbc_server_result(self._h, int(rid), ctypes.c_void_p(pos.ctypes.data),
                                               ctypes.c_void_p(vel.ctypes.data), ctypes.byref(info)))
        return pos, vel, info

    def close(self):
        if getattr(self, "_h", None):
            load().vbc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Systems advanced together (vbc_batch_*): their two-step graphs captured
    side by side into one CUDA graph; bitwise the same as stepping each alone.
    The systems must outlive the batch."""

    def __init__(self, systems):
        self._systems = list(systems)
        arr = (ctypes.c_void_p * len(self._systems))(*[s._h.value if isinstance(s._h, ctypes.c_void_p) else s._h
                                                       for s in self._systems])
        h = ctypes.c_void_p()
        _check(load().vbc_batch_create(arr, len(self._systems), ctypes.byref(h)))
        self._h = h

    def set_mode(self, mode: int = VBC_BATCH_FUSED, wait_limit: int = -1):
        """VBC_BATCH_FUSED (one cooperative launch per iteration for all systems) or
        VBC_BATCH_GRAPHS; wait_limit bounds each grid-wide wait (< 0: the default)."""
        _check(load().vbc_batch_set_mode(self._h, int(mode), int(wait_limit)))

    def fused_launches(self) -> int:
        return int(load().vbc_batch_fused_launches(self._h))

    def step(self, nsteps: int, dt: float, kT, gamma: float):
        """kT: one temperature for all systems, or one per system."""
        t = np.broadcast_to(np.asarray(kT, dtype=np.float64), (len(self._systems),)).copy()
        _check(load().vbc_batch_step(self._h, int(nsteps), dt, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     gamma))

    def close(self):
        if getattr(self, "_h", None):
            load().vbc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
