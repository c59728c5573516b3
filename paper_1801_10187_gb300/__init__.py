"""Python binding of libmpcd: the SRD step of multiparticle collision dynamics
(arXiv:1801.10187) on one NVIDIA GB300.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libmpcd.so`` (built in place by ``__graft_entry__.build()``).  There is
no CPU fallback; without the library or a CUDA device the calls raise.

    box = Box(n=(100, 100, 100), precision="mixed", seed=2)
    box.set_state(pos, vel)          # (N, 3) float64 arrays, input order kept
    box.step(1000)                   # asynchronous on the box's stream
    pos, vel, *_ = box.get_state()
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpcd.so")

MPCD_OK, MPCD_EINVAL, MPCD_ENOMEM, MPCD_ECUDA, MPCD_EDEVICE, MPCD_ESTATE = 0, -1, -2, -3, -4, -5
FP64, MIXED = 0, 1
SRD, AT = 0, 1  # collision rules (Eq. srd, Eq. at)


class MpcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmpcd error {code}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("precision", ctypes.c_int32),
        ("a", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("thermostat", ctypes.c_int32),
        ("sort_period", ctypes.c_int32),
        ("walls_z", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("body_force", ctypes.c_double * 3),
        ("virt_density", ctypes.c_double),
        ("chain_len", ctypes.c_int32),
        ("md_substeps", ctypes.c_int32),
        ("solute_mass", ctypes.c_double),
        ("bond_k", ctypes.c_double),
        ("bond_r0", ctypes.c_double),
        ("angular", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
        ("lj_epsilon", ctypes.c_double),
        ("lj_sigma", ctypes.c_double),
    ]


class _Obs(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_double * 3),
        ("KE", ctypes.c_double),
        ("T_kin", ctypes.c_double),
        ("T_cell_mean", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("n", ctypes.c_int64),
        ("occupied_cells", ctypes.c_int64),
        ("step", ctypes.c_uint64),
    ]


_lib_handle = None


def lib():
    """Load libmpcd.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    c_int, i32, i64, u64, vp = ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    dp = P(ctypes.c_double)
    L.mpcd_last_error.restype = ctypes.c_char_p
    L.mpcd_create.argtypes = [P(_Params), vp, P(vp)]
    L.mpcd_set_state.argtypes = [vp, i64, dp, dp, i64, dp, dp, u64]
    L.mpcd_set_state_device.argtypes = [vp, i64, vp, vp, u64]
    L.mpcd_set_state_thermal.argtypes = [vp, i64, u64, u64]
    L.mpcd_batch_add_thermal.argtypes = [vp, P(_Params), i64, u64, u64, P(i32)]
    L.mpcd_step.argtypes = [vp, i64]
    L.mpcd_get_state.argtypes = [vp, dp, dp, dp, dp, P(u64)]
    L.mpcd_get_state_device.argtypes = [vp, vp, vp]
    L.mpcd_observables.argtypes = [vp, P(_Obs)]
    L.mpcd_profile.argtypes = [vp, i32, dp]
    L.mpcd_last_cells.argtypes = [vp, P(i32), P(i32)]
    L.mpcd_profile_noalloc.argtypes = [vp, i32, dp]
    L.mpcd_phase_times.argtypes = [vp, i64, dp, i32, P(i32)]
    L.mpcd_phase_name.argtypes = [i32]
    L.mpcd_phase_name.restype = ctypes.c_char_p
    L.mpcd_num_cells.argtypes = [vp]
    L.mpcd_num_cells.restype = i64
    L.mpcd_destroy.argtypes = [vp]
    L.mpcd_destroy.restype = None
    L.mpcd_batch_create.argtypes = [i32, vp, i64, P(vp)]
    L.mpcd_box_footprint.argtypes = [P(_Params), i64]
    L.mpcd_box_footprint.restype = i64
    L.mpcd_batch_add.argtypes = [vp, P(_Params), i64, dp, dp, u64, P(i32)]
    L.mpcd_batch_step.argtypes = [vp, i64]
    L.mpcd_tune.argtypes = [vp, i64, P(i32), dp, P(i64), P(i32), P(i32)]
    L.mpcd_batch_tune.argtypes = [vp, i64, P(i32), dp, P(i64), P(i32), P(i32)]
    L.mpcd_batch_get_state.argtypes = [vp, i32, dp, dp, P(u64)]
    L.mpcd_batch_observables.argtypes = [vp, i32, P(_Obs)]
    L.mpcd_batch_remove.argtypes = [vp, i32]
    L.mpcd_batch_info.argtypes = [vp, P(i32), P(i64)]
    L.mpcd_batch_sync.argtypes = [vp]
    L.mpcd_batch_destroy.argtypes = [vp]
    L.mpcd_batch_destroy.restype = None
    for name in ("mpcd_create", "mpcd_set_state", "mpcd_set_state_device", "mpcd_step",
                 "mpcd_set_state_thermal", "mpcd_batch_add_thermal",
                 "mpcd_get_state", "mpcd_get_state_device", "mpcd_observables", "mpcd_profile",
                 "mpcd_last_cells", "mpcd_phase_times", "mpcd_profile_noalloc", "mpcd_batch_create", "mpcd_batch_add", "mpcd_batch_step",
                 "mpcd_batch_get_state", "mpcd_batch_observables", "mpcd_batch_remove",
                 "mpcd_batch_info", "mpcd_batch_sync", "mpcd_tune", "mpcd_batch_tune"):
        getattr(L, name).restype = c_int
    _lib_handle = L
    return L


def _check(rc):
    if rc != MPCD_OK:
        msg = lib().mpcd_last_error()
        raise MpcdError(rc, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _as3(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3))


def make_params(n=(10, 10, 10), dt=0.1, alpha_deg=130.0, kT=1.0, mass=1.0, seed=1,
                thermostat=False, sort_period=0, walls_z=False, body_force=(0.0, 0.0, 0.0),
                virt_density=0.0, precision="mixed", chain_len=0, md_substeps=0,
                solute_mass=1.0, bond_k=0.0, bond_r0=0.0, alpha=None,
                collision="srd", angular=False, lj_epsilon=0.0, lj_sigma=0.0) -> _Params:
    p = _Params()
    p.n[:] = [int(x) for x in n]
    p.precision = MIXED if precision in ("mixed", MIXED) else FP64
    p.a = 1.0
    p.dt = float(dt)
    p.alpha = float(alpha) if alpha is not None else math.radians(alpha_deg)
    p.kT = float(kT)
    p.mass = float(mass)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.thermostat = int(bool(thermostat))
    p.sort_period = int(sort_period)
    p.walls_z = int(bool(walls_z))
    p.body_force[:] = [float(x) for x in body_force]
    p.virt_density = float(virt_density)
    p.chain_len = int(chain_len)
    p.md_substeps = int(md_substeps)
    p.solute_mass = float(solute_mass)
    p.bond_k = float(bond_k)
    p.bond_r0 = float(bond_r0)
    p.collision = AT if collision in ("at", AT) else SRD
    p.angular = int(bool(angular))
    p.lj_epsilon = float(lj_epsilon)
    p.lj_sigma = float(lj_sigma)
    return p


def _tune(fn, handle, steps_per_candidate):
    bps, ms, taken = ctypes.c_int32(0), ctypes.c_double(0.0), ctypes.c_int64(0)
    chunk, cpw = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(fn(handle, int(steps_per_candidate), ctypes.byref(bps), ctypes.byref(ms),
              ctypes.byref(taken), ctypes.byref(chunk), ctypes.byref(cpw)))
    return bps.value, ms.value, taken.value, chunk.value, cpw.value


def _obs_dict(o: _Obs) -> dict:
    return {"P": np.array(o.P[:]), "KE": o.KE, "T_kin": o.T_kin, "T_cell_mean": o.T_cell_mean,
            "M": o.mass, "n": o.n, "occupied_cells": o.occupied_cells, "step": o.step}


class Box:
    """One SRD box on the current CUDA device (mpcd_create / mpcd_* calls)."""

    def __init__(self, stream=None, **kw):
        self.params = make_params(**kw)
        self.mixed = self.params.precision == MIXED
        self._ctx = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        _check(lib().mpcd_create(ctypes.byref(self.params), st, ctypes.byref(self._ctx)))
        self.n_solvent = 0
        self.n_solute = 0

    def close(self):
        if self._ctx:
            lib().mpcd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_cells(self) -> int:
        return int(lib().mpcd_num_cells(self._ctx))

    def set_state(self, pos, vel, solute_pos=None, solute_vel=None, step=0):
        pos, vel = _as3(pos), _as3(vel)
        sp = _as3(solute_pos) if solute_pos is not None else np.zeros((0, 3))
        sv = _as3(solute_vel) if solute_vel is not None else np.zeros((0, 3))
        self.n_solvent, self.n_solute = pos.shape[0], sp.shape[0]
        _check(lib().mpcd_set_state(self._ctx, pos.shape[0], _dptr(pos), _dptr(vel), sp.shape[0],
                                    _dptr(sp) if sp.size else None,
                                    _dptr(sv) if sv.size else None, int(step)))

    def set_state_device(self, pos, vel, step=0):
        """pos/vel: contiguous CUDA tensors (N, 3) of float32 (mixed) or float64."""
        self.n_solvent, self.n_solute = int(pos.shape[0]), 0
        _check(lib().mpcd_set_state_device(self._ctx, int(pos.shape[0]), ctypes.c_void_p(pos.data_ptr()),
                                           ctypes.c_void_p(vel.data_ptr()), int(step)))

    def set_state_thermal(self, n_solvent: int, init_seed: int, step=0):
        """Thermal initial state drawn on the device (uniform positions, Gaussian
        velocities of variance kT/m, zero total momentum)."""
        self.n_solvent, self.n_solute = int(n_solvent), 0
        _check(lib().mpcd_set_state_thermal(self._ctx, int(n_solvent), int(init_seed) & (2**64 - 1),
                                            int(step)))

    def step(self, nsteps=1):
        _check(lib().mpcd_step(self._ctx, int(nsteps)))

    def tune(self, steps_per_candidate=2):
        """Launch tuner (mpcd_tune): returns (blocks per SM or -1, ms per
        step of the choice, steps the simulation advanced, pass-2 chunk
        depth, cells per warp)."""
        return _tune(lib().mpcd_tune, self._ctx, steps_per_candidate)

    def get_state(self):
        pos = np.empty((self.n_solvent, 3))
        vel = np.empty((self.n_solvent, 3))
        sp = np.empty((self.n_solute, 3))
        sv = np.empty((self.n_solute, 3))
        st = ctypes.c_uint64(0)
        _check(lib().mpcd_get_state(self._ctx, _dptr(pos), _dptr(vel),
                                    _dptr(sp) if self.n_solute else None,
                                    _dptr(sv) if self.n_solute else None, ctypes.byref(st)))
        return pos, vel, sp, sv, st.value

    def get_state_device(self, pos, vel):
        _check(lib().mpcd_get_state_device(self._ctx, ctypes.c_void_p(pos.data_ptr()),
                                           ctypes.c_void_p(vel.data_ptr())))

    def observables(self) -> dict:
        o = _Obs()
        _check(lib().mpcd_observables(self._ctx, ctypes.byref(o)))
        return _obs_dict(o)

    def profile(self, nbins: int) -> np.ndarray:
        out = np.zeros(nbins)
        _check(lib().mpcd_profile(self._ctx, int(nbins), _dptr(out)))
        return out

    def phase_times(self, nsteps: int) -> dict:
        """Mean ms per step of each phase over nsteps eager (event-timed) steps."""
        ms = np.zeros(16)
        k = ctypes.c_int32(0)
        _check(lib().mpcd_phase_times(self._ctx, int(nsteps), _dptr(ms), 16, ctypes.byref(k)))
        return {lib().mpcd_phase_name(i).decode(): float(ms[i]) for i in range(k.value)}

    def profile_noalloc(self, nbins: int) -> np.ndarray:
        """mpcd_profile without any device allocation (static 4096-bin scratch)."""
        out = np.zeros(nbins)
        _check(lib().mpcd_profile_noalloc(self._ctx, int(nbins), _dptr(out)))
        return out

    def footprint_bytes(self) -> int:
        """Device bytes of this box's solvent arrays (mpcd_box_footprint)."""
        return int(lib().mpcd_box_footprint(ctypes.byref(self.params), int(self.n_solvent)))

    def last_cells(self):
        cells = np.empty(self.n_solvent + self.n_solute, dtype=np.int32)
        counts = np.empty(self.num_cells, dtype=np.int32)
        P32 = ctypes.POINTER(ctypes.c_int32)
        _check(lib().mpcd_last_cells(self._ctx, cells.ctypes.data_as(P32), counts.ctypes.data_as(P32)))
        return cells, counts


def box_footprint(n_solvent: int, **kw) -> int:
    p = make_params(**kw)
    return int(lib().mpcd_box_footprint(ctypes.byref(p), int(n_solvent)))


class Batch:
    """Independent boxes advanced together (mpcd_batch_* calls)."""

    def __init__(self, precision="mixed", stream=None, max_bytes=0):
        self._b = ctypes.c_void_p()
        prec = MIXED if precision in ("mixed", MIXED) else FP64
        self.precision = prec
        st = ctypes.c_void_p(stream) if stream else None
        _check(lib().mpcd_batch_create(prec, st, int(max_bytes), ctypes.byref(self._b)))
        self.sizes = {}

    def close(self):
        if self._b:
            lib().mpcd_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, pos, vel, step=0, **kw) -> int:
        kw.setdefault("precision", "mixed" if self.precision == MIXED else "fp64")
        p = make_params(**kw)
        pos, vel = _as3(pos), _as3(vel)
        slot = ctypes.c_int32(-1)
        _check(lib().mpcd_batch_add(self._b, ctypes.byref(p), pos.shape[0], _dptr(pos), _dptr(vel),
                                    int(step), ctypes.byref(slot)))
        self.sizes[slot.value] = pos.shape[0]
        return slot.value

    def add_thermal(self, n_solvent: int, init_seed: int, step=0, **kw) -> int:
        """Admit a box whose thermal initial state is drawn on the device."""
        kw.setdefault("precision", "mixed" if self.precision == MIXED else "fp64")
        p = make_params(**kw)
        slot = ctypes.c_int32(-1)
        _check(lib().mpcd_batch_add_thermal(self._b, ctypes.byref(p), int(n_solvent),
                                            int(init_seed) & (2**64 - 1), int(step),
                                            ctypes.byref(slot)))
        self.sizes[slot.value] = int(n_solvent)
        return slot.value

    def step(self, nsteps=1):
        _check(lib().mpcd_batch_step(self._b, int(nsteps)))

    def tune(self, steps_per_candidate=2):
        """mpcd_batch_tune: (blocks per SM or -1, ms per step, steps taken,
        pass-2 chunk depth, cells per warp)."""
        return _tune(lib().mpcd_batch_tune, self._b, steps_per_candidate)

    def get_state(self, slot: int):
        n = self.sizes[slot]
        pos, vel = np.empty((n, 3)), np.empty((n, 3))
        st = ctypes.c_uint64(0)
        _check(lib().mpcd_batch_get_state(self._b, int(slot), _dptr(pos), _dptr(vel), ctypes.byref(st)))
        return pos, vel, st.value

    def observables(self, slot: int) -> dict:
        o = _Obs()
        _check(lib().mpcd_batch_observables(self._b, int(slot), ctypes.byref(o)))
        return _obs_dict(o)

    def remove(self, slot: int):
        _check(lib().mpcd_batch_remove(self._b, int(slot)))
        self.sizes.pop(slot, None)

    def sync(self):
        _check(lib().mpcd_batch_sync(self._b))

    def info(self):
        n = ctypes.c_int32(0)
        b = ctypes.c_int64(0)
        _check(lib().mpcd_batch_info(self._b, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value
