"""ctypes front end of the plain CPU oracle (``mpcd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module.  The GPU product package
never imports it, and it imports nothing from the product.

The oracle follows arXiv:1801.10187, Sec. 2 (Eqs. stream, srd, thermo) and
Sec. 3.4-3.6 (binning with a random grid shift, cell properties, rotation and
thermostat), one straight loop per stage.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpcd_oracle.c")
_LIB = os.path.join(_HERE, "libmpcd_oracle.so")

FP64 = 0
MIXED = 1
# FP64 model of one mixed-model step: the float state streams in float (as in
# MIXED); binning, sums, draws, xi and the collision are FP64
FP64_FSTREAM = 2

PURPOSE_SHIFT = 0x53484654
PURPOSE_ROT = 0x524F5441
PURPOSE_THERMO = 0x54484D4F
PURPOSE_VIRT = 0x56495254
PURPOSE_AT = 0x414E4452

SRD = 0  # collision rules
AT = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) into this folder."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("dt", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("thermostat", ctypes.c_int32),
        ("walls_z", ctypes.c_int32),
        ("g", ctypes.c_double * 3),
        ("virt_density", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("chain_len", ctypes.c_int32),
        ("md_substeps", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("solute_mass", ctypes.c_double),
        ("bond_k", ctypes.c_double),
        ("bond_r0", ctypes.c_double),
        ("angular", ctypes.c_int32),
        ("pad2_", ctypes.c_int32),
        ("lj_epsilon", ctypes.c_double),
        ("lj_sigma", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i32, i64, u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        _lib.oracle_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32),
                                              P(ctypes.c_uint32)]
        _lib.oracle_shift.argtypes = [u64, u64, P(d)]
        _lib.oracle_cos_sin_turn_f.argtypes = [ctypes.c_uint32, P(ctypes.c_float), P(ctypes.c_float)]
        _lib.oracle_log_f.argtypes = [ctypes.c_float]
        _lib.oracle_log_f.restype = ctypes.c_float
        _lib.oracle_neg_log1m_f.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        _lib.oracle_neg_log1m_f.restype = ctypes.c_float
        _lib.oracle_xi_mixed.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.oracle_xi_mixed.restype = ctypes.c_float
        _lib.oracle_axis.argtypes = [u64, u64, ctypes.c_uint32, i32, P(d)]
        _lib.oracle_gamma_draw.argtypes = [u64, u64, ctypes.c_uint32, i32, d, i32, P(d)]
        _lib.oracle_gamma_draw.restype = i32
        _lib.oracle_at_draw.argtypes = [u64, u64, ctypes.c_uint32, i32, d, i32, P(d)]
        _lib.oracle_solute_forces.argtypes = [P(_Params), i64, P(d), P(d)]
        _lib.oracle_solute_energy.argtypes = [P(_Params), i64, P(d)]
        _lib.oracle_solute_energy.restype = d
        _lib.oracle_step.argtypes = [P(_Params), i64, P(d), P(d), i64, P(d), P(d), P(u64), i64,
                                     P(i32), P(i32)]
        _lib.oracle_step.restype = i32
        _lib.oracle_num_cells.argtypes = [P(_Params)]
        _lib.oracle_num_cells.restype = i64
        _lib.oracle_observables.argtypes = [P(_Params), i64, P(d), P(d), i64, P(d), P(d), P(d)]
        _lib.oracle_observables.restype = i32
        _lib.oracle_profile.argtypes = [P(_Params), i64, P(d), P(d), i32, P(d)]
        _lib.oracle_profile.restype = i32
    return _lib


@dataclass
class Params:
    """SRD parameters in the paper's notation (cell edge a = 1)."""
    n: tuple = (10, 10, 10)
    dt: float = 0.1
    alpha_deg: float = 130.0
    kT: float = 1.0
    mass: float = 1.0
    seed: int = 1
    thermostat: bool = False
    walls_z: bool = False
    g: tuple = (0.0, 0.0, 0.0)
    virt_density: float = 0.0
    precision: int = FP64
    chain_len: int = 0
    md_substeps: int = 0
    solute_mass: float = 1.0
    bond_k: float = 0.0
    bond_r0: float = 0.0
    collision: int = SRD
    angular: bool = False
    lj_epsilon: float = 0.0
    lj_sigma: float = 0.0

    def c(self) -> _Params:
        p = _Params()
        p.n[:] = [int(x) for x in self.n]
        p.dt = self.dt
        p.alpha = math.radians(self.alpha_deg)
        p.kT = self.kT
        p.mass = self.mass
        p.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        p.thermostat = int(bool(self.thermostat))
        p.walls_z = int(bool(self.walls_z))
        p.g[:] = [float(x) for x in self.g]
        p.virt_density = self.virt_density
        p.precision = int(self.precision)
        p.chain_len = int(self.chain_len)
        p.md_substeps = int(self.md_substeps)
        p.solute_mass = self.solute_mass
        p.bond_k = self.bond_k
        p.bond_r0 = self.bond_r0
        p.collision = int(self.collision)
        p.angular = int(bool(self.angular))
        p.lj_epsilon = float(self.lj_epsilon)
        p.lj_sigma = float(self.lj_sigma)
        return p


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def cos_sin_turn_f(w: int):
    """The mixed model's float (cos, sin) of 2 pi w / 2^32."""
    c, s = ctypes.c_float(), ctypes.c_float()
    _load().oracle_cos_sin_turn_f(int(w) & 0xFFFFFFFF, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def log_f(x: float) -> float:
    """The mixed model's float natural logarithm."""
    return _load().oracle_log_f(float(np.float32(x)))


def xi_mixed(ehat: float, ek: float) -> float:
    """The mixed model's thermostat factor sqrt(ehat / ek), float."""
    return _load().oracle_xi_mixed(float(ehat), float(ek))


def neg_log1m_f(hi: int, lo: int) -> float:
    """The mixed model's float -ln(1 - U) for the 53-bit uniform U with words
    (hi, lo): the squared Box-Muller radius over two."""
    return _load().oracle_neg_log1m_f(int(hi) & 0xFFFFFFFF, int(lo) & 0xFFFFFFFF)


def shift(seed: int, t: int) -> np.ndarray:
    s = np.zeros(3)
    _load().oracle_shift(seed, t, _dptr(s))
    return s


def axis(seed: int, t: int, cell: int, precision: int = FP64) -> np.ndarray:
    nv = np.zeros(3)
    _load().oracle_axis(seed, t, cell, precision, _dptr(nv))
    return nv


def gamma_draw(seed: int, t: int, cell: int, nc: int, kT: float, precision: int = FP64):
    e = ctypes.c_double(0.0)
    st = _load().oracle_gamma_draw(seed, t, cell, nc, kT, precision, ctypes.byref(e))
    if st != 0:
        raise RuntimeError(f"oracle_gamma_draw status {st}")
    return e.value


def at_draw(seed: int, t: int, tag: int, kind: int, sigma: float, precision: int = FP64):
    """Random velocity of particle ``tag`` (kind 0 solvent, 1 bead) at step t
    for the Andersen-thermostat rule (Sec. 3.7)."""
    dv = np.zeros(3)
    _load().oracle_at_draw(seed, t, tag, kind, sigma, precision, _dptr(dv))
    return dv


def solute_forces(params: Params, r: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    F = np.zeros_like(r)
    p = params.c()
    _load().oracle_solute_forces(ctypes.byref(p), r.shape[0], _dptr(r), _dptr(F))
    return F


def solute_energy(params: Params, r: np.ndarray) -> float:
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    p = params.c()
    return float(_load().oracle_solute_energy(ctypes.byref(p), r.shape[0], _dptr(r)))


def num_cells(params: Params) -> int:
    p = params.c()
    return int(_load().oracle_num_cells(ctypes.byref(p)))


@dataclass
class State:
    pos: np.ndarray
    vel: np.ndarray
    spos: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    svel: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    step: int = 0

    def copy(self) -> "State":
        return State(self.pos.copy(), self.vel.copy(), self.spos.copy(), self.svel.copy(),
                     self.step)


def step(params: Params, state: State, nsteps: int = 1, want_cells: bool = False):
    """Advance ``state`` in place by ``nsteps`` SRD steps.

    Returns (cell_of_particle, count_per_cell) of the last step when
    ``want_cells``; otherwise None.
    """
    lib = _load()
    p = params.c()
    for name in ("pos", "vel", "spos", "svel"):
        a = getattr(state, name)
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)
        setattr(state, name, a)
    n, nb = state.pos.shape[0], state.spos.shape[0]
    st = ctypes.c_uint64(state.step)
    cells = counts = None
    cptr = kptr = None
    if want_cells:
        cells = np.zeros(n + nb, dtype=np.int32)
        counts = np.zeros(num_cells(params), dtype=np.int32)
        cptr = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        kptr = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    rc = lib.oracle_step(ctypes.byref(p), n, _dptr(state.pos), _dptr(state.vel), nb,
                         _dptr(state.spos), _dptr(state.svel), ctypes.byref(st), nsteps,
                         cptr, kptr)
    state.step = st.value
    if rc != 0:
        raise RuntimeError(f"oracle_step returned {rc}")
    return (cells, counts) if want_cells else None


def observables(params: Params, state: State) -> dict:
    lib = _load()
    p = params.c()
    out = np.zeros(8)
    pos = np.ascontiguousarray(state.pos, dtype=np.float64)
    vel = np.ascontiguousarray(state.vel, dtype=np.float64)
    spos = np.ascontiguousarray(state.spos, dtype=np.float64).reshape(-1, 3)
    svel = np.ascontiguousarray(state.svel, dtype=np.float64).reshape(-1, 3)
    rc = lib.oracle_observables(ctypes.byref(p), pos.shape[0], _dptr(pos), _dptr(vel),
                                spos.shape[0], _dptr(spos), _dptr(svel), _dptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle_observables returned {rc}")
    return {"P": out[0:3].copy(), "KE": out[3], "T_kin": out[4], "T_cell_mean": out[5],
            "occupied_cells": int(out[6]), "M": out[7]}


def profile(params: Params, state: State, nbins: int) -> np.ndarray:
    lib = _load()
    p = params.c()
    out = np.zeros(nbins)
    pos = np.ascontiguousarray(state.pos, dtype=np.float64)
    vel = np.ascontiguousarray(state.vel, dtype=np.float64)
    rc = lib.oracle_profile(ctypes.byref(p), pos.shape[0], _dptr(pos), _dptr(vel), nbins,
                            _dptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle_profile returned {rc}")
    return out
