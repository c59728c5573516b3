"""Pins of the oracle's random streams (CPU only).

* Philox4x32-10 is checked bit for bit against NVIDIA cuRAND's own Philox4_32_10
  host generator, called through its public API (an implementation that shares
  nothing with the oracle).
* The grid shift, the rotation axis (Sec. 3.6, cylindrical projection) and the
  Maxwell-Boltzmann energy draw (Sec. 2 Eq. thermo, Sec. 3.6 Marsaglia-Tsang)
  are checked against the distributions the paper fixes.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

_CURAND_CANDIDATES = ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so",
                      "libcurand.so.10"]


def _curand():
    for name in _CURAND_CANDIDATES:
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    found = ctypes.util.find_library("curand")
    if found:
        return ctypes.CDLL(found)
    pytest.skip("libcurand not available")


def _curand_host_philox(lib, seed, offset, count):
    gen = ctypes.c_void_p()
    PHILOX4_32_10 = 161  # curandRngType_t value of CURAND_RNG_PSEUDO_PHILOX4_32_10
    st = lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10)
    if st != 0:
        pytest.skip(f"curandCreateGeneratorHost status {st}")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xDEADBEEFCAFEF00D, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox emits block b from counter (b // 65536, 0, b % 65536, 0)
    under key (seed_lo, seed_hi); its output must equal the oracle's Philox."""
    lib = _curand()
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for hi_block, lo_block in [(0, 0), (0, 1), (0, 7), (0, 4095), (1, 0), (3, 12345)]:
        block = hi_block * 65536 + lo_block
        got = _curand_host_philox(lib, seed, 4 * block, 8)
        want0 = oracle.philox([hi_block, 0, lo_block, 0], key)
        want1 = oracle.philox([hi_block, 0, lo_block + 1, 0], key)
        assert [int(x) for x in got[:4]] == want0
        assert [int(x) for x in got[4:]] == want1


def test_philox_words_uniform_and_uncorrelated():
    words = np.array([oracle.philox([c, 0, 7, 0], [11, 22]) for c in range(4000)],
                     dtype=np.float64)
    u = words.ravel() / 2.0**32
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # neighbouring words and neighbouring counters are uncorrelated
    assert abs(np.corrcoef(words[:, 0], words[:, 1])[0, 1]) < 0.06
    assert abs(np.corrcoef(words[:-1, 0], words[1:, 0])[0, 1]) < 0.06


def test_grid_shift_uniform_half_open_and_quantised():
    s = np.array([oracle.shift(5, t) for t in range(4000)])
    assert s.min() >= -0.5 and s.max() < 0.5
    assert np.all(s * 2.0**32 == np.round(s * 2.0**32))
    for k in range(3):
        assert stats.kstest(s[:, k] + 0.5, "uniform").pvalue > 1e-4
    # distinct seeds give distinct shifts
    assert not np.allclose(oracle.shift(5, 3), oracle.shift(6, 3))


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_axis_uniform_on_unit_sphere(precision):
    n = np.array([oracle.axis(9, t, c, precision) for t in range(40) for c in range(200)])
    norms = np.linalg.norm(n, axis=1)
    tol = 1e-15 if precision == oracle.FP64 else 3e-7
    assert np.max(np.abs(norms - 1.0)) < 4 * tol
    m = len(n)
    assert np.all(np.abs(n.mean(axis=0)) < 5 * math.sqrt(1 / 3 / m))
    assert np.all(np.abs((n**2).mean(axis=0) - 1 / 3) < 5 * math.sqrt(4 / 45 / m))
    # Archimedes: z uniform in [-1, 1]; azimuth uniform
    assert stats.kstest((n[:, 2] + 1) / 2, "uniform").pvalue > 1e-4
    phi = np.mod(np.arctan2(n[:, 1], n[:, 0]), 2 * np.pi) / (2 * np.pi)
    assert stats.kstest(phi, "uniform").pvalue > 1e-4


def test_mixed_axis_follows_fp64_axis():
    for t in range(5):
        for c in range(50):
            a = oracle.axis(3, t, c, oracle.FP64)
            b = oracle.axis(3, t, c, oracle.MIXED)
            assert np.max(np.abs(a - b)) < 1e-6


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
@pytest.mark.parametrize("nc", [2, 3, 6, 11, 40])
def test_thermostat_energy_is_gamma_distributed(nc, precision):
    """E^ ~ Gamma(3(Nc-1)/2, kT): the MB distribution of the kinetic energy of
    Nc particles about their centre of mass (3(Nc-1) quadratic terms)."""
    kT = 1.7
    e = np.array([oracle.gamma_draw(21, t, c, nc, kT, precision)
                  for t in range(20) for c in range(150)])
    shape = 1.5 * (nc - 1)
    assert stats.kstest(e, "gamma", args=(shape, 0.0, kT)).pvalue > 1e-4
    m = len(e)
    assert abs(e.mean() - shape * kT) < 5 * math.sqrt(shape) * kT / math.sqrt(m)
    assert abs(e.var() / (shape * kT**2) - 1.0) < 0.12


def _ulp32(x):
    x = np.abs(np.asarray(x, dtype=np.float32))
    return np.spacing(np.maximum(x, np.float32(2.0**-126))).astype(np.float64)


def test_float_turn_cos_sin_within_two_ulp():
    """The mixed model's own cos/sin of 2 pi w / 2^32 (octant reduction and
    Taylor series) against numpy's double-precision cos/sin."""
    rng = np.random.default_rng(1)
    words = np.concatenate([rng.integers(0, 2**32, 20000, dtype=np.uint64),
                            np.array([0, 1, 2**29 - 1, 2**29, 2**29 + 1, 2**30, 2**31,
                                      3 * 2**30, 2**32 - 1], dtype=np.uint64)])
    got = np.array([oracle.cos_sin_turn_f(int(w)) for w in words], dtype=np.float64)
    ang = 2 * np.pi * words.astype(np.float64) / 2.0**32
    ref = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    err = np.abs(got - ref)
    # absolute error in units of the float spacing near 1 (the values are <= 1)
    assert err.max() < 2.0 * 2.0**-24
    # exact quadrant points
    assert oracle.cos_sin_turn_f(0) == (1.0, 0.0)
    c, s = oracle.cos_sin_turn_f(2**30)
    assert abs(c) < 1e-7 and s == 1.0


def test_float_log_within_three_ulp():
    rng = np.random.default_rng(2)
    xs = np.concatenate([np.exp(rng.uniform(-85, 85, 20000)), rng.uniform(0.5, 2.0, 20000),
                         [1.0, 2.0, 0.5, 2.0**-32, 1 - 2.0**-24, 1.41421354, 1.41421365]])
    xs = xs.astype(np.float32)
    got = np.array([oracle.log_f(x) for x in xs], dtype=np.float64)
    ref = np.log(xs.astype(np.float64))
    ulps = np.abs(got - ref) / _ulp32(ref)
    assert ulps.max() <= 3.0
    assert oracle.log_f(1.0) == 0.0
    assert oracle.log_f(0.0) == -np.inf
