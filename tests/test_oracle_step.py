"""Pins of the oracle's SRD step (CPU only), each against something the paper or
the mathematics fixes, not against the oracle itself:

* alpha = 0 makes the collision the identity: the trajectory is ballistic and
  equals the closed form r0 + t v dt (mod L)            (Sec. 2, Eq. stream)
* binning equals an independent numpy floor/mod binning (Sec. 3.4)
* each particle's velocity relative to an independently computed cell mean is
  rotated by exactly alpha about the drawn axis, right-handed; cells keep
  momentum and, without thermostat, kinetic energy      (Sec. 2, Eq. srd)
* thermostat: cell energies follow the canonical moments (Sec. 2, Eq. thermo)
* relaxation to a Maxwell-Boltzmann distribution       (Sec. 2)
* two-bead harmonic chain: closed-form oscillation     (Sec. 2, solute MD)
* single-particle cells are unchanged, results do not depend on particle order,
  N steps at once equal N/2 + N/2.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1801_10187_gb300 import inputs


def _state(n=(10, 10, 10), rho=5, seed=1, mixed=False, kT=1.0):
    s = inputs.solvent(n, rho, kT=kT, seed=seed, mixed=mixed)
    return oracle.State(s.pos, s.vel)


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_alpha_zero_is_ballistic_closed_form(precision):
    p = oracle.Params(n=(6, 7, 8), alpha_deg=0.0, precision=precision, seed=3)
    st = _state(p.n, 5, seed=3, mixed=precision == oracle.MIXED)
    r0, v0 = st.pos.copy(), st.vel.copy()
    T = 50
    oracle.step(p, st, T)
    L = np.array(p.n, dtype=float)
    want = np.mod(r0 + T * p.dt * v0, L)
    d = np.abs(st.pos - want)
    d = np.minimum(d, L - d)  # periodic distance
    tol = 1e-12 if precision == oracle.FP64 else 5e-5
    assert d.max() < tol
    vtol = 1e-14 if precision == oracle.FP64 else 2e-6
    assert np.max(np.abs(st.vel - v0)) < vtol * T


@pytest.mark.parametrize("n", [(2, 2, 2), (3, 4, 5)])
@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_binning_matches_independent_floor(n, precision):
    p = oracle.Params(n=n, precision=precision, seed=17)
    st = _state(n, 7, seed=17, mixed=precision == oracle.MIXED)
    t = 5
    st.step = t
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    s = oracle.shift(p.seed, t)
    ijk = np.floor(st.pos - s).astype(np.int64) % np.array(n)
    want = ijk[:, 0] + n[0] * (ijk[:, 1] + n[1] * ijk[:, 2])
    assert np.array_equal(cells, want)
    assert np.array_equal(counts, np.bincount(want, minlength=int(np.prod(n))))


def test_binning_walls_layers():
    n = (4, 3, 5)
    p = oracle.Params(n=n, walls_z=True, thermostat=True, virt_density=5, seed=8)
    st = _state(n, 5, seed=8)
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    s = oracle.shift(p.seed, 0)
    ix = np.floor(st.pos[:, 0] - s[0]).astype(np.int64) % n[0]
    iy = np.floor(st.pos[:, 1] - s[1]).astype(np.int64) % n[1]
    iz = np.floor(st.pos[:, 2] - s[2]).astype(np.int64) + 1
    assert iz.min() >= 0 and iz.max() <= n[2] + 1
    assert np.array_equal(cells, ix + n[0] * (iy + n[1] * iz))
    assert np.all((st.pos[:, 2] >= 0) & (st.pos[:, 2] < n[2]))
    assert len(counts) == n[0] * n[1] * (n[2] + 2)


def _rotation_checks(vbefore, vafter, cells, masses, alpha, seed, t, precision, tol):
    """Independent geometric check of Eq. (srd) for every particle."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    for c in np.unique(cells):
        idx = np.nonzero(cells == c)[0]
        m = masses[idx][:, None]
        u = (m * vbefore[idx]).sum(0) / m.sum()
        u2 = (m * vafter[idx]).sum(0) / m.sum()
        scale = max(1.0, np.abs(vbefore[idx]).max())
        assert np.allclose(u, u2, atol=tol * scale, rtol=0)  # momentum kept per cell
        nax = oracle.axis(seed, t, int(c), precision)
        for i in range(len(idx)):
            d = vbefore[idx[i]] - u
            dp = vafter[idx[i]] - u
            ds = tol * max(1.0, np.linalg.norm(d))
            assert abs(np.linalg.norm(dp) - np.linalg.norm(d)) < ds
            assert abs(nax @ dp - nax @ d) < ds
            dperp = d - (nax @ d) * nax
            dpperp = dp - (nax @ dp) * nax
            q = dperp @ dperp
            if q > 1e-6:
                assert abs(dperp @ dpperp - ca * q) < ds * max(1.0, math.sqrt(q))
                assert abs(np.cross(dperp, dpperp) @ nax - sa * q) < ds * max(1.0, math.sqrt(q))


@pytest.mark.parametrize("precision,tol", [(oracle.FP64, 1e-12), (oracle.MIXED, 2e-6)])
def test_collision_is_rotation_by_alpha_2x2x2(precision, tol):
    n = (2, 2, 2)
    p = oracle.Params(n=n, precision=precision, seed=29, alpha_deg=130.0)
    st = _state(n, 6, seed=29, mixed=precision == oracle.MIXED)
    st.step = 11
    vb = st.vel.copy()
    cells, _ = oracle.step(p, st, 1, want_cells=True)
    _rotation_checks(vb, st.vel, cells, np.ones(len(vb)), math.radians(130.0), p.seed, 11,
                     precision, tol)


def test_collision_with_beads_is_mass_weighted_rotation():
    """Beads (mass 5, single-bead chains without bonds) join the collision; the
    cell mean must be mass weighted for the geometric checks to hold."""
    n = (2, 2, 2)
    p = oracle.Params(n=n, seed=31, chain_len=1, md_substeps=2, solute_mass=5.0,
                      bond_k=0.0, bond_r0=0.5)
    st = _state(n, 4, seed=31)
    rng = np.random.default_rng(5)
    st.spos = rng.random((6, 3)) * 2.0
    st.svel = rng.standard_normal((6, 3)) * math.sqrt(1 / 5)
    vb = np.vstack([st.vel, st.svel])
    cells, _ = oracle.step(p, st, 1, want_cells=True)
    va = np.vstack([st.vel, st.svel])
    masses = np.r_[np.ones(len(st.vel)), 5.0 * np.ones(6)]
    _rotation_checks(vb, va, cells, masses, math.radians(130.0), p.seed, 0, oracle.FP64, 1e-12)
    # unequal masses matter: the unweighted mean would break the checks
    with pytest.raises(AssertionError):
        _rotation_checks(vb, va, cells, np.ones(len(vb)), math.radians(130.0), p.seed, 0,
                         oracle.FP64, 1e-12)


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_cell_momentum_and_energy_conserved(precision):
    p = oracle.Params(n=(10, 10, 10), precision=precision, seed=2)
    st = _state(p.n, 5, seed=2, mixed=precision == oracle.MIXED)
    vb = st.vel.copy()
    cells, _ = oracle.step(p, st, 1, want_cells=True)
    C = oracle.num_cells(p)
    Pb = np.stack([np.bincount(cells, vb[:, k], C) for k in range(3)], 1)
    Pa = np.stack([np.bincount(cells, st.vel[:, k], C) for k in range(3)], 1)
    Kb = np.bincount(cells, 0.5 * (vb**2).sum(1), C)
    Ka = np.bincount(cells, 0.5 * (st.vel**2).sum(1), C)
    denom = np.abs(vb).sum()
    rel = 1e-12 if precision == oracle.FP64 else 3e-6
    # "relative" = |change of the total| / sum m|v|, per cell and in total
    assert np.abs(Pa - Pb).sum() / denom < rel
    assert np.abs(Ka - Kb).sum() / Kb.sum() < (1e-12 if precision == oracle.FP64 else 3e-6)


def test_thermostat_cell_energy_moments():
    """After one thermostatted collision from a hot state (kT 4), each cell's
    energy about its centre of mass has mean 3/2 (Nc-1) kT and variance
    3/2 (Nc-1) kT^2 for the target kT = 1 (Gamma moments)."""
    p = oracle.Params(n=(24, 24, 24), thermostat=True, seed=44)
    st = _state(p.n, 5, seed=44, kT=4.0)
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    C = oracle.num_cells(p)
    P = np.stack([np.bincount(cells, st.vel[:, k], C) for k in range(3)], 1)
    K = np.bincount(cells, 0.5 * (st.vel**2).sum(1), C)
    Ek = K - 0.5 * (P**2).sum(1) / np.maximum(counts, 1)
    for nc in (3, 5, 7):
        e = Ek[counts == nc]
        k = 1.5 * (nc - 1)
        assert abs(e.mean() - k) < 5 * math.sqrt(k / len(e))
        assert abs(e.var() / k - 1.0) < 0.25


def test_relaxes_to_maxwell_boltzmann():
    """SRD gives the Maxwell-Boltzmann velocity distribution: start from uniform
    velocity components of the right variance; after 100 collisions each
    component is Gaussian at the (conserved) temperature."""
    n = (12, 12, 12)
    rng = np.random.default_rng(7)
    N = 10 * 12**3
    pos = rng.random((N, 3)) * 12.0
    vel = (rng.random((N, 3)) * 2 - 1) * math.sqrt(3.0)
    vel -= vel.mean(0)
    st = oracle.State(pos, vel)
    p = oracle.Params(n=n, seed=70)
    assert stats.kstest(st.vel[:, 0] / st.vel[:, 0].std(), "norm").pvalue < 1e-6
    oracle.step(p, st, 100)
    kT = (st.vel**2).sum() / (3 * N)
    for k in range(3):
        assert stats.kstest(st.vel[:, k] / math.sqrt(kT), "norm").pvalue > 1e-3


def test_two_bead_chain_is_a_harmonic_oscillator():
    """Two beads of mass M joined by U = k/2 (r - r0)^2, no solvent, alpha = 0:
    the bond length oscillates as r0 + A cos(omega t), omega = sqrt(2k/M)."""
    M, k, r0, A = 5.0, 1000.0, 0.5, 0.05
    p = oracle.Params(n=(4, 4, 4), alpha_deg=0.0, chain_len=2, md_substeps=50,
                      solute_mass=M, bond_k=k, bond_r0=r0, seed=1)
    st = oracle.State(np.zeros((0, 3)), np.zeros((0, 3)))
    st.spos = np.array([[1.0, 2.0, 2.0], [1.0 + r0 + A, 2.0, 2.0]])
    st.svel = np.zeros((2, 3))
    omega = math.sqrt(2 * k / M)
    for it in range(1, 21):
        oracle.step(p, st, 1)
        r = st.spos[1, 0] - st.spos[0, 0]
        want = r0 + A * math.cos(omega * it * p.dt)
        assert abs(r - want) < 2e-3 * A * it  # velocity-Verlet phase error O(h^2)
    # momentum of the pair stays zero
    assert np.abs(st.svel.sum(0)).max() < 1e-12


def test_single_particle_cell_unchanged():
    p = oracle.Params(n=(5, 5, 5), seed=12)
    rng = np.random.default_rng(1)
    # one particle per cell, each at the centre so shifts never move it out
    idx = np.array([[i, j, k] for i in range(5) for j in range(5) for k in range(5)], float)
    st = oracle.State(idx + 0.5, rng.standard_normal((125, 3)) * 1e-3)
    v0 = st.vel.copy()
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    occupied = counts[cells]
    lone = occupied == 1
    assert lone.sum() > 20
    assert np.max(np.abs(st.vel[lone] - v0[lone])) < 1e-18


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_particle_order_does_not_matter(precision):
    p = oracle.Params(n=(6, 6, 6), precision=precision, thermostat=True, seed=90)
    a = _state(p.n, 5, seed=90, mixed=precision == oracle.MIXED)
    perm = np.random.default_rng(3).permutation(len(a.pos))
    b = oracle.State(a.pos[perm].copy(), a.vel[perm].copy())
    oracle.step(p, a, 3)
    oracle.step(p, b, 3)
    if precision == oracle.MIXED:
        # fixed-point sums are order independent: bit-identical
        assert np.array_equal(a.vel[perm], b.vel)
        assert np.array_equal(a.pos[perm], b.pos)
    else:
        assert np.max(np.abs(a.vel[perm] - b.vel)) < 1e-12


def test_resume_is_bit_exact():
    p = oracle.Params(n=(5, 6, 7), thermostat=True, seed=5)
    a = _state(p.n, 5, seed=5)
    b = a.copy()
    oracle.step(p, a, 10)
    oracle.step(p, b, 4)
    oracle.step(p, b, 6)
    assert a.step == b.step == 10
    assert np.array_equal(a.vel, b.vel) and np.array_equal(a.pos, b.pos)


def test_observables_initial_state():
    p = oracle.Params(n=(10, 10, 10))
    st = _state(p.n, 10, seed=4)
    ob = oracle.observables(p, st)
    assert np.abs(ob["P"]).max() < 1e-10
    assert abs(ob["T_kin"] - 1.0) < 0.03
    assert abs(ob["T_cell_mean"] - 1.0) < 0.05
    assert ob["M"] == 10000
