"""Pins of the oracle's Andersen-thermostat collision rule (CPU only).

Eq. (at), Sec. 2, and Sec. 3.7: every member of a cell draws a Gaussian
random velocity dv_i of variance kT/m_i per component, and
v_i <- u + dv_i - dbar, where dbar = sum m_j dv_j / sum m_j is the cell's
mass-weighted mean random velocity (the paper's (1/Nc) sum dv_j when all
masses are equal).  What fixes the oracle here, independently of its code:
1. the draw: Gaussian components of the stated variance, uncorrelated, keyed
   by (seed, step, tag, kind); the mixed and FP64 draws are the same numbers
   up to float rounding;
2. momentum of every cell conserved, and a cell's u unchanged;
3. starting from a cold flow (all relative velocities zero), the cell's
   kinetic energy about u after one collision is kT/2 times a chi-square
   variable with 3(Nc - 1) degrees of freedom, for any masses: sqrt(m_i) dv_i
   are i.i.d. N(0, kT) and removing the mass-weighted mean is a projection of
   rank Nc - 1 in each component;
4. the transport coefficient: a transverse shear wave decays at the rate
   nu k^2 set by the closed-form MPC-AT viscosity.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from paper_1801_10187_gb300 import inputs

scipy_stats = pytest.importorskip("scipy.stats")


def eta_at(rho, dt, kT=1.0, m=1.0, a=1.0):
    """Closed-form MPC-AT viscosity in 3D with random grid shift (Gompper,
    Ihle, Kroll & Winkler 2009, the review the paper cites for MPCD).
    Kinetic part: rho kT dt / a^3 (rho / (rho - 1 + e^-rho) - 1/2).
    Collisional part: m (rho - 1 + e^-rho) / (12 a dt); it follows from the
    mean momentum change m (u - v_i) of Eq. (at) and the variance a^2 / 12 of
    a uniform coordinate inside a cell (the SRD analogue carries the extra
    factor (2/3)(1 - cos alpha), giving the familiar 1/18)."""
    f = rho - 1.0 + math.exp(-rho)
    return rho * kT * dt / a**3 * (rho / f - 0.5) + m * f / (12.0 * a * dt)


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_at_draw_is_gaussian(precision):
    sigma, N, seed, t = 1.7, 6000, 9, 123
    dv = np.array([oracle.at_draw(seed, t, i, 0, sigma, precision) for i in range(N)])
    z = dv / sigma
    tol_mean = 4.0 / math.sqrt(N)
    assert np.all(np.abs(z.mean(axis=0)) < tol_mean)
    assert np.all(np.abs(z.var(axis=0) - 1.0) < 4.0 * math.sqrt(2.0 / N))
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < tol_mean)
    for k in range(3):
        assert scipy_stats.kstest(z[:, k], "norm").pvalue > 1e-3
    # fourth moment of a normal variable is 3
    assert np.all(np.abs((z**4).mean(axis=0) - 3.0) < 0.35)


def test_at_draw_keys():
    a = oracle.at_draw(5, 7, 11, 0, 1.0)
    assert np.array_equal(a, oracle.at_draw(5, 7, 11, 0, 1.0))  # deterministic
    for other in (oracle.at_draw(5, 8, 11, 0, 1.0), oracle.at_draw(5, 7, 12, 0, 1.0),
                  oracle.at_draw(5, 7, 11, 1, 1.0), oracle.at_draw(6, 7, 11, 0, 1.0)):
        assert np.all(a != other)
    assert np.allclose(oracle.at_draw(5, 7, 11, 0, 3.0), 3.0 * a, rtol=1e-15)


def test_at_draw_mixed_matches_fp64():
    # The float model keeps the high 32 bits of each uniform and rounds 1 - U
    # to float, so a Box-Muller radius near zero (U near 0) is resolved only
    # to about sqrt(2 * 2^-24) = 3.5e-4; elsewhere the two agree to float
    # rounding.
    d = np.array([oracle.at_draw(3, 44, i, i & 1, 1.0, oracle.FP64) for i in range(4000)])
    f = np.array([oracle.at_draw(3, 44, i, i & 1, 1.0, oracle.MIXED) for i in range(4000)])
    err = np.abs(f - d)
    assert err.max() < 5e-4
    assert np.mean(err > 2e-6 * np.maximum(1.0, np.abs(d))) < 0.005


def _cell_sums(cells, ncells, w, x):
    out = np.zeros((ncells, 3))
    for k in range(3):
        out[:, k] = np.bincount(cells, weights=w * x[:, k], minlength=ncells)
    return out


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
@pytest.mark.parametrize("beads", [False, True])
def test_at_conserves_cell_momentum(precision, beads):
    n = (5, 4, 6)
    mixed = precision == oracle.MIXED
    s = inputs.solvent(n, 5.0, seed=21, mixed=mixed)
    pos, vel = s.pos.astype(np.float64), s.vel.astype(np.float64)
    vel = vel + np.array([0.7, -0.3, 0.2])  # a drifting state
    vel[:, 0] += np.sin(pos[:, 2])          # and a shear
    if mixed:
        vel = vel.astype(np.float32).astype(np.float64)
    kw = {}
    st = oracle.State(pos, vel)
    if beads:
        kw = dict(chain_len=10, md_substeps=1, solute_mass=5.0, bond_k=0.0, bond_r0=0.5)
        sp, sv = inputs.chains(n, 3, 10, 0.5, bead_mass=5.0, seed=4)
        st = oracle.State(pos, vel, sp, sv)
    p = oracle.Params(n=n, seed=31, precision=precision, collision=oracle.AT, **kw)
    v0, sv0 = st.vel.copy(), st.svel.copy()
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    nc = oracle.num_cells(p)
    ns = v0.shape[0]
    m = np.concatenate([np.full(ns, 1.0), np.full(sv0.shape[0], 5.0)])
    before = _cell_sums(cells, nc, m, np.vstack([v0, sv0]))
    after = _cell_sums(cells, nc, m, np.vstack([st.vel, st.svel]))
    scale = np.abs(m[:, None] * np.vstack([v0, sv0])).sum()
    tol = 1e-13 if not mixed else 1e-6
    assert np.max(np.abs(after - before)) <= tol * scale
    # the velocities did change (the rule is not the identity)
    assert np.max(np.abs(st.vel - v0)) > 0.1
    # a lone member keeps its velocity: dv - dbar vanishes
    lone = np.where(counts[cells[:ns]] == 1)[0]
    assert lone.size > 0
    assert np.allclose(st.vel[lone], v0[lone], rtol=0, atol=1e-12 if not mixed else 1e-6)


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_at_relative_energy_is_chi_square(precision):
    n = (10, 10, 10)
    rho, kT = 3.0, 1.3
    rng = np.random.default_rng(8)
    N = int(rho * np.prod(n))
    pos = rng.random((N, 3)) * np.array(n, dtype=float)
    u0 = np.array([0.5, -1.25, 0.75])   # exactly representable: a cold uniform flow
    vel = np.tile(u0, (N, 1))
    # solute beads of mass 4 join the cells, also at u0
    nb = 400
    sp = rng.random((nb, 3)) * np.array(n, dtype=float)
    sv = np.tile(u0, (nb, 1))
    if precision == oracle.MIXED:
        pos = pos.astype(np.float32).astype(np.float64)
    p = oracle.Params(n=n, seed=17, kT=kT, precision=precision, collision=oracle.AT,
                      chain_len=1, md_substeps=1, solute_mass=4.0, bond_k=0.0, bond_r0=0.0)
    st = oracle.State(pos, vel, sp, sv)
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    nc = oracle.num_cells(p)
    m = np.concatenate([np.full(N, 1.0), np.full(nb, 4.0)])
    v = np.vstack([st.vel, st.svel])
    M = np.bincount(cells, weights=m, minlength=nc)
    P = _cell_sums(cells, nc, m, v)
    occ = M > 0
    u = np.zeros_like(P)
    u[occ] = P[occ] / M[occ, None]
    tol = 1e-12 if precision == oracle.FP64 else 2e-6
    assert np.max(np.abs(u[occ] - u0)) < tol * 4  # u of every cell unchanged
    d = v - u[cells]
    E = np.bincount(cells, weights=0.5 * m * (d * d).sum(axis=1), minlength=nc)
    sel = counts >= 2
    dof = 3 * (counts[sel] - 1)
    # probability integral transform: uniform on [0, 1] if E ~ (kT/2) chi2(dof)
    pit = scipy_stats.chi2.cdf(2.0 * E[sel] / kT, dof)
    assert scipy_stats.kstest(pit, "uniform").pvalue > 1e-3
    ratio = E[sel] / (0.5 * dof * kT)
    assert abs(ratio.mean() - 1.0) < 4.0 * math.sqrt(2.0 / dof.mean() / sel.sum())


def _shear_wave_eta(dseed):
    """Viscosity from the decay of a transverse shear wave
    v_x = A sin kz, v_y = A cos kz (a z-only flow: no advection term),
    with the thermal state's own projection on those modes removed."""
    n, rho, A, steps, every = (24, 24, 32), 10.0, 1.0, 300, 5
    k = 2 * math.pi / n[2]
    s = inputs.solvent(n, rho, seed=100 + dseed)
    vel = s.vel.copy()
    sn, cs = np.sin(k * s.pos[:, 2]), np.cos(k * s.pos[:, 2])
    vel[:, 0] -= sn * (vel[:, 0] @ sn) / (sn @ sn)
    vel[:, 1] -= cs * (vel[:, 1] @ cs) / (cs @ cs)
    vel[:, 0] += A * sn
    vel[:, 1] += A * cs
    p = oracle.Params(n=n, seed=dseed, collision=oracle.AT)
    st = oracle.State(s.pos.copy(), vel)
    amp = []
    for it in range(steps // every + 1):
        z = st.pos[:, 2]
        amp.append(np.mean(st.vel[:, 0] * np.sin(k * z)) + np.mean(st.vel[:, 1] * np.cos(k * z)))
        if it < steps // every:
            oracle.step(p, st, every)
    t = np.arange(len(amp)) * every * p.dt
    rate = -np.polyfit(t, np.log(np.array(amp)), 1)[0]
    return rate / k**2 * rho  # eta = rho m nu


@pytest.mark.slow
def test_at_shear_wave_recovers_viscosity():
    seeds = list(range(1, 9))
    oracle.build()
    with mp.get_context("spawn").Pool(min(len(seeds), mp.cpu_count())) as pool:
        etas = pool.map(_shear_wave_eta, seeds)
    eta_th = eta_at(10.0, 0.1)
    assert abs(eta_th - 8.111) < 1e-3
    assert abs(np.mean(etas) / eta_th - 1.0) < 0.03, (etas, eta_th)
