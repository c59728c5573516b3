"""Pins of the oracle's angular-momentum-conserving collisions (CPU only).

The paper's collision rules conserve linear momentum only; it cites Noguchi &
Gompper for the constraint that also conserves angular momentum (Sec. 2, after
Eqs. srd and at).  With ``angular`` the oracle adds to each member of a cell
omega x r_c (r_c: position relative to the cell's centre of mass), with
Pi omega = sum m r_c x (v - v') and Pi the cell's inertia tensor.  Fixed
independently of that code:
1. every cell's angular momentum about its centre of mass is the same after
   the collision as before it (and without the option it is not), for SRD
   with and without the thermostat and for the Andersen rule, in both
   arithmetic models; linear momentum stays conserved;
2. Andersen rule from a cold flow: the correction removes the rigid-rotation
   part of the random velocities, so the cell energy about u is kT/2 times a
   chi-square variable with 3 Nc - 6 degrees of freedom (Nc >= 3), 1 for two
   members (rotation about their axis does nothing) and 0 for one;
3. alpha = 0 (no rotation): nothing changes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1801_10187_gb300 import inputs

scipy_stats = pytest.importorskip("scipy.stats")


def cell_frame(pos, cells, n, s):
    """Positions relative to their shifted cell (numpy floor, independent of
    the oracle's arithmetic) and the cell's centre of mass (unit masses)."""
    r = pos - s[None, :]
    r = r - np.floor(r)
    nc = int(np.prod(n))
    cnt = np.bincount(cells, minlength=nc).astype(float)
    com = np.zeros((nc, 3))
    for k in range(3):
        com[:, k] = np.bincount(cells, weights=r[:, k], minlength=nc)
    occ = cnt > 0
    com[occ] /= cnt[occ, None]
    return r - com[cells], cnt


def cell_L(rc, v, cells, nc):
    L = np.cross(rc, v)
    return np.stack([np.bincount(cells, weights=L[:, k], minlength=nc) for k in range(3)], axis=1)


def cell_P(v, cells, nc):
    return np.stack([np.bincount(cells, weights=v[:, k], minlength=nc) for k in range(3)], axis=1)


CASES = [("srd", False), ("srd", True), ("at", False)]


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
@pytest.mark.parametrize("rule,thermo", CASES)
def test_cell_angular_momentum_conserved(precision, rule, thermo):
    n = (6, 5, 7)
    mixed = precision == oracle.MIXED
    s = inputs.solvent(n, 6.0, seed=33, mixed=mixed)
    pos, vel = s.pos.astype(np.float64), s.vel.astype(np.float64)
    vel[:, 0] += 0.8 * np.sin(2 * np.pi * pos[:, 1] / n[1])  # a shear: cells carry spin
    if mixed:
        vel = vel.astype(np.float32).astype(np.float64)
    coll = oracle.AT if rule == "at" else oracle.SRD
    nc = int(np.prod(n))
    out = {}
    for ang in (False, True):
        p = oracle.Params(n=n, seed=44, precision=precision, collision=coll, thermostat=thermo,
                          angular=ang)
        st = oracle.State(pos.copy(), vel.copy(), step=9)
        cells, counts = oracle.step(p, st, 1, want_cells=True)
        sh = oracle.shift(44, 9)
        rc, cnt = cell_frame(st.pos, cells, n, sh)
        out[ang] = (cell_L(rc, vel, cells, nc), cell_L(rc, st.vel, cells, nc),
                    cell_P(vel, cells, nc), cell_P(st.vel, cells, nc), cnt)
    L0, L1, P0, P1, cnt = out[True]
    sel = cnt >= 2
    scale = np.abs(L0[sel]).max()
    tol = 1e-12 if not mixed else 2e-5
    assert np.max(np.abs(L1[sel] - L0[sel])) <= tol * max(scale, 1.0)
    assert np.max(np.abs(P1 - P0)) <= (1e-12 if not mixed else 2e-5) * 10
    # the plain rule does change the cells' angular momenta
    L0p, L1p = out[False][0], out[False][1]
    assert np.max(np.abs(L1p[sel] - L0p[sel])) > 0.05 * scale


@pytest.mark.parametrize("precision", [oracle.FP64, oracle.MIXED])
def test_at_angular_energy_is_chi_square(precision):
    n = (12, 12, 12)
    kT = 0.7
    rng = np.random.default_rng(5)
    N = int(4.0 * np.prod(n))
    pos = rng.random((N, 3)) * np.array(n, dtype=float)
    if precision == oracle.MIXED:
        pos = pos.astype(np.float32).astype(np.float64)
    u0 = np.array([0.25, -0.5, 1.0])
    vel = np.tile(u0, (N, 1))
    p = oracle.Params(n=n, seed=13, kT=kT, precision=precision, collision=oracle.AT, angular=True)
    st = oracle.State(pos, vel)
    cells, counts = oracle.step(p, st, 1, want_cells=True)
    nc = int(np.prod(n))
    d = st.vel - u0
    E = 0.5 * np.bincount(cells, weights=(d * d).sum(axis=1), minlength=nc)
    one = counts == 1
    assert np.max(E[one]) < (1e-20 if precision == oracle.FP64 else 1e-10)
    sel = counts >= 2
    dof = np.where(counts[sel] >= 3, 3 * counts[sel] - 6, 1)
    pit = scipy_stats.chi2.cdf(2.0 * E[sel] / kT, dof)
    assert scipy_stats.kstest(pit, "uniform").pvalue > 1e-3
    # without the correction the same cells follow 3 (Nc - 1) degrees of freedom
    ratio = (2.0 * E[sel] / kT).sum() / dof.sum()
    assert abs(ratio - 1.0) < 4.0 * math.sqrt(2.0 / dof.sum())


def test_angular_with_alpha_zero_changes_nothing():
    n = (5, 5, 5)
    s = inputs.solvent(n, 5.0, seed=2)
    p = oracle.Params(n=n, seed=3, alpha_deg=0.0, angular=True)
    st = oracle.State(s.pos.copy(), s.vel.copy())
    oracle.step(p, st, 3)
    assert np.max(np.abs(st.vel - s.vel)) < 1e-13


def test_angular_rejects_walls_and_solute():
    n = (4, 4, 4)
    s = inputs.solvent(n, 3.0, seed=2)
    with pytest.raises(RuntimeError):
        oracle.step(oracle.Params(n=n, walls_z=True, angular=True, virt_density=3.0),
                    oracle.State(s.pos.copy(), s.vel.copy()), 1)
    sp, sv = inputs.chains(n, 1, 4, 0.5, seed=1)
    with pytest.raises(RuntimeError):
        oracle.step(oracle.Params(n=n, angular=True, chain_len=4, md_substeps=1, solute_mass=5.0,
                                  bond_k=10.0, bond_r0=0.5),
                    oracle.State(s.pos.copy(), s.vel.copy(), sp, sv), 1)
