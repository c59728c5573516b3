"""Pins of the oracle's non-bonded solute forces (CPU only).

Sec. 4.3 runs a bead-spring polymer with non-bonded pair forces from a
neighbour list and only cites the potential; the reading here is the
Weeks-Chandler-Andersen repulsion U(r) = 4 eps ((s/r)^12 - (s/r)^6) + eps
for r < 2^(1/6) s.  Fixed independently of the oracle's force code:
1. two beads: the force at r = s is 24 eps / s along the line of centres,
   U(r_c) = 0 and no force beyond r_c, also across the periodic boundary;
2. forces are minus the gradient of the energy (central differences) for a
   random configuration of chains, and sum to zero (Newton's third law);
3. velocity Verlet conserves energy: beads alone with energy-conserving SRD
   collisions keep KE + U up to an error that falls as h^2.
"""
import math

import numpy as np

import oracle
from paper_1801_10187_gb300 import inputs

EPS, SIG = 1.0, 0.5
RC = 2 ** (1 / 6) * SIG


def params(**kw):
    base = dict(n=(6, 6, 6), chain_len=1, md_substeps=10, solute_mass=5.0, bond_k=0.0,
                bond_r0=0.5, lj_epsilon=EPS, lj_sigma=SIG)
    base.update(kw)
    return oracle.Params(**base)


def test_two_beads_closed_form():
    p = params()
    for r, fmag in ((SIG, 24 * EPS / SIG), (0.9 * RC, None), (RC * 1.0001, 0.0), (2.0, 0.0)):
        pos = np.array([[1.0, 2.0, 3.0], [1.0 + r, 2.0, 3.0]])
        F = oracle.solute_forces(p, pos)
        assert abs(F[0, 1]) + abs(F[0, 2]) < 1e-15
        assert np.allclose(F[0], -F[1], rtol=0, atol=1e-12)
        if fmag is not None:
            assert abs(-F[0, 0] - fmag) <= 1e-12 * max(1.0, fmag)
        else:
            assert -F[0, 0] > 0.0  # repulsive inside the cutoff
    # U vanishes at the cutoff, with its derivative
    pos = np.array([[1.0, 2.0, 3.0], [1.0 + RC * (1 - 1e-9), 2.0, 3.0]])
    assert oracle.solute_energy(p, pos) < 1e-6
    # the nearest image across the box edge
    pos = np.array([[0.1, 3.0, 3.0], [5.95, 3.0, 3.0]])  # 0.15 apart through x = 0
    F = oracle.solute_forces(p, pos)
    assert F[0, 0] > 0.0 and F[1, 0] < 0.0


def test_forces_are_minus_gradient_and_balance():
    # chains of 8 beads along x (spacing about 0.5) on lines 0.55 apart, with
    # jitter: bonds stretched and compressed, neighbouring lines within the
    # cutoff, no extreme overlaps (so that energy differences stay accurate)
    n = (5, 5, 5)
    rng0 = np.random.default_rng(3)
    sp = []
    for iy in range(4):
        for iz in range(3):
            for b in range(8):
                sp.append([0.3 + 0.5 * b, 0.4 + 0.55 * iy, 0.4 + 0.55 * iz])
    sp = np.array(sp) + rng0.uniform(-0.04, 0.04, (len(sp), 3))
    p = params(n=n, chain_len=8, bond_k=100.0)
    F = oracle.solute_forces(p, sp)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-9 * np.abs(F).sum()
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(30):
        i, k = int(rng.integers(len(sp))), int(rng.integers(3))
        a, b = sp.copy(), sp.copy()
        a[i, k] += h
        b[i, k] -= h
        g = -(oracle.solute_energy(p, a) - oracle.solute_energy(p, b)) / (2 * h)
        assert abs(g - F[i, k]) <= 1e-4 * max(1.0, abs(F[i, k])), (i, k, g, F[i, k])
    # the WCA part is present (some pairs are inside the cutoff)
    F0 = oracle.solute_forces(params(n=n, chain_len=8, bond_k=100.0, lj_epsilon=0.0), sp)
    assert np.max(np.abs(F - F0)) > 1.0


def lattice_chains(nlines_y, nlines_z, chain_len, seed, jitter=0.04, spacing=0.55):
    """Chains along x (bead spacing about 0.5) on lines `spacing` apart, with
    jitter: no extreme overlaps, so the energy stays moderate."""
    rng = np.random.default_rng(seed)
    sp = [[0.3 + 0.5 * b, 0.4 + spacing * iy, 0.4 + spacing * iz]
          for iy in range(nlines_y) for iz in range(nlines_z) for b in range(chain_len)]
    return np.array(sp) + rng.uniform(-jitter, jitter, (len(sp), 3))


def _energy_drift(sub):
    n = (6, 6, 6)
    sp = lattice_chains(4, 4, 10, 7, spacing=0.6)
    sv = np.random.default_rng(8).standard_normal(sp.shape) * math.sqrt(1.0 / 5.0)
    p = params(n=n, chain_len=10, bond_k=50.0, md_substeps=sub, dt=0.1)
    st = oracle.State(np.zeros((0, 3)), np.zeros((0, 3)), sp.copy(), sv.copy())
    def E():
        return 0.5 * 5.0 * (st.svel ** 2).sum() + oracle.solute_energy(p, st.spos)
    e0 = E()
    errs = []
    for _ in range(20):
        oracle.step(p, st, 1)
        errs.append(abs(E() - e0))
    return max(errs), e0


def test_verlet_energy_conservation():
    d10, e0 = _energy_drift(10)
    d20, _ = _energy_drift(20)
    assert d10 < 1e-2 * abs(e0)
    assert 3.0 < d10 / d20 < 5.0  # second order in h
