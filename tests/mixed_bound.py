"""Per-particle error bound of one mixed-model step against the FP64 model.

Both models start from the same float state and stream it the same way
(oracle.FP64_FSTREAM streams in float), so they see the same cells; what is
left is the error of the mixed model's float arithmetic in the collision.
With the relative error of particle i defined as
|v_i - v_ref,i| / max(|v_ref,i|, sqrt(kT/m_i)):

  * every rule:     1e-6 (float rounding of v - u, the axis, the rotation and
    u + R(v - u): a few units of 2^-24);
  * thermostat:     + (1 + xi_c) 2^-22 |u_c| / scale_i.  The float u of the
    cell differs from the exact u by at most 2 ulp per component (the
    roundings of the momentum sum's conversion and of the division by M),
    and v' = u + xi R(v - u) carries that error as (I - xi R) e_u; the
    cell's xi (up to ~10^2 in two-member cells whose relative velocity is
    small) scales it;
  * angular:        + 4 * 2^-24 (1 + cond(Pi_c)).  omega solves Pi omega = dL;
    rounding in the float sums of dL and Pi is amplified by the condition
    number of the cell's inertia tensor Pi about its centre of mass (nearly
    collinear three-member cells reach 10^3 and more).  The rank-two branch
    (two members, or all on a line) is well conditioned: cond is taken as 1.

xi_c and u_c are recovered from the FP64 result itself: the collision keeps
each cell's momentum, so u_c is the mass-weighted mean of the cell's
velocities after the step, and |v'_i - u_c| / |v_i - u_c| = xi_c for every
member (R is a rotation).
"""
from __future__ import annotations

import numpy as np

import oracle


def cell_means(cells, vel, mass, ncells):
    """Mass-weighted mean velocity per cell (u) and member counts."""
    M = np.bincount(cells, weights=mass, minlength=ncells)
    u = np.stack([np.bincount(cells, weights=mass * vel[:, k], minlength=ncells)
                  for k in range(3)], axis=1)
    occ = M > 0
    u[occ] /= M[occ, None]
    return u, np.bincount(cells, minlength=ncells)


def inertia_condition(pos, cells, shift, n, ncells):
    """cond(Pi) per cell (Pi about the centre of mass of the solvent members,
    positions in the frame of the shifted cell); 1 where the rank-two branch
    applies (fewer than three members or det Pi <= 1e-6 (tr Pi / 3)^3)."""
    n = np.asarray(n)
    idx = np.stack([cells % n[0], (cells // n[0]) % n[1], cells // (n[0] * n[1])], axis=1)
    L = n.astype(np.float64)
    r = pos - (idx + shift)
    r = (r + 0.5 * L) % L - 0.5 * L  # member of its cell: r in [0, 1) up to rounding
    cnt = np.bincount(cells, minlength=ncells).astype(np.float64)
    S1 = np.stack([np.bincount(cells, weights=r[:, k], minlength=ncells) for k in range(3)], 1)
    S2 = np.zeros((ncells, 3, 3))
    for a in range(3):
        for b in range(a, 3):
            S2[:, a, b] = S2[:, b, a] = np.bincount(cells, weights=r[:, a] * r[:, b],
                                                    minlength=ncells)
    occ = cnt > 0
    com = np.zeros((ncells, 3))
    com[occ] = S1[occ] / cnt[occ, None]
    C = S2 - cnt[:, None, None] * np.einsum("ca,cb->cab", com, com)  # sum r_c r_c^T
    tr = np.trace(C, axis1=1, axis2=2)
    Pi = tr[:, None, None] * np.eye(3) - C
    ev = np.linalg.eigvalsh(Pi)
    trP = ev.sum(axis=1)
    det = ev.prod(axis=1)
    full = (cnt >= 3) & (det > 1e-6 * (trP / 3.0) ** 3)
    cond = np.ones(ncells)
    cond[full] = ev[full, 2] / ev[full, 0]
    return cond


def mixed_step_bound(vel0, vel_ref, cells, *, kT=1.0, m=1.0, thermostat=False,
                     svel_ref=None, bead_cells=None, bead_mass=1.0, angular_cond=None):
    """Bounds (solvent, beads) on the relative error of one mixed step, per
    particle, given the start velocities vel0 (the solvent's velocity before
    the collision; no body force), the FP64 result vel_ref (and svel_ref for
    beads) and the cells of the step."""
    ns = vel_ref.shape[0]
    ncells = int(cells.max(initial=-1)) + 1
    if bead_cells is not None and len(bead_cells):
        ncells = max(ncells, int(bead_cells.max()) + 1)
    scale = np.maximum(np.linalg.norm(vel_ref, axis=1), np.sqrt(kT / m))
    bound = np.full(ns, 1e-6)
    bbound = None
    if svel_ref is not None and len(svel_ref):
        bscale = np.maximum(np.linalg.norm(svel_ref, axis=1), np.sqrt(kT / bead_mass))
        bbound = np.full(len(svel_ref), 1e-6)
    if thermostat:
        allc = cells if bead_cells is None else np.concatenate([cells, bead_cells])
        allv = vel_ref if svel_ref is None else np.concatenate([vel_ref, svel_ref])
        mass = np.concatenate([np.full(ns, m), np.full(len(allc) - ns, bead_mass)])
        u, _ = cell_means(allc, allv, mass, ncells)
        d0 = np.linalg.norm(vel0 - u[cells], axis=1)
        d1 = np.linalg.norm(vel_ref - u[cells], axis=1)
        ratio = np.where(d0 > 0, d1 / np.where(d0 > 0, d0, 1.0), 0.0)
        xi = np.zeros(ncells)
        np.maximum.at(xi, cells, ratio)  # the same for every member up to rounding
        amp = (1.0 + xi) * 2.0**-22 * np.linalg.norm(u, axis=1)
        bound = bound + amp[cells] / scale
        if bbound is not None:
            bbound = bbound + amp[bead_cells] / bscale
    if angular_cond is not None:
        bound = bound + 4.0 * 2.0**-24 * (1.0 + angular_cond[cells]) / scale
    return bound, bbound


def rel_errors(v, ref, kT=1.0, m=1.0):
    scale = np.maximum(np.linalg.norm(ref, axis=1), np.sqrt(kT / m))
    return np.linalg.norm(v - ref, axis=1) / scale


def gamma_flip_cells(seed, t, kT, counts, candidates):
    """Cells among candidates whose float and FP64 Gamma draws differ by more
    than 1e-5 relative: the two samplers accepted different attempts (a
    float decision within rounding of the acceptance boundary)."""
    out = []
    for c in np.unique(candidates):
        nc = int(counts[c])
        if nc < 2:
            continue
        a = oracle.gamma_draw(seed, t, int(c), nc, kT, oracle.FP64)
        b = oracle.gamma_draw(seed, t, int(c), nc, kT, oracle.MIXED)
        if abs(a - b) > 1e-5 * a:
            out.append(int(c))
    return np.array(out, dtype=np.int64)
