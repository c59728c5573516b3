"""GPU parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark times (captured graphs of the fused pass, one
launch per step), against the oracle run on the same states.

  * 100^3 cells at density 10 (10^7 particles), mixed and FP64, and the
    Andersen-rule and angular-correction variants of the mixed box: two steps
    (the stream/bin pass, one fused collide + stream/bin pass, and the
    completing collision), every particle compared.
  * 250^3 cells at density 5 (7.8 * 10^7 particles) with 2000 chains of 50
    beads and the cell thermostat: two steps, every particle compared.
  * the 64-box ensemble (about 1.5 * 10^8 particles) stepped in one batch:
    three boxes compared particle by particle, and for every box the
    momentum conservation that holds at any size.
  * the paper's polymer benchmark (1.25e6 FP64 solvent particles, 1024 chains
    of 50 repelling beads): total momentum and energy conserved.
Tolerances as in the small parity tests: mixed bit-exact, FP64 1e-12
relative per step.

The mixed model's accuracy at full size: one GPU step of the 10^7-particle
box (SRD with and without the thermostat, the Andersen rule, the angular
correction) and of the 7.8 * 10^7-particle solute + thermostat box against
the FP64 model run from the same float state with float streaming (the same
cells), every particle within the bound of tests/mixed_bound.py; cells whose
float and FP64 Gamma samplers accept different attempts are counted and left
out.  The maximum error, the particles above 1e-6 and the flips are shown in
the run's summary.  These runs take a few minutes of oracle time.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1801_10187_gb300 import inputs

from mixed_bound import gamma_flip_cells, inertia_condition, mixed_step_bound, rel_errors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1801_10187_gb300 as pkg  # noqa: E402

W = inputs.WORKLOADS


def rel_err(v, ref, kT=1.0, m=1.0):
    scale = np.maximum(np.linalg.norm(ref, axis=1), math.sqrt(kT / m))
    return (np.linalg.norm(v - ref, axis=1) / scale).max(initial=0.0)


def box_kw(cfg):
    kw = dict(n=cfg["n"], dt=cfg["dt"], alpha_deg=cfg["alpha_deg"], kT=cfg["kT"],
              seed=cfg["seed"], thermostat=cfg["thermostat"], precision=cfg["precision"],
              collision=cfg.get("collision", "srd"), angular=cfg.get("angular", False))
    if cfg.get("n_chains"):
        kw.update(chain_len=cfg["chain_len"], md_substeps=cfg["md_substeps"],
                  solute_mass=cfg["bead_mass"], bond_k=cfg["bond_k"], bond_r0=cfg["bond_r0"])
    return kw


def oracle_params(kw):
    return oracle.Params(
        n=kw["n"], dt=kw["dt"], alpha_deg=kw["alpha_deg"], kT=kw["kT"], seed=kw["seed"],
        thermostat=kw["thermostat"],
        precision=oracle.MIXED if kw["precision"] == "mixed" else oracle.FP64,
        collision=oracle.AT if kw["collision"] == "at" else oracle.SRD,
        chain_len=kw.get("chain_len", 0), md_substeps=kw.get("md_substeps", 0),
        solute_mass=kw.get("solute_mass", 1.0), bond_k=kw.get("bond_k", 0.0),
        bond_r0=kw.get("bond_r0", 0.0), angular=kw["angular"])


def run_full(name, steps=2):
    cfg = W[name]
    kw = box_kw(cfg)
    mixed = cfg["precision"] == "mixed"
    s = inputs.solvent(cfg["n"], cfg["density"], kT=cfg["kT"], seed=cfg["seed"], mixed=mixed)
    sp = sv = None
    if cfg.get("n_chains"):
        sp, sv = inputs.chains(cfg["n"], cfg["n_chains"], cfg["chain_len"], cfg["bond_r0"],
                               kT=cfg["kT"], bead_mass=cfg["bead_mass"], seed=cfg["seed"] + 1000)
    box = pkg.Box(**kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(steps)
    pos, vel, spos, svel, st = box.get_state()
    cells, counts = box.last_cells()
    box.close()
    ref = oracle.State(np.asarray(s.pos, np.float64), np.asarray(s.vel, np.float64),
                       np.zeros((0, 3)) if sp is None else sp.copy(),
                       np.zeros((0, 3)) if sv is None else sv.copy())
    del s
    rc, rk = oracle.step(oracle_params(kw), ref, steps, want_cells=True)
    assert st == ref.step == steps
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_array_equal(counts, rk)
    if mixed:
        np.testing.assert_array_equal(pos, ref.pos)
        np.testing.assert_array_equal(vel, ref.vel)
    else:
        assert rel_err(vel, ref.vel) <= 1e-12 * steps
        assert np.max(np.abs(pos - ref.pos)) <= 1e-10
    return spos, svel, ref


@pytest.mark.parametrize("name", ["srd-100c-rho10-mixed", "srd-100c-rho10-fp64",
                                  "srd-100c-rho10-mixed-at", "srd-100c-rho10-mixed-angular"])
def test_fullsize_10m(name):
    run_full(name)


def test_fullsize_78m_solute_thermostat():
    spos, svel, ref = run_full("srd-250c-rho5-mixed-solute")
    assert rel_err(svel, ref.svel, m=5.0) == 0.0
    assert np.max(np.abs(spos - ref.spos)) <= 1e-11


MIXED_CASES = [("srd-100c-rho10-mixed", False), ("srd-100c-rho10-mixed", True),
               ("srd-100c-rho10-mixed-at", False), ("srd-100c-rho10-mixed-angular", False),
               ("srd-250c-rho5-mixed-solute", True)]


@pytest.mark.parametrize("name,thermostat", MIXED_CASES)
def test_fullsize_mixed_against_fp64_one_step(name, thermostat, report):
    cfg = W[name]
    kw = box_kw(cfg)
    kw["thermostat"] = thermostat
    t0 = 31
    s = inputs.solvent(cfg["n"], cfg["density"], kT=cfg["kT"], seed=cfg["seed"], mixed=True)
    sp = sv = np.zeros((0, 3))
    if cfg.get("n_chains"):
        sp, sv = inputs.chains(cfg["n"], cfg["n_chains"], cfg["chain_len"], cfg["bond_r0"],
                               kT=cfg["kT"], bead_mass=cfg["bead_mass"], seed=cfg["seed"] + 1000)
    box = pkg.Box(**kw)
    box.set_state(s.pos, s.vel, sp if len(sp) else None, sv if len(sv) else None, step=t0)
    box.step(1)
    pos, vel, spos, svel, st = box.get_state()
    cells, counts = box.last_cells()
    box.close()
    p = oracle_params(kw)
    p.precision = oracle.FP64_FSTREAM
    # copies: the oracle steps its state in place, and s.vel is needed below
    ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy(), step=t0)
    rc, rk = oracle.step(p, ref, 1, want_cells=True)
    ns = s.pos.shape[0]
    assert st == ref.step == t0 + 1
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_array_equal(counts, rk)
    np.testing.assert_array_equal(pos, ref.pos)
    if len(sp):
        assert np.max(np.abs(spos - ref.spos)) <= 1e-11
    cond = (inertia_condition(ref.pos, rc[:ns], oracle.shift(kw["seed"], t0), kw["n"], rk.shape[0])
            if kw["angular"] else None)
    M = kw.get("solute_mass", 1.0)
    bound, bbound = mixed_step_bound(s.vel, ref.vel, rc[:ns], kT=kw["kT"], thermostat=thermostat,
                                     svel_ref=ref.svel, bead_cells=rc[ns:], bead_mass=M,
                                     angular_cond=cond)
    err = rel_errors(vel, ref.vel, kT=kw["kT"])
    over = err > bound
    flips = np.zeros(0, dtype=np.int64)
    if thermostat:
        flips = gamma_flip_cells(kw["seed"], t0, kw["kT"], rk, rc[:ns][over])
        over &= ~np.isin(rc[:ns], flips)
    occupied = int(np.count_nonzero(rk))
    keep = ~np.isin(rc[:ns], flips)
    line = (f"mixed vs FP64, one step, {name}{' +thermostat' if thermostat else ''}: "
            f"{ns} particles; outside Gamma-flipped cells: max rel err {err[keep].max():.3g}, "
            f"above 1e-6: {int(np.sum(err[keep] > 1e-6))}, max err/bound "
            f"{np.max(err[keep] / bound[keep]):.3g}; Gamma flips {len(flips)} of {occupied} cells")
    if len(sp):
        eb = rel_errors(svel, ref.svel, kT=kw["kT"], m=M)
        bover = (eb > bbound) & ~np.isin(rc[ns:], flips)
        assert not bover.any()
        line += f", beads max rel err {eb.max():.3g}"
    report.append(line)
    assert not over.any(), line
    assert len(flips) <= 5 + 1e-6 * occupied, line


def test_fullsize_batch64():
    cfg = W["srd-batch64-mixed"]
    specs = inputs.ensemble(cfg["n_boxes"], seed=cfg["ensemble_seed"])
    counts = [int(round(s["density"] * np.prod(s["n"]))) for s in specs]
    batch = pkg.Batch(cfg["precision"])
    slots = []
    for s, n in zip(specs, counts):
        slots.append(batch.add_thermal(n, init_seed=s["seed"], n=s["n"], alpha_deg=s["alpha_deg"],
                                       seed=s["seed"], dt=cfg["dt"], kT=cfg["kT"],
                                       thermostat=cfg["thermostat"]))
    order = np.argsort(counts)
    picked = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    start = {i: batch.get_state(slots[i]) for i in picked}
    ob0 = [batch.observables(sl) for sl in slots]
    steps = 2
    batch.step(steps)
    P1 = [batch.observables(sl)["P"] for sl in slots]
    got = {i: batch.get_state(slots[i]) for i in picked}
    batch.close()
    for i in picked:
        s = specs[i]
        p = oracle.Params(n=s["n"], dt=cfg["dt"], alpha_deg=s["alpha_deg"], kT=cfg["kT"],
                          seed=s["seed"], thermostat=cfg["thermostat"], precision=oracle.MIXED)
        ref = oracle.State(start[i][0].copy(), start[i][1].copy())
        oracle.step(p, ref, steps)
        np.testing.assert_array_equal(got[i][0], ref.pos)
        np.testing.assert_array_equal(got[i][1], ref.vel)
        assert got[i][2] == steps
    # every box: momentum conserved by the collisions up to the float rounding
    # of each stored velocity, |dP| <= steps 2^-24 sum |v| <= steps 2^-24
    # sqrt(2 n KE) (unit mass)
    for n, o, b in zip(counts, ob0, P1):
        bound = steps * 2.0**-24 * math.sqrt(2.0 * n * o["KE"])
        assert np.max(np.abs(o["P"] - b)) <= bound


def test_fullsize_polymer_benchmark_conserves():
    """The paper's polymer benchmark (Sec. 4.3) at full size: 1.25e6 FP64
    solvent particles and 1024 chains of 50 beads with the WCA repulsion.
    The oracle's every-pair loop is too slow here, so the test checks what
    holds at any size: total momentum (collisions and pair forces conserve
    it) and total energy (SRD collisions conserve kinetic energy; velocity
    Verlet with h = 0.002 keeps the rest to well below 1e-4)."""
    cfg = W["srd-50c-rho10-fp64-polymer"]
    kw = box_kw(cfg)
    kw.update(lj_epsilon=cfg["lj_epsilon"], lj_sigma=cfg["lj_sigma"])
    s = inputs.solvent(cfg["n"], cfg["density"], kT=cfg["kT"], seed=cfg["seed"])
    sp, sv = inputs.avoiding_chains(cfg["n"], cfg["n_chains"], cfg["chain_len"], cfg["bond_r0"],
                                    0.9 * cfg["lj_sigma"], bead_mass=cfg["bead_mass"],
                                    seed=cfg["seed"] + 1000)
    p = oracle_params(kw)
    p.lj_epsilon, p.lj_sigma = cfg["lj_epsilon"], cfg["lj_sigma"]
    M = cfg["bead_mass"]

    def totals(vel, spos, svel):
        P = vel.sum(axis=0) + M * svel.sum(axis=0)
        E = 0.5 * (vel ** 2).sum() + 0.5 * M * (svel ** 2).sum() + oracle.solute_energy(p, spos)
        return P, E, np.abs(vel).sum() + M * np.abs(svel).sum()

    P0, E0, scale = totals(s.vel, sp, sv)
    box = pkg.Box(**kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(3)
    pos, vel, spos, svel, st = box.get_state()
    box.close()
    assert st == 3
    P1, E1, _ = totals(vel, spos, svel)
    assert np.max(np.abs(P1 - P0)) <= 1e-10 * scale
    assert abs(E1 - E0) <= 1e-4 * abs(E0)
