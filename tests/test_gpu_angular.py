"""GPU parity of the angular-momentum-conserving collisions (the constraint
the paper cites after Eqs. srd and at, Sec. 2) against the oracle, through
the C ABI.  Mixed model bit-exact (the same float terms summed in int64 fixed
point and the same float 3x3 solve on both sides); FP64 within 1e-12 per step
(summation order and libm), cell ids and counts bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1801_10187_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1801_10187_gb300 as pkg  # noqa: E402


def rel_err(v, ref, kT=1.0, m=1.0):
    scale = np.maximum(np.linalg.norm(ref, axis=1), math.sqrt(kT / m))
    return (np.linalg.norm(v - ref, axis=1) / scale).max(initial=0.0)


def run(n, pos, vel, precision, steps, seed, rule="srd", thermostat=False, step0=0, **kw):
    box = pkg.Box(n=n, seed=seed, precision=precision, collision=rule, thermostat=thermostat,
                  angular=True, **kw)
    box.set_state(pos, vel, step=step0)
    box.step(steps)
    p2, v2, _, _, st = box.get_state()
    cells, counts = box.last_cells()
    box.close()
    okw = {}
    if "body_force" in kw:
        okw["g"] = kw["body_force"]
    p = oracle.Params(n=n, seed=seed, precision=oracle.MIXED if precision == "mixed" else oracle.FP64,
                      collision=oracle.AT if rule == "at" else oracle.SRD, thermostat=thermostat,
                      angular=True, **okw)
    ref = oracle.State(pos.copy(), vel.copy(), step=step0)
    rc, rk = oracle.step(p, ref, steps, want_cells=True)
    assert st == ref.step
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_array_equal(counts, rk)
    if precision == "mixed":
        np.testing.assert_array_equal(p2, ref.pos)
        np.testing.assert_array_equal(v2, ref.vel)
    else:
        assert rel_err(v2, ref.vel) <= 1e-12 * steps
        assert np.max(np.abs(p2 - ref.pos)) <= 1e-11 * steps
    return v2


RULES = [("srd", False), ("srd", True), ("at", False)]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("rule,thermo", RULES)
def test_angular_one_step(precision, rule, thermo):
    s = inputs.solvent((10, 10, 10), 5, seed=7, mixed=precision == "mixed")
    vel = s.vel.copy()
    vel[:, 0] += 0.8 * np.sin(2 * np.pi * s.pos[:, 1] / 10.0)
    if precision == "mixed":
        vel = vel.astype(np.float32).astype(np.float64)
    run((10, 10, 10), s.pos, vel, precision, 1, 7, rule, thermo)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("rule,thermo", RULES)
def test_angular_ragged_multi_step(precision, rule, thermo):
    s = inputs.solvent((23, 17, 9), 7.3, seed=9, mixed=precision == "mixed", n_particles=25699)
    run((23, 17, 9), s.pos, s.vel, precision, 4, 9, rule, thermo, step0=987654321,
        body_force=(0.01, 0.0, -0.02))


def test_angular_mixed_dense_and_overflow():
    # density 12 (rows of 40) over 5 steps, then a cluster beyond the row
    # capacity (overflow list)
    s = inputs.solvent((12, 12, 12), 12, seed=4, mixed=True)
    run((12, 12, 12), s.pos, s.vel, "mixed", 5, 4, "at")
    rng = np.random.default_rng(3)
    s = inputs.solvent((6, 6, 6), 5, seed=5, mixed=True)
    clu = np.full((900, 3), 2.45) + rng.random((900, 3)) * 0.1
    pos = np.vstack([s.pos, clu]).astype(np.float32).astype(np.float64)
    vel = np.vstack([s.vel, rng.standard_normal((900, 3))]).astype(np.float32).astype(np.float64)
    run((6, 6, 6), pos, vel, "mixed", 1, 5, "srd")


def test_angular_box_batched_equal_alone():
    specs = [((9, 9, 9), 5, "srd", True, 301), ((7, 7, 7), 8, "at", False, 302),
             ((8, 8, 8), 5, "srd", False, 303)]
    states = [inputs.solvent(n, rho, seed=sd, mixed=True) for n, rho, _, _, sd in specs]
    batch = pkg.Batch("mixed")
    slots = [batch.add(s.pos, s.vel, n=n, seed=sd, collision=rule, angular=ang)
             for (n, rho, rule, ang, sd), s in zip(specs, states)]
    batch.step(4)
    got = [batch.get_state(sl) for sl in slots]
    batch.close()
    for (n, rho, rule, ang, sd), s, g in zip(specs, states, got):
        box = pkg.Box(n=n, seed=sd, collision=rule, angular=ang, precision="mixed")
        box.set_state(s.pos, s.vel)
        box.step(4)
        pos, vel, *_ = box.get_state()
        box.close()
        np.testing.assert_array_equal(pos, g[0])
        np.testing.assert_array_equal(vel, g[1])


def test_angular_rejects_walls_and_solute():
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(4, 4, 4), angular=True, walls_z=True)
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(4, 4, 4), angular=True, chain_len=4, md_substeps=1, solute_mass=5.0)


def test_angular_mixed_large_velocities_exact():
    # members with |v| >= 1024: the momentum sums and the terms r_c x (v - v')
    # leave the int32 split and take the exact int64 paths
    s = inputs.solvent((6, 6, 6), 5, seed=12, mixed=True)
    vel = s.vel.copy()
    rng = np.random.default_rng(1)
    idx = rng.choice(len(vel), 40, replace=False)
    vel[idx] = rng.uniform(1024.0, 1500.0, (40, 3)) * rng.choice([-1.0, 1.0], (40, 3))
    vel = vel.astype(np.float32).astype(np.float64)
    run((6, 6, 6), s.pos, vel, "mixed", 2, 12, "srd")


def test_angular_two_member_and_lone_cells():
    # a sparse box: most cells hold one or two members (the rank-two branch)
    s = inputs.solvent((8, 8, 8), 1.5, seed=15, mixed=True)
    run((8, 8, 8), s.pos, s.vel, "mixed", 3, 15, "srd")
    s = inputs.solvent((8, 8, 8), 1.5, seed=15)
    run((8, 8, 8), s.pos, s.vel, "fp64", 3, 15, "srd")
