"""GPU parity of the Andersen-thermostat collision rule (Eq. at, Sec. 3.7)
against the oracle, through the C ABI.

Tolerances: mixed model bit-exact (both sides draw the same float Box-Muller
velocities from the same Philox words with their own float series, and sum
them in exact int64 fixed point); FP64 |dv| / max(|v|, sqrt(kT/m)) <= 1e-12
per step (libm against CUDA's log/sin/cos in the draws), cell ids and counts
bit-exact.
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


def run_at(n, pos, vel, precision, steps, seed, step0=0, sp=None, sv=None, kT=1.0, **kw):
    box = pkg.Box(n=n, seed=seed, precision=precision, collision="at", kT=kT, **kw)
    box.set_state(pos, vel, sp, sv, step=step0)
    box.step(steps)
    p2, v2, sp2, sv2, st = box.get_state()
    cells, counts = box.last_cells() if steps > 0 else (None, None)
    box.close()
    okw = {k: v for k, v in kw.items()
           if k in ("chain_len", "md_substeps", "solute_mass", "bond_k", "bond_r0")}
    if "body_force" in kw:
        okw["g"] = kw["body_force"]
    p = oracle.Params(n=n, seed=seed, kT=kT, collision=oracle.AT,
                      precision=oracle.MIXED if precision == "mixed" else oracle.FP64, **okw)
    ref = oracle.State(pos.copy(), vel.copy(),
                       np.zeros((0, 3)) if sp is None else sp.copy(),
                       np.zeros((0, 3)) if sv is None else sv.copy(), step=step0)
    rc, rk = oracle.step(p, ref, steps, want_cells=True)
    return (p2, v2, sp2, sv2, st, cells, counts), (ref, rc, rk)


def check(got, want, precision, tol64=1e-12, steps=1):
    (p2, v2, sp2, sv2, st, cells, counts), (ref, rc, rk) = got, want
    assert st == ref.step
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_array_equal(counts, rk)
    if precision == "mixed":
        np.testing.assert_array_equal(p2, ref.pos)
        np.testing.assert_array_equal(v2, ref.vel)
    else:
        assert rel_err(v2, ref.vel) <= tol64 * steps
        assert np.max(np.abs(p2 - ref.pos)) <= 1e-12 * steps * 10


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_at_one_step_10cube(precision):
    s = inputs.solvent((10, 10, 10), 5, seed=5, mixed=precision == "mixed")
    got, want = run_at((10, 10, 10), s.pos, s.vel, precision, 1, 5)
    check(got, want, precision)
    # the rule changed the velocities
    assert np.max(np.abs(got[1] - s.vel)) > 0.5


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_at_ragged_many_tiles_and_steps(precision):
    # 23 x 17 x 9 cells, an odd particle count, a start step off zero, a body
    # force and several steps through the fused pass
    s = inputs.solvent((23, 17, 9), 7.3, seed=6, mixed=precision == "mixed", n_particles=25699)
    got, want = run_at((23, 17, 9), s.pos, s.vel, precision, 4, 6, step0=123456789012,
                       body_force=(0.01, -0.02, 0.005))
    check(got, want, precision, steps=4)


def test_at_mixed_dense_box_two_stage_blocks():
    # 20^3 cells at 12 per cell: more than 256 members per warp (two staging
    # blocks of pass 1), 10 steps bit-exact
    s = inputs.solvent((20, 20, 20), 12, seed=31, mixed=True)
    got, want = run_at((20, 20, 20), s.pos, s.vel, "mixed", 10, 31)
    check(got, want, "mixed")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_at_overflow_rows(precision):
    # a cluster of 3000 particles in one cell of a density-5 box: the cell's
    # members beyond its row capacity sit in the overflow list, summed per lane
    rng = np.random.default_rng(2)
    s = inputs.solvent((8, 8, 8), 5, seed=3, mixed=precision == "mixed")
    clu = np.full((3000, 3), 2.4) + rng.random((3000, 3)) * 0.2
    pos = np.vstack([s.pos, clu])
    vel = np.vstack([s.vel, rng.standard_normal((3000, 3))])
    if precision == "mixed":
        pos = pos.astype(np.float32).astype(np.float64)
        vel = vel.astype(np.float32).astype(np.float64)
    got, want = run_at((8, 8, 8), pos, vel, precision, 1, 3)
    assert want[2].max() > 500  # far beyond the row capacity (36)
    check(got, want, precision)


def test_at_mixed_exact_int64_paths():
    # |v| >= 1024 for some members (momentum sums leave the int32 split) and
    # kT = 4e6 (random velocities of a few thousand: their sums leave it too)
    s = inputs.solvent((6, 6, 6), 5, seed=12, mixed=True)
    vel = s.vel.copy()
    rng = np.random.default_rng(0)
    idx = rng.choice(len(vel), 40, replace=False)
    vel[idx] = rng.uniform(1024.0, 1500.0, (40, 3)) * rng.choice([-1.0, 1.0], (40, 3))
    vel = vel.astype(np.float32).astype(np.float64)
    for kT in (1.0, 4.0e6):
        got, want = run_at((6, 6, 6), s.pos, vel, "mixed", 2, 12, kT=kT)
        check(got, want, "mixed")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_at_solute_chains(precision):
    n = (8, 8, 8)
    s = inputs.solvent(n, 5, seed=21, mixed=precision == "mixed")
    sp, sv = inputs.chains(n, 6, 10, 0.5, bead_mass=5.0, seed=22)
    kw = dict(chain_len=10, md_substeps=10, solute_mass=5.0, bond_k=1000.0, bond_r0=0.5)
    got, want = run_at(n, s.pos, s.vel, precision, 3, 21, sp=sp, sv=sv, **kw)
    check(got, want, precision, tol64=1e-11)
    ref = want[0]
    tol = 1e-11 if precision == "fp64" else 0.0
    assert rel_err(got[3], ref.svel, m=5.0) <= tol
    assert np.max(np.abs(got[2] - ref.spos)) <= (1e-11 if precision == "fp64" else 0.0)


def test_at_and_srd_boxes_batched_equal_alone():
    specs = [((12, 9, 7), 5, "at", 201), ((5, 5, 5), 10, "srd", 202), ((16, 16, 16), 5, "at", 203)]
    states = [inputs.solvent(n, rho, seed=sd, mixed=True) for n, rho, _, sd in specs]
    batch = pkg.Batch("mixed")
    slots = [batch.add(s.pos, s.vel, n=n, seed=sd, collision=rule)
             for (n, rho, rule, sd), s in zip(specs, states)]
    batch.step(5)
    got = [batch.get_state(sl) for sl in slots]
    batch.close()
    for (n, rho, rule, sd), s, g in zip(specs, states, got):
        box = pkg.Box(n=n, seed=sd, collision=rule, precision="mixed")
        box.set_state(s.pos, s.vel)
        box.step(5)
        pos, vel, *_ = box.get_state()
        box.close()
        np.testing.assert_array_equal(pos, g[0])
        np.testing.assert_array_equal(vel, g[1])


def test_at_invalid_combinations_raise():
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(4, 4, 4), collision="at", thermostat=True)
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(4, 4, 4), collision="at", walls_z=True)
    # solute with rows above 448 records (density 400)
    kw = dict(chain_len=4, md_substeps=1, solute_mass=5.0, bond_k=10.0, bond_r0=0.5)
    box = pkg.Box(n=(2, 2, 2), collision="at", **kw)
    s = inputs.solvent((2, 2, 2), 400, seed=1, mixed=True)
    sp, sv = inputs.chains((2, 2, 2), 1, 4, 0.5, seed=2)
    with pytest.raises(pkg.MpcdError) as e:
        box.set_state(s.pos, s.vel, sp, sv)
    assert e.value.code == pkg.MPCD_EINVAL
    box.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_at_dense_rows_per_cell_kernel(precision):
    # density 400: rows of 524 records, beyond the warp-spread kernel; the
    # Andersen rule runs on the per-cell kernel, same results
    s = inputs.solvent((3, 3, 2), 400, seed=8, mixed=precision == "mixed")
    got, want = run_at((3, 3, 2), s.pos, s.vel, precision, 3, 8)
    check(got, want, precision, steps=3)


def test_at_thermalises_and_conserves_momentum():
    # a hot drifting start relaxes to kT within a few steps (AT thermostats
    # every collision); total momentum stays at its initial value
    n = (16, 16, 16)
    s = inputs.solvent(n, 10, seed=4, kT=4.0)
    vel = s.vel + np.array([0.3, 0.0, -0.1])
    box = pkg.Box(n=n, seed=4, precision="fp64", collision="at", kT=1.0)
    box.set_state(s.pos, vel)
    P0 = vel.sum(axis=0)
    box.step(50)
    ob = box.observables()
    box.close()
    assert np.allclose(ob["P"], P0, rtol=0, atol=1e-9 * np.abs(vel).sum())
    assert abs(ob["T_kin"] - 1.0) < 0.02
    assert abs(ob["T_cell_mean"] - 1.0) < 0.03
