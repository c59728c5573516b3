"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs, element by element.

Tolerances (stated per model):
  FP64  : cell ids and counts bit-exact; positions bit-exact for plain
          streaming; velocities |dv| / max(|v|, sqrt(kT/m)) <= 1e-12.
  mixed : bit-exact against the mixed-model oracle (cell ids, counts,
          positions, velocities): both sides perform the same IEEE float and
          int64 operations, including their own series sin/cos/log; with walls
          the virtual-particle draws use double libm, so those runs compare to
          2e-6.  Against the FP64 model from the same float state with float
          streaming (same cells): within the per-particle bound of
          tests/mixed_bound.py (1e-6, widened by the cell's xi with the
          thermostat).
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


def run_pair(n, rho, precision, steps=1, seed=5, step0=0, n_particles=None, oracle_precision=None,
             **kw):
    mixed = precision == "mixed"
    s = inputs.solvent(n, rho, seed=seed, mixed=mixed, n_particles=n_particles)
    box = pkg.Box(n=n, seed=seed, precision=precision, **kw)
    box.set_state(s.pos, s.vel, step=step0)
    box.step(steps)
    pos, vel, _, _, st = box.get_state()
    cells, counts = box.last_cells() if steps > 0 else (None, None)
    op = oracle_precision if oracle_precision is not None else (oracle.MIXED if mixed else oracle.FP64)
    okw = {k: v for k, v in kw.items() if k in ("thermostat", "walls_z", "g", "virt_density")}
    if "body_force" in kw:
        okw["g"] = kw["body_force"]
    if "alpha_deg" in kw:
        okw["alpha_deg"] = kw["alpha_deg"]
    p = oracle.Params(n=n, seed=seed, precision=op, **okw)
    ref = oracle.State(s.pos.copy(), s.vel.copy(), step=step0)
    rc = oracle.step(p, ref, steps, want_cells=steps > 0)
    box.close()
    return pos, vel, st, cells, counts, ref, rc


@pytest.mark.parametrize("thermostat", [False, True])
def test_fp64_one_step_10cube(thermostat):
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair((10, 10, 10), 5, "fp64",
                                                          thermostat=thermostat)
    assert st == ref.step == 1
    assert np.array_equal(cells, rc)
    assert np.array_equal(counts, rk)
    assert np.array_equal(pos, ref.pos)
    assert rel_err(vel, ref.vel) <= 1e-12


@pytest.mark.parametrize("thermostat", [False, True])
def test_mixed_one_step_10cube(thermostat):
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair((10, 10, 10), 5, "mixed",
                                                          thermostat=thermostat)
    assert np.array_equal(cells, rc)
    assert np.array_equal(counts, rk)
    assert np.array_equal(pos, ref.pos)
    assert np.array_equal(vel, ref.vel)


@pytest.mark.parametrize("thermostat", [False, True])
def test_mixed_against_fp64_oracle(thermostat):
    from mixed_bound import mixed_step_bound, rel_errors
    n = (10, 10, 10)
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair(
        n, 5, "mixed", thermostat=thermostat, oracle_precision=oracle.FP64_FSTREAM)
    assert np.array_equal(cells, rc)
    assert np.array_equal(pos, ref.pos)
    s = inputs.solvent(n, 5, seed=5, mixed=True)
    bound, _ = mixed_step_bound(s.vel, ref.vel, rc, thermostat=thermostat)
    assert np.all(rel_errors(vel, ref.vel) <= bound)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ragged_sizes_many_tiles(precision):
    # 23 x 17 x 9 cells, an odd particle count: several stream tiles and
    # collision tiles with a ragged tail, and a start step off zero.
    tol = 1e-12 if precision == "fp64" else 2e-6
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair(
        (23, 17, 9), 7.3, precision, steps=3, thermostat=True, step0=123456789012,
        n_particles=25699)
    assert st == ref.step
    assert np.array_equal(cells, rc)
    assert np.array_equal(counts, rk)
    if precision == "mixed":
        assert np.array_equal(vel, ref.vel) and np.array_equal(pos, ref.pos)
    assert rel_err(vel, ref.vel) <= tol * 3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_step_trajectory_with_reorders(precision):
    # 40 steps with a reorder every 7 steps: the trajectory still matches
    # (bit for bit in the mixed model).
    tol = 1e-11 if precision == "fp64" else 1e-5
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair(
        (12, 12, 12), 5, precision, steps=40, thermostat=True, sort_period=7, seed=9)
    assert st == 40
    assert np.array_equal(cells, rc)
    if precision == "mixed":
        assert np.array_equal(vel, ref.vel) and np.array_equal(pos, ref.pos)
    assert rel_err(vel, ref.vel) <= tol
    L = 12.0
    d = np.abs(pos - ref.pos)
    d = np.minimum(d, L - d)
    assert d.max() <= (1e-11 if precision == "fp64" else 1e-4)


def test_sort_period_does_not_change_mixed_results():
    """Fixed-point cell sums are order independent: any reorder schedule gives
    bit-identical trajectories."""
    s = inputs.solvent((9, 8, 7), 6, seed=4, mixed=True)
    outs = []
    for sp in (-1, 1, 3, 25):
        box = pkg.Box(n=(9, 8, 7), seed=4, precision="mixed", thermostat=True, sort_period=sp)
        box.set_state(s.pos, s.vel)
        box.step(15)
        outs.append(box.get_state()[:2])
        box.close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_walls_and_body_force(precision):
    tol = 1e-12 if precision == "fp64" else 2e-6
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair(
        (6, 5, 8), 10, precision, steps=4, thermostat=True, walls_z=True,
        body_force=(0.01, 0.0, 0.0), virt_density=10.0, seed=13)
    assert np.array_equal(cells, rc)
    assert np.array_equal(counts, rk)
    assert rel_err(vel, ref.vel) <= tol * 4
    assert np.all((pos[:, 2] >= 0) & (pos[:, 2] < 8))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_clustered_input_takes_cooperative_path(precision):
    """All particles in a few cells: tiles overflow the shared-memory capacity
    and take the block-cooperative path; results still match."""
    rng = np.random.default_rng(2)
    N = 40000
    pos = np.full((N, 3), 2.55) + rng.random((N, 3)) * 0.2  # the 0.2 wide cluster stays
    pos[: N // 3, 0] += 3.0                                   # within one cell per axis
    vel = rng.standard_normal((N, 3))
    vel -= vel.mean(0)
    if precision == "mixed":
        pos = pos.astype(np.float32).astype(np.float64)
        vel = vel.astype(np.float32).astype(np.float64)
    box = pkg.Box(n=(8, 8, 8), seed=3, precision=precision, thermostat=True)
    box.set_state(pos, vel)
    box.step(1)  # one step: the cluster has not spread yet
    p2, v2, *_ = box.get_state()
    cells, counts = box.last_cells()
    box.close()
    ref = oracle.State(pos.copy(), vel.copy())
    rc, rk = oracle.step(oracle.Params(n=(8, 8, 8), seed=3, thermostat=True,
                                       precision=oracle.MIXED if precision == "mixed" else oracle.FP64),
                         ref, 1, want_cells=True)
    assert counts.max() > 4096  # above every tile capacity
    assert np.array_equal(cells, rc)
    assert rel_err(v2, ref.vel) <= (1e-12 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("steps", [1, 3])
def test_rows_overflowing_by_a_few(precision, steps):
    """Tight clusters push some cells a few members past the row capacity (36
    at density 10), three of them in one warp's span: their extra members go
    to the overflow list and come back through it.  Results match the
    oracle."""
    rng = np.random.default_rng(11)
    n = (16, 16, 16)
    s = inputs.solvent(n, 10, seed=12, mixed=precision == "mixed")
    cells = [tuple(c) for c in rng.integers(0, 16, size=(40, 3))]
    cells += [(4, 9, 9), (5, 9, 9), (6, 9, 9)]  # one warp's span, 3 x 40 extra members
    extra_p, extra_v = [], []
    for k, c in enumerate(cells):
        m = 40 if k >= 40 else int(rng.integers(20, 41))
        extra_p.append(np.array(c, float) + 0.45 + 0.1 * rng.random((m, 3)))
        extra_v.append(0.1 * rng.standard_normal((m, 3)))  # slow: the cluster holds
    pos = np.vstack([s.pos] + extra_p)
    vel = np.vstack([s.vel] + extra_v)
    if precision == "mixed":
        pos = pos.astype(np.float32).astype(np.float64)
        vel = vel.astype(np.float32).astype(np.float64)
    box = pkg.Box(n=n, seed=12, precision=precision, thermostat=True)
    box.set_state(pos, vel)
    box.step(steps)
    p2, v2, *_ = box.get_state()
    got_cells, counts = box.last_cells()
    box.close()
    ref = oracle.State(pos.copy(), vel.copy())
    rc, rk = oracle.step(oracle.Params(n=n, seed=12, thermostat=True,
                                       precision=oracle.MIXED if precision == "mixed" else oracle.FP64),
                         ref, steps, want_cells=True)
    # the first collision's cells (one stream of dt = 0.1, grid shift of step
    # 0) hold clustered cells beyond the row capacity
    r1 = np.mod(pos + 0.1 * vel, 16.0)
    c1 = np.mod(np.floor(r1 - oracle.shift(12, 0)), 16).astype(np.int64)
    k1 = np.bincount(c1[:, 0] + 16 * (c1[:, 1] + 16 * c1[:, 2]), minlength=4096)
    assert k1.max() > 36
    assert np.array_equal(got_cells, rc)
    assert np.array_equal(counts, rk)
    if precision == "mixed":
        assert np.array_equal(p2, ref.pos) and np.array_equal(v2, ref.vel)
    else:
        d = np.abs(p2 - ref.pos)
        assert np.minimum(d, 16.0 - d).max() <= 1e-12
        assert rel_err(v2, ref.vel) <= 1e-12 * steps


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases_empty_single_and_one_cell_box(precision):
    # empty state
    box = pkg.Box(n=(3, 3, 3), precision=precision)
    box.set_state(np.zeros((0, 3)), np.zeros((0, 3)))
    box.step(3)
    pos, vel, *_ , st = box.get_state()
    assert pos.shape == (0, 3) and st == 3
    box.close()
    # a single particle keeps its velocity (to rounding) and streams
    box = pkg.Box(n=(3, 3, 3), precision=precision, seed=2)
    box.set_state(np.array([[1.5, 1.5, 1.5]]), np.array([[0.5, -0.25, 1.0]]))
    box.step(4)
    pos, vel, *_ = box.get_state()
    assert np.allclose(vel, [[0.5, -0.25, 1.0]], atol=1e-6)
    assert np.allclose(pos, [[1.7, 1.4, 1.9]], atol=1e-5)
    box.close()
    # a 1 x 1 x 1 box: one cell, every particle collides with all others
    s = inputs.solvent((1, 1, 1), 50, seed=8, mixed=precision == "mixed")
    box = pkg.Box(n=(1, 1, 1), precision=precision, seed=8, thermostat=True)
    box.set_state(s.pos, s.vel)
    box.step(5)
    _, vel, *_ = box.get_state()
    box.close()
    ref = oracle.State(s.pos.copy(), s.vel.copy())
    oracle.step(oracle.Params(n=(1, 1, 1), seed=8, thermostat=True,
                              precision=oracle.MIXED if precision == "mixed" else oracle.FP64), ref, 5)
    assert rel_err(vel, ref.vel) <= (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solute_chains(precision):
    n = (8, 8, 8)
    s = inputs.solvent(n, 5, seed=21, mixed=precision == "mixed")
    sp, sv = inputs.chains(n, 6, 10, 0.5, bead_mass=5.0, seed=22)
    kw = dict(chain_len=10, md_substeps=10, solute_mass=5.0, bond_k=1000.0, bond_r0=0.5)
    box = pkg.Box(n=n, seed=21, precision=precision, thermostat=True, **kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(3)
    pos, vel, spos, svel, st = box.get_state()
    cells, counts = box.last_cells()
    box.close()
    p = oracle.Params(n=n, seed=21, thermostat=True,
                      precision=oracle.MIXED if precision == "mixed" else oracle.FP64, **kw)
    ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy())
    rc, rk = oracle.step(p, ref, 3, want_cells=True)
    assert np.array_equal(cells, rc)
    assert np.array_equal(counts, rk)
    tol = 1e-11 if precision == "fp64" else 3e-6
    assert rel_err(vel, ref.vel) <= tol
    assert rel_err(svel, ref.svel, m=5.0) <= tol
    assert np.max(np.abs(spos - ref.spos)) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solute_many_chains_over_blocks(precision):
    # 701 chains of 10 beads: two chains per MD block, the last block with
    # one; every bond force is computed once and shared by its two beads
    n = (20, 20, 20)
    s = inputs.solvent(n, 5, seed=41, mixed=precision == "mixed")
    sp, sv = inputs.chains(n, 701, 10, 0.5, bead_mass=5.0, seed=42)
    kw = dict(chain_len=10, md_substeps=10, solute_mass=5.0, bond_k=1000.0, bond_r0=0.5)
    box = pkg.Box(n=n, seed=41, precision=precision, **kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(2)
    pos, vel, spos, svel, st = box.get_state()
    cells, counts = box.last_cells()
    box.close()
    p = oracle.Params(n=n, seed=41, precision=oracle.MIXED if precision == "mixed" else oracle.FP64,
                      **kw)
    ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy())
    rc, rk = oracle.step(p, ref, 2, want_cells=True)
    assert np.array_equal(cells, rc)
    assert np.array_equal(counts, rk)
    if precision == "mixed":
        assert np.array_equal(vel, ref.vel)
        assert rel_err(svel, ref.svel, m=5.0) == 0.0
    else:
        assert rel_err(vel, ref.vel) <= 2e-11
        assert rel_err(svel, ref.svel, m=5.0) <= 2e-11
    assert np.max(np.abs(spos - ref.spos)) <= 1e-11


def test_solute_longest_chain():
    # one chain of 1024 beads, the longest allowed: one block of 1024 threads
    # whose positions, bond forces and flags take 53,248 bytes of shared memory
    n = (12, 12, 12)
    s = inputs.solvent(n, 5, seed=43, mixed=True)
    sp, sv = inputs.chains(n, 1, 1024, 0.5, bead_mass=5.0, seed=44)
    kw = dict(chain_len=1024, md_substeps=5, solute_mass=5.0, bond_k=1000.0, bond_r0=0.5)
    box = pkg.Box(n=n, seed=43, precision="mixed", **kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(2)
    pos, vel, spos, svel, st = box.get_state()
    box.close()
    p = oracle.Params(n=n, seed=43, precision=oracle.MIXED, **kw)
    ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy())
    oracle.step(p, ref, 2)
    assert np.array_equal(vel, ref.vel)
    assert rel_err(svel, ref.svel, m=5.0) == 0.0
    assert np.max(np.abs(spos - ref.spos)) <= 1e-11


def test_observables_match_oracle():
    s = inputs.solvent((10, 10, 10), 10, seed=6)
    box = pkg.Box(n=(10, 10, 10), seed=6, precision="fp64", thermostat=True)
    box.set_state(s.pos, s.vel)
    box.step(5)
    ob = box.observables()
    pos, vel, *_ = box.get_state()
    box.close()
    ref = oracle.observables(oracle.Params(n=(10, 10, 10)), oracle.State(pos, vel))
    assert np.allclose(ob["P"], ref["P"], atol=1e-9)
    assert abs(ob["KE"] - ref["KE"]) <= 1e-10 * ref["KE"]
    assert abs(ob["T_kin"] - ref["T_kin"]) <= 1e-10
    assert abs(ob["T_cell_mean"] - ref["T_cell_mean"]) <= 1e-8
    assert ob["occupied_cells"] == ref["occupied_cells"]
    assert ob["step"] == 5


def test_batch_boxes_equal_alone():
    """Boxes of different size, density, angle and seed stepped together give
    bit-identical results to each box alone (mixed model)."""
    specs = [((12, 9, 7), 5, 90.0, 101), ((5, 5, 5), 10, 120.0, 102), ((16, 16, 16), 5, 130.0, 103)]
    states = [inputs.solvent(n, rho, seed=sd, mixed=True) for n, rho, _, sd in specs]
    batch = pkg.Batch("mixed")
    slots = []
    for (n, rho, ang, sd), s in zip(specs, states):
        slots.append(batch.add(s.pos, s.vel, n=n, alpha_deg=ang, seed=sd, thermostat=(sd % 2 == 1)))
    batch.step(6)
    got = [batch.get_state(sl) for sl in slots]
    # remove the middle box and keep stepping the others
    batch.remove(slots[1])
    batch.step(4)
    got_after = [batch.get_state(slots[0]), batch.get_state(slots[2])]
    batch.close()
    for (n, rho, ang, sd), s, g in zip(specs, states, got):
        box = pkg.Box(n=n, alpha_deg=ang, seed=sd, thermostat=(sd % 2 == 1), precision="mixed")
        box.set_state(s.pos, s.vel)
        box.step(6)
        pos, vel, *_ = box.get_state()
        assert np.array_equal(pos, g[0]) and np.array_equal(vel, g[1]) and g[2] == 6
        if sd != 102:
            box.step(4)
            pos, vel, *_ = box.get_state()
            ga = got_after[0 if sd == 101 else 1]
            assert np.array_equal(pos, ga[0]) and np.array_equal(vel, ga[1]) and ga[2] == 10
        box.close()


def test_invalid_arguments_raise():
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(0, 4, 4))
    box = pkg.Box(n=(4, 4, 4))
    with pytest.raises(pkg.MpcdError) as e:
        box.step(1)
    assert e.value.code == pkg.MPCD_ESTATE
    box.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_profile_matches_oracle(precision):
    """mpcd_profile (mean solvent v_x per z slab) against the oracle's profile of
    the same state, in a body-force channel."""
    n = (6, 5, 12)
    s = inputs.solvent(n, 10, seed=17, mixed=precision == "mixed")
    box = pkg.Box(n=n, seed=17, precision=precision, thermostat=True, walls_z=True,
                  body_force=(0.02, 0.0, 0.0), virt_density=10.0)
    box.set_state(s.pos, s.vel)
    box.step(30)
    prof = box.profile(24)
    pos, vel, *_ = box.get_state()
    box.close()
    ref = oracle.profile(oracle.Params(n=n), oracle.State(pos, vel), 24)
    assert np.allclose(prof, ref, rtol=0, atol=1e-12)
    assert prof[12] > 0.0  # the body force drives +x flow in the middle of the channel


@pytest.mark.parametrize("thermostat", [False, True])
def test_mixed_dense_box_many_steps(thermostat):
    """20^3 cells at 12 per cell (rows of 40 records, several member windows
    per warp), 12 steps: bit-exact against the mixed oracle."""
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair((20, 20, 20), 12, "mixed", steps=12,
                                                          seed=31, thermostat=thermostat)
    assert st == 12
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_array_equal(counts, rk)
    np.testing.assert_array_equal(pos, ref.pos)
    np.testing.assert_array_equal(vel, ref.vel)


def test_mixed_large_velocities_exact():
    """Members with |v| >= 1024 leave the int32 split of the fixed-point sums
    and take the exact int64 path: results stay bit-exact."""
    n = (6, 6, 6)
    s = inputs.solvent(n, 5, seed=12, mixed=True)
    vel = s.vel.copy()
    rng = np.random.default_rng(0)
    idx = rng.choice(len(vel), 40, replace=False)
    vel[idx] = rng.uniform(1024.0, 1500.0, (40, 3)) * rng.choice([-1.0, 1.0], (40, 3))
    vel = vel.astype(np.float32).astype(np.float64)
    for thermostat in (False, True):
        box = pkg.Box(n=n, seed=12, precision="mixed", thermostat=thermostat)
        box.set_state(s.pos, vel)
        box.step(2)
        pos, v, _, _, _ = box.get_state()
        box.close()
        ref = oracle.State(s.pos.copy(), vel.copy())
        oracle.step(oracle.Params(n=n, seed=12, thermostat=thermostat, precision=oracle.MIXED), ref, 2)
        np.testing.assert_array_equal(pos, ref.pos)
        np.testing.assert_array_equal(v, ref.vel)


@pytest.mark.parametrize("rho", [320, 340])
def test_mixed_row_capacity_limits(rho):
    """Rows of 432 records (the largest the warp-spread kernel takes) and of
    456 (handled by the per-cell kernel): both bit-exact."""
    pos, vel, st, cells, counts, ref, (rc, rk) = run_pair((3, 3, 3), rho, "mixed", steps=3,
                                                          seed=40, thermostat=True)
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_array_equal(counts, rk)
    np.testing.assert_array_equal(pos, ref.pos)
    np.testing.assert_array_equal(vel, ref.vel)


def test_launch_tuner_keeps_results():
    """mpcd_tune runs real steps under every candidate (grid x cells per warp
    and pass-2 chunk depth: 32 cells with 2, 3, 4 windows, 16 and 8 cells with
    3) and keeps the fastest; the trajectory is bit-identical to plain steps
    (mixed model)."""
    s = inputs.solvent((24, 24, 24), 10, seed=51, mixed=True)
    a = pkg.Box(n=(24, 24, 24), seed=51, precision="mixed", thermostat=True)
    a.set_state(s.pos, s.vel)
    bps, ms, taken, chunk, cpw = a.tune(1)
    assert bps == -1 or bps >= 1
    assert chunk in (2, 3, 4)
    assert cpw in (8, 16, 32) and (cpw == 32 or chunk == 3)
    assert ms > 0.0 and taken >= 2
    a.step(3)
    pa, va, *_, sta = a.get_state()
    a.close()
    b = pkg.Box(n=(24, 24, 24), seed=51, precision="mixed", thermostat=True)
    b.set_state(s.pos, s.vel)
    b.step(taken + 3)
    pb, vb, *_, stb = b.get_state()
    b.close()
    assert sta == stb == taken + 3
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)


@pytest.mark.parametrize("case", ["beads", "ragged_force"])
def test_launch_tuner_cells_per_warp_keeps_results(case):
    """The tuner's candidates with 16 and 8 cells per warp (a 256-cell span
    taken in 2 or 4 parts; lanes without a cell) on the paths they change:
    solute beads (a warp takes only its own cells' beads from the 32-cell bead
    group) and a ragged box (23 x 17 x 9 cells, the last span part partly or
    wholly beyond the grid) with a body force.  Every candidate advances real
    steps; the trajectory equals plain steps bit for bit, beads included."""
    if case == "beads":
        n, rho, seed = (16, 16, 16), 5, 61
        kw = dict(chain_len=10, md_substeps=5, solute_mass=5.0, bond_k=300.0, bond_r0=0.5)
        s = inputs.solvent(n, rho, seed=seed, mixed=True)
        sp, sv = inputs.chains(n, 40, 10, 0.5, bead_mass=5.0, seed=seed + 1)
        box_kw = dict(thermostat=True, **kw)
    else:
        n, rho, seed = (23, 17, 9), 7, 62
        s = inputs.solvent(n, rho, seed=seed, mixed=True)
        sp = sv = None
        box_kw = dict(thermostat=False, body_force=(0.01, -0.02, 0.005))
    a = pkg.Box(n=n, seed=seed, precision="mixed", **box_kw)
    a.set_state(s.pos, s.vel, sp, sv)
    bps, ms, taken, chunk, cpw = a.tune(2)
    assert cpw in (8, 16, 32)
    a.step(3)
    ra = a.get_state()
    a.close()
    b = pkg.Box(n=n, seed=seed, precision="mixed", **box_kw)
    b.set_state(s.pos, s.vel, sp, sv)
    b.step(taken + 3)
    rb = b.get_state()
    b.close()
    assert ra[4] == rb[4] == taken + 3
    for x, y in zip(ra[:4], rb[:4]):
        if x is not None:
            np.testing.assert_array_equal(x, y)
