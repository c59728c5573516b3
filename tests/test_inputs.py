"""The seeded input generators (CPU): what the recipe promises about each
state, checked directly, so that both sides of every parity test start from
what the paper's benchmark set-up describes (Sec. 4, Sec. 4.1)."""
import numpy as np
import pytest

from paper_1801_10187_gb300 import inputs


def min_image(d, L):
    return d - L * np.rint(d / L)


@pytest.mark.parametrize("mixed", [False, True])
def test_solvent_recipe(mixed):
    n = (7, 5, 6)
    s = inputs.solvent(n, 4.5, kT=2.0, seed=3, mixed=mixed)
    L = np.array(n, dtype=float)
    assert s.pos.shape == s.vel.shape == (int(round(4.5 * 7 * 5 * 6)), 3)
    assert np.all(s.pos >= 0.0) and np.all(s.pos < L)
    # zero net momentum: exactly up to the rounding of the mean subtraction,
    # and of the float rounding in the mixed model
    tol = 1e-12 if not mixed else 2.0**-24 * np.abs(s.vel).sum(axis=0).max()
    assert np.all(np.abs(s.vel.sum(axis=0)) <= tol * (1 if mixed else len(s.vel)))
    # variance kT/m per component
    assert np.allclose(s.vel.var(axis=0), 2.0, rtol=0.15)
    if mixed:
        assert np.array_equal(s.pos.astype(np.float32).astype(np.float64), s.pos)
        assert np.array_equal(s.vel.astype(np.float32).astype(np.float64), s.vel)
        assert np.all(s.pos.astype(np.float32) < L.astype(np.float32))
    # the same seed gives the same state, another seed another
    t = inputs.solvent(n, 4.5, kT=2.0, seed=3, mixed=mixed)
    assert np.array_equal(s.pos, t.pos) and np.array_equal(s.vel, t.vel)
    u = inputs.solvent(n, 4.5, kT=2.0, seed=4, mixed=mixed)
    assert not np.array_equal(s.pos, u.pos)


def test_solvent_particle_count_override_and_empty():
    s = inputs.solvent((4, 4, 4), 5, seed=1, n_particles=17)
    assert s.pos.shape == (17, 3)
    e = inputs.solvent((4, 4, 4), 5, seed=1, n_particles=0)
    assert e.pos.shape == (0, 3) and e.vel.shape == (0, 3)


def test_chains_recipe():
    n = (6, 7, 8)
    L = np.array(n, dtype=float)
    sp, sv = inputs.chains(n, 9, 12, 0.5, kT=1.0, bead_mass=5.0, seed=2)
    assert sp.shape == sv.shape == (108, 3)
    assert np.all(sp >= 0.0) and np.all(sp < L)
    bonds = sp.reshape(9, 12, 3)
    d = min_image(bonds[:, 1:] - bonds[:, :-1], L)
    assert np.allclose(np.linalg.norm(d, axis=2), 0.5, rtol=0, atol=1e-12)
    assert np.all(np.abs(sv.sum(axis=0)) <= 1e-12 * len(sv))
    assert np.allclose(sv.var(axis=0), 1.0 / 5.0, rtol=0.35)


def test_avoiding_chains_keep_their_distance():
    n = (5, 5, 5)
    L = np.array(n, dtype=float)
    sp, sv = inputs.avoiding_chains(n, 6, 10, 0.5, 0.45, bead_mass=5.0, seed=7)
    assert sp.shape == sv.shape == (60, 3)
    assert np.all(sp >= 0.0) and np.all(sp < L)
    bonds = sp.reshape(6, 10, 3)
    d = min_image(bonds[:, 1:] - bonds[:, :-1], L)
    assert np.allclose(np.linalg.norm(d, axis=2), 0.5, rtol=0, atol=1e-12)
    # every pair of beads (brute force, minimum image) at least min_dist apart
    dd = min_image(sp[:, None, :] - sp[None, :, :], L)
    r = np.linalg.norm(dd, axis=2)
    r[np.arange(60), np.arange(60)] = np.inf
    assert r.min() >= 0.45 - 1e-12


def test_ensemble_recipe_ranges():
    specs = inputs.ensemble(64, seed=4)
    assert len(specs) == 64
    for i, s in enumerate(specs):
        e = s["n"][0]
        assert s["n"] == (e, e, e) and 16 <= e <= 96
        assert s["density"] in (5, 10)
        assert s["alpha_deg"] in (90.0, 120.0, 130.0)
        assert s["seed"] == 1000 + i
    assert specs == inputs.ensemble(64, seed=4)


def test_box_workloads_name_their_parameters():
    for name, cfg in inputs.WORKLOADS.items():
        if cfg.get("kind", "box") != "box":
            continue
        for key in ("n", "density", "alpha_deg", "dt", "kT", "seed", "thermostat", "precision"):
            assert key in cfg, (name, key)
        assert cfg["precision"] in ("mixed", "fp64")
        if cfg.get("n_chains"):
            for key in ("chain_len", "bead_mass", "bond_k", "bond_r0", "md_substeps"):
                assert key in cfg, (name, key)
