"""GPU parity of the non-bonded solute repulsion (WCA between every pair of
beads, Sec. 4.3 reading) against the oracle, which visits every pair.  Beads
are double in both models: FP64 and mixed runs compare bead states within
1e-10 and the solvent as the solute parity tests do.
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

KW = dict(md_substeps=20, solute_mass=5.0, bond_k=300.0, bond_r0=0.5, lj_epsilon=1.0,
          lj_sigma=0.5)


def rel_err(v, ref, kT=1.0, m=1.0):
    scale = np.maximum(np.linalg.norm(ref, axis=1), math.sqrt(kT / m))
    return (np.linalg.norm(v - ref, axis=1) / scale).max(initial=0.0)


def run(n, rho, nch, cl, precision, steps, seed, thermostat=False, min_dist=0.45, **extra):
    kw = dict(KW, chain_len=cl, **extra)
    s = inputs.solvent(n, rho, seed=seed, mixed=precision == "mixed")
    sp, sv = inputs.avoiding_chains(n, nch, cl, 0.5, min_dist, bead_mass=5.0, seed=seed + 1)
    box = pkg.Box(n=n, seed=seed, precision=precision, thermostat=thermostat, **kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(steps)
    pos, vel, spos, svel, st = box.get_state()
    box.close()
    p = oracle.Params(n=n, seed=seed, thermostat=thermostat,
                      precision=oracle.MIXED if precision == "mixed" else oracle.FP64, **kw)
    ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy())
    oracle.step(p, ref, steps)
    return (pos, vel, spos, svel, st), ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("thermostat", [False, True])
def test_wca_chains_match_oracle(precision, thermostat):
    (pos, vel, spos, svel, st), ref = run((8, 8, 8), 5, 12, 12, precision, 3, 31, thermostat)
    assert st == 3
    d = np.abs(spos - ref.spos)
    d = np.minimum(d, 8.0 - d)
    assert d.max() <= 1e-10
    assert rel_err(svel, ref.svel, m=5.0) <= 1e-10
    tol = 1e-11 if precision == "fp64" else 3e-6
    assert rel_err(vel, ref.vel) <= tol


def test_wca_dense_chains_many_neighbours():
    # 40 chains of 20 beads in a 6^3 box, no two beads closer than sigma:
    # beads at 3.7 per unit volume, about 14 list entries per bead
    (pos, vel, spos, svel, st), ref = run((6, 6, 6), 3, 40, 20, "fp64", 2, 7, min_dist=0.5)
    d = np.abs(spos - ref.spos)
    d = np.minimum(d, 6.0 - d)
    assert d.max() <= 1e-9
    assert rel_err(svel, ref.svel, m=5.0) <= 1e-9


def test_wca_off_is_the_plain_solute_path():
    # lj_epsilon = 0 takes the bonds-only MD kernel; same box with the
    # repulsion on differs from it and each matches its oracle
    n = (8, 8, 8)
    out = []
    for eps in (0.0, 1.0):
        kw = dict(KW, chain_len=10, lj_epsilon=eps)
        s = inputs.solvent(n, 5, seed=41)
        sp, sv = inputs.avoiding_chains(n, 6, 10, 0.5, 0.45, seed=41)
        box = pkg.Box(n=n, seed=41, precision="fp64", **kw)
        box.set_state(s.pos, s.vel, sp, sv)
        box.step(3)
        g = box.get_state()
        box.close()
        p = oracle.Params(n=n, seed=41, precision=oracle.FP64, **kw)
        ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy())
        oracle.step(p, ref, 3)
        assert rel_err(g[3], ref.svel, m=5.0) <= 1e-10
        out.append(g[3])
    assert np.max(np.abs(out[0] - out[1])) > 1e-3


def test_wca_fast_bead_rebuilds_the_list():
    # a bead moving 4 cells per collision step outruns the 0.4 buffer within
    # the step; the list is rebuilt where needed and the result still matches
    n = (6, 6, 6)
    kw = dict(KW, chain_len=5)
    s = inputs.solvent(n, 3, seed=2)
    sp, sv = inputs.avoiding_chains(n, 4, 5, 0.5, 0.45, seed=3)
    sv = sv.copy()
    sv[0] = [40.0, 0.0, 0.0]
    box = pkg.Box(n=n, seed=2, precision="fp64", **kw)
    box.set_state(s.pos, s.vel, sp, sv)
    box.step(2)
    g = box.get_state()
    box.close()
    p = oracle.Params(n=n, seed=2, precision=oracle.FP64, **kw)
    ref = oracle.State(s.pos.copy(), s.vel.copy(), sp.copy(), sv.copy())
    oracle.step(p, ref, 2)
    assert rel_err(g[3], ref.svel, m=5.0) <= 1e-9
    d = np.abs(g[2] - ref.spos)
    assert np.minimum(d, 6.0 - d).max() <= 1e-9


def test_wca_invalid_parameters():
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(8, 8, 8), **dict(KW, chain_len=5, lj_sigma=0.6))  # cutoff + buffer > 1
    with pytest.raises(pkg.MpcdError):
        pkg.Box(n=(2, 8, 8), **dict(KW, chain_len=5))  # fewer than 3 cells on an axis
