"""Thermal initial states drawn on the device, and the continuous-batching
server: every job's result is the same served in the mix as run alone
(bit-exact in the mixed model, whose draws are keyed by seed, step and cell)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1801_10187_gb300 as pkg  # noqa: E402
from paper_1801_10187_gb300 import serve  # noqa: E402


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_thermal_state_statistics(precision):
    n, npart, kT = (20, 16, 12), 200_000, 1.5
    box = pkg.Box(n=n, precision=precision, kT=kT, seed=3)
    box.set_state_thermal(npart, init_seed=77)
    pos, vel, _, _, st = box.get_state()
    box.close()
    assert st == 0 and pos.shape == (npart, 3)
    L = np.array(n, dtype=float)
    assert (pos >= 0).all() and (pos < L).all()
    np.testing.assert_allclose(pos.mean(axis=0) / L, 0.5, atol=0.005)
    # total momentum removed (to the fixed-point rounding of the mean)
    assert np.abs(vel.mean(axis=0)).max() < (1e-6 if precision == "mixed" else 1e-9)
    var = vel.var(axis=0)
    np.testing.assert_allclose(var, kT, rtol=0.02)
    # Gaussian fourth moment: <v^4> = 3 sigma^4
    np.testing.assert_allclose((vel ** 4).mean(axis=0), 3 * kT * kT, rtol=0.05)
    # reproducible
    box2 = pkg.Box(n=n, precision=precision, kT=kT, seed=3)
    box2.set_state_thermal(npart, init_seed=77)
    p2, v2, _, _, _ = box2.get_state()
    box2.close()
    np.testing.assert_array_equal(pos, p2)
    np.testing.assert_array_equal(vel, v2)


def test_batch_add_thermal_equals_box():
    kw = dict(n=(9, 7, 5), alpha_deg=120.0, thermostat=True, seed=11, precision="mixed")
    box = pkg.Box(**kw)
    box.set_state_thermal(3000, init_seed=5)
    box.step(13)
    p1, v1, _, _, s1 = box.get_state()
    box.close()
    b = pkg.Batch("mixed")
    other = b.add_thermal(5000, init_seed=6, n=(11, 11, 11), seed=12)
    slot = b.add_thermal(3000, init_seed=5, **kw)
    b.step(13)
    p2, v2, s2 = b.get_state(slot)
    assert other != slot
    b.close()
    assert s1 == s2 == 13
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(v1, v2)


def test_server_results_equal_alone():
    jobs = serve.poisson_jobs(14, rate=1000.0, seed=9, l_min=4, l_max=14, steps_min=5,
                              steps_max=70, density=5.0)
    big = sorted(jobs, key=lambda j: -j.particles)[:3]
    srv = serve.Server(precision="mixed", max_chunk=16, keep_state=True,
                       max_bytes=sum(pkg.box_footprint(j.particles, precision="mixed",
                                                       **j.box_kwargs()) for j in big))
    stats = srv.run(jobs, realtime=False)
    srv.close()
    assert stats.jobs == len(jobs) and len(stats.latency_s) == len(jobs)
    assert stats.chunks > 1 and stats.max_resident > 1
    assert stats.particle_steps == sum(j.particles * j.steps for j in jobs)
    for j in jobs:
        box = pkg.Box(precision="mixed", **j.box_kwargs())
        box.set_state_thermal(j.particles, init_seed=j.seed)
        box.step(j.steps)
        p, v, _, _, st = box.get_state()
        obs = box.observables()
        box.close()
        jp, jv, jst = j.state
        assert jst == st == j.steps
        np.testing.assert_array_equal(jp, p)
        np.testing.assert_array_equal(jv, v)
        assert math.isclose(j.result["T_kin"], obs["T_kin"], rel_tol=1e-12)
