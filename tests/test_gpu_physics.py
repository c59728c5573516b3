"""Physics of the CUDA path at sizes the oracle cannot reach in seconds.

1. Poiseuille flow between bounce-back walls (body force g along x): the
   time-averaged profile v_x(z) is the parabola rho g z (H - z) / (2 eta), and
   its curvature recovers the closed-form SRD viscosity (8.70 at density 10,
   alpha = 130 deg, dt = 0.1, the paper's benchmark fluid, Sec. 4) within 3%.
   Channel H = 20, L_x = L_y = 50 (5 * 10^5 particles), as a narrow gap keeps
   the start-up transient short.
2. Momentum drift of the mixed model (FP32 particles, float rotation about the
   fixed-point u): over 2000 steps of a 10^5-particle box without thermostat,
   |sum P(t) - sum P(0)| / sum m |v| stays below 1e-7 (printed; the paper's
   concern with float rotations, Sec. 4.1).
3. Energy of the thermostatted mixed model: the kinetic temperature relaxes
   to kT from a hot start.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1801_10187_gb300 as pkg  # noqa: E402
from paper_1801_10187_gb300 import inputs  # noqa: E402


def eta_closed_form(rho, alpha, dt, kT=1.0, m=1.0):
    # kinetic + collisional SRD viscosity with random grid shift (a = 1)
    f = rho - 1.0 + math.exp(-rho)
    ca, c2a = math.cos(alpha), math.cos(2 * alpha)
    eta_kin = rho * kT * dt * (5 * rho / (f * (4 - 2 * ca - 2 * c2a)) - 0.5)
    eta_col = m / (18 * dt) * f * (1 - ca)
    return eta_kin + eta_col


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_poiseuille_viscosity(precision):
    rho, g, H, L = 10.0, 0.005, 20, 50
    n = (L, L, H)
    box = pkg.Box(n=n, precision=precision, walls_z=True, thermostat=True,
                  body_force=(g, 0.0, 0.0), virt_density=rho, seed=21)
    box.set_state_thermal(int(rho * L * L * H), init_seed=21)
    box.step(3000)  # start-up: slowest mode decays in about 470 steps
    nb, chunk, nrep = 40, 10, 500
    prof = np.zeros(nb)
    for _ in range(nrep):
        box.step(chunk)
        prof += box.profile(nb)
    prof /= nrep
    z = (np.arange(nb) + 0.5) * H / nb
    X = np.stack([z * (H - z), np.ones_like(z)], axis=1)
    (A, B), *_ = np.linalg.lstsq(X, prof, rcond=None)
    eta_fit = rho * g / (2 * A)
    eta_th = eta_closed_form(rho, math.radians(130.0), 0.1)
    print(f"\n{precision}: eta fit {eta_fit:.3f}, closed form {eta_th:.3f}, slip {B:.4f}")
    assert abs(eta_fit / eta_th - 1) < 0.03, (eta_fit, eta_th)
    assert abs(B) < 0.05 * prof.max()
    box.close()


def test_mixed_momentum_drift():
    n, rho = (22, 22, 22), 10
    s = inputs.solvent(n, rho, seed=8, mixed=True)
    box = pkg.Box(n=n, precision="mixed", seed=8)
    box.set_state(s.pos, s.vel)
    p0 = box.observables()["P"]
    scale = np.abs(s.vel).sum()  # sum m |v| over components, m = 1
    drift = []
    for _ in range(4):
        box.step(500)
        drift.append(np.abs(box.observables()["P"] - p0).max() / scale)
    box.close()
    print(f"\nmixed momentum drift after 500..2000 steps: {['%.2e' % d for d in drift]}")
    assert max(drift) < 1e-7


def test_thermostat_relaxes_hot_start():
    n, rho = (16, 16, 16), 10
    s = inputs.solvent(n, rho, kT=4.0, seed=9, mixed=True)
    box = pkg.Box(n=n, precision="mixed", thermostat=True, kT=1.0, seed=9)
    box.set_state(s.pos, s.vel)
    assert box.observables()["T_kin"] > 3.5
    box.step(200)
    t = [box.observables()["T_kin"]]
    for _ in range(4):
        box.step(50)
        t.append(box.observables()["T_kin"])
    box.close()
    assert abs(np.mean(t) - 1.0) < 0.01, t
