"""Viscosity pin of the oracle (CPU only, about 20 s).

The paper prints the viscosity of its benchmark fluid: 8.7 (epsilon tau/a^3)
at density 10, alpha = 130 deg, dt = 0.1, kT = 1 (Sec. 4, golden fixture).
1. The closed-form SRD viscosity (kinetic + collisional, random grid shift;
   Gompper et al. 2009 review, cited by the paper) evaluated at those
   parameters reproduces the printed 8.7.
2. A body-force Poiseuille flow between no-slip walls run by the oracle has a
   parabolic profile whose curvature, rho g / eta, recovers that viscosity
   within 3% (fit v(z) = A z (H - z) + B; B absorbs the small wall slip of the
   shifted grid).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1801_10187_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "viscosity_rho10_alpha130.json")


def eta_closed_form(rho, alpha, dt, kT=1.0, m=1.0, a=1.0):
    f = rho - 1.0 + math.exp(-rho)
    ca, c2a = math.cos(alpha), math.cos(2 * alpha)
    eta_kin = rho * kT * dt / a**3 * (5 * rho / (f * (4 - 2 * ca - 2 * c2a)) - 0.5)
    eta_col = m / (18 * a * dt) * f * (1 - ca)
    return eta_kin + eta_col


def test_closed_form_reproduces_printed_viscosity():
    g = json.load(open(GOLDEN))
    eta = eta_closed_form(g["rho"], math.radians(g["alpha_deg"]), g["dt"], g["kT"], g["mass"])
    assert round(eta, 1) == g["eta"]


@pytest.mark.slow
def test_poiseuille_profile_recovers_viscosity():
    rho, g, H, Lx = 10.0, 0.01, 20, 12
    p = oracle.Params(n=(Lx, Lx, H), walls_z=True, thermostat=True, g=(g, 0.0, 0.0),
                      virt_density=rho, seed=11)
    s = inputs.solvent(p.n, rho, seed=11)
    st = oracle.State(s.pos, s.vel)
    oracle.step(p, st, 2000)  # start-up: slowest mode decays as exp(-t pi^2 eta / (rho H^2))
    nb, chunk, nrep = 40, 20, 200
    prof = np.zeros(nb)
    for _ in range(nrep):
        oracle.step(p, st, chunk)
        prof += oracle.profile(p, st, nb)
    prof /= nrep
    z = (np.arange(nb) + 0.5) * H / nb
    X = np.stack([z * (H - z), np.ones_like(z)], axis=1)
    (A, B), *_ = np.linalg.lstsq(X, prof, rcond=None)
    eta_fit = rho * g / (2 * A)
    eta_th = eta_closed_form(rho, math.radians(130.0), 0.1)
    assert abs(eta_fit / eta_th - 1) < 0.03, (eta_fit, eta_th)
    assert abs(B) < 0.05 * prof.max()  # small slip
    # the flow is along x only
    assert np.abs(st.vel[:, 1].mean()) < 0.01 and np.abs(st.vel[:, 2].mean()) < 0.01
