"""Closed-form flow pins of the oracle (CPU only).

* Poiseuille between halfway bounce-back walls is exact at steady state for
  the TRT model with Lambda = 3/16 (Sec. 2.1.2), for any viscosity.
* Couette flow driven by a moving wall (Eq. (14) with delta = 1/2) is exact.
* Bounce-back walls conserve mass; the body force adds a * N_fluid of momentum
  per step in a periodic box.
* A shear wave decays at the rate nu k^2 with nu from Eq. (7).
"""
import numpy as np
import pytest

from oracle import Domain, Params, Simulation
from oracle.lbm import equilibrium

rng = np.random.default_rng(7)


@pytest.mark.parametrize("tau,steps", [(0.8, 2000), (1.3, 1500)])
def test_poiseuille_is_exact(tau, steps):
    H, a = 10, 1e-6
    dom = Domain(1, 1, H, periodic=(True, True, False))
    sim = Simulation(dom, Params(tau=tau, body_force=(a, 0, 0)))
    nu = (tau - 0.5) / 3
    z = np.arange(H) + 0.5
    exact = a / (2 * nu) * z * (H - z)
    u0 = np.zeros((3, H, 1, 1))
    u0[0] = exact[:, None, None]
    sim.set_pdfs(equilibrium(np.ones((H, 1, 1)), u0))
    sim.step(steps)
    rho, u = sim.fields()
    assert np.abs(u[0, :, 0, 0] - exact).max() / exact.max() < 1e-9
    assert np.abs(u[1:]).max() < 1e-13


def test_couette_is_exact():
    H, uw = 10, 0.01
    dom = Domain(1, 1, H, periodic=(True, True, False),
                 wall_vel_hi=[[0, 0, 0], [0, 0, 0], [uw, 0, 0]])
    sim = Simulation(dom, Params(tau=1.3))
    sim.step(1500)
    rho, u = sim.fields()
    z = np.arange(H) + 0.5
    assert np.abs(u[0, :, 0, 0] - uw * z / H).max() / uw < 1e-9
    assert np.abs(rho - 1).max() < 1e-12


def test_bounce_back_walls_conserve_mass():
    dom = Domain(6, 5, 7, periodic=(False, True, False),
                 wall_vel_hi=[[0, 0, 0.0], [0, 0, 0], [0.02, 0.01, 0]])
    sim = Simulation(dom, Params(tau=0.7, body_force=(1e-5, 0, 2e-5)))
    rho0 = 1 + 0.01 * rng.standard_normal((7, 5, 6))
    u0 = 0.02 * rng.standard_normal((3, 7, 5, 6))
    sim.set_pdfs(equilibrium(rho0, u0))
    m0 = sim.ft.sum()
    sim.step(30)
    assert abs(sim.ft.sum() - m0) / m0 < 1e-14


def test_body_force_momentum_gain_per_step():
    dom = Domain(5, 4, 6)
    a = np.array([3e-5, -1e-5, 2e-5])
    sim = Simulation(dom, Params(tau=0.55, body_force=a))
    sim.set_pdfs(equilibrium(1 + 0.01 * rng.standard_normal((6, 4, 5)),
                             0.03 * rng.standard_normal((3, 6, 4, 5))))
    from oracle.lbm import momentum
    j0 = momentum(sim.ft).reshape(3, -1).sum(1)
    sim.step(1)
    j1 = momentum(sim.ft).reshape(3, -1).sum(1)
    assert np.abs(j1 - j0 - a * 120).max() < 1e-14


def test_shear_wave_decay_rate_matches_viscosity():
    L, U, tau = 32, 1e-4, 0.8
    nu = (tau - 0.5) / 3
    k = 2 * np.pi / L
    dom = Domain(1, 1, L)
    sim = Simulation(dom, Params(tau=tau))
    z = np.arange(L) + 0.5
    u0 = np.zeros((3, L, 1, 1))
    u0[0] = U * np.sin(k * z)[:, None, None]
    sim.set_pdfs(equilibrium(np.ones((L, 1, 1)), u0))
    sim.step(20)
    amp0 = np.abs(sim.fields()[1][0, :, 0, 0]).max()
    n = 200
    sim.step(n)
    amp1 = np.abs(sim.fields()[1][0, :, 0, 0]).max()
    rate = -np.log(amp1 / amp0) / n
    assert abs(rate / (nu * k * k) - 1) < 5e-3
