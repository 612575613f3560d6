"""Pins of the oracle's particle part: lubrication, contact, integrator (CPU only).

* lubrication (Sec. 3.1): equal-sphere and plane-wall limits against the
  classical leading-order coefficients (normal 1/4 for equal spheres;
  wall 1, 8/15, 1/10, 2/15, 2/5), Newton's third law, the step function,
  the minimum gap of Eq. (56) against Table 6;
* contact (Sec. 4.1.2): Eq. (43) reproduces e_dry and T_c of the damped
  linear oscillator; dry normal impacts on a wall and between two spheres
  give e_dry; a dry oblique impact in gross sliding follows rigid-body
  impulse theory, Psi_out = Psi_in - (1 + e) mu (1 + 1/K), K = 2/5;
* sticking contact (Eqs. (45), (49), (50)): an undamped sticking contact
  oscillates at sqrt(k_t (1/m + r_c^2/I)) with first-order amplitude growth in
  dt_p; a rigidly rotating pair keeps its spring length and force (the Eq. (49)
  rescale); a sphere on an incline rolls at 5/7 g sin(theta) below
  tan(theta) = 7/2 mu_p and slides (Coulomb, slip rate g (sin - 7/2 mu cos))
  above it;
* Velocity Verlet (Eqs. (37)-(38)) is exact for a constant force.
"""
import math
import os

import numpy as np
import pytest

from oracle import Domain, Params, Simulation
from oracle.particles import (lubrication_on_i, lubrication_min_gap, contact_coefficients,
                              collision_time)

HERE = os.path.dirname(os.path.abspath(__file__))
rng = np.random.default_rng(3)
MU = 0.05


def lub(Ri, Rj, delta, n, u, oi, oj, tangential=True):
    return lubrication_on_i(Ri, Rj, delta, n, u, oi, oj, MU, 2 / 3, 0.5, 0.5, 1e-3, tangential)


def test_min_gap_matches_table6():
    rows = np.loadtxt(os.path.join(HERE, 'golden', 'lub_min_gap_table6.txt'))
    for D, printed in rows:
        assert round(lubrication_min_gap(D / 2), 3) == pytest.approx(printed, abs=1e-12)


def test_normal_lubrication_equal_spheres():
    R, d = 4.0, 0.2
    n = np.array([0.0, 0.0, 1.0])
    u = np.array([0.0, 0.0, -0.01])
    F, T = lub(R, R, d, n, u, np.zeros(3), np.zeros(3), tangential=False)
    expect = -1.5 * math.pi * MU * R * R * (1 / d - 1.5) * u
    assert np.allclose(F, expect, rtol=1e-14, atol=0)
    assert np.abs(T).max() == 0


def test_tangential_equal_sphere_log_coefficient():
    # leading log coefficient of the tangential resistance of equal spheres is 1/6
    R, d = 3.0, 0.1
    n = np.array([1.0, 0.0, 0.0])
    u = np.array([0.0, 0.02, 0.0])
    F, _ = lub(R, R, d, n, u, np.zeros(3), np.zeros(3))
    assert np.allclose(F, 6 * math.pi * MU * R * (1 / 6) * math.log(d / 0.5) * u, rtol=1e-14)


def test_wall_limits_of_the_lubrication_terms():
    R, d = 5.0, 0.05
    n = np.array([0.0, 0.0, 1.0])
    u = np.array([0.01, -0.02, -0.03])
    om = np.array([1e-3, 2e-3, 5e-4])
    Fw, Tw = lub(R, None, d, n, u, om, np.zeros(3))
    Fb, Tb = lub(R, 1e9 * R, d, n, u, om, np.zeros(3))
    assert np.allclose(Fw, Fb, rtol=1e-7)
    assert np.allclose(Tw, Tb, rtol=1e-7)
    # classical wall coefficients: normal 1, tangential 8/15 and 1/10, rotation 2/15 and 2/5
    un = (u @ n) * n
    ut = u - un
    lt = math.log(d / 0.5)
    ln_ = -6 * math.pi * MU * R * R * (1 / d - 1.5) * un
    ftt = 6 * math.pi * MU * R * (8 / 15) * lt * ut
    ftr = -6 * math.pi * MU * R * R * (2 / 15) * lt * np.cross(om, n)
    ttt = 8 * math.pi * MU * R * R * (1 / 10) * lt * np.cross(u, n)
    ttr = 8 * math.pi * MU * R ** 3 * (2 / 5) * lt * (om - (om @ n) * n)
    assert np.allclose(Fw, ln_ + ftt + ftr, rtol=1e-13)
    assert np.allclose(Tw, ttt + ttr, rtol=1e-13)


def test_lubrication_forces_obey_newtons_third_law():
    for _ in range(20):
        Ri, Rj = rng.uniform(2, 8, 2)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        u = 0.01 * rng.standard_normal(3)
        oi, oj = 1e-3 * rng.standard_normal((2, 3))
        d = rng.uniform(0.01, 0.45)
        Fi, _ = lub(Ri, Rj, d, n, u, oi, oj)
        Fj, _ = lub(Rj, Ri, d, -n, -u, oj, oi)
        assert np.allclose(Fi + Fj, 0, atol=1e-16 + 1e-12 * np.abs(Fi).max())


def test_lubrication_step_function_and_gap_cap():
    n = np.array([0.0, 1.0, 0.0])
    u = np.array([0.01, -0.01, 0.0])
    om = np.array([0.0, 0.0, 1e-3])
    for d in (0.0, -0.01, 2 / 3, 0.7):
        F, T = lub(4.0, 4.0, d, n, u, om, om)
        assert np.abs(F).max() == 0 and np.abs(T).max() == 0
    F1, T1 = lub(4.0, 4.0, 1e-3, n, u, om, om)
    F2, T2 = lub(4.0, 4.0, 5e-4, n, u, om, om)
    assert np.array_equal(F1, F2) and np.array_equal(T1, T2)
    # between the tangential cut-off 1/2 and the normal one 2/3 only the normal term acts
    F3, T3 = lub(4.0, 4.0, 0.6, n, u, om, om)
    assert F3[0] == 0 and np.abs(T3).max() == 0 and F3[1] != 0


def test_contact_coefficients_reproduce_the_damped_oscillator():
    m, e, Tc = 123.0, 0.83, 37.0
    kn, dn, kt, dt = contact_coefficients(m, e, Tc, 0.22)
    gamma = dn / (2 * m)
    wd = math.sqrt(kn / m - gamma ** 2)
    assert abs(wd * Tc - math.pi) < 1e-12
    assert abs(math.exp(-gamma * Tc) - e) < 1e-14
    kappa = 2 * (1 - 0.22) / (2 - 0.22)
    assert abs(kt / kn - kappa) < 1e-15 and abs(dt / dn - math.sqrt(kappa)) < 1e-15
    assert abs(collision_time(20.0, 0.0) - 2.31 * 20 * math.sqrt(3)) < 1e-12


def dry_sim(dom, X, U, Om, R, rho, n_sub, **kw):
    p = Params(tau=0.8, n_sub=n_sub, lubrication=False, **kw)
    sim = Simulation(dom, p)
    sim.X = np.asarray(X, float)
    sim.U = np.asarray(U, float)
    sim.Om = np.asarray(Om, float)
    sim.R = np.asarray(R, float)
    sim.rho_p = np.asarray(rho, float)
    N = len(sim.R)
    sim.F_prev, sim.T_prev = sim.dem_forces(np.zeros((N, 3)), np.zeros((N, 3)), 0.0, False)
    return sim


def run_dry(sim, steps):
    N = len(sim.R)
    hist = []
    for _ in range(steps):
        sim.dem_subcycles(np.zeros((N, 3)), np.zeros((N, 3)))
        hist.append((sim.X.copy(), sim.U.copy(), sim.Om.copy()))
    return hist


def test_dry_normal_wall_impact_gives_e_dry_and_Tc():
    dom = Domain(32, 32, 32, periodic=(True, True, False))
    R, v, Tc = 4.0, 0.05, 20.0
    sim = dry_sim(dom, [[16, 16, R + 0.02]], [[0, 0, -v]], [[0, 0, 0]], [R], [8.0], 40,
                  Tc=Tc, e_dry=0.97)
    hist = run_dry(sim, 40)
    gaps = np.array([h[0][0, 2] - R for h in hist])
    in_contact = np.nonzero(gaps < 0)[0]
    duration = (in_contact[-1] - in_contact[0] + 1)
    assert abs(duration - Tc) <= 1.0
    u_after = hist[-1][1][0, 2]
    assert abs(u_after / v - 0.97) < 2e-3


def test_dry_head_on_sphere_collision_gives_e_dry():
    dom = Domain(40, 20, 20)
    R, v = 3.0, 0.04
    sim = dry_sim(dom, [[20 - R - 0.01, 10, 10], [20 + R + 0.01, 10, 10]],
                  [[v, 0, 0], [-v, 0, 0]], np.zeros((2, 3)), [R, R], [2.5, 2.5], 40,
                  Tc=15.0, e_dry=0.9)
    hist = run_dry(sim, 40)
    U = hist[-1][1]
    assert abs((U[1, 0] - U[0, 0]) / (2 * v) - 0.9) < 2e-3
    assert abs(U[0, 0] + U[1, 0]) < 1e-15


def test_dry_oblique_impact_in_gross_sliding():
    dom = Domain(32, 32, 32, periodic=(True, True, False))
    R, un, psi_in, e, mu = 4.0, 0.02, 5.0, 0.97, 0.15
    # a stiff contact (small T_c) keeps the overlap, and with it the shortening of
    # the lever arm R + delta/2, small against R
    sim = dry_sim(dom, [[16, 16, R + 0.005]], [[psi_in * un, 0, -un]], [[0, 0, 0]], [R], [2.5],
                  200, Tc=5.0, e_dry=e, mu_p=mu, nu_p=0.22)
    hist = run_dry(sim, 12)
    X, U, Om = hist[-1]
    assert X[0, 2] - R > 0
    u_t_out = U[0, 0] - R * Om[0, 1]
    psi_out = u_t_out / un
    assert abs(psi_out - (psi_in - (1 + e) * mu * (1 + 1 / 0.4))) < 0.005


def test_velocity_verlet_is_exact_for_constant_force():
    dom = Domain(64, 64, 64)
    g = np.array([1e-5, -2e-5, -3e-5])
    sim = dry_sim(dom, [[10.0, 20.0, 60.0]], [[0.01, 0.0, 0.02]], [[0, 0, 0]], [3.0], [3.0], 7,
                  gravity=g)
    run_dry(sim, 30)
    acc = g * (3.0 - 1.0) / 3.0
    t = 30.0
    x = np.array([10.0, 20.0, 60.0]) + np.array([0.01, 0, 0.02]) * t + 0.5 * acc * t * t
    x = np.mod(x, 64.0)
    assert np.allclose(sim.X[0], x, atol=1e-12)
    assert np.allclose(sim.U[0], np.array([0.01, 0, 0.02]) + acc * t, atol=1e-15)


# ---------------------------------------------------------------------------
# sticking branch of the tangential contact (Sec. 4.1.2, Eqs. (45), (49), (50))
# ---------------------------------------------------------------------------

def resting_on_wall(R, rho, g_vec, Tc, e, mu, nu, n_sub, u0=(0.0, 0.0, 0.0)):
    """A dry sphere resting on the wall z = 0 at the equilibrium overlap of its
    weight's normal part (no lubrication, no fluid)."""
    dom = Domain(64, 64, 64, periodic=(True, True, False))
    m = rho * math.pi * (2 * R) ** 3 / 6
    kn, _, _, _ = contact_coefficients(m, e, Tc, nu)
    f_ext = math.pi * (2 * R) ** 3 / 6 * (rho - 1.0) * np.asarray(g_vec, float)
    delta0 = f_ext[2] / kn                        # < 0: weight pressing into the wall
    sim = dry_sim(dom, [[32.0, 32.0, R + delta0]], [u0], [[0, 0, 0]], [R], [rho], n_sub,
                  Tc=Tc, e_dry=e, mu_p=mu, nu_p=nu, gravity=tuple(g_vec))
    return sim, m, delta0


def contact_slip(sim, delta):
    """Tangential velocity of the contact point of a sphere on the wall z = 0
    (Eq. (B.7) with the lever arm R + delta/2 of the wall contact point)."""
    rc = sim.R[0] + 0.5 * delta
    return sim.U[0, 0] - rc * sim.Om[0, 1], rc


def sticking_oscillation(n_sub, steps=120):
    """Slip velocity of the contact point, one sample per time step, of an
    undamped sphere set sliding at 5e-4 along a wall it rests on."""
    R, rho, Tc, mu, nu = 4.0, 8.0, 20.0, 0.15, 0.23
    sim, m, delta0 = resting_on_wall(R, rho, (0.0, 0.0, -1e-3), Tc, 1.0, mu, nu, n_sub,
                                     u0=(5e-4, 0.0, 0.0))
    _, _, kt, dt_ = contact_coefficients(m, 1.0, Tc, nu)
    assert dt_ == 0.0
    rc = R + 0.5 * delta0
    I = 0.4 * m * R * R
    omega_t = math.sqrt(kt * (1.0 / m + rc * rc / I))
    slip = []
    for k in range(steps):
        s, _ = contact_slip(sim, delta0)
        slip.append(s)
        sim.dem_subcycles(np.zeros((1, 3)), np.zeros((1, 3)))
        # still sticking: the spring force stays inside the Coulomb cone
        d = sim.hist[(0, 'wall', 2, 0)]
        assert kt * math.sqrt(d @ d) < mu * m * (rho - 1) / rho * 1e-3
    return np.array(slip), omega_t


def test_sticking_contact_oscillates_at_the_tangential_spring_frequency():
    # Undamped (e_dry = 1) sticking contact: the spring delta_t integrates the
    # contact-point velocity (Eq. (50)) and pulls back with -k_t delta_t
    # (Eq. (45)). With F_x = -k_t delta_t acting at the contact point, the slip
    # velocity obeys d^2 delta_t / dt^2 = -k_t (1/m + r_c^2 / I) delta_t, a
    # harmonic oscillator of angular frequency sqrt(k_t (1/m + r_c^2 / I)).
    slip, omega_t = sticking_oscillation(40)
    t = np.arange(len(slip), dtype=float)
    # zero crossings of u0 cos(omega_t t) lie at (j + 1/2) pi / omega_t
    z = [t[k] + slip[k] / (slip[k] - slip[k + 1]) for k in range(len(t) - 1)
         if slip[k] > 0 >= slip[k + 1] or slip[k] < 0 <= slip[k + 1]]
    assert len(z) >= 8
    half_period = (z[-1] - z[0]) / (len(z) - 1)
    assert abs(half_period / (math.pi / omega_t) - 1.0) < 0.01
    assert abs(z[0] / (0.5 * math.pi / omega_t) - 1.0) < 0.02
    # The spring is integrated explicitly with the velocity of the start of
    # each subcycle and pulls with the value it had there, so the undamped
    # oscillation gains energy at a rate proportional to dt_p: halving dt_p
    # halves the amplitude's growth over the same time (first order).
    g40 = np.abs(slip[-25:]).max() / 5e-4 - 1.0
    slip80, _ = sticking_oscillation(80)
    g80 = np.abs(slip80[-25:]).max() / 5e-4 - 1.0
    assert 0.0 < g80 < g40 < 0.3
    assert abs(g40 / g80 - 2.0) < 0.25


@pytest.mark.parametrize('t0', [(0.0, 2e-3, 0.0), (0.0, 2e-3, 1e-3)])
def test_rigidly_rotating_contact_keeps_its_spring_length(t0):
    # Two spheres in sticking contact rotate together as one rigid body about
    # the z axis through their midpoint: the contact point has no relative
    # velocity, so the stored spring must only turn with the contact frame
    # (Eq. (49): projection on the new tangent plane, rescaled to the old
    # length), never shrink or grow, and its force -k_t delta_t keeps its size.
    # A spring in the plane of rotation turns exactly with the pair.
    R, eps, Om = 3.0, 0.02, 0.01
    dom = Domain(40, 40, 40)
    c = np.array([20.0, 20.0, 20.0])
    half = R - 0.5 * eps
    p = Params(tau=0.8, n_sub=10, lubrication=False, e_dry=0.97, Tc=15.0, mu_p=0.5, nu_p=0.23)
    sim = Simulation(dom, p)
    sim.R = np.array([R, R])
    sim.rho_p = np.array([2.5, 2.5])
    t0 = np.array(t0)
    sim.hist[(0, 1)] = t0.copy()
    dth = 0.1
    m = sim.mass[0]
    kn, _, kt, _ = contact_coefficients(0.5 * m, p.e_dry, 15.0, p.nu_p)
    assert kt * np.linalg.norm(t0) < p.mu_p * kn * eps
    for k in range(1, 16):
        th = k * dth
        n = np.array([math.cos(th), math.sin(th), 0.0])
        sim.X = np.array([c + half * n, c - half * n])
        w = np.array([0.0, 0.0, Om])
        sim.U = np.array([np.cross(w, sim.X[0] - c), np.cross(w, sim.X[1] - c)])
        sim.Om = np.array([w, w])
        F, T = sim.dem_forces(np.zeros((2, 3)), np.zeros((2, 3)), 0.1, update_history=True)
        d = sim.hist[(0, 1)]
        assert abs(np.linalg.norm(d) / np.linalg.norm(t0) - 1.0) < 1e-12
        assert abs(d @ n) < 1e-15
        if t0[2] == 0.0:
            tang = np.array([-math.sin(th), math.cos(th), 0.0])
            assert np.allclose(d, t0[1] * tang, rtol=0, atol=1e-12 * np.linalg.norm(t0))
        # contact force on sphere 0: the normal spring plus -k_t times the
        # turned tangential spring (no damping: no relative velocity)
        Fn = -kn * (-eps) * n
        assert np.allclose(F[0], Fn - kt * d, rtol=0, atol=1e-13)


@pytest.mark.parametrize('ratio,sticks', [(0.9, True), (1.1, False)])
def test_sphere_on_an_incline_rolls_below_and_slides_above_the_friction_limit(ratio, sticks):
    # A sphere on a plane inclined at theta (gravity tilted against the wall
    # z = 0) rolls without slipping while the friction it needs,
    # (2/7) m g sin(theta), stays below mu_p m g cos(theta), i.e. for
    # tan(theta) < 7/2 mu_p: the contact sticks (Eq. (50)) and the centre
    # accelerates at 5/7 g sin(theta). Above that limit it slides with the
    # Coulomb force mu_p |F_n| (Eq. (47)): the centre accelerates at
    # g (sin - mu_p cos) and the contact point slips at the rate
    # g (sin - 7/2 mu_p cos).
    R, rho, Tc, mu, nu, g = 4.0, 8.0, 20.0, 0.15, 0.23, 2e-4
    th = math.atan(ratio * 3.5 * mu)
    g_vec = (g * math.sin(th), 0.0, -g * math.cos(th))
    sim, m, delta0 = resting_on_wall(R, rho, g_vec, Tc, 0.3, mu, nu, 20)
    geff = g * (rho - 1.0) / rho
    U0, S0 = None, None
    t1, t2 = 150, 350
    for k in range(t2 + 1):
        if k == t1:
            U0 = sim.U[0, 0]
            S0, _ = contact_slip(sim, delta0)
        if k >= t1:
            s, _ = contact_slip(sim, delta0)
            if sticks:
                assert abs(s) < 1e-3 * geff * k
        sim.dem_subcycles(np.zeros((1, 3)), np.zeros((1, 3)))
    a = (sim.U[0, 0] - U0) / (t2 - t1 + 1)
    S1, _ = contact_slip(sim, delta0)
    if sticks:
        assert abs(a / (5.0 / 7.0 * geff * math.sin(th)) - 1.0) < 0.01
    else:
        assert abs(a / (geff * (math.sin(th) - mu * math.cos(th))) - 1.0) < 0.01
        rate = (S1 - S0) / (t2 - t1 + 1)
        assert abs(rate / (geff * (math.sin(th) - 3.5 * mu * math.cos(th))) - 1.0) < 0.02
