"""Pins of the oracle's fluid-particle coupling (CPU only).

* mapping (Sec. 2.2): cell counts against an independent lattice-point count,
  lowest-index ownership, periodic images;
* link fraction delta_q (Eq. (14)): closed form on axis and diagonal links;
* momentum exchange (Eqs. (15)-(17)) with the missing-link term: an isolated
  sphere and a close pair in fluid at rest feel exactly zero force;
* momentum balance: with particles at rest the fluid loses exactly the
  momentum the particles gain;
* torque sign and size for a sphere spinning in fluid at rest;
* Stokes drag on a periodic array of spheres, C_ref = 2.842 (Sec. 2.4),
  independent of the relaxation time;
* refill (Eq. (18)): uniform flow gives the equilibrium, a linear velocity
  field gives its exact strain rate, central differences are exact for a
  quadratic field, one-sided next to a solid cell;
* prescribed motion (Sec. 2.3.3) moves a sphere by the set velocity;
* the complete step (Algorithm 1): a sphere carried by a uniform flow keeps
  the flow in its equilibrium with zero force, prescribed on an oblique
  path or free (DEM) on a mirror-symmetric one, where it moves at constant
  velocity without spinning;
* interacting particles (contact, lubrication, walls, periodic sides,
  refill): the complete trajectory is invariant under a cyclic permutation
  of the axes (a rotation of the lattice), under a mirror of one axis, under
  a translation by whole cells along the periodic axes and under a new
  order of the particles.
"""
import itertools

import numpy as np
import pytest

from oracle import Domain, Params, Simulation
from oracle.d3q19 import C, W
from oracle.lbm import density, equilibrium, momentum
from oracle.coupling import stream_and_couple, missing_links, refill
from oracle.particles import map_cells, cell_centres, link_fraction, dist2

rng = np.random.default_rng(11)


def lattice_points(r2):
    """Number of integer points n with |n|^2 <= r2 (independent brute force)."""
    k = int(np.ceil(np.sqrt(r2))) + 1
    return sum(1 for n in itertools.product(range(-k, k + 1), repeat=3)
               if n[0] ** 2 + n[1] ** 2 + n[2] ** 2 <= r2)


@pytest.mark.parametrize("r2", [1, 2, 3, 4, 5, 9, 10, 17])
def test_mapping_counts_lattice_points(r2):
    dom = Domain(16, 16, 16)
    X = np.array([[8.5, 8.5, 8.5]])
    R = np.array([np.sqrt(r2)])
    # make R*R exactly r2 where sqrt rounds: the tie must count as inside
    owner, shell = map_cells(cell_centres(dom), X, R, dom, 2.0)
    n_inside = (owner == 0).sum()
    if R[0] * R[0] == r2:
        assert n_inside == lattice_points(r2)
    else:
        assert lattice_points(r2 - 1) <= n_inside <= lattice_points(r2)
    rs2 = (R[0] + 2.0) ** 2
    n_shell = lattice_points(rs2) - n_inside
    assert shell.sum() == n_shell


def test_mapping_lowest_index_wins_and_periodic_image():
    dom = Domain(12, 10, 14)
    X = np.array([[6.0, 5.0, 7.0], [7.5, 5.0, 7.0], [0.2, 9.9, 13.8]])
    R = np.array([2.5, 2.5, 2.2])
    owner, shell = map_cells(cell_centres(dom), X, R, dom, 2.0)
    centres = cell_centres(dom)
    for (z, y, x), o in np.ndenumerate(owner):
        c = centres[z, y, x]
        inside = []
        for i in range(3):
            d = c - X[i]
            d = d - np.array(dom.shape) * np.round(d / np.array(dom.shape))
            if d @ d <= R[i] ** 2:
                inside.append(i)
        assert o == (min(inside) if inside else -1)
    # the sphere across the corner has the same cell count as an interior copy
    owner2, _ = map_cells(cell_centres(dom), np.array([[6.2, 4.9, 6.8]]), R[2:], dom, 2.0)
    assert (owner == 2).sum() == (owner2 == 0).sum()


def test_link_fraction_closed_form():
    dom = Domain(20, 20, 20)
    xp = np.array([10.0, 10.25, 10.5])
    x = np.array([[6.5, 10.25, 10.5]])
    # axis link towards the centre: surface at distance 3.5 - R
    assert np.allclose(link_fraction(x, (1, 0, 0), xp, 3.0, dom), 0.5, atol=1e-15)
    # diagonal link: |r + t c|^2 = R^2 solved by hand
    x = np.array([[8.5, 8.5, 10.5]])
    r = x[0] - xp
    c = np.array([1.0, 1.0, 0.0])
    R = 1.8
    a, b, cc = 2.0, 2 * r @ c, r @ r - R * R
    t = (-b - np.sqrt(b * b - 4 * a * cc)) / (2 * a)
    assert abs(link_fraction(x, c, xp, R, dom)[0] - t) < 1e-15
    assert abs(np.linalg.norm(r + t * c) - R) < 1e-14


def rest_state(dom):
    nx, ny, nz = dom.shape
    return equilibrium(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))


def test_isolated_sphere_in_fluid_at_rest_feels_no_force():
    dom = Domain(16, 14, 15)
    X = np.array([[7.3, 6.9, 7.6]])
    R = np.array([3.7])
    owner, _ = map_cells(cell_centres(dom), X, R, dom, 2.0)
    _, F, T = stream_and_couple(rest_state(dom), dom, owner, X, np.zeros((1, 3)),
                                np.zeros((1, 3)), R)
    Fm, Tm = missing_links(dom, owner, X, R)
    assert np.abs(Fm).max() == 0 and np.abs(Tm).max() == 0
    assert np.abs(F).max() < 1e-14


def test_missing_links_close_pair_and_wall():
    dom = Domain(24, 14, 16, periodic=(True, True, False))
    R = np.array([3.5, 3.6, 3.0])
    # pair along x with surface gap 0.2; third sphere 0.1 above the wall z = 0
    X = np.array([[4.4, 7.5, 11.5], [4.4 + 7.1 + 0.2, 7.5, 11.5], [19.0, 7.0, 3.1]])
    owner, _ = map_cells(cell_centres(dom), X, R, dom, 2.0)
    assert all((owner == i).any() for i in range(3))
    _, F, T = stream_and_couple(rest_state(dom), dom, owner, X, np.zeros((3, 3)),
                                np.zeros((3, 3)), R)
    Fm, Tm = missing_links(dom, owner, X, R)
    # without the correction the close bodies attract each other
    assert F[0, 0] > 1e-2 and F[1, 0] < -1e-2 and F[2, 2] < -1e-2
    assert np.abs(F + Fm).max() < 1e-13


def test_missing_links_cancel_the_torque_of_an_oblique_pair():
    # off-axis neighbours: the fluid at rest exerts a torque on each body of a
    # close pair (and on a sphere near a wall) through the links it lacks; the
    # missing-link terms (Sec. 2.2), applied at points of the same lattice
    # lines, cancel force and torque exactly
    dom = Domain(24, 14, 16, periodic=(True, True, False))
    R = np.array([3.5, 3.6, 3.0])
    X = np.array([[4.9, 7.2, 11.3], [4.9 + 7.1 + 0.15, 8.1, 12.0], [18.6, 6.8, 3.08]])
    owner, _ = map_cells(cell_centres(dom), X, R, dom, 2.0)
    _, F, T = stream_and_couple(rest_state(dom), dom, owner, X, np.zeros((3, 3)),
                                np.zeros((3, 3)), R)
    Fm, Tm = missing_links(dom, owner, X, R)
    assert np.abs(T).max() > 0.1
    assert np.abs(F + Fm).max() < 1e-13 and np.abs(T + Tm).max() < 1e-13


def test_momentum_balance_with_resting_particles():
    dom = Domain(18, 16, 17)
    X = np.array([[5.2, 8.1, 8.4], [12.9, 7.7, 9.0]])
    R = np.array([3.1, 2.7])
    owner, _ = map_cells(cell_centres(dom), X, R, dom, 2.0)
    nx, ny, nz = dom.shape
    ft = equilibrium(1 + 0.01 * rng.standard_normal((nz, ny, nx)),
                     0.02 * rng.standard_normal((3, nz, ny, nx)))
    ft[:, owner >= 0] = 0.0
    f, F, T = stream_and_couple(ft, dom, owner, X, np.zeros((2, 3)), np.zeros((2, 3)), R)
    j0 = momentum(ft).reshape(3, -1).sum(1)
    j1 = momentum(f).reshape(3, -1).sum(1)
    assert np.abs(j1 - j0 + F.sum(0)).max() < 1e-13
    assert np.abs(F).max() > 1e-3


def test_spinning_sphere_torque_opposes_rotation():
    L, R, om, tau = 24, 3.0, 1e-4, 1.3
    dom = Domain(L, L, L)
    sim = Simulation(dom, Params(tau=tau, fixed_particles=True))
    sim.add_spheres([[12.0, 12.0, 12.0]], [[0, 0, 0]], [[0, 0, om]], [R], [1.0])
    sim.step(250)
    mu = (tau - 0.5) / 3
    Tz = sim.Tfp[0, 2]
    assert Tz < 0
    assert abs(sim.Tfp[0, 0]) < 1e-3 * abs(Tz) and abs(sim.Tfp[0, 1]) < 1e-3 * abs(Tz)
    rotlet = 8 * np.pi * mu * R ** 3 * om
    assert 0.8 < -Tz / rotlet < 1.25
    assert np.abs(sim.Ffp[0]).max() < 1e-3 * abs(Tz)


def stokes_C(tau, D=8.0, a=1e-7, max_blocks=40):
    L = int(2 * D)
    dom = Domain(L, L, L)
    sim = Simulation(dom, Params(tau=tau, body_force=(a, 0, 0), fixed_particles=True))
    sim.add_spheres([[L / 2, L / 2, L / 2]], [[0, 0, 0]], [[0, 0, 0]], [D / 2], [1.0])
    nu = (tau - 0.5) / 3
    prev = None
    for _ in range(max_blocks):
        sim.step(100)
        rho, u = sim.fields()
        ubar = u[0].sum() / L ** 3
        Cn = (sim.Ffp[0, 0] + np.pi / 6 * D ** 3 * a) / (3 * np.pi * nu * D * ubar)
        if prev is not None and abs(Cn - prev) < 1e-7 * abs(Cn):
            return Cn
        prev = Cn
    raise AssertionError("Stokes drag did not converge")


def test_stokes_drag_periodic_array():
    c1 = stokes_C(1.3)
    c2 = stokes_C(2.0)
    assert abs(c1 / 2.842 - 1) < 0.02
    # TRT with the magic parameter: boundary location independent of viscosity
    assert abs(c1 - c2) / c1 < 1e-5


def test_refill_uniform_flow_gives_equilibrium():
    dom = Domain(9, 9, 9)
    u0 = np.array([0.02, -0.01, 0.015])
    rho0 = 1.01
    ft = equilibrium(np.full((9, 9, 9), rho0), np.broadcast_to(u0[:, None, None, None], (3, 9, 9, 9)))
    owner_old = np.full((9, 9, 9), -1)
    owner_old[4, 4, 4] = 0
    owner_new = np.full((9, 9, 9), -1)
    X = np.array([[4.5, 4.5, 3.9]])
    cells = refill(ft, dom, owner_old, owner_new, X, u0[None], np.zeros((1, 3)), 1 / 0.7,
                   np.zeros(3))
    assert cells == [(4, 4, 4)]
    cu = C @ u0
    expect = W * rho0 * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u0 @ u0)
    assert np.abs(ft[:, 4, 4, 4] - expect).max() < 1e-15


def test_refill_linear_field_uses_exact_strain():
    n = 9
    dom = Domain(n, n, n)
    G = np.array([[0.0, 2e-3, 0.0], [0.0, 0.0, -1e-3], [5e-4, 0.0, 0.0]])
    centres = cell_centres(dom)
    u = np.einsum('ab,zyxb->azyx', G, centres - 4.5)
    ft = equilibrium(np.ones((n, n, n)), u)
    owner_old = np.full((n, n, n), -1)
    owner_old[4, 4, 4] = 0
    X = np.array([[4.5, 4.5, 4.5]])
    s_nu = 1 / 0.8
    refill(ft, dom, owner_old, np.full((n, n, n), -1), X, np.zeros((1, 3)), np.zeros((1, 3)),
           s_nu, np.zeros(3))
    S = G + G.T
    expect = np.zeros(19)
    for q in range(19):
        cq = C[q].astype(float)
        expect[q] = W[q] * (1 - 1.5 / s_nu * (cq @ S @ cq - np.trace(S) / 3))
    # rho_bar of the linear equilibrium neighbours is exactly 1
    assert np.abs(ft[:, 4, 4, 4] - expect).max() < 1e-15


def brute_force_solid_count(dom, X, R):
    """Cells whose centre lies within R of X (minimum image), by plain loops."""
    n = 0
    for k, j, i in itertools.product(range(dom.shape[2]), range(dom.shape[1]), range(dom.shape[0])):
        d = np.array([i + 0.5, j + 0.5, k + 0.5]) - X
        d -= np.array(dom.shape) * np.round(d / np.array(dom.shape))
        n += d @ d <= R * R
    return n


def test_prescribed_motion_moves_by_the_set_velocity():
    # prescribed motion (Sec. 2.3.3 sets a sphere's velocity every step):
    # x advances by u per step, the mapping follows, uncovered cells refill
    dom = Domain(12, 12, 12)
    sim = Simulation(dom, Params(tau=0.8, prescribed_motion=True))
    X0 = np.array([[6.25, 6.0, 5.9]])
    R = 2.6
    sim.add_spheres(X0, [[0, 0, 0]], [[0, 0, 0]], [R], [1.0])
    refills = 0
    U = np.array([[0.35, -0.2, 0.1]])
    for k in range(1, 9):
        sim.U = U.copy()
        sim.step(1)
        refills += len(sim.refilled)
    X = (X0 + 8 * U) % 12.0
    assert np.abs(sim.X - X).max() < 1e-12
    assert int((sim.owner >= 0).sum()) == brute_force_solid_count(dom, X[0], R)
    assert refills > 0
    # the stored velocity is the one set: no DEM forces act on it
    assert np.array_equal(sim.U, U)


def test_prescribed_motion_at_rest_equals_fixed_particles():
    runs = []
    for mode in ('prescribed', 'fixed'):
        dom = Domain(12, 12, 12)
        sim = Simulation(dom, Params(tau=0.8, body_force=(1e-5, 0, 0),
                                     prescribed_motion=mode == 'prescribed', fixed_particles=mode == 'fixed'))
        sim.add_spheres([[6.25, 6.0, 5.9]], [[0, 0, 0]], [[0, 0, 0]], [2.6], [1.0])
        sim.step(5)
        runs.append(sim)
    assert np.array_equal(runs[0].ft, runs[1].ft)
    assert np.array_equal(runs[0].Ffp, runs[1].Ffp)


def refill_expect(S, s_nu, u_t=np.zeros(3), rho_bar=1.0):
    """Eq. (18) written out for a given strain S = grad u + grad u^T."""
    out = np.zeros(19)
    for q in range(19):
        cq = C[q].astype(float)
        cu = cq @ u_t
        out[q] = W[q] * (rho_bar + 3 * rho_bar * cu + 4.5 * rho_bar * cu * cu - 1.5 * rho_bar * u_t @ u_t
                         - 1.5 / s_nu * rho_bar * (cq @ S @ cq - np.trace(S) / 3))
    return out


def test_refill_gradient_is_central_for_a_quadratic_field():
    # Eq. (18) with second-order central differences: exact for a quadratic
    # velocity field (a one-sided difference would pick up the curvature)
    n = 9
    dom = Domain(n, n, n)
    d = cell_centres(dom) - 4.5
    u = np.stack([2e-3 * d[..., 1] + 3e-4 * d[..., 1] ** 2,
                  -1e-3 * d[..., 2] + 2e-4 * d[..., 0] ** 2,
                  5e-4 * d[..., 0] - 4e-4 * d[..., 2] ** 2])
    ft = equilibrium(np.ones((n, n, n)), u)
    owner_old = np.full((n, n, n), -1)
    owner_old[4, 4, 4] = 0
    s_nu = 1 / 0.9
    refill(ft, dom, owner_old, np.full((n, n, n), -1), np.array([[4.5, 4.5, 4.5]]), np.zeros((1, 3)),
           np.zeros((1, 3)), s_nu, np.zeros(3))
    G = np.array([[0.0, 2e-3, 0.0], [0.0, 0.0, -1e-3], [5e-4, 0.0, 0.0]])   # gradient at the cell
    rho_bar = np.mean([density(ft)[4 + C[q][2], 4 + C[q][1], 4 + C[q][0]] for q in range(1, 19)])
    assert np.abs(ft[:, 4, 4, 4] - refill_expect(G + G.T, s_nu, rho_bar=rho_bar)).max() < 1e-14


def test_refill_falls_back_to_one_sided_differences_next_to_a_solid():
    # a solid neighbour in +x: d u / d x from the cell's own (particle) velocity
    # and the -x neighbour, exact for a linear field whose value at the cell is
    # the particle velocity there
    n = 9
    dom = Domain(n, n, n)
    d = cell_centres(dom) - 4.5
    G = np.array([[1e-3, 0.0, 2e-4], [-5e-4, 3e-4, 0.0], [0.0, 1e-3, -4e-4]])
    u0 = np.array([0.01, -0.02, 0.005])
    u = u0[:, None, None, None] + np.einsum('ab,zyxb->azyx', G, d)
    ft = equilibrium(np.ones((n, n, n)), u)
    owner_old = np.full((n, n, n), -1)
    owner_old[4, 4, 4] = 0
    owner_new = np.full((n, n, n), -1)
    owner_new[4, 4, 5] = 1                      # the +x neighbour is (still) solid
    ft[:, 4, 4, 5] = equilibrium(np.array(1.2), np.array([0.1, 0.1, 0.1]))   # and its PDFs unusable
    X = np.array([[4.5, 4.5, 4.5], [6.5, 4.5, 4.5]])
    s_nu = 1 / 0.75
    refill(ft, dom, owner_old, owner_new, X, np.stack([u0, u0]), np.zeros((2, 3)), s_nu, np.zeros(3))
    fluid_nbrs = [q for q in range(1, 19) if not (C[q][0] == 1 and C[q][1] == 0 and C[q][2] == 0)
                  and owner_new[4 + C[q][2], 4 + C[q][1], 4 + C[q][0]] < 0]
    rho_bar = np.mean([density(ft)[4 + C[q][2], 4 + C[q][1], 4 + C[q][0]] for q in fluid_nbrs])
    got = ft[:, 4, 4, 4]
    assert np.abs(got - refill_expect(G + G.T, s_nu, u_t=u0, rho_bar=rho_bar)).max() < 1e-14



def carried_sphere(U, X0, tau, prescribed, steps=16, n=14, R=2.7):
    """A sphere moving with a uniform flow U in a fully periodic box, run
    through the complete coupled step (Algorithm 1)."""
    dom = Domain(n, n, n)
    sim = Simulation(dom, Params(tau=tau, prescribed_motion=prescribed))
    sim.set_pdfs(equilibrium(np.ones((n, n, n)), np.broadcast_to(U[:, None, None, None], (3, n, n, n))))
    sim.add_spheres([X0], [U], [[0, 0, 0]], [R], [1.7])
    refills, covers = 0, set()
    for _ in range(steps):
        if prescribed:
            sim.U = U[None].copy()
        sim.step(1)
        refills += len(sim.refilled)
        covers.add(tuple(np.flatnonzero(sim.owner.ravel() >= 0)))
    assert refills > 0 and len(covers) > 3          # the sphere crossed cells
    fluid = sim.owner < 0
    feq = equilibrium(np.array(1.0), U)
    assert np.abs(sim.ft[:, fluid] - feq[:, None]).max() < 1e-14
    assert np.abs(sim.Ffp).max() < 1e-13
    assert np.abs(sim.X - (np.asarray(X0) + steps * U) % n).max() < 1e-12
    assert int((~fluid).sum()) == brute_force_solid_count(dom, sim.X[0], R)
    return sim


@pytest.mark.parametrize("tau", [0.6, 1.3])
def test_sphere_carried_by_uniform_flow_keeps_it_uniform(tau):
    # moving with the flow, the sphere leaves the fluid in its equilibrium:
    # the moving-wall CLI value (Eq. (14)) of a uniform field is that field's
    # equilibrium, no collision (Eq. (5)) changes an equilibrium, and the
    # refill (Eq. (18)) of the uncovered cells gives the same equilibrium. The
    # link pairs of each lattice line through the closed surface cancel in the
    # momentum exchange (Eqs. (15)-(17)): zero force. (The torque of the
    # Galilean term -u_b (f_p - f_pbar) is O(U^2) and not zero on a discrete
    # sphere whose chords differ between lattice directions, so the oblique
    # motion here is prescribed, Sec. 2.3.3.)
    carried_sphere(np.array([0.071, -0.043, 0.029]), [6.8, 7.3, 6.6], tau, prescribed=True)


@pytest.mark.parametrize("X0", [[6.8, 7.0, 7.0], [6.8, 7.5, 6.5]])
def test_free_sphere_carried_by_uniform_flow_moves_with_it(X0):
    # the same with the DEM (Eqs. (37)-(38)) moving the sphere: motion along x
    # with the centre on mirror planes of the lattice in y and z, so the
    # mapped body keeps both mirror symmetries, the torque cancels too, and the
    # sphere moves with the flow at constant velocity without spinning
    U = np.array([0.083, 0.0, 0.0])
    sim = carried_sphere(U, X0, 0.8, prescribed=False)
    assert np.abs(sim.Tfp).max() < 1e-13
    assert np.abs(sim.U - U).max() < 1e-14 and np.abs(sim.Om).max() < 1e-15


# Three spheres with spin in a box periodic in x, y and bounded by walls in z,
# under gravity: a pair that comes into contact (through lubrication) across
# the periodic side x = 0, and a sphere across the periodic side y = 0 rising
# against gravity into the top wall's lubrication range.
PAIR_WALL = dict(shape=np.array([16, 14, 18]), periodic=np.array([1, 1, 0]),
                 g=np.array([0.0, 0.0, -2e-4]),
                 X=np.array([[13.6, 7.2, 8.0], [2.75, 6.9, 8.3], [8.0, 1.0, 15.72]]),
                 U=np.array([[0.05, 0.002, 0.0], [-0.05, 0.0, -0.004], [0.0, -0.01, 0.08]]),
                 Om=np.array([[0.0, 0.01, 0.002], [0.003, 0.0, -0.01], [0.0, 0.0, 0.0]]),
                 R=np.array([2.6, 2.4, 2.2]), rho=np.array([8.0, 6.0, 9.0]))


def run_pair_wall(shape, periodic, g, X, U, Om, R, rho, steps=30, watch=None):
    """The complete coupled step, `steps` times, for PAIR_WALL (or a
    transformed copy of it); watch(sim) is called after every step."""
    dom = Domain(*shape, periodic=tuple(bool(v) for v in periodic))
    sim = Simulation(dom, Params(tau=0.8, gravity=tuple(g), Tc=10.0))
    sim.add_spheres(X, U, Om, R, rho)
    for _ in range(steps):
        sim.step(1)
        if watch:
            watch(sim)
    return sim


def close(a, b):
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(x).max())


def rotated_run(perm):
    """PAIR_WALL with its axes renamed by perm (a cyclic permutation is a
    rotation of the lattice); returns the final particle state and velocity
    field with the axes named back, and the smallest pair and wall gaps."""
    c = PAIR_WALL
    p = list(perm)
    gaps = [np.inf, np.inf]

    def watch(sim):
        gaps[0] = min(gaps[0], np.sqrt(dist2(sim.X[0], sim.X[1], sim.dom)) - c['R'][0] - c['R'][1])
        gaps[1] = min(gaps[1], c['shape'][2] - sim.X[2, p.index(2)] - c['R'][2])

    sim = run_pair_wall(c['shape'][p], c['periodic'][p], c['g'][p], c['X'][:, p], c['U'][:, p],
                        c['Om'][:, p], c['R'], c['rho'], watch=watch)
    back = np.argsort(p)
    state = [a[:, back] for a in (sim.X, sim.U, sim.Om, sim.Ffp, sim.Tfp)]
    # the velocity field with its components and array axes named back (array
    # axis j holds coordinate 2 - j)
    _, u = sim.fields()
    u = np.transpose(u[back], [0] + [1 + 2 - back[2 - j] for j in range(3)])
    return state + [u], gaps


@pytest.mark.parametrize("perm", [(2, 0, 1), (1, 2, 0)])
def test_interacting_particles_are_invariant_under_axis_rotation(perm):
    # D3Q19, the mapping, the boundary conditions, the refill, the lubrication
    # and contact laws and the walls are all invariant under a rotation of the
    # lattice that permutes the axes cyclically (Secs. 2-4). A general
    # trajectory of interacting particles has no closed form, but it must be
    # the same, to rounding, in the rotated frame: this catches any axis that
    # is treated differently from the others
    a, (pair_gap, wall_gap) = rotated_run((0, 1, 2))
    b, gaps_b = rotated_run(perm)
    assert a[-1].shape == (3, 18, 14, 16) and b[-1].shape == a[-1].shape
    assert pair_gap < 0 and wall_gap < 0.05          # contact, and wall lubrication
    assert np.allclose(gaps_b, (pair_gap, wall_gap), rtol=0, atol=1e-12)
    close(a, b)


def shifted_run(shift):
    """PAIR_WALL translated by whole cells along the periodic axes x and y;
    the final state and field are translated back."""
    c = PAIR_WALL
    shift = np.array([shift[0], shift[1], 0])
    sim = run_pair_wall(c['shape'], c['periodic'], c['g'], (c['X'] + shift) % c['shape'], c['U'], c['Om'],
                        c['R'], c['rho'])
    _, u = sim.fields()
    u = np.roll(u, shift=(-shift[1], -shift[0]), axis=(2, 3))
    return [(sim.X - shift) % c['shape'], sim.U, sim.Om, sim.Ffp, sim.Tfp, u]


@pytest.mark.parametrize("shift", [(5, -3), (-13, 7)])
def test_interacting_particles_are_invariant_under_a_periodic_shift(shift):
    # a translation by whole cells along periodic axes is a symmetry of the
    # periodic box: the collisions that happen across the periodic sides in
    # PAIR_WALL happen inside the box after the shift (and the reverse), with
    # the same result to rounding
    close(shifted_run((0, 0)), shifted_run(shift))


def relabelled_run(order):
    """PAIR_WALL's spheres inserted in another order; the final state is put
    back into the original order."""
    c = PAIR_WALL
    p = list(order)
    sim = run_pair_wall(c['shape'], c['periodic'], c['g'], c['X'][p], c['U'][p], c['Om'][p], c['R'][p],
                        c['rho'][p])
    back = np.argsort(p)
    _, u = sim.fields()
    return [sim.X[back], sim.U[back], sim.Om[back], sim.Ffp[back], sim.Tfp[back], u]


@pytest.mark.parametrize("order", [(1, 0, 2), (2, 1, 0)])
def test_interacting_particles_do_not_depend_on_their_labels(order):
    # no cell lies inside two spheres here, so the particle index enters
    # nothing but bookkeeping: the two members of a colliding or lubricated
    # pair must get the same forces and torques whichever of them comes first
    # (Eqs. (25)-(33), (39)-(50) act on i and on j alike)
    close(relabelled_run((0, 1, 2)), relabelled_run(order))


def mirrored_run(axis):
    """PAIR_WALL's spheres, gravity and walls mirrored on the plane
    x_axis = L_axis / 2 (None: not mirrored); the final state is mirrored
    back. Vectors flip their axis component, pseudovectors (angular velocity,
    torque) the two others."""
    c = PAIR_WALL
    shape = c['shape']
    sv = np.ones(3)                  # sign of a vector's components
    X = c['X'].copy()
    if axis is not None:
        sv[axis] = -1.0
        X[:, axis] = shape[axis] - X[:, axis]
    sp = sv * np.prod(sv)            # sign of a pseudovector's components
    sim = run_pair_wall(shape, c['periodic'], c['g'] * sv, X, c['U'] * sv, c['Om'] * sp, c['R'], c['rho'])
    _, u = sim.fields()
    Xb = sim.X.copy()
    if axis is None:
        return [Xb, sim.U, sim.Om, sim.Ffp, sim.Tfp, u]
    Xb[:, axis] = shape[axis] - Xb[:, axis]
    if c['periodic'][axis]:
        Xb[:, axis] %= shape[axis]
    u = np.flip(u * sv[:, None, None, None], axis=1 + 2 - axis)
    return [Xb, sim.U * sv, sim.Om * sp, sim.Ffp * sv, sim.Tfp * sp, u]


@pytest.mark.parametrize("axis", [0, 2])
def test_interacting_particles_are_invariant_under_a_mirror(axis):
    # D3Q19 and every law of the step are symmetric under a reflection of one
    # axis (Secs. 2-4): PAIR_WALL mirrored on a periodic (x) or walled (z)
    # axis equals the original to rounding. This catches code that treats +c
    # and -c differently (one branch of a one-sided difference, one of the two
    # walls)
    close(mirrored_run(None), mirrored_run(axis))
