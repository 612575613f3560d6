"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Tolerances:
  * flags and owners (integer work): bit-exact;
  * float64 storage: relative L2 <= 1e-11 on PDFs, velocity, density and
    particle state for runs of up to 40 steps, <= 1e-10 for 300 steps (both
    sides are float64; only the summation order of the per-particle sums and
    the contraction into FMAs differ, each adding ~1e-16 per step, and the
    coupled dynamics carry these differences along);
  * float32 storage (and float32 collision): relative L2 <= 1e-6 on velocity
    and density, <= 1e-5 on particle positions, the targets of the float32
    path.
"""
import numpy as np
import pytest

from cases import build_gpu, build_oracle, spheres, rel_l2
from oracle.lbm import equilibrium

pytestmark = pytest.mark.gpu

F64_TOL = 1e-11


@pytest.fixture(scope='module')
def L():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2003_01490_gb300 import lbmdem
    lbmdem.load_library()
    return lbmdem


def random_state(shape, seed, amp_u=0.03):
    nx, ny, nz = shape
    r = np.random.default_rng(seed)
    f = equilibrium(1 + 0.01 * r.standard_normal((nz, ny, nx)), amp_u * r.standard_normal((3, nz, ny, nx)))
    return f * (1 + 0.02 * r.standard_normal(f.shape))


def random_spheres(shape, periodic, n, rmin, rmax, seed, gap=0.3):
    r = np.random.default_rng(seed)
    pos, rad = [], []
    L = np.array(shape, float)
    while len(rad) < n:
        R = r.uniform(rmin, rmax)
        p = r.uniform(0, 1, 3) * L
        ok = True
        for a in range(3):
            if not periodic[a] and (p[a] - R < 0.6 or p[a] + R > L[a] - 0.6):
                ok = False
        for q, Rq in zip(pos, rad):
            d = p - q
            for a in range(3):
                if periodic[a]:
                    d[a] -= L[a] * np.round(d[a] / L[a])
            if np.linalg.norm(d) < R + Rq + gap:
                ok = False
        if ok:
            pos.append(p)
            rad.append(R)
    return np.array(pos), np.array(rad)


# ---------------------------------------------------------------- mapping

@pytest.mark.parametrize('periodic', [(1, 1, 0), (1, 1, 1), (0, 1, 0)])
def test_mapping_is_bit_exact(L, periodic):
    shape = (70, 37, 41)            # not a multiple of the 32 x 4 x 4 tiles
    pos, rad = random_spheres(shape, periodic, 14, 2.2, 7.5, seed=sum(periodic))
    case = dict(shape=shape, periodic=periodic, tau=0.7, storage='f32',
                spheres=spheres(pos, rad, density=np.full(len(rad), 1.5)),
                dem=dict(fixed_particles=1))
    ora = build_oracle(case)
    ctx = build_gpu(case)
    _, _, flags = L.lbm_get_fields(ctx)
    owner = L.lbm_get_owner(ctx)
    solid = (flags & L.FLAG_SOLID) != 0
    assert np.array_equal(solid, ora.owner >= 0)
    assert np.array_equal(owner[solid], ora.owner[solid])
    assert np.array_equal((flags & L.FLAG_SHELL) != 0, ora.shell)
    # NEAR covers every fluid cell with a solid neighbour; MISS every solid
    # cell next to another body or a wall
    from oracle.d3q19 import C
    nx, ny, nz = shape
    fluid = ~solid
    need_near = np.zeros_like(fluid)
    need_miss = np.zeros_like(fluid)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
    for c in C[1:]:
        xs = [x + c[0], y + c[1], z + c[2]]
        out = np.zeros_like(fluid)
        for a, n in enumerate(shape):
            if periodic[a]:
                xs[a] = xs[a] % n
            else:
                out |= (xs[a] < 0) | (xs[a] >= n)
                xs[a] = np.clip(xs[a], 0, n - 1)
        nb_solid = solid[xs[2], xs[1], xs[0]] & ~out
        nb_owner = np.where(nb_solid, ora.owner[xs[2], xs[1], xs[0]], -1)
        need_near |= fluid & nb_solid
        need_miss |= solid & (out | (nb_solid & (nb_owner != ora.owner)))
    assert not (need_near & ((flags & L.FLAG_NEAR) == 0)).any()
    assert not (need_miss & ((flags & L.FLAG_MISS) == 0)).any()


# ---------------------------------------------------------------- fluid only

def test_fluid_with_moving_walls_f64(L):
    shape = (37, 20, 23)
    case = dict(shape=shape, periodic=(1, 0, 0), tau=0.62, storage='f64', body_force=(2e-5, 0, -1e-5),
                wall_vel_hi=[[0, 0, 0], [0.01, 0, 0.005], [0.02, -0.01, 0]],
                wall_vel_lo=[[0, 0, 0], [0, 0, 0], [-0.01, 0, 0]],
                relax=dict(lambda_b_bulk=3.0), init_pdfs=random_state(shape, 1))
    ora = build_oracle(case)
    ctx = build_gpu(case)
    ora.step(15)
    L.lbm_step(ctx, 15)
    f = L.lbm_get_pdfs(ctx)
    assert rel_l2(f - 1, ora.ft - 1) < F64_TOL
    rho, u, _ = L.lbm_get_fields(ctx)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o) < F64_TOL and rel_l2(rho, r_o) < F64_TOL


# ---------------------------------------------------------------- fixed particles

def fixed_particle_case(storage, shape=(40, 36, 30)):
    R = np.array([5.2, 4.6, 3.7])
    pos = np.array([[10.3, 17.9, 15.2], [10.3 + 5.2 + 4.6 + 0.35, 18.4, 14.6], [30.0, 6.0, 3.1 + 0.9]])
    vel = np.array([[0.01, -0.004, 0.002], [0.0, 0.006, -0.003], [-0.005, 0.0, 0.0]])
    om = np.array([[0.0, 0.001, -0.002], [0.003, 0.0, 0.0], [0.0, 0.0, 0.004]])
    return dict(shape=shape, periodic=(1, 1, 0), tau=0.58, storage=storage, body_force=(1e-5, 0, 0),
                spheres=spheres(pos, R, vel=vel, omega=om), dem=dict(fixed_particles=1),
                init_pdfs=random_state(shape, 2, amp_u=0.01))


def test_fixed_moving_boundaries_f64(L):
    case = fixed_particle_case('f64')
    ora = build_oracle(case)
    ctx = build_gpu(case)
    for _ in range(3):
        ora.step(3)
        L.lbm_step(ctx, 3)
        st = L.lbm_get_particle_state(ctx)
        assert rel_l2(st['force_hyd'], ora.Ffp) < F64_TOL
        assert rel_l2(st['torque_hyd'], ora.Tfp) < F64_TOL
    fluid = ora.owner < 0
    f = L.lbm_get_pdfs(ctx)
    assert rel_l2(f[:, fluid], ora.ft[:, fluid]) < F64_TOL


def test_fixed_moving_boundaries_f32(L):
    case = fixed_particle_case('f32')
    ora = build_oracle(case)
    ctx = build_gpu(case)
    ora.step(6)
    L.lbm_step(ctx, 6)
    st = L.lbm_get_particle_state(ctx)
    assert rel_l2(st['force_hyd'], ora.Ffp) < 1e-5
    assert rel_l2(st['torque_hyd'], ora.Tfp) < 1e-5
    rho, u, _ = L.lbm_get_fields(ctx)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o) < 1e-6 and rel_l2(rho, r_o) < 1e-6


# ---------------------------------------------------------------- moving particles

def collision_case(storage):
    shape = (34, 30, 36)
    R = np.array([4.0, 3.5, 3.2])
    # sphere 0 falls onto the wall z = 0; spheres 1 and 2 approach each other
    pos = np.array([[9.0, 9.5, 4.0 + 0.3], [22.3, 15.0, 18.0], [22.0, 15.2, 18.0 + 3.5 + 3.2 + 0.3]])
    vel = np.array([[0.01, 0.0, -0.06], [0.0, 0.0, 0.05], [0.0, 0.0, -0.05]])
    om = np.array([[0.0, 0.002, 0.0], [0.0, 0.0, 0.0], [0.001, 0.0, 0.0]])
    return dict(shape=shape, periodic=(1, 1, 0), tau=0.6, storage=storage,
                spheres=spheres(pos, R, density=np.array([10.0, 8.0, 8.0]), vel=vel, omega=om),
                dem=dict(gravity=(0.0, 0.0, -2e-4), Tc=8.0))


def test_moving_particles_collisions_f64(L):
    case = collision_case('f64')
    ora = build_oracle(case)
    ctx = build_gpu(case)
    contacts, refills = set(), 0
    for _ in range(8):
        for _ in range(5):
            ora.step(1)
            contacts |= {k[1] == 'wall' for k in ora.hist}
            refills += len(ora.refilled)
        L.lbm_step(ctx, 5)
        st = L.lbm_get_particle_state(ctx)
        assert rel_l2(st['pos'], ora.X) < F64_TOL
        assert rel_l2(st['vel'], ora.U) < F64_TOL
        assert rel_l2(st['omega'], ora.Om) < 1e-10
    rho, u, flags = L.lbm_get_fields(ctx)
    assert np.array_equal((flags & L.FLAG_SOLID) != 0, ora.owner >= 0)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o) < F64_TOL and rel_l2(rho, r_o) < F64_TOL
    # the case exercised sphere-wall and sphere-sphere contacts and refills
    assert contacts == {True, False} and refills > 0


def test_moving_particles_collisions_f32(L):
    case = collision_case('f32')
    ora = build_oracle(case)
    ctx = build_gpu(case)
    ora.step(40)
    L.lbm_step(ctx, 40)
    st = L.lbm_get_particle_state(ctx)
    assert rel_l2(st['pos'], ora.X) < 1e-5
    rho, u, flags = L.lbm_get_fields(ctx)
    both = (ora.owner < 0) & ((flags & L.FLAG_SOLID) == 0)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o, both) < 1e-6 and rel_l2(rho, r_o, both) < 1e-6


def prescribed_case(storage):
    # a sphere accelerated towards -z by a prescribed velocity (the artificial
    # acceleration of Sec. 2.3.3, scaled to a small box: u_s = 0.05, fast ramp),
    # spinning, between no-slip walls in x and y, periodic in z
    return dict(shape=(24, 24, 40), periodic=(0, 0, 1), tau=0.6, storage=storage,
                spheres=spheres([[12.0, 12.0, 20.0]], [4.5]), dem=dict(fixed_particles=2))


def prescribed_velocity(t, u_s=0.05, t_acc=8.0):
    return np.array([[0.0, 0.0, -u_s * (1.0 - np.exp(-t / t_acc))]])


@pytest.mark.parametrize('storage,tol', [('f64', F64_TOL), ('f32', 1e-6)])
def test_prescribed_motion(L, storage, tol):
    case = prescribed_case(storage)
    ora = build_oracle(case)
    ctx = build_gpu(case)
    om = np.array([[0.0, 0.002, 0.0]])
    refills = 0
    for t in range(1, 41):
        u = prescribed_velocity(t)
        ora.U, ora.Om = u.copy(), om.copy()
        L.lbm_set_particle_velocity(ctx, u, om)
        ora.step(1)
        L.lbm_step(ctx, 1)
        refills += len(ora.refilled)
    st = L.lbm_get_particle_state(ctx)
    assert np.abs(st['pos'] - ora.X).max() < 1e-12
    assert np.array_equal(st['vel'], ora.U) and np.array_equal(st['omega'], ora.Om)
    rho, u, flags = L.lbm_get_fields(ctx)
    assert np.array_equal((flags & L.FLAG_SOLID) != 0, ora.owner >= 0)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o) < tol and rel_l2(rho, r_o) < tol
    assert rel_l2(st['force_hyd'], ora.Ffp) < 100 * tol
    assert refills > 0


@pytest.mark.parametrize('storage,tol', [('f64', 1e-13), ('f32', 1e-6)])
@pytest.mark.parametrize('prescribed', [True, False])
def test_sphere_carried_by_uniform_flow(L, storage, tol, prescribed):
    # an exact solution of the coupled step (Algorithm 1): a sphere moving with
    # a uniform flow in a periodic box leaves the fluid in that flow's
    # equilibrium with zero force while it crosses cells; prescribed on an
    # oblique path, free (DEM) along x through mirror planes of the lattice
    n, steps = 14, 16
    U = np.array([0.071, -0.043, 0.029]) if prescribed else np.array([0.083, 0.0, 0.0])
    X0 = np.array([6.8, 7.3, 6.6]) if prescribed else np.array([6.8, 7.0, 7.0])
    f0 = equilibrium(np.ones((n, n, n)), np.broadcast_to(U[:, None, None, None], (3, n, n, n)))
    case = dict(shape=(n, n, n), periodic=(1, 1, 1), tau=0.8, storage=storage, init_pdfs=f0,
                spheres=spheres([X0], [2.7], density=[1.7], vel=[U]),
                dem=dict(fixed_particles=2 if prescribed else 0))
    ora = build_oracle(case)
    ctx = build_gpu(case)
    ora.step(steps)
    L.lbm_step(ctx, steps)
    st = L.lbm_get_particle_state(ctx)
    _, _, flags = L.lbm_get_fields(ctx)
    solid = (flags & L.FLAG_SOLID) != 0
    assert np.array_equal(solid, ora.owner >= 0)
    assert np.abs(st['pos'][0] - (X0 + steps * U) % n).max() < (1e-12 if storage == 'f64' else 1e-6)
    f = L.lbm_get_pdfs(ctx)
    feq = equilibrium(np.array(1.0), U)
    assert np.abs(f[:, ~solid] - feq[:, None]).max() < tol
    assert np.abs(st['force_hyd']).max() < 1e3 * tol
    if not prescribed:
        assert np.abs(st['vel'][0] - U).max() < 1e3 * tol
        assert np.abs(st['torque_hyd']).max() < 1e3 * tol


def test_prescribed_approach_then_free_motion_f64(L):
    # Sec. 4.4: the approach velocity is prescribed, then the sphere moves
    # freely (DEM with gravity) from the current state on
    case = prescribed_case('f64')
    case['dem'] = dict(fixed_particles=2, gravity=(0.0, 0.0, -2e-5))
    ora = build_oracle(case)
    ctx = build_gpu(case)
    for t in range(1, 16):
        u = prescribed_velocity(t)
        ora.U = u.copy()
        L.lbm_set_particle_velocity(ctx, u)
        ora.step(1)
        L.lbm_step(ctx, 1)
    ora.set_motion(dem=True)
    L.lbm_set_motion(ctx, L.MOTION_DEM)
    for _ in range(3):
        ora.step(5)
        L.lbm_step(ctx, 5)
        st = L.lbm_get_particle_state(ctx)
        assert rel_l2(st['pos'], ora.X) < F64_TOL
        assert rel_l2(st['vel'], ora.U) < 1e-10
    rho, u, flags = L.lbm_get_fields(ctx)
    assert np.array_equal((flags & L.FLAG_SOLID) != 0, ora.owner >= 0)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o) < F64_TOL and rel_l2(rho, r_o) < F64_TOL


def test_sphere_wall_workload_first_300_steps_f64(L):
    from paper_2003_01490_gb300 import workloads
    w = workloads.sphere_wall()
    case = dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage='f64',
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                dem=w['dem'])
    ora = build_oracle(case)
    ctx = build_gpu(case)
    ora.step(300)
    L.lbm_step(ctx, 300)
    st = L.lbm_get_particle_state(ctx)
    assert rel_l2(st['pos'], ora.X) < 10 * F64_TOL
    assert rel_l2(st['vel'], ora.U) < 10 * F64_TOL
    rho, u, _ = L.lbm_get_fields(ctx)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o) < 10 * F64_TOL and rel_l2(rho, r_o) < 10 * F64_TOL


# ---------------------------------------------------------------- suspension workload

def suspension_case(storage):
    from paper_2003_01490_gb300 import workloads
    w = workloads.reduced_suspension(storage=storage)
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=storage,
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                dem=w['dem'])


@pytest.fixture(scope='module')
def suspension_oracle():
    """Float64 oracle of the 64 x 64 x 128 suspension (150 spheres), 6 steps."""
    ora = build_oracle(suspension_case('f64'))
    ora.step(6)
    return ora


@pytest.mark.parametrize('storage,tol_u,tol_x', [('f64', F64_TOL, F64_TOL), ('f32', 1e-6, 1e-5)])
def test_reduced_suspension(L, suspension_oracle, storage, tol_u, tol_x):
    ora = suspension_oracle
    ctx = build_gpu(suspension_case(storage))
    L.lbm_step(ctx, 6)
    st = L.lbm_get_particle_state(ctx)
    assert rel_l2(st['pos'], ora.X) < tol_x
    rho, u, flags = L.lbm_get_fields(ctx)
    both = (ora.owner < 0) & ((flags & L.FLAG_SOLID) == 0)
    r_o, u_o = ora.fields()
    assert rel_l2(u, u_o, both) < tol_u and rel_l2(rho, r_o, both) < tol_u
    if storage == 'f64':
        assert np.array_equal((flags & L.FLAG_SOLID) != 0, ora.owner >= 0)
        assert rel_l2(st['force_hyd'], ora.Ffp) < 1e-10


@pytest.fixture(scope='module')
def full_size(L):
    """The 256 x 256 x 512 suspension (10,000 spheres) in the float32 launch
    configuration bench.py times, spheres held in place with the workload's
    velocities and seeded angular velocities, no gravity."""
    from paper_2003_01490_gb300 import workloads
    w = workloads.suspension()
    om = np.random.default_rng(17).normal(0.0, 1e-4, size=(len(w['radius']), 3))
    case = dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage='f32',
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], om),
                dem=dict(w['dem'], fixed_particles=1, gravity=(0.0, 0.0, 0.0), fluid_counterforce=0))
    ctx = build_gpu(case)
    return dict(w=w, omega=om, ctx=ctx, case=case)


def test_full_size_suspension_mapping_sampled(L, full_size):
    """256 x 256 x 512 cells, 10,000 spheres: the flags and owners of sampled
    cells equal a brute-force float64 evaluation over every nearby sphere."""
    from scipy.spatial import cKDTree
    from oracle import Domain
    from oracle.particles import map_cells
    w, ctx = full_size['w'], full_size['ctx']
    _, _, flags = L.lbm_get_fields(ctx)
    owner = L.lbm_get_owner(ctx)
    nx, ny, nz = w['shape']
    r = np.random.default_rng(5)
    cells = [r.integers(0, (nx, ny, nz), size=(40000, 3))]
    for i in r.choice(len(w['radius']), 12, replace=False):
        lo = np.floor(w['pos'][i] - 9).astype(int)
        g = np.stack(np.meshgrid(*[np.arange(lo[a], lo[a] + 19) for a in range(3)], indexing='ij'), -1)
        cells.append(g.reshape(-1, 3) % np.array([nx, ny, nz]))
    cells = np.unique(np.concatenate(cells), axis=0)
    tree = cKDTree(w['pos'], boxsize=np.array([nx, ny, nz], float))
    dom = Domain(nx, ny, nz)
    cand = tree.query_ball_point(cells + 0.5, r=w['radius'].max() + 2.0 + 0.1)
    for (x, y, z), js in zip(cells, cand):
        js = sorted(js)
        o, sh = map_cells(np.array([[x + 0.5, y + 0.5, z + 0.5]]), w['pos'][js], w['radius'][js], dom, 2.0)
        want_owner = js[o[0]] if o[0] >= 0 else -1
        fl = flags[z, y, x]
        assert bool(fl & L.FLAG_SOLID) == (want_owner >= 0), (x, y, z)
        if want_owner >= 0:
            assert owner[z, y, x] == want_owner, (x, y, z)
        assert bool(fl & L.FLAG_SHELL) == bool(sh[0]), (x, y, z)


def test_full_size_suspension_first_step_sampled(L, full_size):
    """The same full-size launch, one step from rest: the post-collision PDFs
    of sampled fluid cells next to sphere surfaces (particle links with CLI
    values of moving, spinning walls) and of random fluid cells equal the
    oracle's stream, boundary condition and collision evaluated on the 3x3x3
    neighbourhood of each cell (its own mapping of the nearby spheres, its own
    rest equilibrium as the start), and the force and torque of sampled spheres
    against the oracle on the box around each."""
    from scipy.spatial import cKDTree
    from oracle import Domain, Params
    from oracle.coupling import stream_and_couple
    from oracle.lbm import collide
    from oracle.particles import cell_centres, map_cells
    w, ctx, om = full_size['w'], full_size['ctx'], full_size['omega']
    nx, ny, nz = w['shape']
    L.lbm_step(ctx, 1)
    f_gpu = L.lbm_get_pdfs(ctx).reshape(19, nz, ny, nx)
    r = np.random.default_rng(23)
    # cells half a cell outside random sphere surfaces, and random cells
    k = r.choice(len(w['radius']), 240, replace=False)
    d = r.normal(size=(240, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    near = np.floor(w['pos'][k] + (w['radius'][k] + 0.6)[:, None] * d).astype(int)
    cells = np.concatenate([near, r.integers(0, (nx, ny, nz), size=(80, 3))]) % np.array([nx, ny, nz])
    L3 = np.array([nx, ny, nz], float)
    tree = cKDTree(w['pos'], boxsize=L3)
    dom_w = Domain(3, 3, 3, periodic=(False, False, False))
    centres_w = cell_centres(dom_w)
    s_bulk, s_shell = Params(tau=w['tau']).rates()
    ft_w = equilibrium(np.ones((3, 3, 3)), np.zeros((3, 3, 3, 3)))
    checked = links_seen = 0
    for x, y, z in cells:
        js = sorted(tree.query_ball_point([x + 0.5, y + 0.5, z + 0.5], r=w['radius'].max() + 2.0 + 2.0))
        origin = np.array([x - 1, y - 1, z - 1], float)
        Xw = w['pos'][js] - origin
        Xw -= L3 * np.round((Xw - 1.5) / L3)            # image nearest to the window
        Rw, Uw, Ow = w['radius'][js], w['vel'][js], om[js]
        owner_w, shell_w = map_cells(centres_w, Xw, Rw, dom_w, 2.0)
        if owner_w[1, 1, 1] >= 0:
            continue
        f_w, _, _ = stream_and_couple(ft_w, dom_w, owner_w, Xw, Uw, Ow, Rw)
        links_seen += int((owner_w >= 0).any())
        want = collide(f_w[:, 1:2, 1, 1], np.zeros(3), s_bulk, s_shell, shell_w[1:2, 1, 1])[:, 0]
        got = f_gpu[:, z, y, x]
        assert np.abs(got - want).max() < 1e-8, (x, y, z, np.abs(got - want).max())
        checked += 1
    assert checked > 200 and links_seen > 150
    # the momentum-exchange force and torque of sampled spheres (Eqs. (15)-(17)
    # with the missing links), from the oracle on the box around each sphere
    from oracle.coupling import missing_links
    st = L.lbm_get_particle_state(ctx)
    for i in r.choice(len(w['radius']), 12, replace=False):
        R = w['radius'][i]
        h = int(np.ceil(R)) + 3
        base = np.floor(w['pos'][i]).astype(int) - h
        dom_b = Domain(2 * h + 1, 2 * h + 1, 2 * h + 1, periodic=(False, False, False))
        js = sorted(tree.query_ball_point(w['pos'][i], r=R + w['radius'].max() + 2 * h))
        Xb = w['pos'][js] - base
        Xb -= L3 * np.round((Xb - (h + 0.5)) / L3)
        owner_b, _ = map_cells(cell_centres(dom_b), Xb, w['radius'][js], dom_b, 2.0)
        ft_b = equilibrium(np.ones(owner_b.shape), np.zeros((3,) + owner_b.shape))
        _, F, T = stream_and_couple(ft_b, dom_b, owner_b, Xb, w['vel'][js], om[js], w['radius'][js])
        Fm, Tm = missing_links(dom_b, owner_b, Xb, w['radius'][js])
        me = js.index(i)
        want_F, want_T = F[me] + Fm[me], T[me] + Tm[me]
        assert np.abs(st['force_hyd'][i] - want_F).max() < 1e-5 * np.abs(want_F).max() + 1e-9, i
        assert np.abs(st['torque_hyd'][i] - want_T).max() < 1e-5 * np.abs(want_T).max() + 1e-9, i


@pytest.mark.parametrize('storage,bound', [('f16', 2e-2), ('bf16', 1e-1)])
def test_reduced_precision_storage_error(L, suspension_oracle, storage, bound):
    """Shifted f16 / bf16 PDF storage (float32 collision, float64 particles):
    the measured error against the float64 oracle after 6 steps stays within
    a bound set by the storage precision (2^-11 and 2^-8 relative rounding of
    f_q - w_q); the measured error is printed beside the bound."""
    ora = suspension_oracle
    ctx = build_gpu(suspension_case(storage))
    L.lbm_step(ctx, 6)
    st = L.lbm_get_particle_state(ctx)
    rho, u, flags = L.lbm_get_fields(ctx)
    both = (ora.owner < 0) & ((flags & L.FLAG_SOLID) == 0)
    r_o, u_o = ora.fields()
    e_u, e_r = rel_l2(u, u_o, both), rel_l2(rho - 1, r_o - 1, both)
    e_x = np.sqrt(((st['pos'] - ora.X) ** 2).sum(1).mean()) / (2 * ora.R.mean())
    print('%s storage after 6 steps: rel L2 u %.3e, rel L2 (rho-1) %.3e, RMS position error / D %.3e'
          % (storage, e_u, e_r, e_x))
    assert e_u < bound and e_x < 1e-6
