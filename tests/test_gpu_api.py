"""Argument checks of the C ABI that need a device context (lbm_create
allocates on the GPU): sphere insertion rules of lbm_add_spheres, capacity,
state, and the NaN marker that solid cells show through lbm_get_pdfs."""
import numpy as np
import pytest

from cases import build_gpu, spheres

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def L():
    from paper_2003_01490_gb300 import lbmdem
    lbmdem.load_library()
    return lbmdem


def fresh(L, shape=(40, 36, 30), periodic=(1, 1, 0), max_particles=8, storage='f32'):
    return build_gpu(dict(shape=shape, periodic=periodic, tau=0.6, storage=storage), max_particles=max_particles)


def add(L, ctx, pos, R):
    sp = spheres(pos, R)
    return L.lbm_add_spheres(ctx, sp['pos'], sp['vel'], sp['omega'], sp['radius'], sp['density'])


def test_overlap_across_the_periodic_side_is_rejected(L):
    ctx = fresh(L)
    add(L, ctx, [[2.0, 18.0, 15.0]], [4.0])
    # centre distance 2 + 40 - 35 = 7 < 8 through the periodic x side
    with pytest.raises(L.LbmError) as e:
        add(L, ctx, [[35.0, 18.0, 15.0]], [4.0])
    assert e.value.status == L.STATUS_CODES['LBM_ERR_INVALID']
    # 8.5 apart: accepted, also within one call
    add(L, ctx, [[33.5, 18.0, 15.0], [14.0, 18.0, 15.0]], [4.0, 4.0])


def test_overlap_within_one_call_is_rejected(L):
    ctx = fresh(L)
    with pytest.raises(L.LbmError):
        add(L, ctx, [[10.0, 10.0, 10.0], [17.9, 10.0, 10.0]], [4.0, 4.0])


def test_wall_crossing_short_periodic_side_and_capacity(L):
    ctx = fresh(L, max_particles=2)
    with pytest.raises(L.LbmError):
        add(L, ctx, [[10.0, 10.0, 2.0]], [3.0])       # crosses the z wall
    ctx2 = fresh(L, shape=(40, 20, 30), max_particles=2)
    with pytest.raises(L.LbmError):
        add(L, ctx2, [[10.0, 10.0, 15.0]], [8.0])     # 2 R + 4 >= 20 on periodic y
    add(L, ctx, [[10.0, 10.0, 10.0], [25.0, 25.0, 15.0]], [3.0, 3.0])
    with pytest.raises(L.LbmError) as e:
        add(L, ctx, [[30.0, 10.0, 15.0]], [3.0])
    assert e.value.status == L.STATUS_CODES['LBM_ERR_CAPACITY']


def test_radius_outside_one_to_hundred_cells_is_rejected(L):
    # the exact integer link sums of a particle stay inside 32 bits up to R = 100
    ctx = fresh(L, shape=(208, 208, 208), periodic=(1, 1, 1), max_particles=2)
    for R in (0.5, 100.5):
        with pytest.raises(L.LbmError) as e:
            add(L, ctx, [[104.0, 104.0, 104.0]], [R])
        assert e.value.status == L.STATUS_CODES['LBM_ERR_INVALID']
    add(L, ctx, [[104.0, 104.0, 104.0]], [100.0])


def test_spheres_only_before_the_first_step(L):
    ctx = fresh(L)
    add(L, ctx, [[10.0, 10.0, 10.0]], [3.0])
    L.lbm_step(ctx, 1)
    with pytest.raises(L.LbmError) as e:
        add(L, ctx, [[25.0, 25.0, 15.0]], [3.0])
    assert e.value.status == L.STATUS_CODES['LBM_ERR_STATE']


@pytest.mark.parametrize('storage', ['f64', 'f32', 'f16', 'bf16'])
def test_solid_cells_hold_the_marker(L, storage):
    ctx = fresh(L, storage=storage)
    add(L, ctx, [[12.3, 17.6, 14.9]], [5.2])
    L.lbm_step(ctx, 3)
    f = L.lbm_get_pdfs(ctx)
    solid = L.lbm_get_owner(ctx) >= 0
    assert solid.sum() > 0
    assert np.isnan(f[:, solid]).all()
    assert np.isfinite(f[:, ~solid]).all()
    # values uploaded for solid cells are replaced by the marker
    g = np.where(np.isnan(f), 0.05, f)
    L.lbm_set_pdfs(ctx, g)
    h = L.lbm_get_pdfs(ctx)
    assert np.isnan(h[:, solid]).all()
    assert np.array_equal(h[:, ~solid], g[:, ~solid])


def test_graph_replayed_steps_equal_plain_launches(L):
    """Steps after the first replay a captured CUDA graph; with phase timing on,
    the same steps run as plain launches. Float32 sums are order-independent
    (fixed point), so both give identical PDFs and particle states."""
    from cases import spheres as mk
    R = np.array([4.5, 3.8, 4.1])
    pos = np.array([[10.2, 12.7, 9.9], [20.3, 13.1, 10.4], [14.8, 24.6, 16.2]])
    vel = np.array([[0.01, 0.0, -0.004], [-0.008, 0.002, 0.0], [0.0, -0.006, 0.003]])
    case = dict(shape=(34, 36, 30), periodic=(1, 1, 0), tau=0.6, storage='f32',
                body_force=(1e-5, 0.0, 0.0), spheres=mk(pos, R, vel=vel),
                dem=dict(gravity=(0.0, 0.0, -2e-5)))
    a = build_gpu(case)
    b = build_gpu(case)
    L.lbm_profile(b, 1)
    for n in (1, 4, 7):          # odd and even step counts from both buffer parities
        L.lbm_step(a, n)
        L.lbm_step(b, n)
    assert np.array_equal(L.lbm_get_pdfs(a), L.lbm_get_pdfs(b), equal_nan=True)
    sa, sb = L.lbm_get_particle_state(a), L.lbm_get_particle_state(b)
    for k in ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd'):
        assert np.array_equal(sa[k], sb[k]), k
    assert L.lbm_launch_count(a) == L.lbm_launch_count(b)


def test_concurrent_contexts_equal_each_run_alone(L):
    """Independent contexts on their own streams (the batched mode of
    bench.py) give exactly the results of each box run by itself."""
    import torch
    from paper_2003_01490_gb300 import workloads
    inst = workloads.batched(n=3, seed=77, storage='f32', steps_divisor=200)

    def make(w):
        case = dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=w['storage'],
                    spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                    dem=w['dem'])
        return build_gpu(case)

    alone = []
    for w in inst:
        ctx = make(w)
        L.lbm_step(ctx, w['steps'])
        alone.append((L.lbm_get_pdfs(ctx), L.lbm_get_particle_state(ctx)))
    streams = [torch.cuda.Stream() for _ in inst]
    ctxs = []
    for w, st in zip(inst, streams):
        with torch.cuda.stream(st):
            ctxs.append(make(w))
    left = [w['steps'] for w in inst]
    while any(left):
        for k, (ctx, st) in enumerate(zip(ctxs, streams)):
            if left[k]:
                n = min(3, left[k])
                with torch.cuda.stream(st):
                    L.lbm_step(ctx, n)
                left[k] -= n
    torch.cuda.synchronize()
    for (f, s), ctx in zip(alone, ctxs):
        assert np.array_equal(L.lbm_get_pdfs(ctx), f, equal_nan=True)
        s2 = L.lbm_get_particle_state(ctx)
        for k in ('pos', 'vel', 'omega'):
            assert np.array_equal(s2[k], s[k]), k


def test_served_jobs_equal_each_run_alone(L):
    """Continuous batching (jobs admitted over time, advanced in rounds on
    their own streams) leaves every job's result exactly as if it ran alone."""
    from paper_2003_01490_gb300 import serve, workloads
    jobs = workloads.served(n=4, seed=5, storage='f16', steps_divisor=400, max_side=48, gap=0.001)
    mixed = serve.serve(jobs, budget_bytes=1 << 34, chunk=3, keep_state=True)
    alone = serve.fifo(jobs, keep_state=True)
    for a, b in zip(mixed, alone):
        for k in ('pos', 'vel', 'omega'):
            assert np.array_equal(a['state'][k], b['state'][k]), (a['name'], k)
    summ = serve.summary(mixed)
    assert summ['jobs'] == 4 and summ['p99_latency_s'] >= summ['p50_latency_s'] > 0


def checkpoint_case():
    from paper_2003_01490_gb300 import workloads
    w = workloads.suspension(shape=(48, 48, 64), n=24, D=12.0, seed=20030149, storage='f32', steps=0)
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage='f32',
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']), dem=w['dem'])


def state(L, ctx):
    st = L.lbm_get_particle_state(ctx)
    return [st[k] for k in ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd')] + [L.lbm_get_pdfs(ctx)]


def test_checkpoint_restore_continues_bit_for_bit(L):
    case = checkpoint_case()
    ctx = build_gpu(case)
    L.lbm_step(ctx, 10)
    buf = L.lbm_save(ctx)
    L.lbm_step(ctx, 15)
    a = state(L, ctx)
    # back into the same context, and into a fresh one created the same way
    L.lbm_restore(ctx, buf)
    L.lbm_step(ctx, 15)
    fresh = build_gpu(case)
    L.lbm_restore(fresh, buf)
    L.lbm_step(fresh, 15)
    for b in (state(L, ctx), state(L, fresh)):
        for x, y in zip(a, b):
            assert np.array_equal(x, y, equal_nan=True)


def test_restore_rejects_other_contexts_and_garbage(L):
    ctx = build_gpu(checkpoint_case())
    buf = L.lbm_save(ctx)
    other = fresh(L)
    with pytest.raises(L.LbmError) as e:
        L.lbm_restore(other, buf)
    assert e.value.status == L.STATUS_CODES['LBM_ERR_INVALID']
    with pytest.raises(L.LbmError):
        L.lbm_restore(ctx, np.zeros(64, dtype=np.uint8))


def test_unstable_runs_and_fast_particles_are_reported(L):
    # failure detection without a GPU fault: the device status word turns a
    # blown-up density and a particle faster than 0.5 cells per step into
    # errors at the next synchronising call
    ctx = build_gpu(dict(shape=(24, 24, 24), periodic=(1, 1, 0), tau=0.505, storage='f32',
                         body_force=(0.02, 0.0, 0.0), spheres=spheres([[12.0, 12.0, 12.0]], [4.0]),
                         dem=dict(fixed_particles=1)))
    L.lbm_step(ctx, 500)
    with pytest.raises(L.LbmError) as e:
        L.lbm_sync(ctx)
    assert e.value.status == L.STATUS_CODES['LBM_ERR_UNSTABLE']
    # the error is sticky in its context; a new context is unaffected
    with pytest.raises(L.LbmError):
        L.lbm_sync(ctx)
    ctx2 = fresh(L)
    add(L, ctx2, [[20.0, 18.0, 15.0]], [3.0])
    L.lbm_set_particle_velocity(ctx2, np.array([[0.6, 0.0, 0.0]]))
    L.lbm_step(ctx2, 1)
    with pytest.raises(L.LbmError) as e:
        L.lbm_sync(ctx2)
    assert e.value.status == L.STATUS_CODES['LBM_ERR_UNSTABLE']


def test_density_probe_interpolates_a_linear_field_exactly(L):
    # lbm_sample_density: trilinear interpolation of the cell-centred density;
    # a density linear in x (equilibrium at rest) is reproduced at any point
    # between cell centres
    shape = (24, 20, 16)
    ctx = build_gpu(dict(shape=shape, periodic=(1, 1, 1), tau=0.7, storage='f32'))
    nx, ny, nz = shape
    rho_x = 1.0 + 1e-3 * np.arange(nx)
    W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = W[:, None, None, None] * rho_x[None, None, None, :] * np.ones((1, nz, ny, 1))
    L.lbm_set_pdfs(ctx, f.reshape(19, -1))
    pts = np.random.default_rng(3).uniform([0.5, 0.0, 0.0], [nx - 0.5, ny, nz], size=(50, 3))
    got = L.lbm_sample_density(ctx, pts)
    assert np.abs(got - (1.0 + 1e-3 * (pts[:, 0] - 0.5))).max() < 1e-6


def test_async_particle_state_read_out_equals_the_synchronous_one(L):
    # one read-out queued after every step into page-locked buffers (later
    # copies overwrite earlier ones in stream order); after lbm_sync the
    # buffers hold the state of the last step, equal to the synchronous
    # read-out of a twin context; a buffer of the wrong size is refused
    import torch
    case = checkpoint_case()
    a, b = build_gpu(case), build_gpu(case)
    n = len(case['spheres']['radius'])
    keys = ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd')
    pinned = {k: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy() for k in keys}
    for _ in range(12):
        L.lbm_step(a, 1)
        L.lbm_get_particle_state_async(a, pinned)
    L.lbm_sync(a)
    L.lbm_step(b, 12)
    ref = L.lbm_get_particle_state(b)
    for k in keys:
        assert np.array_equal(pinned[k], ref[k]), k
    # only some of the arrays
    L.lbm_get_particle_state_async(a, {'vel': pinned['vel']})
    L.lbm_sync(a)
    with pytest.raises(ValueError):
        L.lbm_get_particle_state_async(a, {'pos': np.zeros((n, 2))})
