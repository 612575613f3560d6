"""The batched form: many independent boxes advanced in lock step, one CUDA
graph per step with the dense kernels of all instances in one persistent
launch (lbm_batch_*).

* Every instance of a batch ends bit for bit where the same box ends when
  stepped alone, given the same tile and chunk of the dense kernel (the
  per-cell arithmetic is the same; the per-particle force sums of the 4- and
  2-byte formats are exact integer sums).
* A float64 instance inside a batch matches the float64 oracle (the batched
  dense kernel does Algorithm 1's step as the single-box one does).
* A deactivated instance is not touched; instances of different sizes, step
  counts and parameters coexist; the autotuner picks a launch shape.
"""
import numpy as np
import pytest

from cases import build_gpu, build_oracle, spheres, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def L():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2003_01490_gb300 import lbmdem
    lbmdem.load_library()
    return lbmdem


def sphere_wall_case(s, D, ratio, tau, storage, seed):
    r = np.random.default_rng(seed)
    g = 2e-4 * r.uniform(0.5, 1.5)
    return dict(shape=(s, s, 2 * s), periodic=(1, 1, 0), tau=tau, storage=storage,
                spheres=spheres([[s / 2 + r.uniform(-1, 1), s / 2 + r.uniform(-1, 1), 1.2 * s]], [D / 2],
                                density=[ratio], vel=[[0.0, 0.0, -0.01]], omega=[[0.0, 1e-3, 0.0]]),
                dem=dict(gravity=(0.0, 0.0, -g)))


def suspension_case(shape, n, storage, seed):
    from paper_2003_01490_gb300 import workloads
    w = workloads.suspension(shape=shape, n=n, D=10.0, seed=seed, storage=storage)
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=storage,
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']), dem=w['dem'])


def solo_launch(shape, sms):
    """Tile width and z chunk of the single-box dense launch (the library's rule)."""
    nx, ny, nz = shape
    bx = 128 if nx >= 128 else ((nx + 31) // 32) * 32
    by = 256 // bx
    bxy = ((nx + bx - 1) // bx) * ((ny + by - 1) // by)
    zc = (bxy * nz) // (4 * sms)
    return bx, max(1, min(24, zc))


def state(L, ctx):
    st = L.lbm_get_particle_state(ctx)
    return L.lbm_get_pdfs(ctx), st['pos'], st['vel'], st['omega']


@pytest.mark.parametrize('storage', ['f32', 'f16'])
def test_batch_equals_each_instance_alone(L, storage):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cases = [sphere_wall_case(32, 8.0, 4.0, 0.6, storage, 1), sphere_wall_case(40, 10.0, 2.0, 0.7, storage, 2),
             suspension_case((48, 48, 96), 30, storage, 3), sphere_wall_case(64, 16.0, 8.0, 0.55, storage, 4)]
    steps = 30
    solo = []
    for c in cases:
        ctx = build_gpu(c)
        L.lbm_step(ctx, steps)
        solo.append(state(L, ctx))
        del ctx
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)               # the first step of each instance runs on its own
    b = L.lbm_batch_create(ctxs)
    for i, c in enumerate(cases):
        bx, zc = solo_launch(c['shape'], sms)
        L.lbm_batch_set_launch(b, i, bx, zc, 4)
    L.lbm_batch_step(b, steps - 1)
    L.lbm_batch_sync(b)
    for i, ctx in enumerate(ctxs):
        got = state(L, ctx)
        for g, s_ in zip(got, solo[i]):
            assert np.array_equal(np.nan_to_num(g, nan=7.0), np.nan_to_num(s_, nan=7.0)), i
    # every instance has at most 32 particles, so each step is 11 gang
    # launches for all instances together: body force and missing links,
    # bin reset, bins, neighbour lists, the persistent dense launch, force
    # finalisation, the DEM steps, counter reset, tile scatter, mapping, refill
    assert L.lbm_batch_launch_count(b) == 11 * (steps - 1)


def test_float64_instance_in_a_batch_matches_the_oracle(L):
    case = dict(shape=(24, 20, 26), periodic=(1, 1, 0), tau=0.65, storage='f64',
                spheres=spheres([[8.0, 10.0, 4.3], [16.5, 9.5, 14.0]], [3.8, 3.0],
                                density=[3.0, 2.0], vel=[[0.0, 0.0, -0.02], [0.01, 0.0, 0.0]]),
                dem=dict(gravity=(0.0, 0.0, -1e-4)))
    others = [sphere_wall_case(32, 8.0, 4.0, 0.6, 'f64', 5), suspension_case((32, 32, 32), 6, 'f64', 6)]
    ora = build_oracle(case)
    ctxs = [build_gpu(case)] + [build_gpu(c) for c in others]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    ora.step(1)
    b = L.lbm_batch_create(ctxs)
    L.lbm_batch_step(b, 15)
    L.lbm_batch_sync(b)
    ora.step(15)
    st = L.lbm_get_particle_state(ctxs[0])
    rho, u, _ = L.lbm_get_fields(ctxs[0])
    r_o, u_o = ora.fields()
    assert rel_l2(st['pos'], ora.X) < 1e-11
    assert rel_l2(st['vel'], ora.U) < 1e-10
    assert rel_l2(u, u_o) < 1e-11 and rel_l2(rho, r_o) < 1e-11


def test_batch_of_widths_that_are_not_powers_of_two(L):
    # 96- and 72-cell wide boxes run in 128-wide tiles: same result as alone
    # within float32 rounding of the per-lane force sums (other tile shapes)
    cases = [sphere_wall_case(96, 24.0, 2.0, 0.6, 'f32', 13), sphere_wall_case(72, 18.0, 3.0, 0.6, 'f32', 14)]
    steps = 20
    solo = []
    for c in cases:
        ctx = build_gpu(c)
        L.lbm_step(ctx, steps)
        solo.append(state(L, ctx))
        del ctx
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    b = L.lbm_batch_create(ctxs)
    L.lbm_batch_step(b, steps - 1)
    L.lbm_batch_sync(b)
    for i, ctx in enumerate(ctxs):
        f, x, u, om = state(L, ctx)
        fluid = ~np.isnan(f)
        assert np.array_equal(fluid, ~np.isnan(solo[i][0]))
        assert rel_l2(f[fluid], solo[i][0][fluid]) < 1e-6
        assert rel_l2(x, solo[i][1]) < 1e-9 and rel_l2(u, solo[i][2]) < 1e-5


def test_inactive_instance_is_untouched_and_finished_instances_drop_out(L):
    cases = [sphere_wall_case(32, 8.0, 4.0, 0.6, 'f32', 7), sphere_wall_case(48, 12.0, 3.0, 0.6, 'f32', 8),
             sphere_wall_case(40, 10.0, 5.0, 0.62, 'f32', 9)]
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    b = L.lbm_batch_create(ctxs)
    L.lbm_batch_step(b, 5)
    L.lbm_batch_sync(b)
    before = state(L, ctxs[1])
    L.lbm_batch_set_active(b, 1, 0)
    L.lbm_batch_step(b, 7)
    L.lbm_batch_sync(b)
    after = state(L, ctxs[1])
    for x, y in zip(before, after):
        assert np.array_equal(np.nan_to_num(x, nan=7.0), np.nan_to_num(y, nan=7.0))
    # the others kept moving
    assert not np.array_equal(state(L, ctxs[0])[1], before[1])
    L.lbm_batch_set_active(b, 1, 1)
    L.lbm_batch_step(b, 2)
    L.lbm_batch_sync(b)


def test_batch_refuses_instances_that_never_stepped(L):
    ctxs = [build_gpu(sphere_wall_case(32, 8.0, 4.0, 0.6, 'f32', 10))]
    b = L.lbm_batch_create(ctxs)
    with pytest.raises(L.LbmError) as err:
        L.lbm_batch_step(b, 1)
    assert err.value.status == -7


def test_autotuner_picks_and_caches_a_launch_shape(L, tmp_path, monkeypatch):
    from paper_2003_01490_gb300 import tune
    monkeypatch.setattr(tune, 'CACHE', str(tmp_path / 'cache.json'))
    cases = [sphere_wall_case(32, 8.0, 4.0, 0.6, 'f32', 11), sphere_wall_case(64, 16.0, 3.0, 0.6, 'f32', 12)]
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    b = L.lbm_batch_create(ctxs)
    cands = [(0, 8, 4), (0, 16, 2), (32, 32, 3)]
    best = tune.tune_batch(b, 'f32', steps=2, cands=cands, restore=True)
    assert best['source'] == 'timed' and (best['tile_bx'], best['zchunk'], best['blocks_per_sm']) in cands
    again = tune.tune_batch(b, 'f32', steps=2, cands=cands)
    assert again['source'] == 'cache' and again['zchunk'] == best['zchunk']
    L.lbm_batch_step(b, 3)
    L.lbm_batch_sync(b)


def test_two_batches_on_their_own_streams_equal_each_instance_alone(L):
    # disjoint instances in two batches that run concurrently, each on its own
    # stream (ordered against the contexts' stream by events)
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cases = [sphere_wall_case(32, 8.0, 4.0, 0.6, 'f32', 21), sphere_wall_case(40, 10.0, 2.0, 0.7, 'f32', 22),
             sphere_wall_case(48, 12.0, 3.0, 0.6, 'f32', 23), sphere_wall_case(64, 14.0, 5.0, 0.65, 'f32', 24)]
    steps = 25
    solo = []
    for c in cases:
        ctx = build_gpu(c)
        L.lbm_step(ctx, steps)
        solo.append(state(L, ctx))
        del ctx
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    batches = [L.lbm_batch_create(ctxs[0::2], stream=streams[0]), L.lbm_batch_create(ctxs[1::2], stream=streams[1])]
    for b, part in zip(batches, (cases[0::2], cases[1::2])):
        for i, c in enumerate(part):
            bx, zc = solo_launch(c['shape'], sms)
            L.lbm_batch_set_launch(b, i, bx, zc, 2)
    for b in batches:
        L.lbm_batch_step(b, steps - 1)
    for b in batches:
        L.lbm_batch_sync(b)
    for i, ctx in enumerate(ctxs):      # read on the contexts' stream: ordered after the batches
        for g, s_ in zip(state(L, ctx), solo[i]):
            assert np.array_equal(np.nan_to_num(g, nan=7.0), np.nan_to_num(s_, nan=7.0)), i


def test_contexts_moved_to_their_batch_streams_run_concurrently_and_equal_each_alone(L):
    # tune.make_groups moves each batch's contexts onto its stream
    # (lbm_set_stream), so the batches share no stream; the results stay those
    # of each instance alone, and the contexts' later work follows the batches
    import torch
    from paper_2003_01490_gb300 import tune
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cases = [sphere_wall_case(32, 8.0, 4.0, 0.6, 'f32', 31), sphere_wall_case(40, 10.0, 2.0, 0.7, 'f32', 32),
             sphere_wall_case(48, 12.0, 3.0, 0.6, 'f32', 33), sphere_wall_case(64, 14.0, 5.0, 0.65, 'f32', 34)]
    steps = 25
    solo = []
    for c in cases:
        ctx = build_gpu(c)
        L.lbm_step(ctx, steps + 3)
        solo.append(state(L, ctx))
        del ctx
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    groups = tune.make_groups(ctxs, 2)
    for g, (b, _) in enumerate(groups):
        for i, c in enumerate(cases[g::2]):
            bx, zc = solo_launch(c['shape'], sms)
            L.lbm_batch_set_launch(b, i, bx, zc, 2)
    for b, _ in groups:
        L.lbm_batch_step(b, steps - 1)
    for ctx in ctxs:                    # plain steps on the contexts' new streams
        L.lbm_step(ctx, 3)
    for b, _ in groups:
        L.lbm_batch_sync(b)
    for i, ctx in enumerate(ctxs):
        for g, s_ in zip(state(L, ctx), solo[i]):
            assert np.array_equal(np.nan_to_num(g, nan=7.0), np.nan_to_num(s_, nan=7.0)), i


@pytest.mark.parametrize('kind', ['fixed', 'many', 'prescribed'])
def test_every_kind_of_instance_in_gang_launches_equals_itself_alone(L, kind):
    # beside a one-sphere instance (one-block DEM): 'fixed', an instance with
    # held particles (no DEM, mapping or refill); 'many', one with 40
    # particles (the multi-block DEM: first position update, one launch per
    # subcycle); 'prescribed', one moved by its set velocities
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    other = suspension_case((48, 48, 96), 40 if kind == 'many' else 12, 'f32', 41)
    if kind != 'many':
        other['dem'] = dict(other['dem'], fixed_particles=1 if kind == 'fixed' else 2)
    cases = [sphere_wall_case(32, 8.0, 4.0, 0.6, 'f32', 42), other]
    steps = 20
    solo = []
    for c in cases:
        ctx = build_gpu(c)
        L.lbm_step(ctx, steps)
        solo.append(state(L, ctx))
        del ctx
    ctxs = [build_gpu(c) for c in cases]
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    b = L.lbm_batch_create(ctxs)
    for i, c in enumerate(cases):
        bx, zc = solo_launch(c['shape'], sms)
        L.lbm_batch_set_launch(b, i, bx, zc, 4)
    L.lbm_batch_step(b, steps - 1)
    L.lbm_batch_sync(b)
    for i, ctx in enumerate(ctxs):
        got = state(L, ctx)
        assert np.array_equal(np.nan_to_num(got[0], nan=7.0), np.nan_to_num(solo[i][0], nan=7.0)), (kind, i)
        for g, s_ in zip(got[1:], solo[i][1:]):
            if kind == 'many' and i == 1:
                # the multi-block DEM runs in another compiled kernel in a gang
                # launch than alone, whose float64 contractions may differ: its
                # particle state agrees to rounding (the fluid, which sees the
                # particles through float32 views, bit for bit)
                err = np.abs(g - s_).max() / max(np.abs(s_).max(), 1e-300)
                print('multi-block DEM in a gang launch: max relative difference %.1e' % err)
                assert err < 1e-10, err
            else:
                assert np.array_equal(g, s_), (kind, i)
    # 11 gang launches a step, plus the first position update and the 10
    # subcycles of the multi-block DEM, or the prescribed move
    extra = {'fixed': 0, 'many': 11, 'prescribed': 1}[kind]
    assert L.lbm_batch_launch_count(b) == (11 + extra) * (steps - 1)
