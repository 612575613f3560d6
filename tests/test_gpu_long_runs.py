"""Parity with the float64 oracle at the stated step counts.

* The 32 x 32 x 64 sphere-wall collision in float64 over its whole 2000
  steps: the sphere settles, enters the wall's lubrication range and hits the
  wall (first contact at step 1564 in the oracle), so contact, lubrication
  and the wall laws of Secs. 3.1 and 4.1 are all compared. Particle state
  after every step, fields after steps 1000 and 2000.
  Tolerance: both sides compute in float64 and differ only in summation order
  and FMA contraction (~1e-16 relative per operation). Over 40 steps that
  shows as ~1e-12 relative in the fields, over 300 steps ~1e-11 (the dynamics
  carry the differences along, see test_gpu_parity.py); 2000 steps with a
  stiff contact (T_c = 32 steps) amplify them further, so the bounds sit at
  1e-9 (fields, trajectory) -- still seven orders below the float32 path.
* The 64 x 64 x 128 suspension (150 spheres of D = 12) at step 1000 (and
  5000 where the oracle run has reached it) against two floors, both from
  float64 oracle runs (tests/golden/make_long_runs.py, oracle only):
  - the predictability floor: the divergence of two runs whose inputs differ
    by 1e-12 in one position (suspension_64x64x128_floor.txt);
  - the storage floor: the divergence caused by storing f - w in the format
    alone, the oracle's PDFs rounded to it after every step
    (suspension_64x64x128_storage_floor.txt).
  Where both floors lie below the float32 targets (relative L2 1e-6 on
  velocity and density, 1e-5 on positions) the targets are asserted; where a
  floor lies above a target no implementation storing that format can meet
  it, and the error is held to a small multiple of the floor (the kernels
  also round their arithmetic, which the storage floor leaves out).
* The precision forms (float16 / bfloat16 storage of f - w) on the same
  suspension, errors against their storage floors.
"""
import os

import numpy as np
import pytest

from cases import build_gpu, spheres

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, 'golden')


@pytest.fixture(scope='module')
def L():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2003_01490_gb300 import lbmdem
    lbmdem.load_library()
    return lbmdem


def rel_l2(a, b, mask=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    return float(np.sqrt(((a - b) ** 2).sum()) / np.sqrt((b * b).sum()))


def sphere_wall_case(storage):
    from paper_2003_01490_gb300 import workloads
    w = workloads.sphere_wall()
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=storage,
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']), dem=w['dem'])


def test_sphere_wall_collision_over_its_2000_steps_f64(L):
    gold = np.load(os.path.join(GOLDEN, 'sphere_wall_2000.npz'))
    ref = gold['states']                      # per step: x, u, omega, F^fp, T^fp
    ctx = build_gpu(sphere_wall_case('f64'))
    got = []
    fields = {}
    for step in range(1, 2001):
        L.lbm_step(ctx, 1)
        st = L.lbm_get_particle_state(ctx)
        got.append(np.concatenate([st['pos'][0], st['vel'][0], st['omega'][0]]))
        if step in (1000, 2000):
            rho, u, flags = L.lbm_get_fields(ctx)
            fields[step] = (rho, u, (flags & L.FLAG_SOLID) != 0)
    got = np.array(got)
    R = 4.0
    gap_gpu, gap_ref = got[:, 2] - R, ref[:, 2] - R
    # the run reaches the wall: contact (overlap) on both sides, at the same step
    assert gap_ref.min() < 0 and gap_gpu.min() < 0
    first_ref, first_gpu = int(np.argmax(gap_ref < 0)), int(np.argmax(gap_gpu < 0))
    assert first_gpu == first_ref
    e_x = rel_l2(got[:, :3], ref[:, :3])
    e_u = rel_l2(got[:, 3:6], ref[:, 3:6])
    e_gap = np.abs(gap_gpu - gap_ref).max() / np.abs(gap_ref).max()
    errs = {}
    for step in (1000, 2000):
        rho, u, solid = fields[step]
        both = ~solid & ~gold['solid_%d' % step]
        errs[step] = (rel_l2(u, gold['u_%d' % step], both), rel_l2(rho, gold['rho_%d' % step], both),
                      rel_l2(rho - 1.0, gold['rho_%d' % step] - 1.0, both))
    print('sphere-wall f64, 2000 steps: trajectory rel L2 x %.2e, u %.2e, gap %.2e; fields at 1000: u %.2e, '
          'rho %.2e, rho-1 %.2e; at 2000: u %.2e, rho %.2e, rho-1 %.2e'
          % ((e_x, e_u, e_gap) + errs[1000] + errs[2000]))
    assert e_x < 1e-9 and e_u < 1e-9 and e_gap < 1e-9
    for step in (1000, 2000):
        # rho - 1 is ~1e-5 at rest, so its relative error is the most sensitive
        # number here (1.3e-9 measured at step 2000 on GB300)
        assert errs[step][0] < 1e-9 and errs[step][1] < 1e-12 and errs[step][2] < 1e-8


# ------------------------------------------------------------ suspension at 1000 / 5000 steps

def load_rows(name, keyed_by_format=False):
    p = os.path.join(GOLDEN, name)
    if not os.path.exists(p):
        pytest.skip('%s not stored yet (tests/golden/make_long_runs.py)' % name)
    rows = {}
    for line in open(p):
        if line.startswith('#') or not line.strip():
            continue
        v = line.split()
        key = (v[0], int(v[1])) if keyed_by_format else int(v[0])
        vals = v[2:] if keyed_by_format else v[1:]
        rows[key] = dict(zip(('u', 'rho', 'rho1', 'pos', 'pos_d', 'vel'), map(float, vals)))
    return rows


def suspension_case(storage):
    from paper_2003_01490_gb300 import workloads
    w = workloads.reduced_suspension(storage=storage)
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=storage,
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']), dem=w['dem'])


def errors_against(L, ctx, gold, step):
    """Errors of the context's state against an oracle file at `step`: fields
    over cells fluid on both sides (rho - 1 from the file's float32 rho - 1,
    or from its float32 rho where only that is stored), particle state with
    periodic images."""
    shape = np.array([64.0, 64.0, 128.0])
    st = L.lbm_get_particle_state(ctx)
    rho, u, flags = L.lbm_get_fields(ctx)
    both = ((flags & L.FLAG_SOLID) == 0) & ~gold['solid_%d' % step]
    if 'drho_%d' % step in gold.files:
        d_ref = gold['drho_%d' % step].astype(np.float64)
    else:
        d_ref = gold['rho_%d' % step].astype(np.float64) - 1.0
    k = list(gold['state_steps']).index(step)
    xr = gold['states'][k][:, :3]
    d = st['pos'] - xr
    d -= shape * np.round(d / shape)
    return dict(u=rel_l2(u, gold['u_%d' % step], both), rho=rel_l2(rho, 1.0 + d_ref, both),
                rho1=rel_l2(rho - 1.0, d_ref, both),
                pos=float(np.sqrt((d * d).sum() / (xr * xr).sum())),
                pos_d=float(np.sqrt((d * d).sum(1).mean()) / 12.0),
                vel=rel_l2(st['vel'], gold['states'][k][:, 3:6]))


def report(label, e, floors):
    keys = ('u', 'rho', 'rho1', 'pos', 'pos_d', 'vel')
    print('%s: ' % label + ', '.join('%s %.2e' % (k, e[k]) for k in keys))
    for name, f in floors.items():
        print('    %s floor: ' % name + ', '.join('%s %.2e' % (k, f[k]) for k in keys))


def run_to_1000(L, storage):
    path = os.path.join(GOLDEN, 'suspension_64x64x128_1000.npz')
    if not os.path.exists(path):
        pytest.skip('oracle run not stored yet (tests/golden/make_long_runs.py storage)')
    gold = np.load(path)
    ctx = build_gpu(suspension_case(storage))
    L.lbm_step(ctx, 1000)
    return ctx, errors_against(L, ctx, gold, 1000)


# where a target lies below a floor, the error is held to this multiple of
# the floor: the kernels' float32 arithmetic adds rounding of its own
# (measured on GB300 at step 1000: float16 1.04 x its storage floor in u,
# bfloat16 1.00 x)
ARITH_FACTOR = 1.5


def test_reduced_suspension_f32_at_1000_steps_against_the_floors(L):
    chaos = load_rows('suspension_64x64x128_floor.txt')[1000]
    storage = load_rows('suspension_64x64x128_storage_floor.txt', keyed_by_format=True)[('f32', 1000)]
    _, e = run_to_1000(L, 'f32')
    report('f32 step 1000', e, {'predictability': chaos, 'f32 storage': storage})
    # the float32 copies of rho in the predictability runs resolve no density
    # difference below 6e-8: that floor's rho columns are not used. Measured
    # on GB300: u 3.4e-7, rho 4.1e-10, positions 1.0e-9 (all floors lie
    # below the targets, so the targets are asserted)
    for key, tol in (('u', 1e-6), ('rho', 1e-6), ('pos', 1e-5)):
        floor = storage[key] if key.startswith('rho') else max(storage[key], chaos[key])
        if floor < tol:
            assert e[key] < tol, (key, e[key], floor)
        else:
            assert e[key] < ARITH_FACTOR * floor, (key, e[key], floor)


@pytest.mark.parametrize('storage', ['f16', 'bf16'])
def test_precision_form_errors_at_1000_steps_against_their_storage_floor(L, storage):
    floor = load_rows('suspension_64x64x128_storage_floor.txt', keyed_by_format=True)[(storage, 1000)]
    _, e = run_to_1000(L, storage)
    report('%s step 1000' % storage, e, {storage + ' storage': floor})
    for key in ('u', 'rho1', 'pos_d', 'vel'):
        assert e[key] < ARITH_FACTOR * floor[key], (key, e[key], floor[key])


def test_reduced_suspension_f32_at_5000_steps_against_the_predictability_floor(L):
    path = os.path.join(GOLDEN, 'suspension_64x64x128_5000.npz')
    if not os.path.exists(path) or 'u_5000' not in np.load(path).files:
        pytest.skip('oracle run has not reached step 5000 (tests/golden/make_long_runs.py suspension)')
    gold = np.load(path)
    rows = load_rows('suspension_64x64x128_floor.txt')
    if 5000 not in rows:
        pytest.skip('predictability floor at step 5000 not written yet (tests/golden/make_long_runs.py floor)')
    chaos = rows[5000]
    ctx = build_gpu(suspension_case('f32'))
    L.lbm_step(ctx, 5000)
    e = errors_against(L, ctx, gold, 5000)
    report('f32 step 5000', e, {'predictability': chaos})
    # a float32 run is a perturbation of ~1e-7 of every value, the floor's of
    # 1e-12 of one position: where chaos has amplified the latter beyond the
    # targets, the former is held to 1e5 times it
    for key, tol in (('u', 1e-6), ('pos', 1e-5)):
        if chaos[key] >= tol:
            assert e[key] < 1e5 * chaos[key], (key, e[key], chaos[key])
