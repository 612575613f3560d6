"""Writes the float64 oracle's long runs that the GPU parity tests compare
against at the stated step counts. Uses only the oracle and the seeded input
generators. Run from the repository root:

    python tests/golden/make_long_runs.py sphere-wall            # minutes
    python tests/golden/make_long_runs.py suspension [SCRATCH]   # hours, two processes
    python tests/golden/make_long_runs.py floor [SCRATCH]        # floor from what exists
    python tests/golden/make_long_runs.py storage [SCRATCH]      # hours, four processes

The suspension runs save their results after each of the field steps, so
the step-1000 comparison exists long before step 5000 is reached; `floor`
recomputes the floor file from the steps both runs have saved.

sphere-wall: the 32 x 32 x 64 sphere-wall collision (one sphere of D = 8,
density ratio 8, tau = 0.6, walls at the z faces, gravity for a terminal
Stokes number of about 10; the sphere-wall tests of Sec. 4.4 in shape) over
its 2000 steps: particle state after every step and the fields (rho, u) after
steps 1000 and 2000, float64 -> sphere_wall_2000.npz.

suspension: the 64 x 64 x 128 periodic suspension (150 spheres of D = 12,
27 % solids, the parameters of the 256 x 256 x 512 suspension) over 5000
steps: particle state every 100 steps, fields after steps 1000 and 5000
(float32 copies: the float32 comparisons they serve sit at 1e-6, far above
the 6e-8 rounding of the copy) -> suspension_64x64x128_5000.npz. A second
oracle run from the same inputs, with particle 0 displaced by 1e-12 along x,
gives the predictability floor (the divergence of two float64 runs that
differ by 1e-12 in one input, Algorithm 1 being chaotic in a dense
suspension) -> suspension_64x64x128_floor.txt.

storage: the same suspension over 1000 steps, four oracle runs at once: the
float64 reference, saved with rho - 1 (not rho) so that density deviations of
1e-5 keep their digits -> suspension_64x64x128_1000.npz; and three runs whose
stored post-collision PDFs are rounded after every step to the storage
formats of the precision forms (f - w rounded to nearest in float32; float16
and bfloat16 from that float32 value) -> the storage floor
suspension_64x64x128_storage_floor.txt: the error that storing f - w in that
format causes by itself, whatever the arithmetic around it.
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, 'tests'))

SPHERE_WALL = os.path.join(HERE, 'sphere_wall_2000.npz')
SUSPENSION = os.path.join(HERE, 'suspension_64x64x128_5000.npz')
FLOOR = os.path.join(HERE, 'suspension_64x64x128_floor.txt')
SUSPENSION_1000 = os.path.join(HERE, 'suspension_64x64x128_1000.npz')
STORAGE_FLOOR = os.path.join(HERE, 'suspension_64x64x128_storage_floor.txt')
STORAGE_FORMATS = ('f32', 'f16', 'bf16')
SUSP_FIELD_STEPS = (1000, 5000)
SUSP_STATE_EVERY = 100
PERTURBATION = 1e-12


def sphere_wall_case(storage='f64'):
    from cases import spheres
    from paper_2003_01490_gb300 import workloads
    w = workloads.sphere_wall()
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=storage,
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                dem=w['dem'])


def suspension_case(storage='f64', perturb=0.0):
    from cases import spheres
    from paper_2003_01490_gb300 import workloads
    w = workloads.reduced_suspension(storage=storage)
    pos = np.array(w['pos'], dtype=np.float64)
    pos[0, 0] += perturb
    return dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage=storage,
                spheres=spheres(pos, w['radius'], w['density'], w['vel'], w['omega']), dem=w['dem'])


def run_sphere_wall():
    from cases import build_oracle
    sim = build_oracle(sphere_wall_case())
    states, fields = [], {}
    t0 = time.time()
    for step in range(1, 2001):
        sim.step()
        states.append(np.concatenate([sim.X[0], sim.U[0], sim.Om[0], sim.Ffp[0], sim.Tfp[0]]))
        if step in (1000, 2000):
            rho, u = sim.fields()
            fields[step] = (rho, u, sim.owner >= 0)
        if step % 100 == 0:
            print('sphere-wall step %d (%.0f s), z = %.4f' % (step, time.time() - t0, sim.X[0, 2]), flush=True)
    np.savez_compressed(SPHERE_WALL, states=np.array(states),
                        rho_1000=fields[1000][0], u_1000=fields[1000][1], solid_1000=fields[1000][2],
                        rho_2000=fields[2000][0], u_2000=fields[2000][1], solid_2000=fields[2000][2])


def _suspension_run(perturb, out):
    os.environ.setdefault('OMP_NUM_THREADS', '2')
    from cases import build_oracle
    sim = build_oracle(suspension_case(perturb=perturb))
    states = {}
    arrays = {}
    t0 = time.time()
    last = max(SUSP_FIELD_STEPS)
    for step in range(1, last + 1):
        sim.step()
        if step % SUSP_STATE_EVERY == 0:
            states[step] = np.concatenate([sim.X, sim.U, sim.Om], axis=1)
            print('suspension (perturbation %g) step %d (%.0f s)' % (perturb, step, time.time() - t0), flush=True)
        if step in SUSP_FIELD_STEPS:
            rho, u = sim.fields()
            arrays['rho_%d' % step] = rho.astype(np.float32)
            arrays['u_%d' % step] = u.astype(np.float32)
            arrays['solid_%d' % step] = sim.owner >= 0
            steps = sorted(states)
            tmp = out + '.tmp.npz'
            np.savez_compressed(tmp, state_steps=np.array(steps), states=np.array([states[s] for s in steps]),
                                **arrays)
            os.replace(tmp, out)


def round_storage(v, fmt):
    """v rounded to the storage format: float32 (nearest even), float16 and
    bfloat16 (nearest even, from the float32 value)."""
    v32 = np.asarray(v, np.float64).astype(np.float32)
    if fmt == 'f32':
        return v32.astype(np.float64)
    if fmt == 'f16':
        return v32.astype(np.float16).astype(np.float64)
    bits = v32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def _storage_run(fmt, out):
    """1000 oracle steps; fmt None keeps float64, else the fluid cells'
    post-collision PDFs are stored as w + round(f - w) after every step."""
    os.environ['OMP_NUM_THREADS'] = '1'
    from cases import build_oracle
    from oracle.d3q19 import W
    sim = build_oracle(suspension_case())
    w = W.reshape(19, 1)
    states = {}
    t0 = time.time()
    for step in range(1, 1001):
        sim.step()
        if fmt is not None:
            fluid = sim.owner < 0
            sim.ft[:, fluid] = w + round_storage(sim.ft[:, fluid] - w, fmt)
        if step % SUSP_STATE_EVERY == 0:
            states[step] = np.concatenate([sim.X, sim.U, sim.Om], axis=1)
            print('suspension (%s storage) step %d (%.0f s)' % (fmt or 'f64', step, time.time() - t0), flush=True)
    rho, u = sim.fields()
    steps = sorted(states)
    tmp = out + '.tmp.npz'
    np.savez_compressed(tmp, state_steps=np.array(steps), states=np.array([states[k] for k in steps]),
                        drho_1000=np.where(sim.owner < 0, rho - 1.0, 0.0).astype(np.float32),
                        u_1000=u.astype(np.float32), solid_1000=sim.owner >= 0)
    os.replace(tmp, out)


def run_storage(scratch):
    ctx = mp.get_context('spawn')
    jobs = [(None, SUSPENSION_1000)] + [(f, os.path.join(scratch, 'suspension_storage_%s.npz' % f))
                                        for f in STORAGE_FORMATS]
    procs = [ctx.Process(target=_storage_run, args=j) for j in jobs]
    for p in procs:
        p.start()
    for p in procs:
        p.join()
        if p.exitcode != 0:
            raise SystemExit('oracle run failed')
    write_storage_floor(scratch)


def write_storage_floor(scratch):
    a = np.load(SUSPENSION_1000)
    shape = suspension_case()['shape']
    lines = ['# storage floor of the 64x64x128 suspension (150 spheres D=12) at step 1000: the float64',
             '# oracle with its fluid PDFs stored as w + round(f - w) in the format after every step,',
             '# against the plain float64 oracle. Relative L2 of u, of rho and of rho-1 over cells fluid in',
             '# both runs, relative L2 of the positions, RMS position distance / D, relative L2 of the',
             '# particle velocities.',
             '# format step rel_u rel_rho rel_rho-1 rel_pos rms_pos/D rel_vel']
    for fmt in STORAGE_FORMATS:
        path = os.path.join(scratch, 'suspension_storage_%s.npz' % fmt)
        if not os.path.exists(path):
            continue
        b = np.load(path)
        both = ~a['solid_1000'] & ~b['solid_1000']
        da, db = a['drho_1000'].astype(np.float64), b['drho_1000'].astype(np.float64)
        ru = rel_l2(b['u_1000'], a['u_1000'], both)
        rr = rel_l2(1.0 + db, 1.0 + da, both)
        rr1 = rel_l2(db, da, both)
        k = list(a['state_steps']).index(1000)
        xa, xb = a['states'][k][:, :3], b['states'][k][:, :3]
        rp, dp = position_error(xb, xa, shape, 12.0)
        ua, ub = a['states'][k][:, 3:6], b['states'][k][:, 3:6]
        rv = float(np.linalg.norm(ub - ua) / np.linalg.norm(ua))
        lines.append('%s 1000 %.6e %.6e %.6e %.6e %.6e %.6e' % (fmt, ru, rr, rr1, rp, dp, rv))
    with open(STORAGE_FLOOR, 'w') as fh:
        fh.write('\n'.join(lines) + '\n')
    print('\n'.join(lines))


def rel_l2(a, b, mask):
    a = np.asarray(a, np.float64)[..., mask]
    b = np.asarray(b, np.float64)[..., mask]
    return float(np.sqrt(((a - b) ** 2).sum()) / np.sqrt((b * b).sum()))


def position_error(xa, xb, shape, D):
    """(relative L2 of the positions, RMS distance / D) with periodic images."""
    L = np.array(shape, np.float64)
    d = xa - xb
    d -= L * np.round(d / L)
    return float(np.sqrt((d * d).sum() / (xb * xb).sum())), float(np.sqrt((d * d).sum(1).mean()) / D)


def run_suspension(scratch):
    perturbed = os.path.join(scratch, 'suspension_perturbed.npz')
    ctx = mp.get_context('spawn')
    procs = [ctx.Process(target=_suspension_run, args=(0.0, SUSPENSION)),
             ctx.Process(target=_suspension_run, args=(PERTURBATION, perturbed))]
    for p in procs:
        p.start()
    for p in procs:
        p.join()
        if p.exitcode != 0:
            raise SystemExit('oracle run failed')
    write_floor(scratch)


def write_floor(scratch):
    perturbed = os.path.join(scratch, 'suspension_perturbed.npz')
    a, b = np.load(SUSPENSION), np.load(perturbed)
    shape = suspension_case()['shape']
    lines = ['# predictability floor of the float64 oracle on the 64x64x128 suspension (150 spheres D=12):',
             '# the same run with particle 0 displaced by %g along x. Per step: relative L2 of u and of rho'
             % PERTURBATION,
             '# and of rho-1 over cells fluid in both runs, relative L2 of the positions, RMS position',
             '# distance / D, relative L2 of the particle velocities.',
             '# step rel_u rel_rho rel_rho-1 rel_pos rms_pos/D rel_vel']
    for step in SUSP_FIELD_STEPS:
        if 'u_%d' % step not in a.files or 'u_%d' % step not in b.files:
            continue
        both = ~a['solid_%d' % step] & ~b['solid_%d' % step]
        ru = rel_l2(b['u_%d' % step], a['u_%d' % step], both)
        rr = rel_l2(b['rho_%d' % step], a['rho_%d' % step], both)
        rr1 = rel_l2(b['rho_%d' % step].astype(np.float64) - 1.0, a['rho_%d' % step].astype(np.float64) - 1.0,
                     both)
        k = list(a['state_steps']).index(step)
        xa, xb = a['states'][k][:, :3], b['states'][k][:, :3]
        rp, dp = position_error(xb, xa, shape, 12.0)
        ua, ub = a['states'][k][:, 3:6], b['states'][k][:, 3:6]
        rv = float(np.linalg.norm(ub - ua) / np.linalg.norm(ua))
        lines.append('%d %.6e %.6e %.6e %.6e %.6e %.6e' % (step, ru, rr, rr1, rp, dp, rv))
    with open(FLOOR, 'w') as fh:
        fh.write('\n'.join(lines) + '\n')
    print('\n'.join(lines))


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else ''
    if what == 'sphere-wall':
        run_sphere_wall()
    elif what in ('suspension', 'floor', 'storage', 'storage-floor'):
        scratch = sys.argv[2] if len(sys.argv) > 2 else HERE
        {'suspension': run_suspension, 'floor': write_floor, 'storage': run_storage,
         'storage-floor': write_storage_floor}[what](scratch)
    else:
        raise SystemExit(__doc__)


if __name__ == '__main__':
    main()
