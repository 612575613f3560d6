#!/usr/bin/env python
"""Throughput benchmark of the coupled LBM-DEM time step (one JSON line).

Default workload: the dense periodic suspension, 256 x 256 x 512 cells with
10,000 spheres of D = 12 (27 % solids), float32 PDF storage, Algorithm 1 per
step (fused stream/boundary/collision, force averaging, 10 DEM subcycles,
mapping, refill). Metric: MLUPS = cells x steps / time / 1e6 over all cells.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 the script runs under torch.distributed.run, one rank per GPU,
each rank advancing its own independent replica (weak scaling); rank 0 prints
the line with the max-over-ranks time. --impl reference times the float64
CPU oracle on a bounded sample of the same workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129e6
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=1000)
    ap.add_argument('--warmup', type=int, default=20)
    ap.add_argument('--impl', default='ours', choices=('ours', 'reference'))
    ap.add_argument('--workload', default='suspension', choices=('suspension', 'sphere-wall', 'batched', 'served'))
    ap.add_argument('--instances', type=int, default=64, help='batched: number of boxes')
    ap.add_argument('--steps-divisor', type=int, default=20,
                    help='batched: divide each instance step count (2000-10000) by this')
    ap.add_argument('--storage', default=None, choices=(None, 'f64', 'f32', 'f16', 'bf16'))
    ap.add_argument('--shape', default=None, help='NXxNYxNZ of the suspension box (default 256x256x512)')
    ap.add_argument('--particles', type=int, default=None, help='sphere count (default: 27 %% solids)')
    ap.add_argument('--e2e-steps', type=int, default=200)
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--cpu-sample', action='store_true', help=argparse.SUPPRESS)
    ap.add_argument('--cpu-seconds', type=float, default=15.0)
    ap.add_argument('--sample-shape', default='64x64x128', help=argparse.SUPPRESS)
    ap.add_argument('--reference-budget', type=float, default=150.0,
                    help='seconds the reference arm may spend on its timed steps')
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def workload(name, storage=None, seed_offset=0, shape=None, particles=None):
    import math
    from paper_2003_01490_gb300 import workloads
    if name == 'suspension' and shape:
        sh = tuple(int(v) for v in shape.split('x'))
        n = particles or max(1, int(round(0.2696 * sh[0] * sh[1] * sh[2] / (math.pi * 12.0 ** 3 / 6.0))))
        w = workloads.suspension(shape=sh, n=n, seed=20030149 + seed_offset, storage=storage or 'f32')
    elif name == 'suspension':
        w = workloads.suspension(seed=20030149 + seed_offset, storage=storage or 'f32')
    else:
        w = workloads.sphere_wall()
        if storage:
            w['storage'] = storage
            w['name'] = w['name'].rsplit(', ', 1)[0] + ', ' + storage
    return w


def make_context(w):
    from paper_2003_01490_gb300 import lbmdem as L
    r, d = L.lbm_default_params()
    r.tau = w['tau']
    for k, v in w['dem'].items():
        if k == 'gravity':
            for a in range(3):
                d.gravity[a] = v[a]
        else:
            setattr(d, k, v)
    g = L.make_grid(w['shape'], w['periodic'])
    return L.lbm_create(g, r, w['body_force'], d, w['storage'], len(w['radius']))


def add_spheres(ctx, w):
    from paper_2003_01490_gb300 import lbmdem as L
    L.lbm_add_spheres(ctx, w['pos'], w['vel'], w['omega'], w['radius'], w['density'])


# float64 roofline of the dense kernel: algorithmic FLOPs per fluid cell
# (population-form TRT + Guo forcing + rank-2 bulk correction, ~200-260) and
# per particle link (link fraction root, CLI value, momentum-exchange force
# and torque), and the float64 peak from the unit counts and clocks
FLOP_PER_FLUID_CELL = 230
FLOP_PER_LINK = 75
FP64_PEAK_TFLOPS = round(152 * 2.07e9 * 2 * 2 / 1e12, 3)


def bytes_per_cell(storage):
    es = {'f64': 8, 'f32': 4, 'f16': 2, 'bf16': 2}[storage]
    return 2 * 19 * es + 1, 1          # fluid cell, solid cell (flag byte only)


def measured_peak():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    try:
        with open(p) as fh:
            return float(json.load(fh)['hbm_gbs']), 'measured'
    except Exception:
        return FALLBACK_HBM_GBS, 'fallback'


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ('stream_collide.cu', 'links.cuh', 'common.cuh'):
        with open(os.path.join(ROOT, 'paper_2003_01490_gb300', 'csrc', f), 'rb') as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(storage, workload_name):
    """DRAM bytes per launch of the stream/collide kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, 'profiles', 'stream_collide_%s_%s.md' % (workload_name, storage))
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ':' in line and line.strip().startswith(('traffic_bytes_per_launch', 'source_sha256')):
            k, v = line.split(':', 1)
            vals[k.strip()] = v.strip().strip('`')
    if vals.get('source_sha256') != kernel_source_hash():
        return None
    try:
        return float(vals['traffic_bytes_per_launch'])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.idx), '--query-gpu=' + self.FIELDS,
                 '--format=csv,noheader,nounits', '-lms', '100'],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ('hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap')
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(',')]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == 'active':
                    reasons.add(n)
        if not sm:
            return None
        return {'sm_mhz': statistics.median(sm), 'sm_max_mhz': max(smax), 'samples': len(sm),
                'reasons': sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle

SAMPLE_SHAPES = ((64, 64, 128), (48, 48, 96), (32, 32, 64), (24, 24, 48), (16, 16, 32))


def sample_workload(shape):
    """The suspension's parameters on a smaller periodic box at the same solid
    fraction (27 %, spheres of D = 12)."""
    import math
    from paper_2003_01490_gb300 import workloads
    cells = shape[0] * shape[1] * shape[2]
    n = max(1, int(round(0.2696 * cells / (math.pi * 12.0 ** 3 / 6.0))))
    return workloads.suspension(shape=shape, n=n, storage='f64', steps=0)


def cpu_sample(seconds, steps=None, warmup=0, shape=(64, 64, 128)):
    """Time the float64 oracle on a bounded sample of the suspension workload."""
    sys.path.insert(0, os.path.join(ROOT, 'tests'))
    from cases import build_oracle, spheres
    w = sample_workload(tuple(shape))
    case = dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage='f64',
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                dem=w['dem'])
    sim = build_oracle(case)
    for _ in range(warmup):
        sim.step()
    t0 = time.perf_counter()
    n = 0
    while (steps is None and (n < 2 or time.perf_counter() - t0 < seconds)) or \
            (steps is not None and n < steps):
        sim.step()
        n += 1
    dt = time.perf_counter() - t0
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    return {'value': cells * n / dt / 1e6, 'unit': 'MLUPS', 'cores': 1, 'kind': 'oracle',
            'steps': n, 'seconds': dt,
            'sample': 'float64 numpy oracle, %dx%dx%d periodic box, %d spheres D=12 (solid '
                      'fraction and parameters of the 256x256x512 suspension), %d timed steps, '
                      'one thread' % (tuple(w['shape']) + (len(w['radius']), n))}


def run_cpu_subprocess(seconds, steps=None, warmup=0, shape=(64, 64, 128)):
    env = dict(os.environ, OMP_NUM_THREADS='1', OPENBLAS_NUM_THREADS='1', MKL_NUM_THREADS='1')
    cmd = [sys.executable, os.path.abspath(__file__), '--cpu-sample', '--cpu-seconds', str(seconds),
           '--sample-shape', 'x'.join(str(v) for v in shape)]
    if steps is not None:
        cmd += ['--steps', str(steps), '--warmup', str(warmup)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError('oracle sample failed: ' + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ main arms

def dist_setup(n):
    import torch
    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    if world > 1:
        import torch.distributed as dist
        backend = 'nccl' if torch.cuda.is_available() else 'gloo'
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def allreduce_max(v, world):
    """Largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = 'cuda' if dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells_per_rank, steps, ms_max):
    """Cell updates of all ranks' replicas over the slowest rank's time."""
    return world * cells_per_rank * steps / (ms_max * 1e-3) / 1e6


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def count_links(solid, periodic):
    """Particle links of the mapping: (fluid cell x, direction q) pairs whose
    upstream cell x - c_q is solid. solid is indexed [z, y, x]; on a
    non-periodic axis the cells beyond the box are walls, not particles."""
    import numpy as np
    c = [(0, 1, 0), (0, -1, 0), (-1, 0, 0), (1, 0, 0), (0, 0, 1), (0, 0, -1), (-1, 1, 0), (1, 1, 0),
         (-1, -1, 0), (1, -1, 0), (0, 1, 1), (0, -1, 1), (-1, 0, 1), (1, 0, 1), (0, 1, -1), (0, -1, -1),
         (-1, 0, -1), (1, 0, -1)]
    fluid = ~solid
    n = 0
    for cx, cy, cz in c:
        up = np.roll(solid, shift=(cz, cy, cx), axis=(0, 1, 2))
        for axis, cc in ((2, cx), (1, cy), (0, cz)):
            if cc and not periodic[2 - axis]:
                sl = [slice(None)] * 3
                sl[axis] = 0 if cc > 0 else -1
                up[tuple(sl)] = False
        n += int(np.count_nonzero(fluid & up))
    return n


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2003_01490_gb300 import lbmdem as L
    w = workload(args.workload, args.storage, seed_offset=rank, shape=args.shape,
                 particles=args.particles)
    storage = w['storage']
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    ctx = make_context(w)
    add_spheres(ctx, w)
    L.lbm_step(ctx, args.warmup)
    L.lbm_sync(ctx)
    stream = torch.cuda.current_stream()
    # timed region 1 (the value): the production path, steady-state steps
    # replayed as CUDA graphs
    launches0 = L.lbm_launch_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.lbm_step(ctx, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    L.lbm_sync(ctx)
    ms = e0.elapsed_time(e1)
    launches = L.lbm_launch_count(ctx) - launches0
    # timed region 2 (the phase split and the kernel time of the roofline):
    # the same steps with CUDA events between the phases (plain launches)
    L.lbm_profile(ctx, 1)
    L.lbm_step(ctx, args.steps)
    L.lbm_sync(ctx)
    phases, nsteps = L.lbm_profile_read(ctx)
    L.lbm_profile(ctx, 0)
    _, _, flags = L.lbm_get_fields(ctx)
    solid = (flags & L.FLAG_SOLID) != 0
    n_solid = int(solid.sum())
    n_links = count_links(solid, w['periodic'])
    ms_max = allreduce_max(ms, world)
    value = whole_job_mlups(world, cells, args.steps, ms_max)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean launch time
    bf, bs = bytes_per_cell(storage)
    # per link the kernel also reads f~_p(x) and f~_q(x) at the cell itself
    # (CLI, Eq. (14)), values no pull reads
    es = {'f64': 8, 'f32': 4}.get(storage, 2)
    alg_bytes = (cells - n_solid) * bf + n_solid * bs + n_links * 2 * es
    k_ms = phases['stream_collide'] / max(nsteps, 1)
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    traffic = recorded_traffic(storage, args.workload)
    share = {k: round(v / sum(phases.values()), 4) for k, v in phases.items()} if sum(phases.values()) else {}
    roofline = {'bound': 'hbm', 'achieved': round(achieved, 1), 'peak': peak, 'unit': 'GB/s',
                'frac': round(achieved / peak, 4), 'traffic': traffic,
                'kernel': 'stream_collide_kernel (pull stream with the particle links: CLI condition and '
                          'momentum exchange; wall bounce-back; TRT+aB collision)',
                'kernel_ms_per_launch': round(k_ms, 5), 'alg_bytes_per_launch': int(alg_bytes),
                'links_per_launch': int(n_links),
                'peak_source': peak_kind + ' (MEASURED_PEAKS.json hbm_gbs)' if peak_kind == 'measured'
                else 'fallback 6.8 TB/s', 'phase_share': share}
    if storage == 'f64':
        # float64: GB300's float64 units (1.26 TFLOP/s) bind before HBM
        # (305 B and ~230 FLOP per fluid cell)
        flops = (cells - n_solid) * FLOP_PER_FLUID_CELL + n_links * FLOP_PER_LINK
        achieved_tf = flops / (k_ms * 1e-3) / 1e12
        roofline.update({'bound': 'alu', 'achieved': round(achieved_tf, 4), 'peak': FP64_PEAK_TFLOPS,
                         'unit': 'TFLOP/s', 'frac': round(achieved_tf / FP64_PEAK_TFLOPS, 4),
                         'alg_flops_per_launch': int(flops),
                         'peak_source': 'derived: 152 SMs x 2.07 GHz x 2 float64 FMA per clock x 2 FLOP',
                         'hbm': {'achieved': round(achieved, 1), 'peak': peak, 'unit': 'GB/s',
                                 'frac': round(achieved / peak, 4)}})

    e2e = None
    if not args.no_e2e:
        del ctx
        torch.cuda.synchronize()
        e2e = run_e2e(args, w, world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = run_cpu_subprocess(args.cpu_seconds)
            cpu = {k: cpu[k] for k in ('value', 'unit', 'cores', 'kind', 'sample')}
        except Exception as ex:  # reported, not fatal
            cpu = {'value': None, 'error': str(ex)[:200]}
    line = {
        'metric': 'MLUPS', 'value': round(value, 1), 'unit': 'MLUPS', 'n_gpus': world,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': round(ms_max / args.steps, 5),
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': storage,
        'data': 'synthetic',
        'config': {'workload': w['name'], 'cells': cells, 'particles': len(w['radius']),
                   'solid_cells': n_solid, 'storage': storage,
                   'l2': 'working set %.1f GB of PDFs > 129 MB L2, no flush needed'
                         % (2 * 19 * cells * {'f64': 8, 'f32': 4}.get(storage, 2) / 1e9),
                   'parallelism': 'replicas' if world > 1 else 'single GPU'},
        'roofline': roofline, 'cpu_baseline': cpu, 'e2e': e2e, 'clocks': clk,
        'gpu_launches': int(launches),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(args, w, world):
    """Same metric through the public API with host buffers: sphere upload
    (host -> device) and, every step, lbm_step + particle-state read-back into
    pinned host memory, all inside the timed region."""
    import numpy as np
    import torch
    from paper_2003_01490_gb300 import lbmdem as L
    n = len(w['radius'])
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    ctx = make_context(w)
    pinned = {k: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
              for k in ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd')}
    host = {k: np.ascontiguousarray(w[k]) for k in ('pos', 'vel', 'omega', 'radius', 'density')}
    K = args.e2e_steps
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.lbm_add_spheres(ctx, host['pos'], host['vel'], host['omega'], host['radius'], host['density'])
    for _ in range(K):
        L.lbm_step(ctx, 1)
        L.lbm_get_particle_state(ctx, out=pinned)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = allreduce_max(dt, world)
    h2d = sum(host[k].nbytes for k in host) / K
    d2h = 5 * 3 * 8 * n
    del ctx
    return {'value': round(world * cells * K / dt / 1e6, 1), 'unit': 'MLUPS',
            'h2d_bytes_per_step': int(h2d), 'd2h_bytes_per_step': int(d2h), 'steps': K,
            'includes': 'sphere upload + mapping, per step lbm_step + particle-state read-back'}


def run_reference(args, rank, world):
    """The float64 oracle as it stands, K timed steps after W warm-up steps, on
    the largest sample box of the suspension whose K + W steps fit the budget."""
    if rank != 0:
        return
    w = workload(args.workload)
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    probe = run_cpu_subprocess(0.0, steps=2, warmup=1, shape=SAMPLE_SHAPES[-1])
    t_cell = probe['seconds'] / probe['steps'] / (16 * 16 * 32)
    shape = SAMPLE_SHAPES[-1]
    for sh in SAMPLE_SHAPES:
        if (args.steps + args.warmup) * t_cell * sh[0] * sh[1] * sh[2] <= args.reference_budget:
            shape = sh
            break
    res = run_cpu_subprocess(0.0, steps=args.steps, warmup=args.warmup, shape=shape)
    line = {
        'impl': 'reference', 'metric': 'MLUPS', 'value': round(res['value'], 4), 'unit': 'MLUPS',
        'n_gpus': world, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': round(res['seconds'] / max(res['steps'], 1) * 1e3, 3),
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
        'data': 'synthetic',
        'config': {'workload': w['name'], 'cells': cells, 'sample': res['sample']},
        'cpu_baseline': {'value': round(res['value'], 4), 'unit': 'MLUPS', 'cores': res['cores'],
                         'kind': 'oracle', 'sample': res['sample']},
        'e2e': {'value': round(res['value'], 4), 'unit': 'MLUPS', 'h2d_bytes_per_step': 0,
                'd2h_bytes_per_step': 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local):
    """Many small independent boxes: every instance has its own context and
    CUDA stream, and all of them advance concurrently (steady-state steps are
    graph launches). The value is the aggregate MLUPS over all instances; the
    same work run one instance at a time (the plain per-job loop) is reported
    beside it."""
    import torch
    from paper_2003_01490_gb300 import lbmdem as L
    from paper_2003_01490_gb300 import workloads
    inst = workloads.batched(n=args.instances, seed=20030149 + 1000 * rank,
                             storage=args.storage or 'f32', steps_divisor=args.steps_divisor)
    work = sum(w['shape'][0] * w['shape'][1] * w['shape'][2] * w['steps'] for w in inst)

    def build():
        ctxs = []
        for w in inst:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                ctx = make_context(w)
                add_spheres(ctx, w)
                L.lbm_step(ctx, 3)   # warm-up: first step and the graph captures
            ctxs.append((ctx, st))
        torch.cuda.synchronize()
        return ctxs

    # the plain per-job loop: one instance at a time
    ctxs = build()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (ctx, st), w in zip(ctxs, inst):
        with torch.cuda.stream(st):
            L.lbm_step(ctx, w['steps'])
        st.synchronize()
    t_seq = allreduce_max(time.perf_counter() - t0, world)
    del ctxs
    torch.cuda.synchronize()
    # all instances concurrently, queued in rounds of `chunk` steps
    ctxs = build()
    launches0 = sum(L.lbm_launch_count(c) for c, _ in ctxs)
    left = [w['steps'] for w in inst]
    chunk = 25
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while any(left):
        for k, (ctx, st) in enumerate(ctxs):
            if left[k]:
                n = min(chunk, left[k])
                with torch.cuda.stream(st):
                    L.lbm_step(ctx, n)
                left[k] -= n
    torch.cuda.synchronize()
    t_bat = allreduce_max(time.perf_counter() - t0, world)
    clk = clocks.stop()
    for ctx, _ in ctxs:
        L.lbm_sync(ctx)
    launches = sum(L.lbm_launch_count(c) for c, _ in ctxs) - launches0
    value = world * work / t_bat / 1e6
    cells = [w['shape'][0] * w['shape'][1] * w['shape'][2] for w in inst]
    line = {
        'metric': 'MLUPS', 'value': round(value, 1), 'unit': 'MLUPS', 'n_gpus': world,
        'steps': sum(w['steps'] for w in inst), 'warmup': 3, 'ms_per_step': None,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': args.storage or 'f32', 'data': 'synthetic',
        'config': {'workload': 'batched: %d sphere-wall boxes, sides 32-96 (s x s x 2s), %d-%d cells, '
                               'steps 2000-10000 / %d' % (len(inst), min(cells), max(cells), args.steps_divisor),
                   'cell_updates': int(work), 'streams': len(inst),
                   'l2': 'working set %.1f GB of PDFs > 129 MB L2' % (sum(cells) * 2 * 19 * 4 / 1e9),
                   'parallelism': 'replicas' if world > 1 else 'single GPU'},
        'sequential': {'value': round(world * work / t_seq / 1e6, 1), 'unit': 'MLUPS',
                       'kind': 'the same instances one at a time (plain per-job loop)'},
        'wall_s': {'batched': round(t_bat, 3), 'sequential': round(t_seq, 3)},
        'clocks': clk, 'gpu_launches': int(launches),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_served(args, rank, world, local):
    """A seeded stream of jobs (Poisson arrivals; sphere-wall and suspension
    cubes of 32^3 to 128^3) served with continuous batching in float16
    storage, against the plain float32 FIFO loop on the same trace."""
    import torch
    from paper_2003_01490_gb300 import serve, workloads
    jobs = workloads.served(n=args.instances if '--instances' in sys.argv else 48,
                            seed=20030149 + 1000 * rank, storage=args.storage or 'f16',
                            steps_divisor=args.steps_divisor if '--steps-divisor' in sys.argv else 50)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    clocks = ClockSampler(local)
    clocks.start()
    rec = serve.serve(jobs, budget)
    clk = clocks.stop()
    base_jobs = [dict(j, storage='f32') for j in jobs]
    base = serve.fifo(base_jobs)
    s_srv, s_fifo = serve.summary(rec), serve.summary(base)
    line = {
        'metric': 'MLUPS', 'value': s_srv['mlups'], 'unit': 'MLUPS', 'n_gpus': world,
        'steps': sum(j['steps'] for j in jobs), 'warmup': 0, 'ms_per_step': None,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': args.storage or 'f16', 'data': 'synthetic',
        'config': {'workload': 'served: %d jobs, Poisson arrivals (mean gap 4 ms), sphere-wall and suspension '
                               'cubes 32^3-128^3, steps 1000-20000 / 50' % len(jobs),
                   'budget_bytes': budget, 'parallelism': 'replicas' if world > 1 else 'single GPU'},
        'served': s_srv, 'fifo_f32': s_fifo, 'clocks': clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.cpu_sample:
        steps = args.steps if '--steps' in sys.argv else None
        shape = tuple(int(v) for v in args.sample_shape.split('x'))
        print(json.dumps(cpu_sample(args.cpu_seconds, steps, args.warmup if steps else 0, shape)))
        return
    if args.impl == 'reference':
        rank = int(os.environ.get('RANK', '0'))
        world = int(os.environ.get('WORLD_SIZE', '1'))
        run_reference(args, rank, world)
        return
    rank, world, local = dist_setup(args.gpus)
    if args.workload == 'batched':
        run_batched(args, rank, world, local)
    elif args.workload == 'served':
        run_served(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
