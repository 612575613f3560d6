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
# many concurrent streams (batched and served forms): let CUDA map them onto
# its 32 hardware work queues instead of the default 8 (read at CUDA start)
os.environ.setdefault('CUDA_DEVICE_MAX_CONNECTIONS', '32')

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
    ap.add_argument('--e2e-steps', type=int, default=None, help='end-to-end steps (default: --steps, at least 200)')
    ap.add_argument('--trace-file', default=None, help='served: write the arrival trace (JSON) here')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-configs', action='store_true',
                    help='skip the sphere-wall, precision, batched and served lines of the default run')
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
    for f in ('stream_collide.cu', 'stream_collide_staged.cu', 'sc_common.cuh', 'links.cuh', 'common.cuh'):
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


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_cpu_all_cores(seconds, shape=(64, 64, 128)):
    """One single-threaded oracle replica per host core, all running at once
    on the same sample box; the value is the sum of their rates (the oracle
    is a serial program, so its all-core throughput is that of independent
    replicas)."""
    n = host_cores()
    env = dict(os.environ, OMP_NUM_THREADS='1', OPENBLAS_NUM_THREADS='1', MKL_NUM_THREADS='1')
    cmd = [sys.executable, os.path.abspath(__file__), '--cpu-sample', '--cpu-seconds', str(seconds),
           '--sample-shape', 'x'.join(str(v) for v in shape)]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(n)]
    res = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError('oracle sample failed: ' + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    value = sum(r['value'] for r in res)
    return {'value': value, 'unit': 'MLUPS', 'cores': n, 'kind': 'oracle',
            'sample': '%d concurrent single-thread replicas of: %s' % (n, res[0]['sample'])}


def cpu_baseline_both(seconds):
    """The oracle timed on one core and on all host cores (value: all cores)."""
    one = run_cpu_subprocess(seconds)
    one = {k: one[k] for k in ('value', 'unit', 'cores', 'kind', 'sample')}
    try:
        allc = run_cpu_all_cores(seconds)
    except Exception as ex:   # reported, not fatal
        allc = dict(one, all_cores_error=str(ex)[:200])
    out = dict(allc)
    out['one_core'] = one
    return out


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


def measure_box(w, steps, warmup, world, local, profile_steps=None):
    """Time `steps` steady-state steps of one context (CUDA graphs, CUDA events
    on the context's stream, clocks sampled meanwhile), then the same number of
    steps (or profile_steps) as plain launches with CUDA events between the
    phases. Returns a dict of the measurements and the final mapping."""
    import torch
    from paper_2003_01490_gb300 import lbmdem as L
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    ctx = make_context(w)
    add_spheres(ctx, w)
    L.lbm_step(ctx, warmup)
    L.lbm_sync(ctx)
    stream = torch.cuda.current_stream()
    launches0 = L.lbm_launch_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.lbm_step(ctx, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    L.lbm_sync(ctx)
    ms = e0.elapsed_time(e1)
    launches = L.lbm_launch_count(ctx) - launches0
    L.lbm_profile(ctx, 1)
    L.lbm_step(ctx, profile_steps or steps)
    L.lbm_sync(ctx)
    phases, nsteps = L.lbm_profile_read(ctx)
    L.lbm_profile(ctx, 0)
    _, _, flags = L.lbm_get_fields(ctx)
    solid = (flags & L.FLAG_SOLID) != 0
    n_solid = int(solid.sum())
    n_links = count_links(solid, w['periodic'])
    del ctx
    torch.cuda.synchronize()
    ms_max = allreduce_max(ms, world)
    return dict(cells=cells, ms=ms_max, value=whole_job_mlups(world, cells, steps, ms_max), clocks=clk,
                launches=launches, phases=phases, nsteps=nsteps, n_solid=n_solid, n_links=n_links)


_FP64_PEAK = None


def fp64_peak():
    """Measured float64 FMA throughput (TFLOP/s) of this device, once per run."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        from paper_2003_01490_gb300 import lbmdem as L
        try:
            _FP64_PEAK = (L.lbm_fp64_fma_rate(), 'measured: lbm_fp64_fma_rate (8 independent FMA chains per '
                                                 'thread, 8 x 256 threads per SM, CUDA events, best of 3)')
        except Exception as ex:
            _FP64_PEAK = (FP64_PEAK_TFLOPS, 'derived (measurement failed: %s): 152 SMs x 2.07 GHz x 2 '
                                            'float64 FMA per clock x 2 FLOP' % str(ex)[:80])
    return _FP64_PEAK


def dense_roofline(m, storage, workload_name):
    """Roofline of the dense kernel: algorithmic bytes per launch (fluid cells
    x (2 x 19 PDFs + 1 flag byte), solid cells x 1 flag byte) over its mean
    launch time from the CUDA events of the profiled region."""
    cells, n_solid, n_links, phases, nsteps = m['cells'], m['n_solid'], m['n_links'], m['phases'], m['nsteps']
    bf, bs = bytes_per_cell(storage)
    alg_bytes = (cells - n_solid) * bf + n_solid * bs
    # not algorithmic: per link the kernel also reads f~_p(x) and f~_q(x) at
    # the cell itself (CLI, Eq. (14)), values no pull reads
    es = {'f64': 8, 'f32': 4}.get(storage, 2)
    k_ms = phases['stream_collide'] / max(nsteps, 1)
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    traffic = recorded_traffic(storage, workload_name)
    share = {k: round(v / sum(phases.values()), 4) for k, v in phases.items()} if sum(phases.values()) else {}
    roofline = {'bound': 'hbm', 'achieved': round(achieved, 1), 'peak': peak, 'unit': 'GB/s',
                'frac': round(achieved / peak, 4), 'traffic': traffic,
                'kernel': 'stream_collide_kernel (pull stream with the particle links: CLI condition and '
                          'momentum exchange; wall bounce-back; TRT+aB collision)',
                'kernel_ms_per_launch': round(k_ms, 5), 'alg_bytes_per_launch': int(alg_bytes),
                'links_per_launch': int(n_links), 'link_bytes_per_launch': int(n_links * 2 * es),
                'peak_source': peak_kind + ' (MEASURED_PEAKS.json hbm_gbs)' if peak_kind == 'measured'
                else 'fallback 6.8 TB/s', 'phase_share': share}
    if storage == 'f64':
        # float64: GB300's float64 units bind before HBM (305 B and ~230 FLOP
        # per fluid cell)
        fpk, fsrc = fp64_peak()
        flops = (cells - n_solid) * FLOP_PER_FLUID_CELL + n_links * FLOP_PER_LINK
        achieved_tf = flops / (k_ms * 1e-3) / 1e12
        roofline.update({'bound': 'alu', 'achieved': round(achieved_tf, 4), 'peak': round(fpk, 4),
                         'unit': 'TFLOP/s', 'frac': round(achieved_tf / fpk, 4),
                         'alg_flops_per_launch': int(flops), 'peak_source': fsrc,
                         'hbm': {'achieved': round(achieved, 1), 'peak': peak, 'unit': 'GB/s',
                                 'frac': round(achieved / peak, 4)}})
    return roofline


def run_ours(args, rank, world, local):
    import torch
    w = workload(args.workload, args.storage, seed_offset=rank, shape=args.shape,
                 particles=args.particles)
    storage = w['storage']
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    m = measure_box(w, args.steps, args.warmup, world, local)
    value, ms_max, clk, launches, n_solid = m['value'], m['ms'], m['clocks'], m['launches'], m['n_solid']
    roofline = dense_roofline(m, storage, args.workload)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, w, world)
    configs = None
    if not args.no_configs and args.workload == 'suspension' and not args.shape:
        configs = measure_configs(args, rank, world, local)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_both(args.cpu_seconds)
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
    if configs is not None:
        line['configs'] = configs
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(args, w, world):
    """Same metric through the public API with host buffers: sphere upload
    (host -> device) and, every step, lbm_step + particle-state read-back into
    pinned host memory (queued on the context's stream after the step, so the
    host does not wait per step), all inside the timed region, which ends
    with lbm_sync."""
    import numpy as np
    import torch
    from paper_2003_01490_gb300 import lbmdem as L
    n = len(w['radius'])
    cells = w['shape'][0] * w['shape'][1] * w['shape'][2]
    ctx = make_context(w)
    pinned = {k: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
              for k in ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd')}
    host = {k: np.ascontiguousarray(w[k]) for k in ('pos', 'vel', 'omega', 'radius', 'density')}
    K = args.e2e_steps or max(args.steps, 200)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.lbm_add_spheres(ctx, host['pos'], host['vel'], host['omega'], host['radius'], host['density'])
    for _ in range(K):
        L.lbm_step(ctx, 1)
        L.lbm_get_particle_state_async(ctx, pinned)
    L.lbm_sync(ctx)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = allreduce_max(dt, world)
    h2d = sum(host[k].nbytes for k in host) / K
    d2h = 5 * 3 * 8 * n
    del ctx
    return {'value': round(world * cells * K / dt / 1e6, 1), 'unit': 'MLUPS',
            'h2d_bytes_per_step': int(h2d), 'd2h_bytes_per_step': int(d2h), 'steps': K,
            'includes': 'sphere upload + mapping, per step lbm_step + particle-state read-back '
                        '(lbm_get_particle_state_async into pinned memory), lbm_sync at the end'}


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


def measure_batched(n_inst, steps_divisor, storage, rank, world, local):
    """Many small independent boxes. The batched form: all instances in one
    batch (lbm_batch_*), one CUDA graph per step with the dense kernels of all
    active instances in one persistent launch, its launch shape picked by the
    autotuner (tune.py); every instance runs its own step count (a finished
    instance drops out of the batch). Beside it the plain per-job loop: the
    same instances one at a time, lbm_step() per job. Both timed regions cover
    every step of every instance (the first step of each instance runs on its
    own in both)."""
    import torch
    from paper_2003_01490_gb300 import lbmdem as L
    from paper_2003_01490_gb300 import tune, workloads
    inst = workloads.batched(n=n_inst, seed=20030149 + 1000 * rank, storage=storage,
                             steps_divisor=steps_divisor)
    work = sum(w['shape'][0] * w['shape'][1] * w['shape'][2] * w['steps'] for w in inst)
    cells = [w['shape'][0] * w['shape'][1] * w['shape'][2] for w in inst]

    def build():
        ctxs = []
        for w in inst:
            ctx = make_context(w)
            add_spheres(ctx, w)
            ctxs.append(ctx)
        torch.cuda.synchronize()
        return ctxs

    # the plain per-job loop: one instance at a time
    ctxs = build()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ctx, w in zip(ctxs, inst):
        L.lbm_step(ctx, w['steps'])
    torch.cuda.synchronize()
    t_seq = allreduce_max(time.perf_counter() - t0, world)
    for ctx in ctxs:
        L.lbm_sync(ctx)
    del ctxs
    torch.cuda.synchronize()
    # autotune the number of concurrent batches and their launch shape on
    # instances of the same shapes
    ctxs = build()
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    best = tune.tune_batched(ctxs, storage)
    del ctxs
    torch.cuda.synchronize()
    # the batched form
    ctxs = build()
    launches0 = sum(L.lbm_launch_count(c) for c in ctxs)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ctx in ctxs:
        L.lbm_step(ctx, 1)
    G = best['groups']
    groups = tune.make_groups(ctxs, G)
    segments = 0
    for g, (b, _) in enumerate(groups):
        L.lbm_batch_set_launch(b, -1, best['tile_bx'], best['zchunk'], best['blocks_per_sm'])
        # every batch runs its own instances' step counts; a finished instance
        # leaves its batch (all queued without waiting)
        left = [w['steps'] - 1 for w in inst[g::G]]
        for i, l in enumerate(left):
            if l == 0:
                L.lbm_batch_set_active(b, i, 0)
        while any(left):
            n = min(l for l in left if l > 0)
            L.lbm_batch_step(b, n)
            segments += 1
            for i in range(len(left)):
                if left[i] > 0:
                    left[i] -= n
                    if left[i] == 0:
                        L.lbm_batch_set_active(b, i, 0)
    torch.cuda.synchronize()
    t_bat = allreduce_max(time.perf_counter() - t0, world)
    clk = clocks.stop()
    launches = sum(L.lbm_launch_count(c) for c in ctxs) - launches0
    n_capt, capt_ms = 0, 0.0
    for b, _ in groups:
        L.lbm_batch_sync(b)
        launches += L.lbm_batch_launch_count(b)
        c_, m_ = L.lbm_batch_capture_stats(b)
        n_capt += c_
        capt_ms += m_
    del groups, ctxs
    torch.cuda.synchronize()
    return {
        'value': round(world * work / t_bat / 1e6, 1), 'unit': 'MLUPS',
        'workload': 'batched: %d sphere-wall boxes, sides 32-96 (s x s x 2s), %d-%d cells, steps 2000-10000 / %d, %s'
                    % (len(inst), min(cells), max(cells), steps_divisor, storage),
        'cell_updates': int(work), 'steps': sum(w['steps'] for w in inst), 'instances': len(inst),
        'form': '%d concurrent batches (one stream each); per batch and step one CUDA graph with the dense '
                'kernels of its active instances in one persistent launch and their DEM steps in one launch; '
                '%d segments (an instance leaves its batch when its steps are done)' % (G, segments),
        'launch_shape': {k: best[k] for k in ('groups', 'tile_bx', 'zchunk', 'blocks_per_sm', 'source')},
        'graph_captures': {'count': n_capt, 'host_ms': round(capt_ms, 1)},
        'l2': 'working set %.1f GB of PDFs > 129 MB L2' % (sum(cells) * 2 * 19 * 4 / 1e9),
        'sequential': {'value': round(world * work / t_seq / 1e6, 1), 'unit': 'MLUPS',
                       'kind': 'the same instances one at a time (plain per-job loop, lbm_step per job)'},
        'wall_s': {'batched': round(t_bat, 3), 'sequential': round(t_seq, 3)},
        'clocks': clk, 'gpu_launches': int(launches)}


def run_batched(args, rank, world, local):
    storage = args.storage or 'f32'
    r = measure_batched(args.instances, args.steps_divisor, storage, rank, world, local)
    line = {
        'metric': 'MLUPS', 'value': r['value'], 'unit': 'MLUPS', 'n_gpus': world,
        'steps': r['steps'], 'warmup': 3, 'ms_per_step': None,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': storage, 'data': 'synthetic',
        'config': {'workload': r['workload'], 'cell_updates': r['cell_updates'], 'instances': r['instances'],
                   'form': r['form'], 'launch_shape': r['launch_shape'], 'l2': r['l2'],
                   'parallelism': 'replicas' if world > 1 else 'single GPU'},
        'sequential': r['sequential'], 'wall_s': r['wall_s'], 'clocks': r['clocks'],
        'gpu_launches': r['gpu_launches'],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_served(n_jobs, steps_divisor, rank, local, max_side=256, trace_file=None):
    """The served form: a seeded stream of independent jobs (half sphere-wall
    collisions, half periodic suspensions; cubes of 32^3 to max_side^3 cells,
    0-2000 spheres of D = 8-16, 1000-20000 steps divided by steps_divisor)
    with Poisson arrivals, served with continuous batching (admission by a
    memory budget of 0.8 of the free device memory). The arrival rate follows
    Little's law from a calibration pass: the aggregate throughput R (cell
    updates per second) of the first jobs served all at once, and
    lambda = 0.9 R / (mean work per job), i.e. arrivals at 90 % of the
    capacity the GPU showed. The same trace is served in float16 and in
    float32 storage and run by the plain float32 FIFO loop: float16-served
    against float32-served isolates the precision gain, float32-served against
    the float32 FIFO loop the concurrency gain at equal accuracy."""
    import torch
    from paper_2003_01490_gb300 import lbmdem as L, serve, workloads
    gap0 = 0.004
    jobs = workloads.served(n=n_jobs, seed=20030149 + 1000 * rank, storage='f16', steps_divisor=steps_divisor,
                            max_side=max_side, gap=gap0)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    work = [j['shape'][0] * j['shape'][1] * j['shape'][2] * j['steps'] for j in jobs]
    mean_work = sum(work) / len(work)
    # calibration: the first min(16, n) jobs all at once, float16
    k = min(16, len(jobs))
    cal = [dict(j, arrival=0.0) for j in jobs[:k]]
    t0 = time.perf_counter()
    serve.serve(cal, budget)
    R = sum(work[:k]) / (time.perf_counter() - t0)
    lam = 0.9 * R / mean_work
    # the same Poisson draws with mean gap 1 / lambda
    scale = (1.0 / lam) / gap0
    for j in jobs:
        j['arrival'] *= scale
    mean_bytes = sum(serve.job_bytes(j) for j in jobs) / len(jobs)
    if trace_file:
        with open(trace_file, 'w') as fh:
            json.dump([{k_: (list(v) if isinstance(v, tuple) else v) for k_, v in j.items()
                        if k_ in ('name', 'shape', 'periodic', 'steps', 'arrival', 'tau')} for j in jobs], fh)
    out = {'workload': 'served: %d jobs (a stated tenth of the 2000-job stream when n = 200), Poisson arrivals, '
                       'sphere-wall and suspension cubes 32^3-%d^3 with 0-2000 spheres of D 8-16, steps 1000-20000 / %d'
                       % (len(jobs), max_side, steps_divisor),
           'budget_bytes': budget, 'cell_updates': int(sum(work)),
           'arrival_rate': {'jobs_per_s': round(lam, 3), 'rule': "Little's law: 0.9 x calibrated throughput / "
                            "mean work per job", 'calibrated_mlups': round(R / 1e6, 1),
                            'mean_cell_updates_per_job': round(mean_work),
                            'resident_jobs_for_0.8_of_memory': round(budget / mean_bytes, 1)},
           'trace_file': trace_file}
    for key, storage, fn in (('served_f16', 'f16', 'serve'), ('served_f32', 'f32', 'serve'),
                             ('fifo_f32', 'f32', 'fifo')):
        js = [dict(j, storage=storage) for j in jobs]
        clocks = ClockSampler(local)
        clocks.start()
        rec = serve.serve(js, budget) if fn == 'serve' else serve.fifo(js)
        clk = clocks.stop()
        out[key] = dict(serve.summary(rec), clocks=clk)
        torch.cuda.synchronize()
    return out


def run_served(args, rank, world, local):
    n = args.instances if '--instances' in sys.argv else 200
    div = args.steps_divisor if '--steps-divisor' in sys.argv else 50
    r = measure_served(n, div, rank, local, trace_file=args.trace_file)
    s_srv = r['served_f16']
    line = {
        'metric': 'MLUPS', 'value': s_srv['mlups'], 'unit': 'MLUPS', 'n_gpus': world,
        'steps': None, 'warmup': 0, 'ms_per_step': None,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': 'f16', 'data': 'synthetic',
        'config': {'workload': r['workload'], 'budget_bytes': r['budget_bytes'], 'arrival_rate': r['arrival_rate'],
                   'cell_updates': r['cell_updates'], 'parallelism': 'replicas' if world > 1 else 'single GPU'},
        'served': s_srv, 'served_f32': r['served_f32'], 'fifo_f32': r['fifo_f32'], 'clocks': s_srv['clocks'],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_configs(args, rank, world, local):
    """The other workloads, each in a short timed region with its own clocks
    record: the float64 sphere-wall collision over its 2000 steps, the
    suspension in float16 and bfloat16 storage, the batched boxes and the
    served job stream."""
    out = {}
    try:
        w = workload('sphere-wall')
        m = measure_box(w, 2000, 5, world, local, profile_steps=200)
        out['sphere_wall_f64'] = {'workload': w['name'] + ', 2000 steps', 'value': round(m['value'], 1),
                                  'unit': 'MLUPS', 'us_per_step': round(m['ms'] / 2000 * 1e3, 2),
                                  'roofline': dense_roofline(m, 'f64', 'sphere-wall'), 'clocks': m['clocks'],
                                  'gpu_launches': int(m['launches'])}
    except Exception as ex:   # reported, not fatal
        out['sphere_wall_f64'] = {'error': str(ex)[:300]}
    for st in ('f16', 'bf16'):
        try:
            w = workload('suspension', st)
            m = measure_box(w, 200, 5, world, local, profile_steps=100)
            out['suspension_' + st] = {'workload': w['name'], 'value': round(m['value'], 1), 'unit': 'MLUPS',
                                       'ms_per_step': round(m['ms'] / 200, 5),
                                       'roofline': dense_roofline(m, st, 'suspension'), 'clocks': m['clocks'],
                                       'gpu_launches': int(m['launches'])}
        except Exception as ex:
            out['suspension_' + st] = {'error': str(ex)[:300]}
    try:
        out['batched'] = measure_batched(64, 20, 'f32', rank, world, local)
    except Exception as ex:
        out['batched'] = {'error': str(ex)[:300]}
    try:
        out['served'] = measure_served(100, 100, rank, local)
    except Exception as ex:
        out['served'] = {'error': str(ex)[:300]}
    return out


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
    if args.gpus > 1 and 'WORLD_SIZE' not in os.environ:
        # not under torch.distributed.run yet: launch one rank per GPU
        import socket
        with socket.socket() as so:
            so.bind(('127.0.0.1', 0))
            port = so.getsockname()[1]
        cmd = [sys.executable, '-m', 'torch.distributed.run', '--nnodes=1', '--nproc-per-node', str(args.gpus),
               '--master-addr', '127.0.0.1', '--master-port', str(port), os.path.abspath(__file__)] + sys.argv[1:]
        os.execv(sys.executable, cmd)
    if int(os.environ.get('WORLD_SIZE', '1')) != args.gpus:
        sys.exit('bench.py: --gpus %d but WORLD_SIZE=%s ranks were launched'
                 % (args.gpus, os.environ.get('WORLD_SIZE')))
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
