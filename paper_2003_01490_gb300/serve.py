"""Continuous batching of independent LBM-DEM jobs on one GPU.

Jobs arrive over time. A job is admitted as soon as it has arrived and its
device memory fits the budget; each admitted job gets its own context and
CUDA stream, and the loop advances every admitted job in rounds of `chunk`
time steps (steady-state steps are CUDA-graph launches, so one host thread
keeps many small boxes in flight). A finished job's particle state is read
back, its context is released and its memory returns to the budget for the
next arrival. A job may be cancelled at a given time: if it is still waiting
it is dropped from the queue; if it is running, the loop waits for the steps
already queued on its stream, releases its context and returns its memory
to the budget. `fifo` runs the same trace one job at a time, in arrival
order: the plain per-job loop.
"""
import time

import numpy as np

from . import lbmdem as L


def make_context(job):
    r, d = L.lbm_default_params()
    r.tau = job['tau']
    for k, v in job['dem'].items():
        if k == 'gravity':
            for a in range(3):
                d.gravity[a] = v[a]
        else:
            setattr(d, k, v)
    g = L.make_grid(job['shape'], job['periodic'])
    ctx = L.lbm_create(g, r, job['body_force'], d, job['storage'], max(1, len(job['radius'])))
    if len(job['radius']):
        L.lbm_add_spheres(ctx, job['pos'], job['vel'], job['omega'], job['radius'], job['density'])
    return ctx


def job_bytes(job):
    g = L.make_grid(job['shape'], job['periodic'])
    return L.lbm_required_bytes(g, job['storage'], max(1, len(job['radius'])))


def _record(job, t_arrive, t_admit, t_done, state, steps=None, cancelled=False):
    cells = job['shape'][0] * job['shape'][1] * job['shape'][2]
    done = job['steps'] if steps is None else steps
    return {'name': job['name'], 'arrival': t_arrive, 'admit': t_admit, 'done': t_done,
            'latency': t_done - t_arrive, 'cell_updates': cells * done, 'state': state,
            'cancelled': cancelled}


def admissions(pending, arrival, need, now, used, budget_bytes):
    """Jobs to admit now: the waiting jobs in arrival order, as long as the
    next one has arrived and its memory fits the budget (the first that does
    not fit waits at the head of the queue). Returns (admitted, used)."""
    admitted = []
    for k in pending:
        if arrival[k] > now or used + need[k] > budget_bytes:
            break
        admitted.append(k)
        used += need[k]
    return admitted, used


def cancellations(pending, running, cancel_at, now):
    """Jobs whose cancellation time has come: (waiting jobs to drop, running
    jobs to stop), each in the order given. cancel_at maps a job index to a
    time in seconds from the start; jobs not in it run to completion, and a
    job that already finished is in neither list."""
    due = {k for k, t in cancel_at.items() if t <= now}
    return [k for k in pending if k in due], [k for k in running if k in due]


def serve(jobs, budget_bytes, chunk=25, keep_state=False, cancel_at=None):
    """Run `jobs` (each with an 'arrival' time in seconds from the start) with
    continuous batching; returns one record per job in arrival order.
    cancel_at: optional {job index: time in seconds from the start} at which
    that job is cancelled (its record then has 'cancelled' True and counts
    the steps it ran)."""
    import torch
    order = sorted(range(len(jobs)), key=lambda k: jobs[k]['arrival'])
    need = [job_bytes(j) for j in jobs]
    too_big = [jobs[k]['name'] for k in order if need[k] > budget_bytes]
    if too_big:
        # such a job would wait at the head of the queue for ever
        raise ValueError('jobs larger than the memory budget of %d bytes: %s'
                         % (budget_bytes, ', '.join(too_big[:5])))
    arrival = [j['arrival'] for j in jobs]
    pending = list(order)
    running = []          # [job index, ctx, stream, steps left, admit time, done event]
    used = 0
    out = {}
    cancel_at = dict(cancel_at or {})
    t0 = time.perf_counter()
    while pending or running:
        now = time.perf_counter() - t0
        if cancel_at:
            drop_wait, drop_run = cancellations(pending, [item[0] for item in running], cancel_at, now)
            for k in drop_wait:
                pending.remove(k)
                out[k] = _record(jobs[k], jobs[k]['arrival'], None, now, None, steps=0, cancelled=True)
            still = []
            for item in running:
                if item[0] in drop_run:
                    k, ctx, st, left, t_adm = item[0], item[1], item[2], item[3], item[4]
                    st.synchronize()      # none of its steps still in flight
                    out[k] = _record(jobs[k], jobs[k]['arrival'], t_adm, time.perf_counter() - t0, None,
                                     steps=jobs[k]['steps'] - left, cancelled=True)
                    used -= need[k]
                    item[1] = None        # the context and its arena go
                    del ctx
                else:
                    still.append(item)
            running = still
            for k in drop_wait + drop_run:
                del cancel_at[k]
        # admission: arrived jobs in order, while the budget allows
        admitted, used = admissions(pending, arrival, need, now, used, budget_bytes)
        for k in admitted:
            pending.remove(k)
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                ctx = make_context(jobs[k])
            running.append([k, ctx, st, jobs[k]['steps'], time.perf_counter() - t0, None])
        if not running:
            if pending:   # nothing admitted yet: wait for the next arrival
                time.sleep(max(0.0, min(1e-3, jobs[pending[0]]['arrival'] - now)))
            continue
        # one round: every running job advances by up to `chunk` steps
        for item in running:
            k, ctx, st, left = item[0], item[1], item[2], item[3]
            if left > 0:
                n = min(chunk, left)
                L.lbm_step(ctx, n)
                item[3] -= n
                if item[3] == 0:
                    ev = torch.cuda.Event()
                    ev.record(st)
                    item[5] = ev
        # completions
        still = []
        for item in running:
            k, ctx, st, left, t_adm, ev = item
            if left == 0 and ev is not None and ev.query():
                state = L.lbm_get_particle_state(ctx) if keep_state else None
                L.lbm_sync(ctx)
                out[k] = _record(jobs[k], jobs[k]['arrival'], t_adm, time.perf_counter() - t0, state)
                used -= need[k]
                del ctx
            else:
                still.append(item)
        running = still
    return [out[k] for k in order]


def fifo(jobs, keep_state=False):
    """The same trace, one job at a time in arrival order."""
    import torch
    order = sorted(range(len(jobs)), key=lambda k: jobs[k]['arrival'])
    out = {}
    t0 = time.perf_counter()
    for k in order:
        now = time.perf_counter() - t0
        if jobs[k]['arrival'] > now:
            time.sleep(jobs[k]['arrival'] - now)
        t_adm = time.perf_counter() - t0
        ctx = make_context(jobs[k])
        L.lbm_step(ctx, jobs[k]['steps'])
        state = L.lbm_get_particle_state(ctx) if keep_state else None
        L.lbm_sync(ctx)
        torch.cuda.current_stream().synchronize()
        out[k] = _record(jobs[k], jobs[k]['arrival'], t_adm, time.perf_counter() - t0, state)
        del ctx
    return [out[k] for k in order]


def summary(records):
    """Makespan and MLUPS over all records (the steps of cancelled jobs count as
    work done); jobs/s and latency percentiles over the completed jobs."""
    done = [r for r in records if not r.get('cancelled')]
    span = max(r['done'] for r in records) - min(r['arrival'] for r in records)
    work = sum(r['cell_updates'] for r in records)
    lat = np.array([r['latency'] for r in done]) if done else np.zeros(1)
    return {'jobs': len(done), 'cancelled': len(records) - len(done), 'makespan_s': round(span, 4),
            'jobs_per_s': round(len(done) / span, 2), 'mlups': round(work / span / 1e6, 1),
            'p50_latency_s': round(float(np.percentile(lat, 50)), 4),
            'p99_latency_s': round(float(np.percentile(lat, 99)), 4)}
