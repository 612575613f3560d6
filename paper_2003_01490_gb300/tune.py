"""Autotuner of the batched dense kernel's launch shape.

A batch (``lbm_batch_create``) runs the stream/collide kernels of all its
instances as one persistent launch over a table of work items (instance,
tile of tile_bx x 256/tile_bx cells, chunk of zchunk planes). Which tile width,
chunk depth and number of resident blocks per multiprocessor is fastest
depends on the mix of box sizes and on the GPU, so this module measures it:
every candidate is set with ``lbm_batch_set_launch``, warmed up (its graph is
captured) and timed over a few batched steps with CUDA events on the batch's
stream; the fastest is set on the batch and stored in a JSON cache keyed by
the GPU, the storage format and the sorted box shapes, so a later batch of the
same kind starts from it without timing again.

Timing advances the instances by the steps it runs (as a warm-up would); pass
``restore=True`` to put every instance back to its state before tuning
(checkpoint and restore of each context).
"""
import hashlib
import json
import os

from . import lbmdem as L

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), '_tune', 'batch_launch.json')


def candidates(shapes):
    """Launch shapes to try: (tile_bx, zchunk, blocks_per_sm); tile_bx 0 is
    the automatic width (the box width rounded up to whole warps, at most 128)."""
    max_nx = max(s[0] for s in shapes)
    widths = [0] + ([64] if max_nx > 64 else []) + ([32] if max_nx > 32 else [])
    out = []
    for bx in widths:
        for zc in (8, 16, 32, 64):
            for bps in (2, 3, 4):
                out.append((bx, zc, bps))
    return out


def signature(ctxs, storage):
    import torch
    shapes = sorted(tuple(c.shape) for c in ctxs)
    dev = torch.cuda.get_device_name()
    h = hashlib.sha256(repr((dev, storage, shapes)).encode()).hexdigest()[:16]
    return h, dev, shapes


def _load_cache():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save_cache(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + '.tmp'
    with open(tmp, 'w') as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_steps(batch, steps):
    """Milliseconds of `steps` batched steps (CUDA events on the current stream)."""
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    L.lbm_batch_step(batch, steps)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1)


def tune_batch(batch, storage, steps=6, use_cache=True, restore=False, cands=None):
    """Pick and set the fastest launch shape of `batch`; returns
    {'tile_bx', 'zchunk', 'blocks_per_sm', 'ms_per_step', 'source', 'tried'}."""
    ctxs = batch.ctxs
    key, dev, shapes = signature(ctxs, storage)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        L.lbm_batch_set_launch(batch, -1, c['tile_bx'], c['zchunk'], c['blocks_per_sm'])
        return dict(c, source='cache')
    saved = None
    if restore:
        saved = [L.lbm_save(c) for c in ctxs]
    results = []
    for bx, zc, bps in (cands or candidates(shapes)):
        L.lbm_batch_set_launch(batch, -1, bx, zc, bps)
        L.lbm_batch_step(batch, 1)            # capture
        ms = time_steps(batch, steps) / steps
        results.append((ms, bx, zc, bps))
    L.lbm_batch_sync(batch)
    ms, bx, zc, bps = min(results)
    L.lbm_batch_set_launch(batch, -1, bx, zc, bps)
    if restore:
        for c, buf in zip(ctxs, saved):
            L.lbm_restore(c, buf)
    best = {'tile_bx': bx, 'zchunk': zc, 'blocks_per_sm': bps, 'ms_per_step': round(ms, 5),
            'gpu': dev, 'storage': storage, 'instances': len(ctxs), 'tried': len(results)}
    if use_cache:
        cache = _load_cache()
        cache[key] = best
        _save_cache(cache)
    return dict(best, source='timed')


def make_groups(ctxs, G):
    """G batches over the contexts (round robin), each on its own stream; the
    contexts of a batch move to its stream first, so that no stream they
    share orders one batch after another."""
    import torch
    groups = []
    for g in range(G):
        part = ctxs[g::G]
        if not part:
            continue
        st = torch.cuda.Stream()
        for c in part:
            L.lbm_set_stream(c, st)
        groups.append((L.lbm_batch_create(part, stream=st), st))
    return groups


def time_groups(groups, steps):
    """Wall milliseconds of `steps` steps of every batch, all running at once."""
    import time
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b, _ in groups:
        L.lbm_batch_step(b, steps)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3


def tune_batched(ctxs, storage, steps=4, groups=(1, 2, 4, 8, 16, 32, 64), use_cache=True):
    """Number of concurrent batches and the launch shape for running `ctxs`
    (every one stepped once already): first the group count with the
    automatic shape, then the shape for that count. The contexts advance by
    the steps timed. Returns {'groups', 'tile_bx', 'zchunk', 'blocks_per_sm',
    'ms_per_step', 'source'}."""
    key, dev, shapes = signature(ctxs, storage)
    key = 'groups-' + key
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return dict(cache[key], source='cache')
    res = []
    for G in groups:
        if G > len(ctxs):
            continue
        gs = make_groups(ctxs, G)
        for b, _ in gs:
            L.lbm_batch_step(b, 1)          # capture
        res.append((time_groups(gs, steps) / steps, G))
        del gs
    _, G = min(res)
    gs = make_groups(ctxs, G)
    shapes_ms = []
    for bx, zc, bps in [(bx, zc, bps) for bx in (0, 32) for zc in (8, 16, 32) for bps in (2, 4)]:
        for b, _ in gs:
            L.lbm_batch_set_launch(b, -1, bx, zc, bps)
            L.lbm_batch_step(b, 1)
        shapes_ms.append((time_groups(gs, steps) / steps, bx, zc, bps))
    for b, _ in gs:
        L.lbm_batch_sync(b)
    ms, bx, zc, bps = min(shapes_ms)
    best = {'groups': G, 'tile_bx': bx, 'zchunk': zc, 'blocks_per_sm': bps, 'ms_per_step': round(ms, 5),
            'gpu': dev, 'storage': storage, 'instances': len(ctxs),
            'tried': {'groups': [[g, round(m, 4)] for m, g in res], 'shapes': len(shapes_ms)}}
    if use_cache:
        cache = _load_cache()
        cache[key] = best
        _save_cache(cache)
    return dict(best, source='timed')
