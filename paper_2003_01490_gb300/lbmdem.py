"""Python binding of the C ABI in ``include/lbmdem.h`` (ctypes, marshalling only).

The functions keep the C names: :func:`lbm_create`, :func:`lbm_add_spheres`,
:func:`lbm_step`, :func:`lbm_get_particle_state`, :func:`lbm_get_fields` and
the helpers around them. Every numerical step runs in the CUDA library
``_lib/liblbmdem.so``; this module only converts numpy arrays and parameter
structs. Device memory comes from PyTorch (one arena tensor per context, see
:func:`lbm_create`) and the work is queued on PyTorch's current CUDA stream.
There is no CPU fallback: if the library is missing or CUDA is unavailable
the calls raise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, '_lib', 'liblbmdem.so')

STORAGE = {'f64': 0, 'f32': 1, 'f16': 2, 'bf16': 3}
# lbm_dem.fixed_particles: particles moved by the DEM, held fixed, or moved by prescribed velocities
MOTION_DEM, MOTION_FIXED, MOTION_PRESCRIBED = 0, 1, 2
FLAG_SOLID, FLAG_SHELL, FLAG_NEAR, FLAG_MISS, FLAG_NEWFLUID, FLAG_MULTI = 0x01, 0x02, 0x04, 0x08, 0x10, 0x20
STATUS = {0: 'LBM_OK', -1: 'LBM_ERR_INVALID', -2: 'LBM_ERR_OOM', -3: 'LBM_ERR_CUDA',
          -4: 'LBM_ERR_UNSTABLE', -5: 'LBM_ERR_CAPACITY', -6: 'LBM_ERR_TIMEOUT', -7: 'LBM_ERR_STATE'}
STATUS_CODES = {v: k for k, v in STATUS.items()}
EXPORTS = ('lbm_default_params', 'lbm_required_bytes', 'lbm_create', 'lbm_create_in_arena',
           'lbm_add_spheres', 'lbm_step', 'lbm_get_particle_state', 'lbm_get_particle_state_async',
           'lbm_set_particle_velocity',
           'lbm_set_motion', 'lbm_checkpoint_bytes', 'lbm_save', 'lbm_restore', 'lbm_sample_density',
           'lbm_get_fields',
           'lbm_get_owner', 'lbm_get_pdfs', 'lbm_set_pdfs', 'lbm_sync', 'lbm_set_stream', 'lbm_profile',
           'lbm_profile_read', 'lbm_map_spheres_noalloc', 'lbm_fp64_fma_rate', 'lbm_batch_create',
           'lbm_batch_set_launch', 'lbm_batch_set_active', 'lbm_batch_step', 'lbm_batch_sync',
           'lbm_batch_launch_count', 'lbm_batch_capture_stats', 'lbm_batch_last_error', 'lbm_batch_destroy', 'lbm_launch_count',
           'lbm_last_error',
           'lbm_destroy')

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t


class LbmGrid(ctypes.Structure):
    _fields_ = [('nx', c_int), ('ny', c_int), ('nz', c_int), ('periodic', c_int * 3),
                ('wall_vel_lo', (c_double * 3) * 3), ('wall_vel_hi', (c_double * 3) * 3)]


class LbmRelax(ctypes.Structure):
    _fields_ = [('tau', c_double), ('magic', c_double), ('lambda_b_shell', c_double),
                ('lambda_b_bulk', c_double), ('shell_width', c_double)]


class LbmDem(ctypes.Structure):
    _fields_ = [('e_dry', c_double), ('Tc', c_double), ('nu_p', c_double), ('mu_p', c_double),
                ('n_sub', c_int), ('lub_cut_n', c_double), ('lub_cut_tt', c_double),
                ('lub_cut_tr', c_double), ('lub_min_a', c_double), ('lub_min_b', c_double),
                ('gravity', c_double * 3), ('lubrication', c_int), ('tangential_lubrication', c_int),
                ('force_averaging', c_int), ('fluid_counterforce', c_int),
                ('fixed_particles', c_int), ('missing_links', c_int)]


class LbmError(RuntimeError):
    """A C call returned a non-zero lbm_status."""

    def __init__(self, status, message):
        super().__init__('%s: %s' % (STATUS.get(status, status), message))
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load ``liblbmdem.so`` and declare the C signatures. Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError('liblbmdem.so is not built (%s); run paper_2003_01490_gb300.build' % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp = P(c_double)
    lib.lbm_default_params.argtypes = [P(LbmRelax), P(LbmDem)]
    lib.lbm_required_bytes.argtypes = [P(LbmGrid), c_int, c_int, P(c_size_t)]
    lib.lbm_create.argtypes = [P(LbmGrid), P(LbmRelax), dp, P(LbmDem), c_int, c_int, c_void_p,
                               P(c_void_p)]
    lib.lbm_create_in_arena.argtypes = [P(LbmGrid), P(LbmRelax), dp, P(LbmDem), c_int, c_int,
                                        c_void_p, c_void_p, c_size_t, P(c_void_p)]
    lib.lbm_add_spheres.argtypes = [c_void_p, c_int, dp, dp, dp, dp, dp, P(c_int)]
    lib.lbm_step.argtypes = [c_void_p, c_int]
    lib.lbm_get_particle_state.argtypes = [c_void_p, c_int, dp, dp, dp, dp, dp, P(c_int)]
    lib.lbm_get_particle_state_async.argtypes = [c_void_p, c_int, dp, dp, dp, dp, dp, P(c_int)]
    lib.lbm_set_particle_velocity.argtypes = [c_void_p, c_int, dp, dp]
    lib.lbm_set_motion.argtypes = [c_void_p, c_int]
    lib.lbm_sample_density.argtypes = [c_void_p, c_int, dp, dp]
    lib.lbm_checkpoint_bytes.argtypes = [c_void_p, P(c_size_t)]
    lib.lbm_save.argtypes = [c_void_p, c_void_p, c_size_t]
    lib.lbm_restore.argtypes = [c_void_p, c_void_p, c_size_t]
    lib.lbm_get_fields.argtypes = [c_void_p, dp, dp, P(ctypes.c_ubyte)]
    lib.lbm_get_owner.argtypes = [c_void_p, P(c_int)]
    lib.lbm_get_pdfs.argtypes = [c_void_p, dp]
    lib.lbm_set_pdfs.argtypes = [c_void_p, dp]
    lib.lbm_sync.argtypes = [c_void_p]
    lib.lbm_set_stream.argtypes = [c_void_p, c_void_p]
    lib.lbm_profile.argtypes = [c_void_p, c_int]
    lib.lbm_profile_read.argtypes = [c_void_p, dp, P(ctypes.c_longlong)]
    lib.lbm_map_spheres_noalloc.argtypes = [P(LbmGrid), c_double, c_int, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p]
    lib.lbm_fp64_fma_rate.argtypes = [c_int, dp]
    lib.lbm_batch_create.argtypes = [P(c_void_p), c_int, c_void_p, P(c_void_p)]
    lib.lbm_batch_set_launch.argtypes = [c_void_p, c_int, c_int, c_int, c_int]
    lib.lbm_batch_set_active.argtypes = [c_void_p, c_int, c_int]
    lib.lbm_batch_step.argtypes = [c_void_p, c_int]
    lib.lbm_batch_sync.argtypes = [c_void_p]
    lib.lbm_batch_capture_stats.argtypes = [c_void_p, P(c_int), dp]
    lib.lbm_batch_launch_count.argtypes = [c_void_p]
    lib.lbm_batch_launch_count.restype = ctypes.c_longlong
    lib.lbm_batch_last_error.argtypes = [c_void_p]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    lib.lbm_batch_destroy.argtypes = [c_void_p]
    lib.lbm_batch_destroy.restype = None
    lib.lbm_launch_count.argtypes = [c_void_p]
    lib.lbm_launch_count.restype = ctypes.c_longlong
    lib.lbm_last_error.argtypes = [c_void_p]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_destroy.argtypes = [c_void_p]
    lib.lbm_destroy.restype = None
    for name in EXPORTS:
        if name not in ('lbm_launch_count', 'lbm_last_error', 'lbm_destroy', 'lbm_batch_launch_count',
                        'lbm_batch_last_error', 'lbm_batch_destroy'):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != 0:
        msg = load_library().lbm_last_error(ctx).decode()
        raise LbmError(status, msg)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(c_double)) if a is not None else None


def _vec(a, n, width):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(n * width))


def lbm_default_params():
    """Paper defaults (tau = 0.6): returns (LbmRelax, LbmDem)."""
    r, d = LbmRelax(), LbmDem()
    _check(load_library().lbm_default_params(ctypes.byref(r), ctypes.byref(d)))
    return r, d


def make_grid(shape, periodic=(1, 1, 1), wall_vel_lo=None, wall_vel_hi=None):
    """LbmGrid from (nx, ny, nz); wall velocities are [axis][component] arrays."""
    g = LbmGrid()
    g.nx, g.ny, g.nz = (int(v) for v in shape)
    for a in range(3):
        g.periodic[a] = int(bool(periodic[a]))
        for c in range(3):
            g.wall_vel_lo[a][c] = 0.0 if wall_vel_lo is None else float(wall_vel_lo[a][c])
            g.wall_vel_hi[a][c] = 0.0 if wall_vel_hi is None else float(wall_vel_hi[a][c])
    return g


class Context:
    """Handle of one simulation context; owns the PyTorch arena tensor."""

    def __init__(self, handle, arena, shape):
        self.handle = handle
        self.arena = arena
        self.shape = shape

    @property
    def ncells(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def __del__(self):
        if getattr(self, 'handle', None):
            load_library().lbm_destroy(self.handle)
            self.handle = None


def lbm_required_bytes(grid, storage, max_particles):
    out = c_size_t(0)
    _check(load_library().lbm_required_bytes(ctypes.byref(grid), STORAGE[storage],
                                             int(max_particles), ctypes.byref(out)))
    return out.value


def lbm_create(grid, relax, body_force, dem, storage='f32', max_particles=0, device=None):
    """Create a context whose device memory is one PyTorch uint8 tensor (the arena)
    on the current CUDA device, with work queued on PyTorch's current stream."""
    import torch
    lib = load_library()
    if not torch.cuda.is_available():
        raise RuntimeError('CUDA device required: the library has no CPU path')
    nbytes = lbm_required_bytes(grid, storage, max_particles)
    dev = torch.device('cuda') if device is None else torch.device(device)
    arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = arena.data_ptr()
    pad = (-base) % 256
    stream = torch.cuda.current_stream(dev).cuda_stream
    bf = (c_double * 3)(*(body_force if body_force is not None else (0.0, 0.0, 0.0)))
    h = c_void_p()
    _check(lib.lbm_create_in_arena(ctypes.byref(grid), ctypes.byref(relax), bf, ctypes.byref(dem),
                                   STORAGE[storage], int(max_particles), c_void_p(stream),
                                   c_void_p(base + pad), c_size_t(nbytes), ctypes.byref(h)))
    return Context(h.value, arena, (grid.nx, grid.ny, grid.nz))


def lbm_add_spheres(ctx, pos, vel, omega, radius, density):
    """Add spheres; arrays are (n, 3) or (n,) float64. Returns the first new index."""
    radius = np.ascontiguousarray(np.asarray(radius, dtype=np.float64).reshape(-1))
    n = len(radius)
    pos, vel, omega = _vec(pos, n, 3), _vec(vel, n, 3), _vec(omega, n, 3)
    density = np.ascontiguousarray(np.asarray(density, dtype=np.float64).reshape(n))
    first = c_int(0)
    _check(load_library().lbm_add_spheres(ctx.handle, n, _dptr(pos), _dptr(vel), _dptr(omega),
                                          _dptr(radius), _dptr(density), ctypes.byref(first)),
           ctx.handle)
    return first.value


def lbm_set_particle_velocity(ctx, vel=None, omega=None):
    """Replace the velocities of particles 0 .. n-1 ((n, 3) float64 each, either None)."""
    arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3))
            for a in (vel, omega)]
    n = max([len(a) for a in arrs if a is not None] or [0])
    for a in arrs:
        if a is not None and len(a) != n:
            raise ValueError('vel and omega need the same number of rows')
    _check(load_library().lbm_set_particle_velocity(ctx.handle, n, _dptr(arrs[0]), _dptr(arrs[1])), ctx.handle)


def lbm_set_motion(ctx, mode):
    """Move particles by the DEM (MOTION_DEM), hold them (MOTION_FIXED) or move them by their set
    velocities (MOTION_PRESCRIBED) from the next step on."""
    _check(load_library().lbm_set_motion(ctx.handle, int(mode)), ctx.handle)


def lbm_sample_density(ctx, pos):
    """Density at points pos ((n, 3) lattice units) by trilinear interpolation."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    out = np.zeros(len(pos))
    _check(load_library().lbm_sample_density(ctx.handle, len(pos), _dptr(pos), _dptr(out)), ctx.handle)
    return out


def lbm_save(ctx):
    """The whole simulation state as a uint8 array (a checkpoint)."""
    lib = load_library()
    n = c_size_t(0)
    _check(lib.lbm_checkpoint_bytes(ctx.handle, ctypes.byref(n)), ctx.handle)
    buf = np.empty(n.value, dtype=np.uint8)
    _check(lib.lbm_save(ctx.handle, buf.ctypes.data_as(c_void_p), n.value), ctx.handle)
    return buf


def lbm_restore(ctx, buf):
    """Put a checkpoint of lbm_save back (same grid, storage and capacity)."""
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().lbm_restore(ctx.handle, buf.ctypes.data_as(c_void_p), buf.size), ctx.handle)


def lbm_step(ctx, n_steps=1):
    _check(load_library().lbm_step(ctx.handle, int(n_steps)), ctx.handle)


def lbm_sync(ctx):
    _check(load_library().lbm_sync(ctx.handle), ctx.handle)


def lbm_set_stream(ctx, stream=None):
    """Queue the context's later work on `stream` (a torch.cuda.Stream; None:
    PyTorch's current stream) after the work queued so far."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(load_library().lbm_set_stream(ctx.handle, c_void_p(st.cuda_stream)), ctx.handle)


def lbm_get_particle_state(ctx, out=None):
    """Return dict of (n, 3) arrays pos, vel, omega, force_hyd, torque_hyd.

    ``out`` may hold preallocated (pinned) float64 arrays under the same keys."""
    lib = load_library()
    n = c_int(0)
    _check(lib.lbm_get_particle_state(ctx.handle, 0, None, None, None, None, None, ctypes.byref(n)),
           ctx.handle)
    n = n.value
    keys = ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd')
    res = {}
    for k in keys:
        if out is not None and k in out:
            res[k] = out[k]
        else:
            res[k] = np.zeros((n, 3))
    _check(lib.lbm_get_particle_state(ctx.handle, n, *[_dptr(res[k]) for k in keys], None),
           ctx.handle)
    return res


def lbm_get_particle_state_async(ctx, out):
    """Queue copies of the particle state into the arrays of ``out`` (keys
    pos, vel, omega, force_hyd, torque_hyd, any subset; C-contiguous float64
    with n x 3 entries, page-locked for the copies to overlap host work) and
    return without waiting; the values are there once lbm_sync(ctx) returns.
    The arrays must stay alive until then."""
    lib = load_library()
    n = c_int(0)
    _check(lib.lbm_get_particle_state_async(ctx.handle, 0, None, None, None, None, None, ctypes.byref(n)),
           ctx.handle)
    n = n.value
    keys = ('pos', 'vel', 'omega', 'force_hyd', 'torque_hyd')
    ptrs = []
    for k in keys:
        a = out.get(k)
        if a is not None:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags['C_CONTIGUOUS']
                    and a.size >= 3 * n):
                raise ValueError('%s: expected a C-contiguous float64 array of %d x 3 values' % (k, n))
        ptrs.append(_dptr(a))
    _check(lib.lbm_get_particle_state_async(ctx.handle, n, *ptrs, None), ctx.handle)


def lbm_get_fields(ctx):
    """Return rho (nz, ny, nx), u (3, nz, ny, nx) and flags (nz, ny, nx) as numpy arrays."""
    nx, ny, nz = ctx.shape
    rho = np.zeros(ctx.ncells)
    u = np.zeros(3 * ctx.ncells)
    flags = np.zeros(ctx.ncells, dtype=np.uint8)
    _check(load_library().lbm_get_fields(ctx.handle, _dptr(rho), _dptr(u),
                                         flags.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))),
           ctx.handle)
    return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx), flags.reshape(nz, ny, nx)


def lbm_get_owner(ctx):
    nx, ny, nz = ctx.shape
    owner = np.zeros(ctx.ncells, dtype=np.int32)
    _check(load_library().lbm_get_owner(ctx.handle, owner.ctypes.data_as(ctypes.POINTER(c_int))),
           ctx.handle)
    return owner.reshape(nz, ny, nx)


def lbm_get_pdfs(ctx):
    nx, ny, nz = ctx.shape
    f = np.zeros(19 * ctx.ncells)
    _check(load_library().lbm_get_pdfs(ctx.handle, _dptr(f)), ctx.handle)
    return f.reshape(19, nz, ny, nx)


def lbm_set_pdfs(ctx, f):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
    if f.size != 19 * ctx.ncells:
        raise ValueError('expected 19 x cells values')
    _check(load_library().lbm_set_pdfs(ctx.handle, _dptr(f)), ctx.handle)


PHASES = ('boundary', 'stream_collide', 'force_finalize', 'dem', 'mapping', 'refill')


def lbm_profile(ctx, enable):
    _check(load_library().lbm_profile(ctx.handle, int(bool(enable))), ctx.handle)


def lbm_profile_read(ctx):
    """Return ({phase: total ms}, timed steps) of the CUDA-event phase timing."""
    ms = (c_double * len(PHASES))()
    steps = ctypes.c_longlong(0)
    _check(load_library().lbm_profile_read(ctx.handle, ms, ctypes.byref(steps)), ctx.handle)
    return dict(zip(PHASES, list(ms))), steps.value


def lbm_map_spheres_noalloc(grid, shell_width, pos, radius, flags, owner):
    """Map spheres into caller-owned device buffers without any device allocation.

    pos (n x 3 float64), radius (n float64), flags (cells uint8) and owner
    (cells int32) are CUDA tensors; the work runs on PyTorch's current stream.
    """
    import torch
    n = radius.numel()
    # sizes first (the C side writes nx*ny*nz flag bytes and owners and reads
    # 3n positions, so an undersized buffer must be refused here)
    ncells = int(grid.nx) * int(grid.ny) * int(grid.nz)
    if pos.numel() != 3 * n:
        raise ValueError('pos must hold 3 x %d values (one centre per radius), got %d' % (n, pos.numel()))
    if flags.numel() != ncells or owner.numel() != ncells:
        raise ValueError('flags and owner must hold nx*ny*nz = %d cells, got %d and %d'
                         % (ncells, flags.numel(), owner.numel()))
    for t, dt in ((pos, torch.float64), (radius, torch.float64), (flags, torch.uint8), (owner, torch.int32)):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt):
            raise ValueError('expected contiguous CUDA tensors of the documented dtypes')
    dev = flags.device
    if any(t.device != dev for t in (pos, radius, owner)):
        raise ValueError('pos, radius, flags and owner must be on one device')
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev).cuda_stream
        _check(load_library().lbm_map_spheres_noalloc(ctypes.byref(grid), float(shell_width), int(n),
                                                      c_void_p(pos.data_ptr()), c_void_p(radius.data_ptr()),
                                                      c_void_p(flags.data_ptr()), c_void_p(owner.data_ptr()),
                                                      c_void_p(stream)))


def lbm_fp64_fma_rate(iters=4096):
    """Measured float64 FMA throughput of the current device in TFLOP/s."""
    out = c_double(0.0)
    _check(load_library().lbm_fp64_fma_rate(int(iters), ctypes.byref(out)))
    return out.value


class LbmBatch:
    """Handle of a batch of contexts (see lbm_batch_create); keeps its contexts
    alive and releases the batch before them."""

    def __init__(self, handle, ctxs):
        self.handle = handle
        self.ctxs = list(ctxs)

    def __del__(self):
        if getattr(self, 'handle', None):
            load_library().lbm_batch_destroy(self.handle)
            self.handle = None


def _bcheck(status, b=None):
    if status != 0:
        msg = load_library().lbm_batch_last_error(b.handle if b is not None else None).decode()
        raise LbmError(status, msg)


def lbm_batch_create(ctxs, stream=None):
    """One batch over the contexts (one storage format). stream: a torch CUDA
    stream the batch runs on (None: the contexts' stream, the current one when
    they were created)."""
    arr = (c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    h = c_void_p()
    st = c_void_p(stream.cuda_stream) if stream is not None else None
    _bcheck(load_library().lbm_batch_create(arr, len(ctxs), st, ctypes.byref(h)))
    return LbmBatch(h, ctxs)


def lbm_batch_set_launch(b, instance=-1, tile_bx=0, zchunk=0, blocks_per_sm=0):
    _bcheck(load_library().lbm_batch_set_launch(b.handle, int(instance), int(tile_bx), int(zchunk),
                                                int(blocks_per_sm)), b)


def lbm_batch_set_active(b, instance, active):
    _bcheck(load_library().lbm_batch_set_active(b.handle, int(instance), int(bool(active))), b)


def lbm_batch_step(b, n_steps):
    _bcheck(load_library().lbm_batch_step(b.handle, int(n_steps)), b)


def lbm_batch_sync(b):
    _bcheck(load_library().lbm_batch_sync(b.handle), b)


def lbm_batch_capture_stats(b):
    """(graphs captured, host ms spent capturing and instantiating them)."""
    n, ms = c_int(0), c_double(0.0)
    _bcheck(load_library().lbm_batch_capture_stats(b.handle, ctypes.byref(n), ctypes.byref(ms)), b)
    return n.value, ms.value


def lbm_batch_launch_count(b):
    return int(load_library().lbm_batch_launch_count(b.handle))


def lbm_launch_count(ctx):
    return int(load_library().lbm_launch_count(ctx.handle))
