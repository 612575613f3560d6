"""The allocation-free mapping entry point against the context's own mapping.

lbm_map_spheres_noalloc() exists for callers that cannot call cudaMalloc (a
host framework that owns all device memory, or a loop that cannot afford an
allocation's device synchronisation). It keeps its temporaries in a static
device array, so two calls in a row must both give the flags and owners that
lbm_add_spheres() produces for the same spheres in a new context.
"""
import numpy as np
import pytest

from cases import build_gpu, spheres

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def L():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2003_01490_gb300 import lbmdem
    lbmdem.load_library()
    return lbmdem


def test_no_alloc_mapping_matches_context_mapping(L):
    import torch
    from paper_2003_01490_gb300 import workloads
    w = workloads.reduced_suspension(storage='f32')
    case = dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage='f32',
                spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                dem=dict(w['dem'], fixed_particles=1))
    ctx = build_gpu(case)
    _, _, flags_ref = L.lbm_get_fields(ctx)
    owner_ref = L.lbm_get_owner(ctx)
    assert (flags_ref & L.FLAG_SOLID).any()
    grid = L.make_grid(w['shape'], w['periodic'])
    ncells = int(np.prod(w['shape']))
    pos = torch.tensor(w['pos'].reshape(-1), dtype=torch.float64, device='cuda')
    rad = torch.tensor(w['radius'], dtype=torch.float64, device='cuda')
    flags = torch.full((ncells,), 0xAB, dtype=torch.uint8, device='cuda')
    owner = torch.full((ncells,), 12345, dtype=torch.int32, device='cuda')
    nx, ny, nz = w['shape']
    for _ in range(2):
        L.lbm_map_spheres_noalloc(grid, 2.0, pos, rad, flags, owner)
        torch.cuda.synchronize()
        f = flags.cpu().numpy().reshape(nz, ny, nx)
        o = owner.cpu().numpy().reshape(nz, ny, nx)
        assert np.array_equal(f, flags_ref)
        assert np.array_equal(o, owner_ref)


def test_no_alloc_mapping_rejects_boxes_beyond_its_scratch(L):
    # straight through the C ABI: the box limit is checked before any buffer
    # is touched, so these small buffers are never written
    import ctypes
    import torch
    grid = L.make_grid((1024, 1024, 512))
    pos = torch.zeros(3, dtype=torch.float64, device='cuda')
    rad = torch.ones(1, dtype=torch.float64, device='cuda')
    flags = torch.zeros(8, dtype=torch.uint8, device='cuda')
    owner = torch.zeros(8, dtype=torch.int32, device='cuda')
    st = torch.cuda.current_stream().cuda_stream
    rc = L.load_library().lbm_map_spheres_noalloc(
        ctypes.byref(grid), 2.0, 1, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(rad.data_ptr()),
        ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(owner.data_ptr()), ctypes.c_void_p(st))
    assert rc == -1
    assert 'scratch' in L.load_library().lbm_last_error(None).decode()


def test_no_alloc_mapping_from_two_host_threads(L):
    # Two host threads map different sphere sets on their own streams at the
    # same time; the per-device lock serialises the calls on the shared
    # scratch, so each result equals the context mapping of its own set.
    import threading
    import torch
    from paper_2003_01490_gb300 import workloads
    sets = [workloads.suspension(shape=(64, 64, 128), n=150, seed=20030149 + k, storage='f32') for k in (7, 8)]
    refs = []
    for w in sets:
        case = dict(shape=w['shape'], periodic=w['periodic'], tau=w['tau'], storage='f32',
                    spheres=spheres(w['pos'], w['radius'], w['density'], w['vel'], w['omega']),
                    dem=dict(w['dem'], fixed_particles=1))
        ctx = build_gpu(case)
        _, _, fl = L.lbm_get_fields(ctx)
        refs.append((fl.reshape(-1), L.lbm_get_owner(ctx).reshape(-1)))
        del ctx
    torch.cuda.synchronize()
    grid = L.make_grid(sets[0]['shape'], sets[0]['periodic'])
    ncells = int(np.prod(sets[0]['shape']))
    errors = []

    def worker(k):
        try:
            w = sets[k]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                pos = torch.tensor(w['pos'].reshape(-1), dtype=torch.float64, device='cuda')
                rad = torch.tensor(w['radius'], dtype=torch.float64, device='cuda')
                flags = torch.empty(ncells, dtype=torch.uint8, device='cuda')
                owner = torch.empty(ncells, dtype=torch.int32, device='cuda')
                for _ in range(20):
                    L.lbm_map_spheres_noalloc(grid, 2.0, pos, rad, flags, owner)
                    if not (np.array_equal(flags.cpu().numpy(), refs[k][0]) and
                            np.array_equal(owner.cpu().numpy(), refs[k][1])):
                        errors.append('thread %d: mapping differs' % k)
                        return
        except Exception as ex:   # reported by the main thread
            errors.append('thread %d: %r' % (k, ex))

    threads = [threading.Thread(target=worker, args=(k,)) for k in (0, 1)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
