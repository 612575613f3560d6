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
    import torch
    grid = L.make_grid((1024, 1024, 512))
    pos = torch.zeros(3, dtype=torch.float64, device='cuda')
    rad = torch.ones(1, dtype=torch.float64, device='cuda')
    flags = torch.zeros(8, dtype=torch.uint8, device='cuda')
    owner = torch.zeros(8, dtype=torch.int32, device='cuda')
    with pytest.raises(L.LbmError) as err:
        L.lbm_map_spheres_noalloc(grid, 2.0, pos, rad, flags, owner)
    assert err.value.status == -1
