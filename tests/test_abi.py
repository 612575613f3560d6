"""The C-ABI library builds, loads and exports every declared symbol (CPU only).

No compute call is made here; the struct layouts of the Python binding are
checked against the C compiler's view of include/lbmdem.h.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'lbmdem.h')


@pytest.fixture(scope='module')
def lib():
    from paper_2003_01490_gb300 import build, lbmdem
    if not os.path.exists(lbmdem.LIB_PATH):
        build.build()
    return lbmdem.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r'^\s*(?:lbm_status|void|long long|const char \*)\s*(lbm_\w+)\s*\(',
                                 text, re.M)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ('lbm_create', 'lbm_add_spheres', 'lbm_step', 'lbm_get_particle_state',
              'lbm_get_fields', 'lbm_destroy', 'lbm_sync'):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2003_01490_gb300 import lbmdem
    names = declared_functions()
    assert set(names) == set(lbmdem.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_the_c_compiler(tmp_path, lib):
    from paper_2003_01490_gb300 import lbmdem
    src = tmp_path / 'sizes.c'
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbmdem.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(lbm_grid), '
                   'sizeof(lbm_relax), sizeof(lbm_dem), offsetof(lbm_dem, gravity), '
                   'offsetof(lbm_grid, wall_vel_hi));return 0;}\n')
    exe = tmp_path / 'sizes'
    subprocess.run(['gcc', '-I', os.path.join(ROOT, 'include'), str(src), '-o', str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(lbmdem.LbmGrid), ctypes.sizeof(lbmdem.LbmRelax),
            ctypes.sizeof(lbmdem.LbmDem), lbmdem.LbmDem.gravity.offset,
            lbmdem.LbmGrid.wall_vel_hi.offset]
    assert got == want


def test_default_params_are_the_papers(lib):
    from paper_2003_01490_gb300 import lbmdem
    r, d = lbmdem.lbm_default_params()
    assert r.magic == 3 / 16 and r.lambda_b_shell == 100 and r.lambda_b_bulk == 1 and r.shell_width == 2
    assert d.n_sub == 10 and d.lub_cut_n == 2 / 3 and d.lub_cut_tt == 0.5 and d.lub_cut_tr == 0.5
    assert d.lub_min_a == 0.001 and d.lub_min_b == 0.00007 and d.Tc == 0.0


def test_required_bytes_scales_with_storage(lib):
    from paper_2003_01490_gb300 import lbmdem
    g = lbmdem.make_grid((64, 64, 128))
    b64 = lbmdem.lbm_required_bytes(g, 'f64', 100)
    b32 = lbmdem.lbm_required_bytes(g, 'f32', 100)
    b16 = lbmdem.lbm_required_bytes(g, 'f16', 100)
    n = 64 * 64 * 128
    assert b64 - b32 == pytest.approx(2 * 19 * 4 * n, rel=0.01)
    assert b32 - b16 == pytest.approx(2 * 19 * 2 * n, rel=0.01)
    with pytest.raises(lbmdem.LbmError):
        lbmdem.lbm_required_bytes(lbmdem.make_grid((2, 64, 64)), 'f32', 1)


def raw_create(lib, **change):
    """lbm_create through the raw C call with one parameter changed; the
    argument checks all come before the first CUDA call."""
    from paper_2003_01490_gb300 import lbmdem
    r, d = lbmdem.lbm_default_params()
    shape = change.pop('shape', (16, 16, 32))
    storage = change.pop('storage', 1)
    max_particles = change.pop('max_particles', 4)
    for k, v in change.items():
        setattr(r if hasattr(r, k) else d, k, v)
    g = lbmdem.make_grid(shape)
    h = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(g), ctypes.byref(r), None, ctypes.byref(d), storage,
                        max_particles, None, ctypes.byref(h))
    return st, h.value, lib.lbm_last_error(None).decode()


@pytest.mark.parametrize("change, words", [
    (dict(tau=0.5), 'tau'),
    (dict(storage=4), 'storage'),
    (dict(max_particles=-1), 'max_particles'),
    (dict(max_particles=4000001), 'max_particles'),
    (dict(shape=(2, 16, 16)), 'at least 3'),
    (dict(shape=(2048, 1024, 1024)), '2^31'),
    (dict(n_sub=0), 'n_sub'),
    (dict(e_dry=0.0), 'e_dry'),
    (dict(e_dry=1.5), 'e_dry'),
    (dict(nu_p=1.0), 'nu_p'),
    (dict(mu_p=-0.1), 'mu_p'),
    (dict(lub_cut_tt=0.0), 'cut-offs'),
    (dict(magic=0.0), 'magic'),
    (dict(shell_width=-1.0), 'shell_width'),
    (dict(fixed_particles=3), 'fixed_particles'),
])
def test_create_rejects_invalid_parameters(lib, change, words):
    st, handle, msg = raw_create(lib, **change)
    assert st == -1 and handle is None
    assert words in msg


def test_calls_on_a_null_context_fail_cleanly(lib):
    from paper_2003_01490_gb300 import lbmdem
    P = ctypes.POINTER
    n = ctypes.c_int(0)
    size = ctypes.c_size_t(0)
    dp = P(ctypes.c_double)()
    calls = {
        'lbm_add_spheres': (None, 0, dp, dp, dp, dp, dp, None),
        'lbm_step': (None, 1),
        'lbm_sync': (None,),
        'lbm_set_stream': (None, None),
        'lbm_get_particle_state': (None, 0, dp, dp, dp, dp, dp, ctypes.byref(n)),
        'lbm_get_particle_state_async': (None, 0, dp, dp, dp, dp, dp, ctypes.byref(n)),
        'lbm_set_particle_velocity': (None, 0, dp, dp),
        'lbm_set_motion': (None, 0),
        'lbm_checkpoint_bytes': (None, ctypes.byref(size)),
        'lbm_save': (None, None, 0),
        'lbm_restore': (None, None, 0),
        'lbm_sample_density': (None, 0, dp, dp),
        'lbm_get_fields': (None, dp, dp, None),
        'lbm_get_owner': (None, None),
        'lbm_get_pdfs': (None, dp),
        'lbm_set_pdfs': (None, dp),
        'lbm_profile': (None, 1),
        'lbm_profile_read': (None, dp, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == -1, name
        assert lib.lbm_last_error(None).decode(), name
    assert lib.lbm_launch_count(None) == 0
    lib.lbm_destroy(None)
    for name in lbmdem.EXPORTS:
        assert name in calls or name in (
            'lbm_default_params', 'lbm_required_bytes', 'lbm_create', 'lbm_create_in_arena',
            'lbm_map_spheres_noalloc', 'lbm_fp64_fma_rate', 'lbm_launch_count', 'lbm_last_error',
            'lbm_destroy') or name.startswith('lbm_batch_'), name
    # batch calls on a NULL batch, and batch creation without contexts, fail
    # before any CUDA call
    assert lib.lbm_batch_create(None, 0, None, None) == -1
    h = ctypes.c_void_p()
    assert lib.lbm_batch_create((ctypes.c_void_p * 1)(None), 1, None, ctypes.byref(h)) == -1 and not h.value
    assert lib.lbm_batch_set_launch(None, -1, 0, 0, 0) == -1
    assert lib.lbm_batch_set_active(None, 0, 1) == -1
    assert lib.lbm_batch_step(None, 1) == -1
    assert lib.lbm_batch_sync(None) == -1
    assert lib.lbm_batch_launch_count(None) == 0
    assert lib.lbm_batch_capture_stats(None, None, None) == -1
    assert lib.lbm_batch_last_error(None).decode()
    lib.lbm_batch_destroy(None)
    # the float64 throughput probe checks its arguments before any CUDA call
    out = ctypes.c_double(0.0)
    assert lib.lbm_fp64_fma_rate(0, ctypes.byref(out)) == -1
    assert lib.lbm_fp64_fma_rate(10, None) == -1


def test_create_in_arena_and_mapping_entry_reject_bad_arguments(lib):
    from paper_2003_01490_gb300 import lbmdem
    r, d = lbmdem.lbm_default_params()
    g = lbmdem.make_grid((16, 16, 32))
    h = ctypes.c_void_p()
    assert lib.lbm_create_in_arena(ctypes.byref(g), ctypes.byref(r), None, ctypes.byref(d), 1, 4, None,
                                   None, 0, ctypes.byref(h)) == -1
    assert 'arena' in lib.lbm_last_error(None).decode()
    assert lib.lbm_create(ctypes.byref(g), ctypes.byref(r), None, ctypes.byref(d), 1, 4, None, None) == -1
    # the allocation-free mapping entry checks its arguments before any CUDA call
    buf = ctypes.c_void_p(16)    # never dereferenced: every call below fails its checks first
    for args in [(ctypes.byref(g), 2.0, -1, buf, buf, buf, buf, None),
                 (ctypes.byref(g), 2.0, 1, None, buf, buf, buf, None),
                 (ctypes.byref(g), 2.0, 0, None, None, None, buf, None),
                 (ctypes.byref(lbmdem.make_grid((2, 16, 16))), 2.0, 0, None, None, buf, buf, None),
                 (ctypes.byref(g), -1.0, 0, None, None, buf, buf, None),
                 (ctypes.byref(g), 2.0, 65537, buf, buf, buf, buf, None),
                 (None, 2.0, 0, None, None, buf, buf, None)]:
        assert lib.lbm_map_spheres_noalloc(*args) == -1
    with pytest.raises(lbmdem.LbmError, match='storage'):
        size = ctypes.c_size_t(0)
        lbmdem._check(lib.lbm_required_bytes(ctypes.byref(g), 5, 1, ctypes.byref(size)))


def test_mapping_entry_wrapper_refuses_mismatched_sizes_before_any_gpu_work():
    # the C side writes nx*ny*nz flag bytes and owners and reads 3 n positions:
    # buffers of other sizes are refused by the binding (CPU tensors here, so
    # nothing could have reached a device)
    torch = pytest.importorskip('torch')
    from paper_2003_01490_gb300 import lbmdem
    g = lbmdem.make_grid((16, 16, 32))
    cells = 16 * 16 * 32
    ok = dict(pos=torch.zeros(6, dtype=torch.float64), radius=torch.ones(2, dtype=torch.float64),
              flags=torch.zeros(cells, dtype=torch.uint8), owner=torch.zeros(cells, dtype=torch.int32))
    bad = [dict(ok, pos=torch.zeros(5, dtype=torch.float64)),
           dict(ok, flags=torch.zeros(cells - 1, dtype=torch.uint8)),
           dict(ok, owner=torch.zeros(cells // 2, dtype=torch.int32))]
    for kw in bad:
        with pytest.raises(ValueError, match='pos must|flags and owner'):
            lbmdem.lbm_map_spheres_noalloc(g, 2.0, kw['pos'], kw['radius'], kw['flags'], kw['owner'])
    # right sizes, but host tensors: refused as not CUDA tensors
    with pytest.raises(ValueError, match='CUDA'):
        lbmdem.lbm_map_spheres_noalloc(g, 2.0, ok['pos'], ok['radius'], ok['flags'], ok['owner'])
