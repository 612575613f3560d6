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
