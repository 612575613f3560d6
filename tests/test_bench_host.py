"""Host-side arithmetic of bench.py's measurement (CPU only): the particle
link count behind the algorithmic bytes of the dense kernel, the bytes per
cell, and the rule that the DRAM traffic recorded from an ncu capture is
reported only while the captured kernel source is unchanged."""
import itertools
import json
import os

import numpy as np
import pytest

import bench
from oracle.d3q19 import C


def links_by_loops(solid, periodic):
    """(fluid cell, direction) pairs whose upstream cell is a solid cell, by
    plain loops over D3Q19 (cells beyond a wall are not particles)."""
    nz, ny, nx = solid.shape
    n = 0
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        for q in range(1, 19):
            u = [x - C[q][0], y - C[q][1], z - C[q][2]]
            out = False
            for a, size in enumerate((nx, ny, nz)):
                if not 0 <= u[a] < size:
                    if periodic[a]:
                        u[a] %= size
                    else:
                        out = True
            if not out and solid[u[2], u[1], u[0]]:
                n += 1
    return n


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 1, 0), (0, 1, 0), (0, 0, 0)])
def test_link_count_matches_plain_loops(periodic):
    rng = np.random.default_rng(7)
    solid = rng.random((7, 5, 6)) < 0.3
    assert bench.count_links(solid, periodic) == links_by_loops(solid, periodic)


def test_bytes_per_cell():
    # two PDF arrays of 19 values and the flag byte per fluid cell; a solid
    # cell costs its flag byte only
    assert bench.bytes_per_cell('f64') == (305, 1)
    assert bench.bytes_per_cell('f32') == (153, 1)
    assert bench.bytes_per_cell('f16') == (77, 1)
    assert bench.bytes_per_cell('bf16') == (77, 1)


def test_whole_job_value_counts_every_rank():
    assert bench.whole_job_mlups(4, 1_000_000, 10, 5.0) == pytest.approx(8000.0)


def test_recorded_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    csrc = tmp_path / 'paper_2003_01490_gb300' / 'csrc'
    csrc.mkdir(parents=True)
    for f in ('stream_collide.cu', 'stream_collide_staged.cu', 'sc_common.cuh', 'links.cuh', 'common.cuh'):
        (csrc / f).write_text('// ' + f + '\n')
    (tmp_path / 'profiles').mkdir()
    monkeypatch.setattr(bench, 'ROOT', str(tmp_path))
    h = bench.kernel_source_hash()
    summary = tmp_path / 'profiles' / 'stream_collide_box_f32.md'
    summary.write_text('traffic_bytes_per_launch: 123456\nsource_sha256: `%s`\n' % h)
    assert bench.recorded_traffic('f32', 'box') == 123456.0
    assert bench.recorded_traffic('f16', 'box') is None          # no summary for it
    (csrc / 'links.cuh').write_text('// changed\n')
    assert bench.recorded_traffic('f32', 'box') is None          # kernel changed since


def test_measured_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, 'ROOT', str(tmp_path))
    assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, 'fallback')
    (tmp_path / 'MEASURED_PEAKS.json').write_text(json.dumps({'hbm_gbs': 6691.5}))
    assert bench.measured_peak() == (6691.5, 'measured')


def test_committed_profile_summary_is_well_formed():
    p = os.path.join(bench.ROOT, 'profiles', 'stream_collide_suspension_f32.md')
    text = open(p).read()
    assert 'traffic_bytes_per_launch:' in text and 'source_sha256:' in text
    assert '--clock-control none' in text
