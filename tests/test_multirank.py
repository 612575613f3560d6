"""The multi-rank path of bench.py on the host: two gloo ranks (world size 2,
one process each, as torch.distributed.run starts them) set up the group,
take the slowest rank's time with the max-reduction, meet at the barrier and
report whole-job MLUPS over both replicas; under --impl reference only rank 0
prints. No GPU involved."""
import json
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    if torch.cuda.is_available():   # keep this test on the host
        torch.cuda.is_available = lambda: False
    r, w, _ = bench.dist_setup(world)
    ms = 10.0 + 5.0 * r                       # rank 1 is the slower one
    ms_max = bench.allreduce_max(ms, w)
    bench.barrier(w)
    value = bench.whole_job_mlups(w, 1000, 20, ms_max)
    with open(os.path.join(out_dir, 'rank%d.json' % r), 'w') as fh:
        json.dump(dict(rank=r, world=w, ms_max=ms_max, value=value), fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_time(tmp_path):
    mp = pytest.importorskip('torch.multiprocessing')
    port = free_port()
    mp.start_processes(rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method='spawn')
    res = [json.load(open(tmp_path / ('rank%d.json' % r))) for r in range(2)]
    for r in res:
        assert r['world'] == 2
        assert r['ms_max'] == 15.0
        # two replicas of 1000 cells, 20 steps each, in the slowest rank's 15 ms
        assert abs(r['value'] - 2 * 1000 * 20 / 15e-3 / 1e6) < 1e-12


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = 'suspension'
        steps, warmup, reference_budget = 1, 0, 1.0

    bench.run_reference(Args(), rank=1, world=2)
    assert capsys.readouterr().out == ''


def test_bench_refuses_a_rank_count_other_than_gpus():
    # launched with WORLD_SIZE ranks that differ from --gpus: exit non-zero
    # before any work instead of silently timing fewer replicas
    import subprocess
    env = dict(os.environ, WORLD_SIZE='1', RANK='0', LOCAL_RANK='0')
    r = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--gpus', '2', '--steps', '1'],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode != 0
    assert '--gpus 2 but WORLD_SIZE=1' in r.stderr
