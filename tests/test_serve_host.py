"""Host logic of the served mode (paper_2003_01490_gb300/serve.py), no GPU:
admission in arrival order within the memory budget, and the latency and
throughput summary."""
import numpy as np

from paper_2003_01490_gb300 import serve


def test_admission_in_arrival_order_within_the_budget():
    arrival = [0.0, 0.1, 0.2, 0.3]
    need = [4, 3, 5, 1]
    # at t = 0.25 jobs 0-2 have arrived; the budget of 8 takes 0 and 1, and job 2 (5) does not fit
    admitted, used = serve.admissions([0, 1, 2, 3], arrival, need, now=0.25, used=0, budget_bytes=8)
    assert admitted == [0, 1] and used == 7
    # job 2 blocks the queue head although job 3 would fit (arrival order is kept)
    admitted, used = serve.admissions([2, 3], arrival, need, now=0.5, used=7, budget_bytes=8)
    assert admitted == [] and used == 7
    # once memory is back, both go in order
    admitted, used = serve.admissions([2, 3], arrival, need, now=0.5, used=0, budget_bytes=8)
    assert admitted == [2, 3] and used == 6
    # nothing has arrived yet
    assert serve.admissions([0], arrival, need, now=-1.0, used=0, budget_bytes=100) == ([], 0)


def test_summary_latencies_and_throughput():
    recs = [dict(arrival=0.1 * k, done=0.1 * k + 0.5 + 0.01 * k, latency=0.5 + 0.01 * k, cell_updates=1_000_000)
            for k in range(10)]
    s = serve.summary(recs)
    span = recs[-1]['done'] - recs[0]['arrival']
    assert s['jobs'] == 10
    assert abs(s['makespan_s'] - span) < 1e-4
    assert abs(s['jobs_per_s'] - 10 / span) < 0.01
    assert abs(s['mlups'] - 10 * 1_000_000 / span / 1e6) < 0.1
    lat = np.array([r['latency'] for r in recs])
    assert abs(s['p50_latency_s'] - np.percentile(lat, 50)) < 1e-4
    assert abs(s['p99_latency_s'] - np.percentile(lat, 99)) < 1e-4


def test_a_job_larger_than_the_budget_is_rejected_before_any_work():
    # it could never be admitted and would hold the head of the queue for ever
    import os
    import pytest
    from paper_2003_01490_gb300 import build, lbmdem, workloads
    if not os.path.exists(lbmdem.LIB_PATH):
        build.build()
    jobs = workloads.served(n=3)
    need = [serve.job_bytes(j) for j in jobs]
    with pytest.raises(ValueError, match='memory budget'):
        serve.serve(jobs, budget_bytes=max(need) - 1)
