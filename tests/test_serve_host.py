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


def test_cancellation_picks_due_jobs_that_wait_or_run():
    cancel_at = {0: 0.5, 2: 0.1, 5: 0.2, 7: 9.0}
    # job 2 waits and is due; job 5 runs and is due; job 7 is not due yet;
    # job 0 is due but already finished (neither waiting nor running)
    drop_wait, drop_run = serve.cancellations([2, 3, 7], [4, 5], cancel_at, now=0.6)
    assert drop_wait == [2] and drop_run == [5]
    assert serve.cancellations([2, 3], [5], cancel_at, now=0.05) == ([], [])
    assert serve.cancellations([], [], {}, now=1.0) == ([], [])


def test_summary_counts_cancelled_work_but_not_their_latency():
    recs = [dict(arrival=0.0, done=1.0, latency=1.0, cell_updates=2_000_000),
            dict(arrival=0.0, done=2.0, latency=2.0, cell_updates=2_000_000, cancelled=False),
            dict(arrival=0.5, done=0.7, latency=0.2, cell_updates=500_000, cancelled=True)]
    s = serve.summary(recs)
    assert s['jobs'] == 2 and s['cancelled'] == 1
    assert s['makespan_s'] == 2.0 and s['jobs_per_s'] == 1.0
    assert abs(s['mlups'] - 4.5e6 / 2.0 / 1e6) <= 0.05 + 1e-12      # rounded to 0.1
    assert abs(s['p50_latency_s'] - 1.5) < 1e-9
