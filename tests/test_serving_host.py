"""Scheduling logic of the serving loop without a GPU: a fake runner stands in
for the device work and a fake memory probe for the free device memory."""
import threading
import time

from paper_2203_02369_gb300 import mock
from paper_2203_02369_gb300.serve import Job, ServingLoop, footprint_bytes, poisson_jobs


def _job(k, N=64, n=1000, arrival=0.0, n_traj=3):
    spec = mock.MockSpec(N=N, L=500.0, n_points=n, r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=k)
    return Job(job_id=k, spec=spec, n_traj=n_traj, arrival=arrival)


def test_slots_bound_concurrency_and_every_job_finishes():
    active = [0]
    peak = [0]
    lock = threading.Lock()

    def runner(job):
        with lock:
            active[0] += 1
            peak[0] = max(peak[0], active[0])
        time.sleep(0.02)
        job.traj_latency = [0.001] * job.n_traj
        job.psi = [1.0, 2.0, 1.5, 1.2]
        job.accept = [1, 0, 1, 1]
        with lock:
            active[0] -= 1

    loop = ServingLoop(max_slots=3, reserve_bytes=0, runner=runner, free_bytes=lambda: 1 << 40)
    jobs = [_job(k, arrival=0.001 * k) for k in range(10)]
    stats = loop.run(jobs)
    assert stats["jobs"] == 10 and not stats["errors"]
    assert peak[0] <= 3 and loop.max_active_seen <= 3
    assert peak[0] >= 2          # jobs did overlap
    for j in jobs:
        assert j.admitted >= j.arrival and j.finished >= j.admitted


def test_admission_waits_for_memory():
    # room for one 128^3 job at a time: the second waits for the first
    need = footprint_bytes(128, 1000)
    order = []

    def runner(job):
        order.append(("start", job.job_id))
        time.sleep(0.03)
        order.append(("end", job.job_id))

    loop = ServingLoop(max_slots=8, reserve_bytes=0, runner=runner,
                       free_bytes=lambda: int(1.5 * need) - loop._in_use)
    jobs = [_job(0, N=128), _job(1, N=128)]
    loop.run(jobs)
    assert order.index(("end", 0)) < order.index(("start", 1))


def test_failing_job_is_reported_and_the_loop_keeps_serving():
    def runner(job):
        if job.job_id == 1:
            raise RuntimeError("injected host-side failure")
        job.traj_latency = [0.001]

    loop = ServingLoop(max_slots=2, reserve_bytes=0, runner=runner, free_bytes=lambda: 1 << 40)
    stats = loop.run([_job(k) for k in range(4)])
    assert stats["jobs"] == 4
    assert len(stats["errors"]) == 1 and "injected" in stats["errors"][0]


def test_poisson_stream_shape():
    jobs = poisson_jobs(50, rate_per_s=10.0, seed=3)
    t = [j.arrival for j in jobs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert {j.spec.N for j in jobs} <= {64, 128}
    ns = [j.spec.n_points for j in jobs]
    assert min(ns) >= 1000 and max(ns) <= 100000
