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


# ---------------------------------------------------------------------------
# continuous batching (BatchedServingLoop) with a fake slotted backend
# ---------------------------------------------------------------------------
from paper_2203_02369_gb300.serve import BatchedServingLoop, group_key  # noqa: E402


class FakeSlots:
    """Mirrors hm_slots_* bookkeeping: packed indices, release moves the last
    loaded chain into the freed index; every trajectory advances all loaded jobs."""

    instances = []

    def __init__(self, job, n_slots):
        self.key = group_key(job)
        self.n_slots = n_slots
        self.loaded = []          # job ids by chain index
        self.runs = []            # job ids advanced together by each trajectory
        self.closed = False
        self.lock = threading.Lock()
        FakeSlots.instances.append(self)

    def load(self, job):
        assert group_key(job) == self.key
        assert len(self.loaded) < self.n_slots
        self.loaded.append(job.job_id)
        return len(self.loaded) - 1

    def run(self, k):
        time.sleep(0.002 * k)
        rec = np.zeros((k, len(self.loaded)), dtype=[("psi", float), ("accept", np.int32)])
        for t in range(k):
            self.runs.append(tuple(self.loaded))
            rec["psi"][t] = [float(j) for j in self.loaded]
        rec["accept"] = 1
        return rec

    def adapt_end(self, index):
        return 0.02

    def get(self, index):
        return None, None

    def release(self, index):
        last = len(self.loaded) - 1
        if index != last:
            self.loaded[index] = self.loaded[last]
        self.loaded.pop()
        return last if index != last else -1

    def close(self):
        self.closed = True


def _bloop(**kw):
    FakeSlots.instances = []
    kw.setdefault("free_bytes", lambda: 1 << 40)
    return BatchedServingLoop(reserve_bytes=0, backend_factory=FakeSlots, prepare=lambda j: j, **kw)


import numpy as np  # noqa: E402


def test_batched_jobs_share_launches_and_late_arrivals_join_running_groups():
    loop = _bloop(max_slots=4)
    jobs = [_job(k, N=64, arrival=0.0 if k < 2 else 0.03, n_traj=20) for k in range(4)]
    stats = loop.run(jobs)
    assert stats["jobs"] == 4 and not stats["errors"]
    (be,) = FakeSlots.instances           # one field model, one slotted state
    assert be.closed
    # continuous batching: late arrivals were loaded while the first two ran
    assert any(len(r) == 4 for r in be.runs)
    assert any(len(r) == 2 for r in be.runs)
    for j in jobs:
        assert len(j.traj_latency) == 20 and j.psi == [float(j.job_id)] * 20
        assert j.admitted >= j.arrival and j.finished >= j.admitted


def test_batched_groups_by_field_model_and_bounds_slots():
    loop = _bloop(max_slots=2)
    jobs = [_job(k, N=64 if k % 2 else 128, arrival=0.001 * k, n_traj=5) for k in range(8)]
    stats = loop.run(jobs)
    assert stats["jobs"] == 8 and not stats["errors"]
    assert len(FakeSlots.instances) == 2
    for be in FakeSlots.instances:
        assert max(len(r) for r in be.runs) <= 2
        assert len({group_key(j) for j in jobs if j.spec.N == (64 if be.key[0] == 64 else 128)}) == 1
    assert loop.max_active_seen <= 2


def test_batched_release_moves_keep_each_jobs_records_its_own():
    # jobs of different lengths leave from the middle of the packed indices
    loop = _bloop(max_slots=4)
    jobs = [_job(k, N=64, arrival=0.0, n_traj=3 + 4 * k) for k in range(4)]
    stats = loop.run(jobs)
    assert not stats["errors"]
    for j in jobs:
        assert j.psi == [float(j.job_id)] * j.n_traj


def test_batched_warmup_trajectories_are_not_timed():
    loop = _bloop(max_slots=2)
    j = _job(0, N=64, n_traj=4)
    j.adapt_warmup = 3
    loop.run([j])
    (be,) = FakeSlots.instances
    assert len(be.runs) == 7 and len(j.traj_latency) == 4 and j.eps_used == 0.02


def test_batched_slot_count_follows_free_memory_and_oversize_jobs_fail():
    from paper_2203_02369_gb300.serve import slots_footprint_bytes
    per = slots_footprint_bytes(128, 1, 1000)
    loop = _bloop(max_slots=8, max_points=1000, free_bytes=lambda: 3 * per)
    jobs = [_job(k, N=128, n=500, n_traj=2) for k in range(5)] + [_job(9, N=128, n=5000, n_traj=2)]
    stats = loop.run(jobs)
    assert FakeSlots.instances[0].n_slots == 2
    assert len(stats["errors"]) == 1 and "exceeds the slot room" in stats["errors"][0]


def test_batched_failing_prepare_is_reported():
    FakeSlots.instances = []

    def prep(j):
        if j.job_id == 1:
            raise RuntimeError("injected catalogue failure")
        return j

    loop = BatchedServingLoop(reserve_bytes=0, backend_factory=FakeSlots, prepare=prep, free_bytes=lambda: 1 << 40)
    stats = loop.run([_job(k, n_traj=2) for k in range(3)])
    assert stats["jobs"] == 3 and len(stats["errors"]) == 1 and "injected" in stats["errors"][0]


def test_batched_device_failure_fails_that_groups_jobs_only():
    """A run that fails on the device (here: the fake raises, as a library
    error would surface) ends the jobs then loaded in that group with an
    error; later jobs of the group and other groups are still served."""
    class Flaky(FakeSlots):
        def run(self, k):
            if self.key[0] == 128 and len(self.runs) >= 2 and not getattr(self, "failed", False):
                self.failed = True
                raise RuntimeError("injected device failure")
            return super().run(k)

    FakeSlots.instances = []
    loop = BatchedServingLoop(max_slots=2, reserve_bytes=0, backend_factory=Flaky, prepare=lambda j: j,
                              free_bytes=lambda: 1 << 40)
    jobs = ([_job(k, N=128, arrival=0.0, n_traj=6) for k in range(2)] + [_job(2, N=128, arrival=0.05, n_traj=3)]
            + [_job(k, N=64, arrival=0.0, n_traj=4) for k in (3, 4)])
    stats = loop.run(jobs)
    assert stats["jobs"] == 5
    errs = {j.job_id for j in jobs if j.error}
    assert errs == {0, 1}
    assert all("injected device failure" in jobs[k].error for k in (0, 1))
    assert len(jobs[2].traj_latency) == 3 and all(len(jobs[k].traj_latency) == 4 for k in (3, 4))


def test_batched_grid_slot_policy_and_latency_by_grid():
    # a grid held to one slot serves its jobs one after another while another
    # grid batches; the stats report latency per grid
    loop = _bloop(max_slots=4, grid_slots={128: 1})
    jobs = [_job(k, N=128 if k % 2 else 64, arrival=0.0, n_traj=5) for k in range(6)]
    stats = loop.run(jobs)
    assert stats["jobs"] == 6 and not stats["errors"]
    by = {be.key[0]: be for be in FakeSlots.instances}
    assert by[128].n_slots == 1 and max(len(r) for r in by[128].runs) == 1
    assert by[64].n_slots == 4 and max(len(r) for r in by[64].runs) == 3
    assert set(stats["by_grid"]) == {"64", "128"}
    assert stats["by_grid"]["128"]["jobs"] == 3
    assert stats["by_grid"]["64"]["trajectory_latency_ms"]["p50"] > 0
