"""Serving loops for HAMLET reconstruction jobs.

Jobs (a catalogue on a grid, a number of HMC trajectories) arrive over time
and their chain states stay resident on the device until they finish.

BatchedServingLoop is continuous batching: jobs that share a field model
(grid, box, precision, leapfrog count) are served by one slotted state
(libhamlet's hm_slots_*), which advances every loaded job in the same kernel
launches, one captured CUDA graph per trajectory.  A job arriving while
others run is prepared on a host thread and loaded into a free slot between
two trajectories; a finished job leaves its slot at once.  Each group runs
on its own host thread and CUDA stream, so groups of different grids overlap
on the device.  A group's slot count is set when its first job arrives, from
the free device memory minus a reserve (admission by footprint).

ServingLoop runs each admitted job as a worker thread with its own CUDA
stream (jobs overlap on the device, each in its own launches); with one slot
it is the plain one-job-at-a-time baseline.

Reported by both: latency percentiles per trajectory and per job, aggregate
gradient evaluations/s and effective samples/s.
"""
from __future__ import annotations

import collections
import concurrent.futures
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import mock
from .ess import ess
from .hamlet import Problem, Slots, State


@dataclass
class Job:
    job_id: int
    spec: mock.MockSpec
    n_traj: int
    n_leapfrog: int = 20
    eps: float = 0.025
    seed: int = 0
    arrival: float = 0.0            # seconds after the start of the run
    adapt_warmup: int = 0           # dual-averaging warm-up trajectories before the timed ones
    accept_target: float = 0.70
    sample_sigma_nl: bool = False   # sigma_NL as a chain coordinate, starting at the spec's value
    # filled in by the loop
    admitted: float = float("nan")
    finished: float = float("nan")
    traj_latency: list = field(default_factory=list)
    psi: list = field(default_factory=list)
    accept: list = field(default_factory=list)
    eps_used: float = float("nan")
    final_w: object = None
    final_d: object = None
    error: str = ""


def footprint_bytes(N, n_points, precision="fp32"):
    """Device memory one single-chain job keeps resident: five real grids
    (w, p, grad, saved w, saved grad), six half spectra of workspace, the
    point arrays and bucket records."""
    rsz = 4 if precision == "fp32" else 8
    R = rsz * N ** 3
    S = 2 * rsz * N * N * (N // 2 + 1)
    return 5 * R + 6 * S + n_points * 700 + (8 << 20)


def slots_footprint_bytes(N, n_slots, max_points, precision="fp32"):
    """Device memory of one slotted state: per slot five real grids and six
    half spectra, per point of room about 300 B of catalogue, chain and
    bucket arrays."""
    rsz = 4 if precision == "fp32" else 8
    R = rsz * N ** 3
    S = 2 * rsz * N * N * (N // 2 + 1)
    return n_slots * (5 * R + 6 * S) + n_slots * max_points * 300 + (16 << 20)


class ServingLoop:
    """runner(job) executes one admitted job on the device (default: the
    HAMLET chain below); free_bytes() reports free device memory.  Both are
    injectable so that the scheduling logic can be exercised without a GPU."""

    def __init__(self, max_slots=4, reserve_bytes=2 << 30, device=0, use_graph=True, keep_state=False,
                 runner=None, free_bytes=None):
        self.max_slots = max_slots
        self.reserve = reserve_bytes
        self.device = device
        self.use_graph = use_graph
        self.keep_state = keep_state
        self.runner = runner or self._run_chain
        self.free_bytes = free_bytes or (lambda: torch.cuda.mem_get_info(self.device)[0])
        self._lock = threading.Lock()
        self._in_use = 0          # bytes admitted and not yet released
        self._active = 0
        self.max_active_seen = 0
        self.admission_log = []   # (time, job_id, active after admission)

    def _run_job(self, job: Job, t0: float, done: "queue.Queue"):
        try:
            self.runner(job)
        except Exception as exc:   # reported per job; the loop keeps serving
            job.error = repr(exc)
        job.finished = time.perf_counter() - t0
        done.put(job)

    def _run_chain(self, job: Job):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(stream):
            cat = mock.make_catalog(job.spec)
            prob = Problem.from_mock(job.spec, cat, device=self.device)
            st = State(prob, [cat["d_init"]], seed=job.seed, chain_ids=[job.job_id])
            if job.sample_sigma_nl:
                st.sample_sigma_nl(True, job.spec.sigma_nl)
            eps = job.eps
            if job.adapt_warmup > 0:
                # the job's own step size, tuned to the target acceptance
                e, _ = st.adapt_step_size(job.adapt_warmup, job.n_leapfrog, job.eps, target=job.accept_target)
                eps = float(e[0])
            job.eps_used = eps
            for _ in range(job.n_traj):
                a = time.perf_counter()
                tr = st.run_chain(1, job.n_leapfrog, eps, use_graph=self.use_graph, trace=True)
                job.traj_latency.append(time.perf_counter() - a)
                job.psi.append(float(tr[0, 0]["psi"]))
                job.accept.append(int(tr[0, 0]["accept"]))
            if self.keep_state:
                g = st.get(0)
                stream.synchronize()
                job.final_w = g["w"].cpu()
                job.final_d = g["d"].cpu()
            st.close()
            prob.close()
            stream.synchronize()

    def run(self, jobs):
        """Serve `jobs` (arrival times in seconds from now); returns stats."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        waiting = []
        done = queue.Queue()
        threads = []
        finished = []
        t0 = time.perf_counter()
        i = 0
        while len(finished) < len(jobs):
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                waiting.append(pending[i])
                i += 1
            # admit in arrival order while a slot and memory are available
            while waiting:
                j = waiting[0]
                need = footprint_bytes(j.spec.N, j.spec.n_points, j.spec.precision)
                with self._lock:
                    ok = self._active < self.max_slots and need + self.reserve <= self.free_bytes()
                    if ok:
                        self._active += 1
                        self._in_use += need
                        self.max_active_seen = max(self.max_active_seen, self._active)
                if not ok:
                    break
                waiting.pop(0)
                j.admitted = time.perf_counter() - t0
                self.admission_log.append((j.admitted, j.job_id, self._active))
                th = threading.Thread(target=self._run_job, args=(j, t0, done), daemon=True)
                th.start()
                threads.append(th)
            try:
                j = done.get(timeout=0.002)
                with self._lock:
                    self._active -= 1
                    self._in_use -= footprint_bytes(j.spec.N, j.spec.n_points, j.spec.precision)
                finished.append(j)
            except queue.Empty:
                pass
        for th in threads:
            th.join()
        makespan = time.perf_counter() - t0
        return summarize(finished, makespan)


def group_key(job):
    """Jobs that can share a slotted state."""
    sp = job.spec
    return (sp.N, float(sp.L), sp.precision, job.n_leapfrog, tuple(sorted(vars(sp.cosmo).items())))


class SlotsBackend:
    """One slotted state on its own CUDA stream (the device side of a group)."""

    def __init__(self, job, n_slots, max_points, seed, device=0, use_graph=True, priority=0):
        torch.cuda.set_device(device)
        # a lower number is a higher priority: the device schedules the CTAs
        # of this group's pending kernels ahead of lower-priority streams
        self.stream = torch.cuda.Stream(device=device, priority=int(priority))
        sp = job.spec
        self.n_leapfrog = job.n_leapfrog
        self.use_graph = use_graph
        with torch.cuda.stream(self.stream):
            self.template = Problem(sp.N, sp.L, sp.cosmo, sp.sigma_nl, sp.precision, device=device)
            self.slots = Slots(self.template, n_slots, max_points, seed=seed)

    def load(self, job):
        with torch.cuda.stream(self.stream):
            return self.slots.load(job._prob, job._cat["d_init"], job.job_id, job.eps,
                                   job.accept_target if job.adapt_warmup > 0 else 0.0,
                                   job.spec.sigma_nl if job.sample_sigma_nl else 0.0)

    def run(self, n_traj):
        with torch.cuda.stream(self.stream):
            return self.slots.run(n_traj, self.n_leapfrog, self.use_graph)

    def adapt_end(self, index):
        with torch.cuda.stream(self.stream):
            return self.slots.adapt_end(index)

    def get(self, index):
        with torch.cuda.stream(self.stream):
            g = self.slots.get(index)
            self.stream.synchronize()
            return g["w"].cpu(), g["d"].cpu()

    def release(self, index):
        with torch.cuda.stream(self.stream):
            return self.slots.release(index)

    def close(self):
        with torch.cuda.stream(self.stream):
            self.slots.close()
            self.template.close()
            self.stream.synchronize()


def _prepare_job(job, device):
    """Host side of an arrival: the catalogue and its problem (tables, copies)."""
    torch.cuda.set_device(device)
    job._cat = mock.make_catalog(job.spec)
    job._prob = Problem.from_mock(job.spec, job._cat, device=device)
    return job


class BatchedServingLoop:
    """Continuous batching over slotted states (see the module docstring).

    backend_factory(job, n_slots) -> backend with load/run/adapt_end/get/
    release/close, prepare(job) -> job and free_bytes() are injectable so the
    scheduling can be exercised without a GPU.

    While no job waits for a slot of a group, one call runs as many
    trajectories (at most max_batch_traj) as the loaded job closest to an
    event (end of its warm-up or of its run) still needs, so the host's
    bookkeeping is paid once per call; the trajectory latency recorded is
    the call's time divided by its trajectories.

    grid_slots maps a grid size N to the most jobs its group batches (the
    rest wait for a slot): a grid whose single chain already fills the GPU
    gains little from sharing launches and pays for it in trajectory
    latency, so it can be held to one or two slots while small grids batch
    up to max_slots.  grid_priority maps N to its group's CUDA stream
    priority (lower is higher): the group's job loads, refreshes and step
    adaptation go ahead of a large grid's kernels.  The trajectories
    themselves replay from captured graphs on the slotted state's own stream,
    at the default priority."""

    def __init__(self, max_slots=8, max_points=100_000, reserve_bytes=2 << 30, device=0, use_graph=True,
                 keep_state=False, seed=0, backend_factory=None, prepare=None, free_bytes=None, prep_threads=2,
                 max_batch_traj=4, grid_slots=None, grid_priority=None):
        self.max_batch_traj = max(1, int(max_batch_traj))
        self.grid_slots = dict(grid_slots or {})
        self.grid_priority = dict(grid_priority or {})
        self.max_slots = max_slots
        self.max_points = max_points
        self.reserve = reserve_bytes
        self.device = device
        self.keep_state = keep_state
        self.seed = seed
        self.backend_factory = backend_factory or (
            lambda job, n: SlotsBackend(job, n, max_points, seed, device=device, use_graph=use_graph,
                                        priority=self.grid_priority.get(job.spec.N, 0)))
        self.prepare = prepare or (lambda job: _prepare_job(job, device))
        self.free_bytes = free_bytes or (lambda: torch.cuda.mem_get_info(self.device)[0])
        self.prep_threads = prep_threads
        self._cv = threading.Condition()
        self.groups = {}            # key -> dict(backend, ready deque, slots, thread)
        self.max_active_seen = 0
        self.admission_log = []     # (time, job_id, group slots in use after admission)

    def _group_worker(self, g, t0, done):
        be = g["backend"]
        active = {}                 # chain index -> job
        while True:
            with self._cv:
                while not g["ready"] and not active and not g["stop"]:
                    self._cv.wait(timeout=0.05)
                if g["stop"] and not g["ready"] and not active:
                    return
                admit = []
                while g["ready"] and len(active) + len(admit) < g["slots"]:
                    admit.append(g["ready"].popleft())
            for job in admit:
                try:
                    idx = be.load(job)
                except Exception as exc:   # reported per job; the group keeps serving
                    job.error = repr(exc)
                    job.finished = time.perf_counter() - t0
                    done.put(job)
                    continue
                job.admitted = time.perf_counter() - t0
                job._warm = job.adapt_warmup
                job.eps_used = job.eps
                active[idx] = job
                with self._cv:
                    self.admission_log.append((job.admitted, job.job_id, len(active)))
                    self.max_active_seen = max(self.max_active_seen, len(active))
            if not active:
                continue

            def left(j):
                return j._warm if j._warm > 0 else j.n_traj - len(j.traj_latency)
            with self._cv:
                waiting = bool(g["ready"])
            k = 1 if waiting else max(1, min(self.max_batch_traj, min(left(j) for j in active.values())))
            a = time.perf_counter()
            try:
                rows = be.run(k)
            except Exception as exc:
                # the jobs loaded in this group fail with the error; their
                # slots are released so that later arrivals can be served
                for idx in sorted(active, reverse=True):
                    job = active.pop(idx)
                    try:
                        be.release(idx)
                    except Exception:
                        pass
                    job.error = repr(exc)
                    job.finished = time.perf_counter() - t0
                    done.put(job)
                continue
            dt = (time.perf_counter() - a) / k
            finished = []
            for idx in sorted(active):
                job = active[idx]
                for t in range(k):
                    rec = rows[t][idx]
                    if job._warm > 0:
                        job._warm -= 1
                        if job._warm == 0:
                            job.eps_used = be.adapt_end(idx)
                        continue
                    job.traj_latency.append(dt)
                    job.psi.append(float(rec["psi"]))
                    job.accept.append(int(rec["accept"]))
                if len(job.traj_latency) >= job.n_traj:
                    finished.append(idx)
            # release from the highest index down: each release moves the
            # last loaded chain into the freed index
            for idx in sorted(finished, reverse=True):
                job = active.pop(idx)
                if self.keep_state:
                    job.final_w, job.final_d = be.get(idx)
                moved = be.release(idx)
                if moved >= 0:
                    active[idx] = active.pop(moved)
                job.finished = time.perf_counter() - t0
                prob = getattr(job, "_prob", None)
                if prob is not None and hasattr(prob, "close"):
                    prob.close()
                done.put(job)

    def _group_for(self, job, t0, done):
        """The job's group, created (with its slot count from the free
        memory) on first use; None while it does not fit."""
        key = group_key(job)
        g = self.groups.get(key)
        if g is not None:
            return g
        sp = job.spec
        per = slots_footprint_bytes(sp.N, 1, self.max_points, sp.precision)
        room = self.free_bytes() - self.reserve - (16 << 20)
        cap = min(self.max_slots, int(self.grid_slots.get(sp.N, self.max_slots)))
        n = min(cap, int(room // per)) if room > 0 else 0
        if n < 1:
            return None
        g = {"backend": self.backend_factory(job, n), "ready": collections.deque(), "slots": n, "stop": False}
        g["thread"] = threading.Thread(target=self._group_worker, args=(g, t0, done), daemon=True)
        self.groups[key] = g
        g["thread"].start()
        return g

    def run(self, jobs):
        """Serve `jobs` (arrival times in seconds from now); returns stats."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        done = queue.Queue()
        finished = []
        blocked = []                # prepared jobs whose group does not fit yet
        preps = []
        t0 = time.perf_counter()
        i = 0
        pool = concurrent.futures.ThreadPoolExecutor(max_workers=self.prep_threads)
        try:
            while len(finished) < len(jobs):
                now = time.perf_counter() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    j = pending[i]
                    i += 1
                    if j.spec.n_points > self.max_points:
                        j.error = f"catalogue of {j.spec.n_points} points exceeds the slot room {self.max_points}"
                        j.finished = now
                        finished.append(j)
                        continue
                    preps.append(pool.submit(self._prepare_safe, j))
                still = []
                for f in preps:
                    if not f.done():
                        still.append(f)
                        continue
                    j = f.result()
                    if j.error:
                        j.finished = time.perf_counter() - t0
                        finished.append(j)
                    else:
                        blocked.append(j)
                preps = still
                keep = []
                for j in blocked:
                    g = self._group_for(j, t0, done)
                    if g is None:
                        if not self.groups:
                            j.error = "does not fit in device memory"
                            j.finished = time.perf_counter() - t0
                            finished.append(j)
                        else:
                            keep.append(j)
                        continue
                    with self._cv:
                        g["ready"].append(j)
                        self._cv.notify_all()
                blocked = keep
                try:
                    finished.append(done.get(timeout=0.002))
                except queue.Empty:
                    pass
        finally:
            pool.shutdown(wait=True)
            with self._cv:
                for g in self.groups.values():
                    g["stop"] = True
                self._cv.notify_all()
            for g in self.groups.values():
                g["thread"].join()
                g["backend"].close()
        makespan = time.perf_counter() - t0
        return summarize(finished, makespan)

    def _prepare_safe(self, job):
        try:
            return self.prepare(job)
        except Exception as exc:   # reported per job; the loop keeps serving
            job.error = repr(exc)
            return job


def latency_by_grid(jobs):
    """Trajectory and job latency percentiles of the jobs of each grid size."""
    out = {}
    for N in sorted({j.spec.N for j in jobs}):
        js = [j for j in jobs if j.spec.N == N and not j.error]
        lat = np.array([x for j in js for x in j.traj_latency])
        jl = np.array([j.finished - j.arrival for j in js])
        out[str(N)] = {"jobs": len(js),
                       "trajectory_latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                                                 "p99": float(np.percentile(lat, 99) * 1e3) if lat.size else None},
                       "job_latency_s": {"p50": float(np.percentile(jl, 50)) if jl.size else None,
                                         "p99": float(np.percentile(jl, 99)) if jl.size else None}}
    return out


def summarize(jobs, makespan):
    lat = np.array([x for j in jobs for x in j.traj_latency]) if jobs else np.zeros(0)
    job_lat = np.array([j.finished - j.arrival for j in jobs])
    evals = sum(len(j.traj_latency) * j.n_leapfrog for j in jobs)
    evals_all = sum((len(j.traj_latency) + j.adapt_warmup) * j.n_leapfrog for j in jobs if not j.error)
    ess_job = [(j, ess(np.array(j.psi))) for j in jobs if len(j.psi) >= 4]
    ess_sum = sum(e for _, e in ess_job)
    # seconds of a job's residence on the device per effective sample it drew
    per_es = np.array([(j.finished - j.admitted) / e for j, e in ess_job if e > 0])
    acc = np.concatenate([np.array(j.accept) for j in jobs]) if jobs else np.zeros(0)
    return {
        "jobs": len(jobs), "errors": [j.error for j in jobs if j.error],
        "makespan_s": makespan,
        "grad_evals_per_s": evals / makespan if makespan > 0 else None,
        "grad_evals_per_s_incl_warmup": evals_all / makespan if makespan > 0 else None,
        "ess_per_s": ess_sum / makespan if makespan > 0 else None,
        "seconds_per_effective_sample": {"p50": float(np.percentile(per_es, 50)) if per_es.size else None,
                                         "p99": float(np.percentile(per_es, 99)) if per_es.size else None},
        "trajectory_latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                                  "p99": float(np.percentile(lat, 99) * 1e3) if lat.size else None},
        "job_latency_s": {"p50": float(np.percentile(job_lat, 50)) if job_lat.size else None,
                          "p99": float(np.percentile(job_lat, 99)) if job_lat.size else None},
        "accept_rate": float(acc.mean()) if acc.size else None,
        "by_grid": latency_by_grid(jobs),
    }


def poisson_jobs(n_jobs, rate_per_s, seed=7, n_traj=30, grids=(64, 128), n_range=(1e3, 1e5), eps=0.025,
                 adapt_warmup=0, accept_target=0.70):
    """Synthetic arrival stream: Poisson arrivals, grid 64^3 or 128^3 (box
    500 Mpc/h) or 256^3 (box 1000 Mpc/h), catalogue sizes log-uniform in
    n_range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for k in range(n_jobs):
        t += rng.exponential(1.0 / rate_per_s)
        N = int(rng.choice(grids))
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        spec = mock.MockSpec(N=N, L=1000.0 if N == 256 else 500.0, n_points=n, r_max=160.0, mask_deg=10.0,
                             sigma_mu=(0.2, 0.45), sigma_nl=250.0, seed=1000 + k)
        jobs.append(Job(job_id=k, spec=spec, n_traj=n_traj, seed=seed, arrival=t, eps=eps,
                        adapt_warmup=adapt_warmup, accept_target=accept_target))
    return jobs
