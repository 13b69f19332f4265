"""Continuous-batching serving loop for HAMLET reconstruction jobs.

Jobs (a catalogue on a grid, a number of HMC trajectories) arrive over time.
A job is admitted as soon as a slot is free and its device-memory footprint
fits the free memory minus a reserve; its chain state then stays resident
on the device until it finishes.  Each slot is a worker thread with its own
CUDA stream: the library's calls release the GIL, so the admitted jobs'
trajectory graphs run concurrently on the GPU while the host admits new
arrivals.  Reported: latency percentiles per trajectory and per job,
aggregate gradient evaluations/s and effective samples/s.
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import mock
from .ess import ess
from .hamlet import Problem, State


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


def summarize(jobs, makespan):
    lat = np.array([x for j in jobs for x in j.traj_latency]) if jobs else np.zeros(0)
    job_lat = np.array([j.finished - j.arrival for j in jobs])
    evals = sum(len(j.traj_latency) * j.n_leapfrog for j in jobs)
    ess_sum = sum(ess(np.array(j.psi)) for j in jobs if len(j.psi) >= 4)
    acc = np.concatenate([np.array(j.accept) for j in jobs]) if jobs else np.zeros(0)
    return {
        "jobs": len(jobs), "errors": [j.error for j in jobs if j.error],
        "makespan_s": makespan,
        "grad_evals_per_s": evals / makespan if makespan > 0 else None,
        "ess_per_s": ess_sum / makespan if makespan > 0 else None,
        "trajectory_latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                                  "p99": float(np.percentile(lat, 99) * 1e3) if lat.size else None},
        "job_latency_s": {"p50": float(np.percentile(job_lat, 50)) if job_lat.size else None,
                          "p99": float(np.percentile(job_lat, 99)) if job_lat.size else None},
        "accept_rate": float(acc.mean()) if acc.size else None,
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
