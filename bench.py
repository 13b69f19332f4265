#!/usr/bin/env python
"""HAMLET hot-path benchmark: HMC gradient evaluations per second (and ESS/s)
on the paper-scale reconstruction -- 128^3 grid, box 500 Mpc/h, 3e4 points,
FP32 fields with FP64 energies, one chain, trajectories of 20 leapfrog steps.

One step = one HMC trajectory (momentum refresh, 20 gradient evaluations with
fused kick/drift, energy, Metropolis test).  Inputs are synthetic (seeded mock
catalogue with the paper's shapes).  L2 is flushed (a 512 MiB write) before
every timed step; each step is timed with CUDA events on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica chain (no
collective on the data path) and value = all ranks' gradient evaluations /
the slowest rank's time.  --impl reference times the FP64 CPU oracle on the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_02369_gb300 import mock  # noqa: E402

METRIC = "HMC grad evals/s & ESS/s at 128³, 3e4 pts vs plain; served p50/p99 latency"
UNIT = "grad_evals/s"
WORKLOAD = "paper-scale plain HMC: 128^3 grid, L=500 Mpc/h, 3e4 points, 1 chain, 20 leapfrog steps/trajectory"
N_LEAPFROG = 20
EPS = 0.025           # frozen step size: acceptance ~0.70 after burn-in on this workload (sweep 0.01-0.03)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--eps", type=float, default=EPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ess", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true", help="run only the 32-chain batched measurement")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-256", action="store_true", help="skip the 256^3 one-chain measurement")
    ap.add_argument("--no-fft-ref", action="store_true", help="skip the cuFFT reference timing")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving mix (64^3/128^3/256^3, 1e3-1e5 points) and print its JSON")
    ap.add_argument("--serve-jobs", type=int, default=60, help="jobs in the serving mix")
    ap.add_argument("--serve-trajectories", type=int, default=50, help="timed trajectories per served job")
    ap.add_argument("--accept-target", type=float, default=0.70,
                    help="acceptance the batched and served chains' step sizes are tuned to (dual averaging)")
    ap.add_argument("--tune-eps", action="store_true", help="print acceptance for a sweep of eps and exit")
    ap.add_argument("--workload", default="grid128_30000pts", choices=["grid128_30000pts", "grid64_5000pts"],
                    help="plain-chain preset (the headline is the 128^3 one; 64^3 for profiling the small grid)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.path = os.path.join(os.environ.get("HM_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel kind (FP32, one chain)
# --------------------------------------------------------------------------
def algorithmic_bytes(N, n, C=1, rsz=4, fo=1.0):
    """Bytes each kernel kind must move per launch if every array it touches
    is read or written once: R = one real N^3 grid, S = one half spectrum,
    plus the per-point records (32 B), partials and catalogue fields.  fo is
    the fraction of x-planes that carry a CIC corner of some point: the
    gather reads, the scatter writes and the adjoint pencil reads only
    those planes of the three component spectra."""
    R = rsz * N ** 3
    S = 2 * rsz * N * N * (N // 2 + 1)
    return {
        "plane_r2c_field": C * (R + S),
        "pencil_velocity": C * (S + 3 * S),
        "plane_c2r_velocity_gather": C * (fo * 3 * S + 3 * 2 * n * (32 + 8)),
        "memset_bucket_counts": 0,
        "points_bucket_count_standalone": C * n * 24,
        "points_bucket_place": C * n * (72 + 48 + 40),
        "points_likelihood_kick": C * n * (104 + 40 + 24),
        "plane_r2c_scatter_adjoint": C * (fo * 3 * S + 3 * 2 * n * 32),
        "pencil_adjoint": C * (fo * 3 * S + S),
        "plane_c2r_gradient_kick": C * (S + 4 * R + S),
        "trajectory_begin": C * (6 * R + 56 * n),
        "finalize_energy": 0,
        "restore_rejected": 0,
    }


def occupied_plane_fraction(prob, d):
    """Fraction of the x-planes holding a CIC corner of some point at
    distances d (planes ix and ix + 1 of every point's cell)."""
    cell, _ = prob.cells(d, sort=False)
    ix = cell.cpu().numpy().astype(np.int64) // (prob.N * prob.N)
    occ = np.zeros(prob.N, dtype=bool)
    occ[ix] = True
    occ[(ix + 1) % prob.N] = True
    return float(occ.mean())


def model_bytes(N, n, rsz=4):
    """Bytes of one gradient evaluation in the reference traffic model: each
    grid-sized array of the method written once and read once (17 real grids
    R + 4 half spectra C per leapfrog step) plus about 300 B per point."""
    R = rsz * N ** 3
    S = 2 * rsz * N * N * (N // 2 + 1)
    return 17 * R + 4 * S + 300 * n


# kernels launched inside one profiled pair of events
KERNELS_PER_PAIR = {"memset_bucket_counts": 0, "trajectory_begin": 3, "restore_rejected": 2}
# kernels on the side stream: their event interval also covers the time their
# CTAs wait for SM room beside the main stream's kernels, so it is not their
# run time; the dominant kernel is taken from the main stream
SIDE_STREAM = {"points_bucket_place"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(kind):
    """dram bytes per launch of a kernel kind from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except Exception:
        return None
    ent = data.get("kernels", {}).get(kind)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2203_02369_gb300", "csrc", ent.get("source", ""))
    try:
        with open(src, "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()
    except Exception:
        return None
    if h != ent.get("source_sha256"):
        return None
    return ent.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------
def oracle_problem(preset="grid128_30000pts"):
    from oracle import hamlet_oracle as O
    spec = mock.PRESETS[preset]
    cat = mock.make_catalog(spec)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    return O, spec, cat, op


def run_oracle_steps(n_steps, eps, preset="grid128_30000pts"):
    """n_steps oracle leapfrog steps (one gradient evaluation each) from the
    mock start state; returns (seconds, evaluations, seconds of each step)."""
    O, spec, cat, op = oracle_problem(preset)
    w = np.zeros((spec.N,) * 3)
    d = cat["d_init"].copy()
    pw, pd = O.draw_momenta(op, 2, 0, 0)
    psi, gw, gd = O.logpost_grad(op, w, d)
    each = []
    t0 = time.perf_counter()
    for _ in range(n_steps):
        t1 = time.perf_counter()
        pw -= 0.5 * eps * gw
        pd -= 0.5 * eps * gd
        w += eps * pw
        d += eps * op.minv_d * pd
        psi, gw, gd = O.logpost_grad(op, w, d)
        pw -= 0.5 * eps * gw
        pd -= 0.5 * eps * gd
        each.append(time.perf_counter() - t1)
    return time.perf_counter() - t0, n_steps, each


def _oracle_worker(args):
    n_steps, eps = args
    _, _, each = run_oracle_steps(n_steps, eps)
    return each


def run_oracle_all_cores(n_per_core, eps):
    """The oracle as it stands on every host core at once: one process per
    core (spawned, so no process inherits a CUDA context), each running
    n_per_core leapfrog steps of the 128^3 workload on its own copy;
    returns (evaluations/s over the wall time of the timed steps, cores)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(1, eps)] * cores)          # import, problem set-up, page-in
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(n_per_core, eps)] * cores)
        wall = time.perf_counter() - t0
    n = sum(len(r) for r in res)
    return n / wall, cores, n, wall


def cpu_baseline_leg(eps):
    """The oracle timed on the host: all cores (the reported value), and one
    core at 128^3 and 64^3 (median of 5 evaluations each)."""
    val, cores, n, wall = run_oracle_all_cores(2, eps)
    _, _, e128 = run_oracle_steps(5, eps)
    _, _, e64 = run_oracle_steps(5, eps, preset="grid64_5000pts")
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle leapfrog steps (one gradient evaluation each) of this workload, numpy FP64, "
                      f"{cores} processes of one thread each (independent copies), {wall:.1f} s wall",
            "single_core_s_per_eval_median": {"grid128_30000pts": float(np.median(e128)),
                                              "grid64_5000pts": float(np.median(e64))},
            "single_core_grad_evals_per_s_128": 1.0 / float(np.median(e128))}


def replica_aggregate(my_ms, units_per_rank, ws, device="cpu"):
    """Whole-job throughput of independent replicas: the slowest rank's timed
    milliseconds (max over ranks, the only collective of the run) and all
    ranks' units divided by that time."""
    import torch
    t = torch.tensor([float(my_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, ws * units_per_rank / (max_ms / 1e3)


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    # every step: one oracle leapfrog step on each host core at once (after
    # a warm-up step per core for imports, problem set-up and page-in)
    val, cores, n, wall = run_oracle_all_cores(args.steps, args.eps)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": 128, "box": 500.0, "points": 30000,
                       "step": f"one oracle leapfrog step (one gradient evaluation) on each of {cores} host cores"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} oracle leapfrog steps (numpy FP64), {cores} processes of one thread"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_batched(args, eps, L, use_graph):
    """32 chains: 8 catalogues (2,000-30,000 points, each from its own seed),
    4 chains each; even catalogues on 128^3, odd on 64^3 (box 500 Mpc/h).
    One state per grid size; both replay their trajectory graphs at once."""
    import torch
    from paper_2203_02369_gb300.hamlet import Problem, State
    from paper_2203_02369_gb300.ess import ess
    specs = mock.batch_presets()
    cats = [mock.make_catalog(s) for s in specs]
    probs = [Problem.from_mock(s, c) for s, c in zip(specs, cats)]
    states = []
    cid = 0
    for N in (128, 64):
        idx = [i for i, s in enumerate(specs) if s.N == N]
        cp, dinit, ids = [], [], []
        for k, i in enumerate(idx):
            for _ in range(4):
                cp.append(k)
                dinit.append(cats[i]["d_init"])
                ids.append(cid)
                cid += 1
        states.append((N, State([probs[i] for i in idx], dinit, seed=4242, chain_problem=cp, chain_ids=ids)))
    nch = sum(s.C for _, s in states)
    mbytes = sum(4 * model_bytes(specs[i].N, specs[i].n_points) for i in range(len(specs)))  # 4 chains each
    stream = torch.cuda.current_stream()
    # burn-in at a small step (the chains start at w = 0), then each chain's
    # step tuned to the plain chain's acceptance by dual averaging, so that
    # both forms are compared at equal acceptance
    for _, s in states:
        s.run_chain(60, L, 0.4 * eps, use_graph=use_graph, trace=False)
    eps_c = {}
    for N, s in states:
        e, _ = s.adapt_step_size(150, L, eps, target=args.accept_target)
        eps_c[N] = e
    torch.cuda.synchronize()
    K = max(4, args.steps // 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for N, s in states:
        s.run_chain(K, L, eps_c[N], use_graph=use_graph, trace=False)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    evals_per_s = nch * K * L / secs
    # per-kernel times of the 128^3 state alone (events inside its graph)
    s128 = states[0][1]
    s128.profile(True)
    s128.run_chain(1, L, eps_c[128], use_graph=use_graph, trace=False)
    torch.cuda.synchronize()
    s128.profile(True)
    for _ in range(5):
        s128.run_chain(1, L, eps_c[128], use_graph=use_graph, trace=False)
        torch.cuda.synchronize()
        s128.profile_collect()
    prof = s128.profile_read()
    s128.profile(False)
    # ESS/s over a continuing run of all chains
    M = 60
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    traces = [s.run_chain(M, L, eps_c[N], use_graph=use_graph, trace=True) for N, s in states]
    e3.record(stream)
    torch.cuda.synchronize()
    msecs = e2.elapsed_time(e3) / 1e3
    ess_tot = sum(ess(tr[:, c]["psi"]) for tr in traces for c in range(tr.shape[1]))
    acc = float(np.mean(np.concatenate([tr["accept"].ravel() for tr in traces])))
    n128 = states[0][1].C
    st128 = states[0][1]
    fo = float(np.mean([occupied_plane_fraction(st128.problems[st128.chain_problem[c]], st128.get(c)["d"]) for c in range(n128)]))
    ab = algorithmic_bytes(128, 30000, C=n128, fo=fo)
    total_k = sum(v[0] for v in prof.values())
    dname, (dms, dl) = max(prof.items(), key=lambda kv: kv[1][0])
    peaks, src = measured_peaks()
    kern = {k: {"us_per_launch": 1e3 * v[0] / v[1] if v[1] else None, "share": v[0] / total_k if total_k else None,
                "gbs_algorithmic": (ab[k] / (v[0] / v[1] / 1e3) / 1e9) if v[1] and v[0] > 0 and ab.get(k) else None}
            for k, v in prof.items()}
    # points per chain differ: the 128^3 roofline uses the bytes of the grid terms only
    ach = ab[dname] / (dms / dl / 1e3) / 1e9 if dl else None
    out = {"chains": nch, "chains_128": n128, "chains_64": nch - n128, "trajectories_timed": K,
           "eps_tuning": {"method": "60 burn-in trajectories at 0.4 eps, then dual averaging over 150 trajectories per chain",
                          "target_accept": args.accept_target,
                          "eps_128_median": float(np.median(eps_c[128])), "eps_64_median": float(np.median(eps_c[64]))},
           "grad_evals_per_s": evals_per_s, "ms_per_trajectory_all_chains": 1e3 * secs / K,
           "ess_psi_sum": ess_tot, "ess_per_s": ess_tot / msecs, "ess_trajectories": M, "accept_rate": acc,
           "kernels_128": kern,
           "model_roofline": {"bytes_per_eval_all_chains": mbytes,
                              "achieved_gbs": mbytes * K * L / secs / 1e9,
                              "frac": mbytes * K * L / secs / 1e9 / peaks.get("hbm_gbs"),
                              "note": "reference traffic model (17R + 4C + 300 B/point per evaluation, each chain "
                                      "at its own grid and catalogue size) x evaluations/s / measured HBM peak"},
           "roofline_128": {"kernel": dname, "achieved": ach, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                            "frac": ach / peaks.get("hbm_gbs") if ach else None,
                            "occupied_plane_fraction": fo,
                            "note": "16 chains of 128^3 in one launch; algorithmic bytes of the grid terms "
                                    "(point terms at 3e4 points per chain, an upper bound for these catalogues)"}}
    for _, s in states:
        s.close()
    for p in probs:
        p.close()
    return out


def run_grid256(L, eps=0.01, K=5):
    """One chain at 256^3 (box 1000 Mpc/h, 1e5 points, r^2 to 160 Mpc/h, the
    serving mix's large grid; its working set is far beyond L2): ms per
    gradient evaluation over K trajectories (CUDA events), and per kernel
    kind the mean launch time (profiled pass) and its algorithmic GB/s."""
    import torch
    from paper_2203_02369_gb300.hamlet import Problem, State
    spec = mock.MockSpec(N=256, L=1000.0, n_points=100000, r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=1007)
    cat = mock.make_catalog(spec)
    prob = Problem.from_mock(spec, cat)
    st = State(prob, [cat["d_init"]], seed=5)
    st.run_chain(3, L, eps, use_graph=True, trace=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tr = st.run_chain(K, L, eps, use_graph=True, trace=True)
    b.record()
    torch.cuda.synchronize()
    ms_eval = a.elapsed_time(b) / (K * L)
    st.profile(True)
    st.run_chain(1, L, eps, use_graph=True, trace=False)
    st.profile(True)
    for _ in range(3):
        st.run_chain(1, L, eps, use_graph=True, trace=False)
        st.profile_collect()
    prof = st.profile_read()
    st.profile(False)
    fo = occupied_plane_fraction(prob, st.get(0)["d"])
    ab = algorithmic_bytes(256, spec.n_points, fo=fo)
    peak = measured_peaks()[0].get("hbm_gbs", 6800.0)
    kern = {}
    for k, (ms, n) in prof.items():
        if not n:
            continue
        us = 1e3 * ms / n
        gbs = ab.get(k, 0) / (us * 1e-6) / 1e9 if ab.get(k) else None
        kern[k] = {"us_per_launch": us, "gbs_algorithmic": gbs, "frac": gbs / peak if gbs else None}
    st.close()
    prob.close()
    return {"workload": "256^3 grid, L=1000 Mpc/h, 1e5 points (r^2 to 160 Mpc/h), 1 chain, 20 leapfrog steps, eps 0.01",
            "ms_per_eval": ms_eval, "grad_evals_per_s": 1e3 / ms_eval, "accept_rate": float(tr["accept"].mean()),
            "occupied_plane_fraction": fo, "kernels": kern,
            "note": "plane kinds are two kernels at 256^3 (z pass over row slabs, y pass over column tiles; the "
                    "gradient epilogue adds the y pass of the drifted field); algorithmic bytes as at 128^3, so "
                    "the extra read and write of the spectra by the two-pass form count as overhead"}


def run_fft_reference(prob, dev, reps=30):
    """The library's 3D r2c/c2r transforms (plane pass + x pencil) against
    cuFFT (torch.fft, unnormalised both ways) on the same 128^3 FP32 grids,
    one and three at a time: each call timed alone with CUDA events, median
    of reps.  A reference only; the hot path fuses its transforms with the
    velocity weights, the CIC work and the leapfrog epilogue."""
    import torch
    N = prob.N
    stream = torch.cuda.current_stream()

    def med(fn):
        ts = []
        for _ in range(reps + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        return float(np.median(ts[3:]))

    out = {}
    dims = (-3, -2, -1)
    for count in (1, 3):
        g = torch.Generator(device=dev).manual_seed(5 + count)
        x = torch.randn((count, N, N, N), device=dev, dtype=torch.float32, generator=g)
        X = prob.fft_r2c(x)
        Xc = torch.fft.rfftn(x, dim=dims)
        y = prob.fft_c2r(X)
        yc = torch.fft.irfftn(Xc, s=(N, N, N), dim=dims, norm="forward")
        out[f"count_{count}"] = {
            "ours_r2c_us": med(lambda: prob.fft_r2c(x)),
            "cufft_r2c_us": med(lambda: torch.fft.rfftn(x, dim=dims)),
            "ours_c2r_us": med(lambda: prob.fft_c2r(X)),
            "cufft_c2r_us": med(lambda: torch.fft.irfftn(Xc, s=(N, N, N), dim=dims, norm="forward")),
            "rel_diff_r2c": float(torch.linalg.vector_norm(X - Xc) / torch.linalg.vector_norm(Xc)),
            "rel_diff_c2r": float(torch.linalg.vector_norm(y - yc) / torch.linalg.vector_norm(yc)),
        }
    out["note"] = ("3D FFT of 128^3 FP32 grids, each call timed alone (CUDA events, median); ours = z-y plane "
                   "pass + x pencil kernels, cuFFT via torch.fft; data L2-resident in both")
    return out


def run_batched_same(prob, d_init, eps, L, use_graph, n_chains=16, K=20, M=60):
    """n_chains chains of the plain workload itself (same catalogue, same
    step, own Philox chain words) in one state: the batched form against the
    plain single chain at equal acceptance and accuracy by construction."""
    import torch
    from paper_2203_02369_gb300.hamlet import State
    from paper_2203_02369_gb300.ess import ess
    st = State(prob, [d_init] * n_chains, seed=99, chain_ids=list(range(100, 100 + n_chains)))
    st.run_chain(60, L, eps, use_graph=use_graph, trace=False)     # burn-in, as the plain chain's warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.run_chain(K, L, eps, use_graph=use_graph, trace=False)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    tr = st.run_chain(M, L, eps, use_graph=use_graph, trace=True)
    e1.record(stream)
    torch.cuda.synchronize()
    msecs = e0.elapsed_time(e1) / 1e3
    ess_tot = sum(ess(tr[:, c]["psi"]) for c in range(n_chains))
    st.close()
    return {"chains": n_chains, "eps": eps, "trajectories_timed": K,
            "grad_evals_per_s": n_chains * K * L / secs, "ms_per_trajectory_all_chains": 1e3 * secs / K,
            "ess_psi_sum": ess_tot, "ess_per_s": ess_tot / msecs, "ess_trajectories": M,
            "accept_rate": float(tr["accept"].mean()),
            "workload": f"{n_chains} chains of the plain workload (same catalogue and step) in one state, "
                        "one captured graph per trajectory; ESS as the plain chain's (Geyer on Psi) after a "
                        "60-trajectory burn-in"}


def run_serving(eps, L, target, grids=(64, 128, 256), n_range=(1e3, 1e5), n_jobs=60, n_timed=50, grid_slots=None,
                grid_priority=None):
    """Poisson stream of reconstruction jobs (64^3 / 128^3 at 500 Mpc/h,
    256^3 at 1000 Mpc/h), all arriving within a fraction of a second so that
    the GPU is saturated.  Served by continuous batching (one slotted state
    per grid, up to 8 jobs advancing in the same launches; grid_slots caps a
    grid's batch) and, for reference, the same jobs one at a time.  Each job
    draws the same chain in both runs (same seed and chain word per job,
    per-job step tuned by the same dual averaging), so acceptance and
    accuracy are equal by construction."""
    from paper_2203_02369_gb300.serve import BatchedServingLoop, ServingLoop, poisson_jobs
    n_warm, seed = 20, 7
    rate = 200.0   # arrivals per second: above both loops' service rates, so both run saturated

    def jobs():
        return poisson_jobs(n_jobs, rate_per_s=rate, seed=seed, n_traj=n_timed, grids=grids, n_range=n_range, eps=eps,
                            adapt_warmup=n_warm, accept_target=target)
    served = BatchedServingLoop(max_slots=8, max_points=int(n_range[1]), seed=seed,
                                grid_slots=grid_slots, grid_priority=grid_priority).run(jobs())
    plain = ServingLoop(max_slots=1).run(jobs())
    served["plain_one_at_a_time"] = {k: plain[k] for k in ("makespan_s", "grad_evals_per_s", "ess_per_s",
                                                           "trajectory_latency_ms", "job_latency_s",
                                                           "grad_evals_per_s_incl_warmup",
                                                           "seconds_per_effective_sample", "accept_rate",
                                                           "errors", "by_grid")}
    served["speedup_vs_plain_evals"] = served["grad_evals_per_s"] / plain["grad_evals_per_s"]
    if served.get("ess_per_s") and plain.get("ess_per_s"):
        served["speedup_vs_plain_ess"] = served["ess_per_s"] / plain["ess_per_s"]
    gs = "/".join(str(x) for x in grids)
    pol = ", ".join([f"{k}^3 at most {v}" for k, v in sorted((grid_slots or {}).items())] +
                    [f"{k}^3 stream priority {v}" for k, v in sorted((grid_priority or {}).items())])
    served["workload"] = (f"{n_jobs} jobs, Poisson arrivals at {rate:.0f}/s, grids {gs}, {n_range[0]:.0e}-{n_range[1]:.0e} points; "
                          f"each job tunes its step by dual averaging ({n_warm} trajectories, target acceptance "
                          f"{target}) and then runs {n_timed} trajectories x {L} steps (the timed ones); served = "
                          "continuous batching over slotted states (up to 8 jobs per grid in one launch"
                          + (f"; {pol}" if pol else "") + "), plain = the same jobs one at a time, each in its own "
                          "one-chain state")
    return served


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2203_02369_gb300.hamlet import Problem, State
    from paper_2203_02369_gb300.ess import ess

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    spec = mock.PRESETS[args.workload]
    cat = mock.make_catalog(spec)
    prob = Problem.from_mock(spec, cat, device=dev)
    state = State(prob, [cat["d_init"]], seed=1000 + rank, chain_ids=[rank])
    L = N_LEAPFROG
    use_graph = not args.no_graph

    if args.tune_eps:
        # burn in at a small step, then measure the acceptance of each step size
        # from the same burnt-in state (position copied into a fresh chain)
        burn = State(prob, [cat["d_init"]], seed=7)
        burn.run_chain(150, L, 0.01, use_graph=use_graph, trace=False)
        g = burn.get(0)
        for e in (0.01, 0.0125, 0.015, 0.0175, 0.02, 0.025, 0.03):
            s2 = State(prob, [cat["d_init"]], seed=8)
            s2.set(0, w=g["w"], d=g["d"])
            s2.refresh()
            tr = s2.run_chain(60, L, e, use_graph=use_graph)
            print(json.dumps({"eps": e, "accept": float(tr["accept"].mean()),
                              "dH_median": float(np.median(np.abs(tr["H_new"] - tr["H_old"]))),
                              "ess_psi": ess(tr[:, 0]["psi"])}), flush=True)
            s2.close()
        return

    if args.batched_only:
        print(json.dumps(run_batched(args, args.eps, L, use_graph)), flush=True)
        return

    if args.serve_only:
        print(json.dumps(run_serving(args.eps, L, args.accept_target, n_jobs=args.serve_jobs,
                                     n_timed=args.serve_trajectories, grid_slots={256: 2},
                                     grid_priority={64: -2, 128: -1})), flush=True)
        return

    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also burns the chain in)
    state.run_chain(args.warmup, L, args.eps, use_graph=use_graph, trace=False)
    barrier()

    # ---- timed region: K trajectories, L2 flushed before each, one event pair per step ----
    clocks = Clocks(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks.start()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        state.run_chain(1, L, args.eps, use_graph=use_graph, trace=False)
        ends[k].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    my_ms = float(np.sum(step_ms))

    # ---- profiled pass: the same K trajectories with an event pair around
    # every kernel launch (on the stream it runs on); gives the per-kernel
    # durations of the roofline and the launch count ----
    state.profile(True)
    state.run_chain(1, L, args.eps, use_graph=use_graph, trace=False)   # capture the profiled graph
    barrier()
    state.profile(True)                                                  # reset the totals
    s_p = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_p = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks_p = Clocks(dev)
    clocks_p.start()
    for k in range(args.steps):
        flush.zero_()
        s_p[k].record(stream)
        state.run_chain(1, L, args.eps, use_graph=use_graph, trace=False)
        e_p[k].record(stream)
        torch.cuda.synchronize()
        state.profile_collect()
    barrier()
    clk_p = clocks_p.stop()
    ms_prof = float(np.mean([s.elapsed_time(e) for s, e in zip(s_p, e_p)]))
    prof = state.profile_read()
    state.profile(False)

    # max over ranks of the timed device time
    max_ms, value = replica_aggregate(my_ms, args.steps * L, ws, dev)

    # ESS/s on the Psi trace of a continuing chain (no flush between trajectories)
    ess_info = None
    if not args.no_ess:
        # one trajectory at a time, each timed on the device; after each, 64
        # fixed field entries and 64 fixed distances are read (outside the
        # timed intervals) for per-coordinate ESS
        M = 2000   # the 128^3 configuration's 2,000 trajectories
        rng = np.random.default_rng(123)
        n_field = spec.N ** 3
        wi = torch.tensor(rng.choice(n_field, 64, replace=False), device=dev)
        di = torch.tensor(rng.choice(spec.n_points, 64, replace=False), device=dev)
        e_s = [torch.cuda.Event(enable_timing=True) for _ in range(M)]
        e_e = [torch.cuda.Event(enable_timing=True) for _ in range(M)]
        recs, ws_, ds_ = [], [], []
        for k in range(M):
            e_s[k].record(stream)
            tr = state.run_chain(1, L, args.eps, use_graph=use_graph, trace=True)
            e_e[k].record(stream)
            recs.append(tr[0, 0])
            g = state.get(0)
            ws_.append(g["w"].reshape(-1)[wi].double())
            ds_.append(g["d"][di])
        torch.cuda.synchronize()
        secs = sum(a.elapsed_time(b) for a, b in zip(e_s, e_e)) / 1e3
        psi = np.array([r["psi"] for r in recs])
        e_psi = ess(psi)
        from paper_2203_02369_gb300.ess import ess_columns
        ew = ess_columns(torch.stack(ws_).cpu().numpy())
        ed = ess_columns(torch.stack(ds_).cpu().numpy())
        ess_info = {"trajectories": M, "ess_psi": e_psi, "ess_per_s": e_psi / secs,
                    "ess_w64": {"min": float(ew.min()), "median": float(np.median(ew))},
                    "ess_d64": {"min": float(ed.min()), "median": float(np.median(ed))},
                    "ess_per_s_min_coordinate": float(min(ew.min(), ed.min())) / secs,
                    "accept_rate": float(np.mean([r["accept"] for r in recs])), "seconds": secs,
                    "note": "Geyer initial-monotone ESS after the warm-up and timed trajectories: of the Psi trace "
                            "(the headline, also used for the batched and served forms) and of 64 fixed field "
                            f"entries and 64 fixed distances (min, median) of the {n_field} and {spec.n_points}; "
                            "seconds = sum of the trajectories' device times"}

    # end to end through the public API: H2D of the chain state from pinned
    # memory, set + refresh, one trajectory, D2H of the new state and trace
    e2e = None
    if not args.no_e2e:
        g = state.get(0)
        w_h = g["w"].cpu().pin_memory()
        d_h = g["d"].cpu().pin_memory()
        w_o = torch.empty_like(w_h).pin_memory()
        d_o = torch.empty_like(d_h).pin_memory()
        ne = min(args.steps, 30)
        s_e = [torch.cuda.Event(enable_timing=True) for _ in range(ne)]
        e_e = [torch.cuda.Event(enable_timing=True) for _ in range(ne)]
        for k in range(ne):
            torch.cuda.synchronize()
            flush.zero_()
            s_e[k].record(stream)
            state.set(0, w=w_h, d=d_h)            # pinned host -> the state, one copy each
            state.refresh()
            trk = state.run_chain(1, L, args.eps, use_graph=use_graph, trace=True)
            state.get(0, out={"w": w_o, "d": d_o})   # the state -> pinned host
            e_e[k].record(stream)
        torch.cuda.synchronize()
        ms_e = float(np.mean([s.elapsed_time(e) for s, e in zip(s_e, e_e)]))
        bi = w_h.numel() * w_h.element_size() + d_h.numel() * 8
        bo = bi + 48
        e2e = {"value": ws * L / (ms_e / 1e3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": ms_e,
               "note": "per step: hm_state_set from pinned host (w, d), hm_state_refresh (one extra gradient "
                       "evaluation, not counted), one trajectory, hm_state_get of (w, d) into pinned host and the "
                       "trace record"}

    # roofline of the dominant kernel (live CUDA-event times from the profiled pass)
    N, n = spec.N, spec.n_points
    fo = occupied_plane_fraction(prob, state.get(0)["d"])
    ab = algorithmic_bytes(N, n, fo=fo)
    total_k = sum(v[0] for v in prof.values())
    dom = max(((k, v) for k, v in prof.items() if k not in SIDE_STREAM), key=lambda kv: kv[1][0])
    dname, (dms, dl) = dom
    peaks, src = measured_peaks()
    avg_s = dms / max(dl, 1) / 1e3
    achieved = ab[dname] / avg_s / 1e9 if avg_s > 0 else None
    peak = peaks.get("hbm_gbs", 6800.0)
    kernels = {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / total_k if total_k else None,
                   "us_per_launch": 1e3 * v[0] / v[1] if v[1] else None,
                   "gbs_algorithmic": (ab[k] / (v[0] / v[1] / 1e3) / 1e9) if v[1] and v[0] > 0 and ab[k] else None}
               for k, v in prof.items()}
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": ncu_traffic(dname),
                "algorithmic_bytes_per_launch": ab[dname], "peak_source": f"{src} hbm_gbs (copy bandwidth)",
                "occupied_plane_fraction": fo,
                "timing": "CUDA events around each launch of the kernel on its stream, averaged over the "
                          "profiled pass of the same K trajectories (L2 flushed before each); dominant = "
                          "largest total among the main-stream kernels",
                "clocks_profiled_pass": clk_p}

    mb = model_bytes(N, n)
    model_roof = {"bytes_per_eval": mb, "achieved_gbs": mb * value / 1e9, "frac": mb * value / 1e9 / peak,
                  "note": "reference traffic model (17R + 4C + 300 B/point per evaluation) x evaluations/s / "
                          "measured HBM peak; the fused kernels move fewer bytes than the model"}

    fft_ref = None
    if not args.no_fft_ref:
        fft_ref = run_fft_reference(prob, dev)

    # CPU baseline: the oracle on a bounded sample, rank 0, N = 1 only
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args.eps)

    batched = None
    if not args.no_batched:
        plain_evals = args.steps * L / (my_ms / 1e3)
        batched = run_batched(args, args.eps, L, use_graph)
        batched["speedup_vs_plain_evals"] = batched["grad_evals_per_s"] / plain_evals
        if ess_info:
            batched["speedup_vs_plain_ess"] = batched["ess_per_s"] / ess_info["ess_per_s"]
        same = run_batched_same(prob, cat["d_init"], args.eps, L, use_graph)
        same["speedup_vs_plain_evals"] = same["grad_evals_per_s"] / plain_evals
        if ess_info:
            same["speedup_vs_plain_ess"] = same["ess_per_s"] / ess_info["ess_per_s"]
            same["plain_accept_rate"] = ess_info["accept_rate"]
        batched["same_workload"] = same

    grid256 = None
    if not args.no_256 and ws == 1:
        grid256 = run_grid256(L)

    serving = None
    if not args.no_serve and ws == 1:
        # the paper-scale serving mix; 256^3 chains fill the GPU alone, so their
        # group batches at most two, and the smaller grids' groups run on
        # higher-priority streams
        serving = run_serving(args.eps, L, args.accept_target, n_jobs=args.serve_jobs, n_timed=args.serve_trajectories,
                              grid_slots={256: 2}, grid_priority={64: -2, 128: -1})
        serving["grid_128_only"] = run_serving(args.eps, L, args.accept_target, grids=(128,), n_range=(3e3, 3e4),
                                               n_jobs=48, n_timed=12)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.workload == "grid128_30000pts" else
                           f"plain HMC: {N}^3 grid, L={spec.L:g} Mpc/h, {n} points, 1 chain, {L} leapfrog steps/trajectory",
                           "grid": N, "box": spec.L, "points": n,
                           "leapfrog_steps": L, "eps": args.eps, "chains_per_gpu": 1,
                           "parallelism": f"replicas{ws}" if ws > 1 else "single",
                           "l2": "flushed (512 MiB write) before every timed step",
                           "graph": use_graph, "energy_dtype": "f64",
                           "ms_per_step_profiled_pass": ms_prof},
                "gpu_launches": int(sum(v[1] * KERNELS_PER_PAIR.get(k, 1) for k, v in prof.items())),
                "clocks": clk, "roofline": roofline, "model_roofline": model_roof, "kernels": kernels,
                "ess": ess_info,
                "e2e": e2e, "cpu_baseline": cpu, "batched": batched, "grid_256": grid256, "serving": serving,
                "fft_reference": fft_ref,
                "wall_s_timed": t_wall}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
