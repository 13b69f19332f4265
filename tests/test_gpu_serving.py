"""Serving on the GPU: a job gives the same result alone and in a mix of
concurrently running jobs (FP64 path: the only difference allowed is the
order of the atomic scatter additions)."""
import numpy as np
import pytest
import torch

from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import serve
    return serve


def _job(S, k, N, n, prec, arrival=0.0, n_traj=4):
    spec = mock.MockSpec(N=N, L=300.0 if N == 32 else 500.0, n_points=n, r_max=96.0 if N == 32 else 160.0,
                         mask_deg=10.0, sigma_mu=(0.2, 0.45), sigma_nl=250.0, seed=500 + k, precision=prec)
    return S.Job(job_id=k, spec=spec, n_traj=n_traj, n_leapfrog=10, eps=0.01, seed=11, arrival=arrival)


def test_job_same_alone_and_in_the_mix(S):
    alone = _job(S, 0, 32, 2000, "fp64")
    S.ServingLoop(max_slots=1, keep_state=True).run([alone])
    mix = [_job(S, 0, 32, 2000, "fp64")] + [_job(S, k, 64, 4000, "fp32", arrival=0.0) for k in (1, 2, 3)]
    loop = S.ServingLoop(max_slots=4, keep_state=True)
    stats = loop.run(mix)
    assert not stats["errors"], stats["errors"]
    assert loop.max_active_seen >= 2
    x = mix[0]
    assert x.accept == alone.accept
    assert np.allclose(x.psi, alone.psi, rtol=1e-12, atol=0)
    w1, w0 = x.final_w.numpy(), alone.final_w.numpy()
    assert np.linalg.norm(w1 - w0) / np.linalg.norm(w0) < 1e-12
    d1, d0 = x.final_d.numpy(), alone.final_d.numpy()
    assert np.linalg.norm(d1 - d0) / np.linalg.norm(d0) < 1e-12


def test_served_stats_are_reported(S):
    jobs = S.poisson_jobs(6, rate_per_s=50.0, seed=5, n_traj=5, grids=(64,), n_range=(1e3, 5e3))
    stats = S.ServingLoop(max_slots=3).run(jobs)
    assert stats["jobs"] == 6 and not stats["errors"]
    assert stats["trajectory_latency_ms"]["p99"] >= stats["trajectory_latency_ms"]["p50"] > 0
    assert stats["grad_evals_per_s"] > 0
