"""The no-allocation gradient entry point against the ordinary one.

hm_logpost_grad_noalloc exists for callers that cannot let the library
allocate device memory (code inside another framework's memory pool, which
accounts for every device byte itself; hosts that budget device memory up
front and allow no allocation once they run); it takes its scratch from one
static device array.  This file is collected last on
purpose, so that a run stopping at its first failure has already run every
other test.  It must pass alone in a fresh process and after the others.
"""
import numpy as np
import pytest
import torch

from paper_2203_02369_gb300 import mock
from paper_2203_02369_gb300._lib import HamletError

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import hamlet
    return hamlet


@pytest.mark.parametrize("N,L,n,prec,seed", [(16, 200.0, 500, "fp64", 0), (32, 300.0, 3001, "fp32", 5)])
def test_noalloc_matches_logpost_grad_twice(H, N, L, n, prec, seed):
    spec = mock.MockSpec(N=N, L=L, n_points=n, r_max=0.32 * L, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=seed, precision=prec)
    cat = mock.make_catalog(spec)
    p = H.Problem.from_mock(spec, cat)
    dt = torch.float32 if prec == "fp32" else torch.float64
    for call in range(2):   # two calls in a row: the shared scratch must not leak state
        w = torch.tensor(mock.white_field(N, seed + 10 * call), dtype=dt, device="cuda")
        d = torch.tensor(cat["d_init"] * (1.0 + 0.01 * call), device="cuda")
        psi_a, gw_a, gd_a = p.logpost_grad(w, d)
        psi_b, gw_b, gd_b = p.logpost_grad_noalloc(w, d)
        torch.cuda.synchronize()
        tol = TOL[prec]
        assert abs(psi_b.item() - psi_a.item()) <= tol * abs(psi_a.item())
        assert rel(gw_b.cpu().numpy(), gw_a.cpu().numpy()) < tol
        assert rel(gd_b.cpu().numpy(), gd_a.cpu().numpy()) < tol


def test_noalloc_rejects_problems_beyond_the_static_scratch(H):
    spec = mock.PRESETS["grid64_5000pts"]
    cat = mock.make_catalog(spec)
    p = H.Problem.from_mock(spec, cat)
    w = torch.zeros((64,) * 3, dtype=torch.float32, device="cuda")
    d = torch.tensor(cat["d_init"], device="cuda")
    with pytest.raises(HamletError, match="too large for the no-allocation path"):
        p.logpost_grad_noalloc(w, d)
