"""The autograd wrapper: its backward pass against central finite differences
(h = 1e-3) along 64 random Fourier-mode directions of the field and on 64
distances, and against the oracle's gradient, on the 64^3 / 5,000-point
configuration (FP64 path so that the differences are not rounding noise).

On the FP32 path a step of 1e-3 is below the rounding of Psi (|w|^2/2 is
~1.3e5 there, Psi carries ~1e-9 relative error), so the FP32 check uses that
Psi is exactly quadratic in w at fixed distances (u is linear in w, the
likelihood Gaussian in u): the central difference then equals the
directional derivative for any step, and h = 1 resolves it."""
import numpy as np
import pytest
import torch

from _parity import check, check_scalar
from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300.hamlet import Problem
    spec = mock.MockSpec(N=64, L=500.0, n_points=5000, r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=1, precision="fp64")
    cat = mock.make_catalog(spec)
    p = Problem.from_mock(spec, cat)
    return spec, cat, p


def test_backward_matches_central_differences(case):
    from paper_2203_02369_gb300.autograd import logpost
    spec, cat, p = case
    N, L = spec.N, spec.L
    rng = np.random.default_rng(3)
    w0 = torch.tensor(mock.white_field(N, 11), device="cuda", requires_grad=True)
    d0 = torch.tensor(cat["d_init"], device="cuda", requires_grad=True)
    psi = logpost(p, w0, d0)
    psi.backward()
    gw, gd = w0.grad.detach(), d0.grad.detach()
    h = 1e-3
    x = np.arange(N) * (L / N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    kf = 2 * np.pi / L
    worst = 0.0
    for _ in range(64):
        n = rng.integers(-N // 2 + 1, N // 2, 3)
        ph = rng.uniform(0, 2 * np.pi)
        e = np.cos(kf * (n[0] * X + n[1] * Y + n[2] * Z) + ph)
        e /= np.linalg.norm(e)
        et = torch.tensor(e, device="cuda")
        with torch.no_grad():
            fp = logpost(p, w0 + h * et, d0).item()
            fm = logpost(p, w0 - h * et, d0).item()
        fd = (fp - fm) / (2 * h)
        an = float(torch.sum(gw * et))
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    assert worst < 1e-6
    # distances away from cell faces (CIC is piecewise linear in d)
    rhat = cat["rhat"]
    t = (L / 2 + cat["d_init"][:, None] * rhat) / (L / N)
    fr = t - np.floor(t)
    margin = 2 * h / (L / N) + 1e-6
    ok = np.nonzero(np.all((fr > margin) & (fr < 1 - margin), axis=1))[0]
    idx = rng.choice(ok, 64, replace=False)
    worst = 0.0
    for i in idx:
        dp = d0.detach().clone()
        dm = d0.detach().clone()
        dp[i] += h
        dm[i] -= h
        with torch.no_grad():
            fd = (logpost(p, w0, dp).item() - logpost(p, w0, dm).item()) / (2 * h)
        worst = max(worst, abs(fd - gd[i].item()) / max(1.0, abs(gd[i].item())))
    assert worst < 1e-5


def test_backward_matches_oracle_gradient(case):
    from paper_2203_02369_gb300.autograd import logpost
    spec, cat, p = case
    w = mock.white_field(spec.N, 12)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    dt = torch.tensor(cat["d_init"], device="cuda", requires_grad=True)
    psi = logpost(p, wt, dt)
    (2.5 * psi).backward()
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    rpsi, rgw, rgd = O.logpost_grad(op, w, cat["d_init"])
    check_scalar("autograd psi", psi.item(), rpsi, 1e-12)
    check("autograd grad_w", wt.grad, 2.5 * rgw, 1e-12)
    check("autograd grad_d", dt.grad, 2.5 * rgd, 1e-12)


def test_backward_fp32_field_directions_central_differences():
    """The 64^3 / 5,000-point configuration on its FP32 path: the backward
    pass along 64 random Fourier-mode directions against central differences
    of the FP32 Psi with h = 1 (exact for a quadratic)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300.autograd import logpost
    from paper_2203_02369_gb300.hamlet import Problem
    spec = mock.MockSpec(N=64, L=500.0, n_points=5000, r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=1, precision="fp32")
    cat = mock.make_catalog(spec)
    p = Problem.from_mock(spec, cat)
    N, L = spec.N, spec.L
    rng = np.random.default_rng(4)
    w0 = torch.tensor(mock.white_field(N, 13), dtype=torch.float32, device="cuda", requires_grad=True)
    d0 = torch.tensor(cat["d_init"], device="cuda")
    psi = logpost(p, w0, d0)
    psi.backward()
    gw = w0.grad.detach().double()
    h = 1.0
    x = np.arange(N) * (L / N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    kf = 2 * np.pi / L
    worst = 0.0
    for _ in range(64):
        n = rng.integers(-N // 2 + 1, N // 2, 3)
        e = np.cos(kf * (n[0] * X + n[1] * Y + n[2] * Z) + rng.uniform(0, 2 * np.pi))
        e /= np.linalg.norm(e)
        et = torch.tensor(e, dtype=torch.float32, device="cuda")
        with torch.no_grad():
            fp = logpost(p, w0 + h * et, d0).item()
            fm = logpost(p, w0 - h * et, d0).item()
        fd = (fp - fm) / (2 * h)
        an = float(torch.sum(gw * et.double()))
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    assert worst < 1e-3
