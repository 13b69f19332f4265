"""On-device chain analytics vs the oracle, through the C ABI: the GPU chain
and the oracle chain start from the same seeded state and run the same
trajectories (their per-trajectory parity is tested in test_gpu_parity.py);
the analytics of the GPU chain are compared with the oracle's analytics of
the oracle chain's states."""
import numpy as np
import pytest
import torch

from _parity import check
from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu

RADII = [12.3, 41.7, 77.9, 130.1]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import hamlet
    return hamlet


def _case(H, N, L, n, prec, seed):
    spec = mock.MockSpec(N=N, L=L, n_points=n, r_max=0.32 * L, mask_deg=0.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=seed, precision=prec)
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(N, L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    return cat, gp, op


def _oracle_states(op, d0, n_traj, eps, n_steps):
    """The oracle chain's states after each trajectory (seed 77, chain 0)."""
    N = op.N
    w, d = np.zeros((N, N, N)), d0.copy()
    psi_grad = O.logpost_grad(op, w, d)
    states = []
    for t in range(n_traj):
        w, d, psi_grad, _ = O.hmc_trajectory(op, w, d, psi_grad, 77, t, 0, eps, n_steps)
        states.append(w.copy())
    return states


def _oracle_analytics(op, states):
    deltas = [O.density_field(op, w) for w in states]
    vels = [O.velocity_field(op, w) for w in states]
    vrs = [O.radial_velocity(op, v) for v in vels]
    md, vd = O.sample_moments(deltas)
    mv, vv = O.sample_moments(vrs)
    met = O.convergence_metric(deltas)
    rows = [O.sphere_moments(op, dl, v, RADII) for dl, v in zip(deltas, vels)]
    sm, sv = O.sample_moments(rows)
    return md, vd, mv, vv, met, sm, sv


@pytest.mark.parametrize("N,L,n,prec,n_traj,eps,n_steps,tol",
                         [(16, 200.0, 500, "fp64", 6, 0.03, 10, 1e-10),
                          (32, 300.0, 800, "fp32", 5, 0.02, 8, 5e-5)])
def test_chain_analytics_vs_oracle(H, N, L, n, prec, n_traj, eps, n_steps, tol):
    cat, gp, op = _case(H, N, L, n, prec, 91)
    st = H.State(gp, [cat["d_init"]], seed=77)
    st.analytics(True, RADII, max_samples=16)
    tr = st.run_chain(n_traj, n_steps, eps)
    states = _oracle_states(op, cat["d_init"], n_traj, eps, n_steps)
    # the two chains took the same decisions (else the comparison is moot)
    g = st.get(0)
    check(f"analytics chain w {prec}", g["w"], states[-1], 1e-10 if prec == "fp64" else 1e-4)
    assert tr[:, 0]["accept"].sum() > 0
    out = st.analytics_read(0)
    md, vd, mv, vv, met, sm, sv = _oracle_analytics(op, states)
    assert out["n_samples"] == n_traj
    check(f"mean delta {prec}", out["mean_delta"], md, tol)
    check(f"var delta {prec}", out["var_delta"], vd, 10 * tol)
    check(f"mean v_r {prec}", out["mean_vr"], mv, tol)
    check(f"var v_r {prec}", out["var_vr"], vv, 10 * tol)
    assert out["metric"].shape == met.shape
    check(f"convergence metric {prec}", out["metric"], met, 10 * tol)
    sph = out["sphere"]
    assert sph.shape == (len(RADII), 5, 2)
    # sphere means are compared against the scale of the quantity (the
    # monopole can sit near zero), variances relatively
    for q in range(5):
        scale = max(np.max(np.abs(sm[:, q])), 1e-30)
        assert np.max(np.abs(sph[:, q, 0] - sm[:, q])) < 10 * tol * scale
        assert rel(sph[:, q, 1], sv[:, q]) < 1e3 * tol


def test_analytics_off_and_warmup_not_sampled(H):
    cat, gp, op = _case(H, 16, 200.0, 300, "fp64", 92)
    st = H.State(gp, [cat["d_init"], cat["d_init"]], seed=5, chain_ids=[0, 1])
    with pytest.raises(H.HamletError):
        st.analytics_read(0)
    st.analytics(True, [30.0, 60.0], max_samples=4)
    st.adapt_step_size(3, 5, 0.02)            # warm-up: no samples
    assert st.analytics_read(1)["n_samples"] == 0
    st.run_chain(6, 5, 0.02, use_graph=True)  # graph replay samples too
    out = st.analytics_read(1)
    assert out["n_samples"] == 6
    assert out["metric"].shape == (4,)         # capped at max_samples
    st.analytics(False)
    with pytest.raises(H.HamletError):
        st.analytics_read(0)
