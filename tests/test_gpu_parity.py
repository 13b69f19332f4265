"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (norm-wise relative, ||x - x_ref|| / ||x_ref||): 1e-12 on the FP64
path and 1e-5 on the FP32 path for Psi and both gradient blocks; bit-exact
for Philox words, cell indices and the cell sort.
"""
import math

import numpy as np
import pytest
import torch

from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    if np.iscomplexobj(a) or np.iscomplexobj(b):
        a = np.concatenate([np.real(a), np.imag(a)])
        b = np.concatenate([np.real(b), np.imag(b)])
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import hamlet
    return hamlet


def make_case(H, N, L, n, precision, seed, mask=0.0, r_max=None, sigma_mu=(0.2, 0.45), sigma_nl=250.0,
              prior=None):
    spec = mock.MockSpec(N=N, L=L, n_points=n, r_max=r_max or 0.32 * L, mask_deg=mask,
                         sigma_mu=sigma_mu, sigma_nl=sigma_nl, seed=seed, precision=precision)
    cat = mock.make_catalog(spec)
    if prior is None:
        prior = ("table", cat["prior_d0"], cat["prior_bin"], cat["prior_logdens"])
    gp = H.Problem.from_mock(spec, cat, prior=prior)
    op = O.problem_from_catalog(N, L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat, prior=prior)
    w = mock.white_field(N, seed + 1000)
    if precision == "fp32":
        w = w.astype(np.float32).astype(np.float64)
    return spec, cat, gp, op, w


# ------------------------------------------------------------------ FFT ----
@pytest.mark.parametrize("N,prec", [(8, "fp32"), (16, "fp32"), (32, "fp32"), (64, "fp32"), (128, "fp32"),
                                    (256, "fp32"), (8, "fp64"), (16, "fp64"), (32, "fp64"), (64, "fp64"),
                                    (128, "fp64")])
def test_fft_roundtrip_vs_numpy(H, N, prec):
    p = H.Problem(N, 100.0, precision=prec)
    rng = np.random.default_rng(N)
    x = rng.normal(size=(2, N, N, N))
    dt = torch.float32 if prec == "fp32" else torch.float64
    xt = torch.tensor(x, dtype=dt, device="cuda")
    X = p.fft_r2c(xt).cpu().numpy()
    ref = np.fft.rfftn(xt.double().cpu().numpy(), axes=(1, 2, 3))
    tol = 2e-6 if prec == "fp32" else 1e-13
    assert rel(X, ref) < tol
    back = p.fft_c2r(torch.tensor(ref, device="cuda")).cpu().numpy() / N ** 3
    assert rel(back, x) < tol


@pytest.mark.parametrize("N,prec", [(8, "fp64"), (32, "fp64"), (128, "fp64"), (64, "fp32"), (128, "fp32"),
                                    (256, "fp32")])
def test_fft_c2r_general_half_spectrum(H, N, prec):
    """A half spectrum that is not the transform of a real field (random
    values everywhere, including the imaginary parts of the kz = 0 and N/2
    lines): c2r keeps the real part of those lines after the complex y and x
    transforms, as numpy's irfftn does."""
    p = H.Problem(N, 100.0, precision=prec)
    rng = np.random.default_rng(N + 5)
    X = rng.normal(size=(1, N, N, N // 2 + 1)) + 1j * rng.normal(size=(1, N, N, N // 2 + 1))
    if prec == "fp32":
        X = X.astype(np.complex64).astype(np.complex128)
    ref = np.fft.irfftn(X, s=(N, N, N), axes=(1, 2, 3)) * N ** 3
    got = p.fft_c2r(torch.tensor(X, device="cuda")).cpu().numpy()
    assert rel(got, ref) < (2e-6 if prec == "fp32" else 1e-13)


# ---------------------------------------------------------- velocity ----
@pytest.mark.parametrize("N,L,prec", [(16, 200.0, "fp64"), (64, 500.0, "fp32"), (32, 300.0, "fp64")])
def test_velocity_field_vs_oracle(H, N, L, prec):
    spec, cat, gp, op, w = make_case(H, N, L, 50, prec, seed=7)
    v = gp.velocity_field(torch.tensor(w, device="cuda")).cpu().numpy()
    ref = O.velocity_field(op, w)
    assert rel(v, ref) < TOL[prec]


# ---------------------------------------------------------- posterior ----
CASES = [
    # N, L, n points, precision, seed, mask
    (16, 200.0, 500, "fp64", 0, 0.0),      # the 16^3 FP64 configuration
    (32, 300.0, 1017, "fp64", 3, 10.0),    # ragged point count, several tiles
    (64, 500.0, 5000, "fp32", 1, 10.0),    # the 64^3 FP32 configuration
    (8, 80.0, 37, "fp32", 4, 0.0),         # smallest grid, ragged pencil tile
]


@pytest.mark.parametrize("N,L,n,prec,seed,mask", CASES)
def test_logpost_grad_vs_oracle(H, N, L, n, prec, seed, mask):
    spec, cat, gp, op, w = make_case(H, N, L, n, prec, seed, mask=mask)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    tol = TOL[prec]
    assert abs(psi.item() - rpsi) / abs(rpsi) < tol
    assert rel(gw.cpu().numpy(), rgw) < tol
    assert rel(gd.cpu().numpy(), rgd) < tol
    # the data part of the field gradient on its own (without the w term)
    assert rel(gw.cpu().numpy() - w, rgw - w) < (50 * tol if prec == "fp32" else tol)


def test_logpost_grad_128_paper_scale_sampled(H):
    """128^3, 3e4 points (the paper-scale configuration): full oracle check."""
    spec = mock.PRESETS["grid128_30000pts"]
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    w = mock.white_field(spec.N, 5).astype(np.float32).astype(np.float64)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    assert abs(psi.item() - rpsi) / abs(rpsi) < 1e-5
    assert rel(gw.cpu().numpy(), rgw) < 1e-5
    assert rel(gd.cpu().numpy(), rgd) < 1e-5


def test_logpost_grad_128_fp64(H):
    """128^3 on the FP64 path (the largest FP64 grid), 1e4 points, 1e-12."""
    spec, cat, gp, op, w = make_case(H, 128, 500.0, 10000, "fp64", 21, mask=10.0, r_max=160.0)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    assert abs(psi.item() - rpsi) <= 1e-12 * abs(rpsi)
    assert rel(gw.cpu().numpy(), rgw) < 1e-12
    assert rel(gd.cpu().numpy(), rgd) < 1e-12


def test_catalog_in_supergalactic_coordinates(H):
    """hm_set_catalog_sg (SGL, SGB in degrees, the paper's data coordinates)
    gives the problem that the unit vectors give."""
    spec, cat, gp, op, w = make_case(H, 16, 200.0, 500, "fp64", 13)
    r = cat["rhat"]
    sgb = np.degrees(np.arcsin(np.clip(r[:, 2], -1, 1)))
    sgl = np.degrees(np.arctan2(r[:, 1], r[:, 0])) % 360.0
    gq = H.Problem(16, 200.0, spec.cosmo, spec.sigma_nl, "fp64",
                   ("table", cat["prior_d0"], cat["prior_bin"], cat["prior_logdens"]))
    gq.set_catalog_sg(sgl, sgb, cat["mu"], cat["sigma_mu"], cat["cz"])
    d = torch.tensor(cat["d_init"], device="cuda")
    wt = torch.tensor(w, device="cuda")
    a = gp.logpost_grad(wt, d)
    b = gq.logpost_grad(wt, d)
    assert abs(a[0].item() - b[0].item()) <= 1e-12 * abs(a[0].item())
    assert rel(b[1].cpu().numpy(), a[1].cpu().numpy()) < 1e-12
    assert rel(b[2].cpu().numpy(), a[2].cpu().numpy()) < 1e-12
    with pytest.raises(Exception, match="SGB"):
        gq.set_catalog_sg(sgl[:3], np.array([0.0, 91.0, 0.0]), cat["mu"][:3], cat["sigma_mu"][:3], cat["cz"][:3])


def test_empty_catalog_is_prior_only(H):
    p = H.Problem(16, 100.0, precision="fp64", prior=("power", 2.0, 0.5, 40.0))
    p.set_catalog(np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros(0))
    w = mock.white_field(16, 3)
    psi, gw, gd = p.logpost_grad(torch.tensor(w, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert abs(psi.item() - 0.5 * np.sum(w * w)) < 1e-10 * np.sum(w * w)
    assert rel(gw.cpu().numpy(), w) < 1e-14


def test_out_of_support_distance_is_infinite(H):
    spec, cat, gp, op, w = make_case(H, 16, 200.0, 40, "fp64", 9, prior=("power", 2.0, 0.5, 90.0))
    d = cat["d_init"].copy()
    d = np.clip(d, 1.0, 80.0)
    d[3] = 95.0
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    assert math.isinf(psi.item()) and psi.item() > 0
    assert gp.last_status() & 1
    assert gd[3].item() == 0.0


# ------------------------------------------------------- index work ----
@pytest.mark.parametrize("N", [16, 64, 128, 256])
def test_cells_and_sort_bit_exact(H, N):
    spec, cat, gp, op, w = make_case(H, N, 400.0, 3001 if N < 128 else 30000, "fp64" if N == 16 else "fp32", 11)
    d = cat["d_init"]
    cell, perm = gp.cells(torch.tensor(d, device="cuda"))
    lin, order = O.cell_sort_order(op, d)
    assert np.array_equal(cell.cpu().numpy(), lin)
    assert np.array_equal(perm.cpu().numpy(), order)


def test_philox_words_bit_exact(H):
    n = 4099
    got = H.philox(0x1234_5678_9ABC, n, 7, 3, 1).cpu().numpy().view(np.uint32).reshape(n, 4)
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n)
    ctr[:, 1], ctr[:, 2], ctr[:, 3] = 7, 3, 1
    ref = O.philox4x32_10(ctr, O.seed_key(0x1234_5678_9ABC))
    assert np.array_equal(got, ref)


# ------------------------------------------------------------- HMC ----
def _state_and_oracle(H, N, L, n, prec, seed):
    spec, cat, gp, op, w = make_case(H, N, L, n, prec, seed)
    st = H.State(gp, [cat["d_init"]], seed=77)
    return spec, cat, gp, op, st


@pytest.mark.parametrize("N,L,n,prec,steps", [(16, 200.0, 500, "fp64", 10), (64, 500.0, 5000, "fp32", 20)])
def test_leapfrog_vs_oracle(H, N, L, n, prec, steps):
    spec, cat, gp, op, st = _state_and_oracle(H, N, L, n, prec, 21)
    rng = np.random.default_rng(5)
    w0 = 0.5 * rng.normal(size=(N, N, N))
    pw0 = rng.normal(size=(N, N, N))
    if prec == "fp32":
        w0 = w0.astype(np.float32).astype(np.float64)
        pw0 = pw0.astype(np.float32).astype(np.float64)
    d0 = cat["d_init"]
    pd0 = rng.normal(size=n) / math.sqrt(op.minv_d)
    st.set(0, w=torch.tensor(w0), d=torch.tensor(d0), pw=torch.tensor(pw0), pd=torch.tensor(pd0))
    st.refresh()
    eps = 0.02
    st.leapfrog(steps, eps)
    g = st.get(0)
    w1, d1, pw1, pd1, psi1, _, _ = O.leapfrog(op, w0, d0, pw0, pd0, eps, steps)
    tol = TOL[prec]
    assert rel(g["w"].cpu().numpy(), w1) < tol
    assert rel(g["d"].cpu().numpy(), d1) < tol
    assert rel(g["pw"].cpu().numpy(), pw1) < tol
    assert rel(g["pd"].cpu().numpy(), pd1) < (tol if prec == "fp64" else 1e-4)
    sc = st.scalars(0)
    assert abs(sc["psi"] - psi1) / abs(psi1) < tol


def test_run_chain_vs_oracle_fp64(H):
    N, L, n = 16, 200.0, 500
    spec, cat, gp, op, st = _state_and_oracle(H, N, L, n, "fp64", 31)
    eps, Lf, ntraj = 0.03, 10, 6
    tr = st.run_chain(ntraj, Lf, eps)
    w, d, recs = O.run_chain(op, np.zeros((N, N, N)), cat["d_init"], seed=77, chain=0, traj0=0,
                             n_traj=ntraj, eps=eps, n_steps=Lf)
    for t in range(ntraj):
        r = recs[t]
        assert abs(tr[t, 0]["H_old"] - r["H_old"]) < 1e-10 * abs(r["H_old"])
        assert abs(tr[t, 0]["H_new"] - r["H_new"]) < 1e-10 * abs(r["H_new"])
        assert abs(tr[t, 0]["logu"] - r["logu"]) < 1e-14
        if abs(r["logu"] - (r["H_old"] - r["H_new"])) > 1e-9:
            assert bool(tr[t, 0]["accept"]) == r["accept"]
    assert tr[:, 0]["accept"].sum() > 0
    g = st.get(0)
    assert rel(g["w"].cpu().numpy(), w) < 1e-10
    assert rel(g["d"].cpu().numpy(), d) < 1e-10


def test_graph_replay_matches_stream_launches(H):
    N, L, n = 32, 300.0, 800
    spec, cat, gp, op, w = make_case(H, N, L, n, "fp32", 41)
    a = H.State(gp, [cat["d_init"]], seed=5)
    b = H.State(gp, [cat["d_init"]], seed=5)
    ta = a.run_chain(5, 8, 0.02, use_graph=False)
    tb = b.run_chain(5, 8, 0.02, use_graph=True)
    assert np.array_equal(ta["accept"], tb["accept"])
    assert np.allclose(ta["H_new"], tb["H_new"], rtol=1e-5)
    ga, gb = a.get(0), b.get(0)
    assert rel(ga["w"].cpu().numpy(), gb["w"].cpu().numpy()) < 1e-5


def test_batched_chains_match_single_chains(H):
    N, L = 32, 300.0
    specs = [mock.MockSpec(N=N, L=L, n_points=n, r_max=96.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                           sigma_nl=250.0, seed=s) for n, s in ((700, 51), (1300, 52))]
    cats = [mock.make_catalog(s) for s in specs]
    probs = [H.Problem.from_mock(s, c) for s, c in zip(specs, cats)]
    batch = H.State(probs, [cats[0]["d_init"], cats[1]["d_init"], cats[1]["d_init"]], seed=9,
                    chain_problem=[0, 1, 1], chain_ids=[0, 1, 2])
    tb = batch.run_chain(4, 6, [0.02, 0.015, 0.015])
    for c, pi in enumerate([0, 1, 1]):
        single = H.State(probs[pi], [cats[pi]["d_init"]], seed=9, chain_ids=[c])
        ts = single.run_chain(4, 6, [0.02, 0.015, 0.015][c])
        assert np.array_equal(ts[:, 0]["accept"], tb[:, c]["accept"])
        assert np.allclose(ts[:, 0]["H_new"], tb[:, c]["H_new"], rtol=1e-5)
        gs, gb = single.get(0), batch.get(c)
        assert rel(gs["w"].cpu().numpy(), gb["w"].cpu().numpy()) < 1e-5
        assert rel(gs["d"].cpu().numpy(), gb["d"].cpu().numpy()) < 1e-6


def test_dual_averaging_matches_oracle_recursion(H):
    spec, cat, gp, op, st = _state_and_oracle(H, 16, 200.0, 500, "fp64", 61)
    eps_out, tr = st.adapt_step_size(40, 10, 0.002, target=0.65)
    da = O.DualAveraging(0.002, delta=0.65)
    for t in range(40):
        assert abs(tr[t, 0]["eps"] - da.eps) <= 1e-12 * da.eps
        da.update(O.accept_probability(tr[t, 0]["H_old"], tr[t, 0]["H_new"]))
    assert abs(eps_out[0] - da.eps_bar) <= 1e-12 * da.eps_bar
    # the tuned step is used by the following run
    tr2 = st.run_chain(3, 10, eps_out)
    assert np.allclose(tr2[:, 0]["eps"], eps_out[0])


def test_sampled_sigma_nl_gradient_and_leapfrog_vs_oracle(H):
    spec, cat, gp, op, st = _state_and_oracle(H, 16, 200.0, 500, "fp64", 71)
    rng = np.random.default_rng(9)
    w0 = 0.5 * rng.normal(size=(16, 16, 16))
    pw0 = rng.normal(size=(16, 16, 16))
    d0 = cat["d_init"]
    pd0 = rng.normal(size=d0.size) / math.sqrt(op.minv_d)
    st.set(0, w=torch.tensor(w0), d=torch.tensor(d0), pw=torch.tensor(pw0), pd=torch.tensor(pd0))
    st.sample_sigma_nl(True, 180.0)
    s, gs = st.sigma_nl()
    psi, gw, gd, rgs = O.logpost_grad_s(op, w0, d0, 180.0)
    assert s[0] == 180.0
    assert abs(gs[0] - rgs) <= 1e-12 * max(1.0, abs(rgs))
    st.leapfrog(8, 0.02)
    g = st.get(0)
    s1, _ = st.sigma_nl()
    w1, d1, rs1, pw1, pd1, ps1, psi1 = O.leapfrog_s(op, w0, d0, 180.0, pw0, pd0, 0.0, 0.02, 8)
    assert rel(g["w"].cpu().numpy(), w1) < 1e-12
    assert rel(g["d"].cpu().numpy(), d1) < 1e-12
    assert abs(s1[0] - rs1) <= 1e-11 * rs1
    assert abs(st.scalars(0)["psi"] - psi1) <= 1e-12 * abs(psi1)
    # a chain with sigma_NL sampled runs and moves it
    tr = st.run_chain(5, 10, 0.02)
    assert np.all(np.isfinite(tr[:, 0]["H_new"]))


def test_logpost_grad_256_cluster_planes(H):
    """256^3 (box 1000 Mpc/h), 2e4 points: the 8-CTA cluster plane passes,
    the posterior gradient and one trajectory against the oracle's."""
    spec = mock.MockSpec(N=256, L=1000.0, n_points=20000, r_max=300.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=81)
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    w = mock.white_field(256, 82).astype(np.float32).astype(np.float64)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    assert abs(psi.item() - rpsi) / abs(rpsi) < 1e-5
    assert rel(gw.cpu().numpy(), rgw) < 1e-5
    assert rel(gd.cpu().numpy(), rgd) < 1e-5
    v = gp.velocity_field(torch.tensor(w, device="cuda")).cpu().numpy()
    assert rel(v, O.velocity_field(op, w)) < 1e-5
    st = H.State(gp, [d], seed=3)
    tr = st.run_chain(1, 3, 0.01, use_graph=True)
    _, _, recs = O.run_chain(op, np.zeros((256,) * 3), d, seed=3, chain=0, traj0=0, n_traj=1, eps=0.01, n_steps=3)
    assert abs(tr[0, 0]["H_new"] - recs[0]["H_new"]) <= 1e-5 * abs(recs[0]["H_new"])
    tr = st.run_chain(2, 5, 0.01, use_graph=True)
    assert np.all(np.isfinite(tr[:, 0]["H_new"]))
