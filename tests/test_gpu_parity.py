"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: 1e-12 on the FP64 path and 1e-5 on the FP32 path for Psi (relative)
and for every vector output, both norm-wise (||x - x_ref|| / ||x_ref||) and
element-wise (max|x - x_ref| / max|x_ref|); bit-exact for Philox words, cell
indices and the cell sort.
"""
import math

import numpy as np
import pytest
import torch

from _parity import check, check_scalar, rel
from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


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
    # prior None: eq. D built from the catalogue's redshifts on both sides
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
    check(f"fft r2c {N} {prec}", X, ref, tol)
    back = p.fft_c2r(torch.tensor(ref, device="cuda")).cpu().numpy() / N ** 3
    check(f"fft c2r {N} {prec}", back, x, tol)


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
    check(f"fft c2r general {N} {prec}", got, ref, 2e-6 if prec == "fp32" else 1e-13)


# ---------------------------------------------------------- velocity ----
@pytest.mark.parametrize("N,L,prec", [(16, 200.0, "fp64"), (64, 500.0, "fp32"), (32, 300.0, "fp64")])
def test_velocity_field_vs_oracle(H, N, L, prec):
    spec, cat, gp, op, w = make_case(H, N, L, 50, prec, seed=7)
    v = gp.velocity_field(torch.tensor(w, device="cuda")).cpu().numpy()
    ref = O.velocity_field(op, w)
    check(f"velocity {N} {prec}", v, ref, TOL[prec])


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
    tag = f"{N}^3/{n}/{prec}"
    check_scalar(f"psi {tag}", psi.item(), rpsi, tol)
    check(f"grad_w {tag}", gw, rgw, tol)
    check(f"grad_d {tag}", gd, rgd, tol)
    # the data part of the field gradient on its own (without the w term)
    check(f"grad_w data part {tag}", gw.cpu().numpy() - w, rgw - w, 50 * tol if prec == "fp32" else tol)


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
    check_scalar("psi 128^3/30000/fp32", psi.item(), rpsi, 1e-5)
    check("grad_w 128^3/30000/fp32", gw, rgw, 1e-5)
    check("grad_d 128^3/30000/fp32", gd, rgd, 1e-5)
    check("grad_w data part 128^3/30000/fp32", gw.cpu().numpy() - w, rgw - w, 5e-4)
    v = gp.velocity_field(torch.tensor(w, device="cuda")).cpu().numpy()
    check("velocity 128^3 fp32", v, O.velocity_field(op, w), 1e-5)


def test_logpost_grad_128_fp64(H):
    """128^3 on the FP64 path (the largest FP64 grid), 1e4 points, 1e-12."""
    spec, cat, gp, op, w = make_case(H, 128, 500.0, 10000, "fp64", 21, mask=10.0, r_max=160.0)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    check_scalar("psi 128^3/10000/fp64", psi.item(), rpsi, 1e-12)
    check("grad_w 128^3/10000/fp64", gw, rgw, 1e-12)
    check("grad_d 128^3/10000/fp64", gd, rgd, 1e-12)


def test_logpost_grad_128_1e5_points(H):
    """The largest 128^3 job of the serving mix (10^5 points, r^2 to 160
    Mpc/h in the 500 Mpc/h box): every plane carries thousands of points."""
    spec, cat, gp, op, w = make_case(H, 128, 500.0, 100000, "fp32", 31, mask=10.0, r_max=160.0)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    check_scalar("psi 128^3/100000/fp32", psi.item(), rpsi, 1e-5)
    check("grad_w 128^3/100000/fp32", gw, rgw, 1e-5)
    check("grad_d 128^3/100000/fp32", gd, rgd, 1e-5)


@pytest.mark.parametrize("N,L,prec", [(64, 500.0, "fp32"), (128, 500.0, "fp32"), (32, 300.0, "fp64"),
                                      (256, 1000.0, "fp32")])
def test_all_points_on_one_x_plane(H, N, L, prec):
    """A degenerate catalogue: every direction lies (almost) in the y-z plane
    through the observer (0 <= rhat_x < 1e-3), so every point's lower CIC
    corner is on the observer's x-plane and one bucket (or one plane's slab
    buckets at 256^3) holds the whole catalogue, a tenth of the directions
    exactly in the plane (the points sit on the cell face, fx = 0)."""
    n = 4000
    spec = mock.MockSpec(N=N, L=L, n_points=n, r_max=0.3 * L, mask_deg=0.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=17, precision=prec)
    cat = mock.make_catalog(spec)
    rng = np.random.default_rng(N)
    rx = rng.uniform(0.0, 1e-3, n)
    rx[: n // 10] = 0.0
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s_ = np.sqrt(1.0 - rx * rx)
    cat["rhat"] = np.ascontiguousarray(np.stack([rx, s_ * np.cos(phi), s_ * np.sin(phi)], axis=1))
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(N, L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    cell, _ = O.cic_cells(op, cat["d_init"])
    assert np.all(cell[:, 0] == N // 2)
    w = mock.white_field(N, 5)
    if prec == "fp32":
        w = w.astype(np.float32).astype(np.float64)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    tag = f"one plane {N}^3/{n}/{prec}"
    check_scalar(f"psi {tag}", psi.item(), rpsi, TOL[prec])
    check(f"grad_w {tag}", gw, rgw, TOL[prec])
    check(f"grad_d {tag}", gd, rgd, TOL[prec])


def test_default_prior_is_the_redshift_distance_histogram(H):
    """Section "Priors": without a caller table the library builds eq. D from
    the catalogue's observed redshifts (d_z by eq. e:dz) at hm_set_catalog;
    the table it reads equals the oracle's, and setting another catalogue
    rebuilds it."""
    spec = mock.PRESETS["grid128_30000pts"]
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    d0, bw, t = gp.prior_table()
    _, od0, obw, ot = op.prior
    assert (d0, bw) == (od0, obw) == (0.0, 5.0)
    assert t.shape == ot.shape
    assert np.max(np.abs(t - ot)) < 1e-12
    ref = O.dz_prior_table(cat["cz"], 0.3, 5.0, 3.0 * op.sigma_v / 100.0)
    assert np.max(np.abs(t - ref)) < 1e-12
    # the chains' start distances sit inside its support
    lp, _ = O.log_prior_d(op, cat["d_init"])
    assert np.all(np.isfinite(lp))
    small = mock.make_catalog(mock.MockSpec(N=128, L=500.0, n_points=800, r_max=60.0, mask_deg=10.0,
                                            sigma_mu=(0.2, 0.45), sigma_nl=250.0, seed=5))
    gp.set_catalog(small["rhat"], small["mu"], small["sigma_mu"], small["cz"], small["sigma_cz"])
    _, _, t2 = gp.prior_table()
    assert np.max(np.abs(t2 - O.dz_prior_table(small["cz"], 0.3, 5.0, 3.0 * op.sigma_v / 100.0))) < 1e-12
    assert t2.shape[0] < t.shape[0]


def test_caller_table_prior(H):
    """A distance-prior table given by the caller (eq. D as a histogram the
    caller built) against the oracle with the same table."""
    spec, cat, gp, op, w = make_case(H, 32, 300.0, 1017, "fp64", 3, mask=10.0,
                                     prior=("table", 0.0, 4.0, -0.01 * np.arange(40.0) - 3.0))
    d = np.clip(cat["d_init"], 1.0, 150.0)
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    check_scalar("psi caller table", psi.item(), rpsi, 1e-12)
    check("grad_w caller table", gw, rgw, 1e-12)
    check("grad_d caller table", gd, rgd, 1e-12)


def test_catalog_in_supergalactic_coordinates(H):
    """hm_set_catalog_sg (SGL, SGB in degrees, the paper's data coordinates)
    gives the problem that the unit vectors give."""
    spec, cat, gp, op, w = make_case(H, 16, 200.0, 500, "fp64", 13)
    r = cat["rhat"]
    sgb = np.degrees(np.arcsin(np.clip(r[:, 2], -1, 1)))
    sgl = np.degrees(np.arctan2(r[:, 1], r[:, 0])) % 360.0
    gq = H.Problem(16, 200.0, spec.cosmo, spec.sigma_nl, "fp64", ("dz", spec.prior_bin, 0.0))
    gq.set_catalog_sg(sgl, sgb, cat["mu"], cat["sigma_mu"], cat["cz"])
    d = torch.tensor(cat["d_init"], device="cuda")
    wt = torch.tensor(w, device="cuda")
    a = gp.logpost_grad(wt, d)
    b = gq.logpost_grad(wt, d)
    check_scalar("psi sg", b[0].item(), a[0].item(), 1e-12)
    check("grad_w sg", b[1], a[1], 1e-12)
    check("grad_d sg", b[2], a[2], 1e-12)
    with pytest.raises(Exception, match="SGB"):
        gq.set_catalog_sg(sgl[:3], np.array([0.0, 91.0, 0.0]), cat["mu"][:3], cat["sigma_mu"][:3], cat["cz"][:3])


def test_empty_catalog_is_prior_only(H):
    p = H.Problem(16, 100.0, precision="fp64", prior=("power", 2.0, 0.5, 40.0))
    p.set_catalog(np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros(0))
    w = mock.white_field(16, 3)
    psi, gw, gd = p.logpost_grad(torch.tensor(w, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert abs(psi.item() - 0.5 * np.sum(w * w)) < 1e-10 * np.sum(w * w)
    check("grad_w prior only", gw, w, 1e-14)


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


@pytest.mark.parametrize("N,L", [(64, 500.0), (128, 500.0), (256, 1000.0)])
def test_cells_next_to_cell_faces_bit_exact(H, N, L):
    """Distances that put a point on a cell face, a few ulp and 1e-12..1e-6
    (relative) to either side of one, and far outside the box (|x/Delta| up
    to ~2600 cells): the cells must still be floor((o + d r)/Delta) mod N
    bit for bit, where the fast screen cannot decide as well as where it can."""
    spec, cat, gp, op, w = make_case(H, N, L, 4000, "fp32", 12)
    r = cat["rhat"]
    rng = np.random.default_rng(N)
    n = r.shape[0]
    ax = np.argmax(np.abs(r), axis=1)
    ra = r[np.arange(n), ax]
    o = op.observer[ax]
    delta = op.delta
    # a face k Delta ahead of the observer along the point's main axis
    steps = rng.integers(1, int(0.3 * N), size=n)
    k = np.where(ra > 0, np.ceil(o / delta) + steps, np.floor(o / delta) - steps)
    d_face = (k * delta - o) / ra
    ds = [d_face]
    for u in (1, 2, 3, 8):
        ds.append(d_face + u * np.spacing(d_face))
        ds.append(d_face - u * np.spacing(d_face))
    for rel_ in (1e-12, 1e-9, 1e-6):
        ds.append(d_face * (1.0 + rel_))
        ds.append(d_face * (1.0 - rel_))
    ds.append(rng.uniform(1.0e3, 1.0e4, size=n))      # far outside the box: the FP64 fallback
    ds.append(rng.uniform(0.0, 1.0e-3, size=n))       # at the observer
    for d in ds:
        cell, _ = gp.cells(torch.tensor(d, device="cuda"), sort=False)
        lin, _ = O.cell_sort_order(op, d)
        assert np.array_equal(cell.cpu().numpy(), lin)


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
    tag = f"leapfrog {N}^3/{n}/{prec}/{steps} steps"
    check(f"w {tag}", g["w"], w1, tol)
    check(f"d {tag}", g["d"], d1, tol)
    check(f"p_w {tag}", g["pw"], pw1, tol)
    check(f"p_d {tag}", g["pd"], pd1, tol if prec == "fp64" else 1e-4)
    sc = st.scalars(0)
    check_scalar(f"psi {tag}", sc["psi"], psi1, tol)


def test_leapfrog_two_chain_state_vs_oracle(H):
    """A launch over several chains evaluates the FP32 path's distance terms
    in FP32 (zbar and mu_i - mu(d) from FP64 differences, the rest FP32):
    both chains of a two-chain 64^3 / 5,000-point state against the oracle."""
    N, L, n, steps = 64, 500.0, 5000, 20
    spec, cat, gp, op, st1 = _state_and_oracle(H, N, L, n, "fp32", 23)
    st = H.State(gp, [cat["d_init"], cat["d_init"]], seed=77, chain_ids=[0, 1])
    rng = np.random.default_rng(6)
    d0 = cat["d_init"]
    starts = []
    for c in range(2):
        w0 = (0.5 * rng.normal(size=(N, N, N))).astype(np.float32).astype(np.float64)
        pw0 = rng.normal(size=(N, N, N)).astype(np.float32).astype(np.float64)
        pd0 = rng.normal(size=n) / math.sqrt(op.minv_d)
        st.set(c, w=torch.tensor(w0), d=torch.tensor(d0), pw=torch.tensor(pw0), pd=torch.tensor(pd0))
        starts.append((w0, pw0, pd0))
    st.refresh()
    for c in range(2):
        gw, gd = st.grad(c)
        rpsi, rgw, rgd = O.logpost_grad(op, starts[c][0], d0)
        check(f"two-chain grad_w chain {c}", gw, rgw, 1e-5)
        check(f"two-chain grad_d chain {c}", gd, rgd, 1e-5)
        check_scalar(f"two-chain psi chain {c}", st.scalars(c)["psi"], rpsi, 1e-5)
    st.leapfrog(steps, 0.02)
    for c in range(2):
        w0, pw0, pd0 = starts[c]
        g = st.get(c)
        w1, d1, pw1, pd1, psi1, _, _ = O.leapfrog(op, w0, d0, pw0, pd0, 0.02, steps)
        tag = f"two-chain leapfrog chain {c}"
        check(f"w {tag}", g["w"], w1, 1e-5)
        check(f"d {tag}", g["d"], d1, 1e-5)
        check(f"p_w {tag}", g["pw"], pw1, 1e-5)
        check(f"p_d {tag}", g["pd"], pd1, 1e-4)
        check_scalar(f"psi {tag}", st.scalars(c)["psi"], psi1, 1e-5)


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
    check("chain w 16^3 fp64", g["w"], w, 1e-10)
    check("chain d 16^3 fp64", g["d"], d, 1e-10)


def _one_trajectory_vs_oracle(H, gp, op, d_init, seed, n_burn, eps, n_steps, tag, tol, tol_pd):
    """n_burn trajectories, then one more replayed as a captured graph exactly
    as bench.py times its steps (one-chain state, Philox key `seed`, chain word
    0); that trajectory against the oracle's from the same start: momenta
    drawn from the same Philox counters, KDK leapfrog, energies, Metropolis
    decision, end point and end momenta (sections "Construction of HMC
    chains" and "Integrating the HMC trajectories")."""
    st = H.State(gp, [d_init], seed=seed, chain_ids=[0])
    if n_burn:
        st.run_chain(n_burn, n_steps, eps, use_graph=True, trace=False)
    g0 = st.get(0)
    w0 = g0["w"].cpu().numpy().astype(np.float64)
    d0 = g0["d"].cpu().numpy()
    traj = st.scalars(0)["traj"]
    assert traj == n_burn
    tr = st.run_chain(1, n_steps, eps, use_graph=True)
    g1 = st.get(0)
    pw0, pd0 = O.draw_momenta(op, seed, traj, 0)
    psi0, gw0, gd0 = O.logpost_grad(op, w0, d0)
    H_old = psi0 + O.kinetic(op, pw0, pd0)
    w1, d1, pw1, pd1, psi1, _, _ = O.leapfrog(op, w0, d0, pw0, pd0, eps, n_steps, grad0=(psi0, gw0, gd0))
    H_new = psi1 + O.kinetic(op, pw1, pd1)
    r = tr[0, 0]
    check_scalar(f"H_old {tag}", r["H_old"], H_old, tol)
    check_scalar(f"H_new {tag}", r["H_new"], H_new, tol)
    logu = O.philox_accept_logu(seed, traj, 0)
    assert abs(r["logu"] - logu) < 1e-14
    accept = bool(np.isfinite(H_new) and logu < H_old - H_new)
    # the decision must agree unless ln U sits within the energies' rounding of H_old - H_new
    if abs(logu - (H_old - H_new)) > 10 * tol * abs(H_old):
        assert bool(r["accept"]) == accept
    acc = bool(r["accept"])
    check(f"w {tag}", g1["w"], w1 if acc else w0, tol)
    check(f"d {tag}", g1["d"], d1 if acc else d0, tol)
    check(f"p_w {tag}", g1["pw"], pw1, tol)
    check(f"p_d {tag}", g1["pd"], pd1, tol_pd)
    return tr


def test_benchmarked_trajectory_128_fp32_vs_oracle(H):
    """The unit bench.py times: the 128^3 / 3e4-point FP32 chain (box 500
    Mpc/h), trajectories of 20 leapfrog steps at eps = 0.025 replayed as a
    captured graph after the bench's 5 warm-up trajectories."""
    spec = mock.PRESETS["grid128_30000pts"]
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    _one_trajectory_vs_oracle(H, gp, op, cat["d_init"], seed=1000, n_burn=5, eps=0.025, n_steps=20,
                              tag="trajectory 128^3/30000/fp32/20 steps", tol=1e-5, tol_pd=1e-4)


def test_trajectory_128_fp64_vs_oracle(H):
    """128^3 on the FP64 path, 1e4 points: one graph-replayed trajectory of
    3 leapfrog steps after one warm-up trajectory, at 1e-12."""
    spec, cat, gp, op, w = make_case(H, 128, 500.0, 10000, "fp64", 21, mask=10.0, r_max=160.0)
    _one_trajectory_vs_oracle(H, gp, op, cat["d_init"], seed=3, n_burn=1, eps=0.02, n_steps=3,
                              tag="trajectory 128^3/10000/fp64/3 steps", tol=1e-12, tol_pd=1e-12)


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
    check("graph vs stream w", gb["w"], ga["w"], 1e-5)


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
        check(f"batched w chain {c}", gb["w"], gs["w"], 1e-5)
        check(f"batched d chain {c}", gb["d"], gs["d"], 1e-6)


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
    check("sigma_NL leapfrog w", g["w"], w1, 1e-12)
    check("sigma_NL leapfrog d", g["d"], d1, 1e-12)
    assert abs(s1[0] - rs1) <= 1e-11 * rs1
    assert abs(st.scalars(0)["psi"] - psi1) <= 1e-12 * abs(psi1)
    # a chain with sigma_NL sampled runs and moves it
    tr = st.run_chain(5, 10, 0.02)
    assert np.all(np.isfinite(tr[:, 0]["H_new"]))


def test_logpost_grad_256_two_pass_planes(H):
    """256^3 (box 1000 Mpc/h), 2e4 points: the z-pass / y-pass plane passes
    and the TMA-staged x pass, the posterior gradient, the velocity field and
    one trajectory against the oracle's."""
    spec = mock.MockSpec(N=256, L=1000.0, n_points=20000, r_max=300.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=81)
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    w = mock.white_field(256, 82).astype(np.float32).astype(np.float64)
    d = cat["d_init"]
    psi, gw, gd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    check_scalar("psi 256^3/20000/fp32", psi.item(), rpsi, 1e-5)
    check("grad_w 256^3/20000/fp32", gw, rgw, 1e-5)
    check("grad_d 256^3/20000/fp32", gd, rgd, 1e-5)
    v = gp.velocity_field(torch.tensor(w, device="cuda")).cpu().numpy()
    check("velocity 256^3 fp32", v, O.velocity_field(op, w), 1e-5)
    st = H.State(gp, [d], seed=3)
    tr = st.run_chain(1, 3, 0.01, use_graph=True)
    _, _, recs = O.run_chain(op, np.zeros((256,) * 3), d, seed=3, chain=0, traj0=0, n_traj=1, eps=0.01, n_steps=3)
    assert abs(tr[0, 0]["H_new"] - recs[0]["H_new"]) <= 1e-5 * abs(recs[0]["H_new"])
    tr = st.run_chain(2, 5, 0.01, use_graph=True)
    assert np.all(np.isfinite(tr[:, 0]["H_new"]))


def test_trajectory_256_bench_workload_vs_oracle(H):
    """The 256^3 workload bench.py times (box 1000 Mpc/h, 1e5 points with r^2
    to 160 Mpc/h, its catalogue seed and chain seed, eps = 0.01): after 3
    warm-up trajectories, one graph-replayed trajectory against the oracle's
    from the same state; 4 leapfrog steps a trajectory rather than the
    bench's 20 keep the oracle's 256^3 transforms to about a minute."""
    spec = mock.MockSpec(N=256, L=1000.0, n_points=100000, r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=1007)
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    _one_trajectory_vs_oracle(H, gp, op, cat["d_init"], seed=5, n_burn=3, eps=0.01, n_steps=4,
                              tag="trajectory 256^3/100000/fp32/4 steps", tol=1e-5, tol_pd=1e-4)


def test_no_bounded_device_wait_gave_up(H):
    """The x pass at FP32 N = 256 waits for tensor copies with a bounded
    poll; after the transforms, gradients and chains above (and one more
    128^3 and 256^3 velocity field here) none may have given up."""
    import ctypes as ct
    for N, L in ((128, 500.0), (256, 1000.0)):
        p = H.Problem(N, L, precision="fp32")
        p.set_catalog(np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros(0))
        v = p.velocity_field(torch.tensor(mock.white_field(N, 3), dtype=torch.float32, device="cuda"))
        assert torch.isfinite(v).all()
    torch.cuda.synchronize()
    n = ct.c_int32(-1)
    assert p.lib.hm_device_wait_timeouts(0, 0, ct.byref(n)) == 0
    assert n.value == 0
