"""Pins of the FP64 oracle against things other than itself: published test
vectors, closed forms, library routines, invariants and brute force."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special, stats

from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock

GOLDEN = __file__.replace("test_oracle_pins.py", "golden/philox4x32_10_kat.txt")

COSMO = dict(omega_m=0.3, omega_b=0.05, h=0.7, n_s=0.96, sigma8=0.8, T_cmb=2.7255)


def tiny_problem(N=8, L=100.0, n=40, seed=3, prior=None, sigma_cz=0.0, r_max=None):
    rng = np.random.default_rng(seed)
    z = 2 * rng.random(n) - 1
    ph = 2 * np.pi * rng.random(n)
    s = np.sqrt(1 - z * z)
    rhat = np.stack([s * np.cos(ph), s * np.sin(ph), z], 1)
    r_max = r_max or 0.4 * L
    d = r_max * (0.2 + 0.8 * rng.random(n))
    mu = 5 * np.log10(d / 0.7) + 25 + 0.2 * rng.normal(size=n)
    cz = 100 * d + 200 * rng.normal(size=n)
    if prior is None:
        prior = ("power", 2.0, 0.5, 0.5 * L)
    p = O.Problem(N, L, COSMO, 150.0, rhat, mu, np.full(n, 0.2), cz,
                  np.full(n, sigma_cz), prior)
    return p, d


# ---------------------------------------------------------------- RNG ----
def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = O.philox4x32_10(np.array([w[:4]], dtype=np.uint64), (w[4], w[5]))[0]
        assert [int(x) for x in out] == w[6:]


def test_uniform53_edges():
    assert O.uniform53(0, 0) == 0.0
    assert O.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # the 53 bits are (a>>5)<<26 | (b>>6)
    assert O.uniform53(1 << 5, 0) == 2.0 ** 26 / 2.0 ** 53
    assert O.uniform53(0, 1 << 6) == 2.0 ** -53


def test_normals_are_standard():
    x = O.philox_normals(200001, seed=11, traj=3, chain=1, tag=O.TAG_FIELD)
    assert abs(x.mean()) < 5 / math.sqrt(x.size)
    assert abs(x.var() - 1) < 5 * math.sqrt(2 / x.size)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # distinct streams differ
    y = O.philox_normals(1000, seed=11, traj=3, chain=1, tag=O.TAG_DIST)
    assert not np.allclose(x[:1000], y)


# ---------------------------------------------------------------- FFT ----
@pytest.mark.parametrize("N", [4, 8])
def test_fft_matches_naive_dft(N):
    rng = np.random.default_rng(N)
    x = rng.normal(size=(N, N, N)) + 1j * rng.normal(size=(N, N, N))
    ref = O.dft3_naive(x, sign=-1)
    assert np.max(np.abs(np.fft.fftn(x) - ref)) < 1e-12 * np.max(np.abs(ref))
    inv = O.dft3_naive(x, sign=+1) / N ** 3
    assert np.max(np.abs(np.fft.ifftn(x) - inv)) < 1e-12 * np.max(np.abs(inv))


def test_parseval_and_hermitian():
    rng = np.random.default_rng(5)
    N = 16
    w = rng.normal(size=(N, N, N))
    X = np.fft.fftn(w)
    assert abs(np.sum(w ** 2) - np.sum(np.abs(X) ** 2) / N ** 3) < 1e-10 * np.sum(w ** 2)
    neg = (-np.arange(N)) % N
    Xm = X[neg][:, neg][:, :, neg]
    assert np.max(np.abs(Xm - np.conj(X))) < 1e-10


# --------------------------------------------------------- cosmology ----
def tophat_j1(x):
    """Top-hat window written independently of the oracle: 3 j1(x)/x with
    scipy's spherical Bessel function (1 at x = 0)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    m = x > 0
    out[m] = 3.0 * special.spherical_jn(1, x[m]) / x[m]
    return out


def test_tophat_window_limits_zero_and_bessel_form():
    # W(x) = 3 j1(x)/x: W -> 1 - x^2/10 as x -> 0, first zero where tan x = x
    for x in (1e-3, 1e-2, 0.1):
        assert abs(O.tophat_window(x) - (1.0 - x * x / 10.0 + x ** 4 / 280.0)) < 1e-9
    x0 = optimize.brentq(lambda x: math.tan(x) - x, 4.0, 4.6)
    assert abs(x0 - 4.493409457909064) < 1e-12
    assert abs(O.tophat_window(x0)) < 1e-12
    x = np.linspace(0.05, 40.0, 2001)
    assert np.max(np.abs(O.tophat_window(x) - tophat_j1(x))) < 1e-12


def test_power_spectrum_normalisation_independent_quadrature():
    # sigma(8 Mpc/h) from adaptive quadrature with the Bessel-form window
    pk = O.PowerSpectrum(**COSMO)
    f = lambda lnk: (lambda k: k ** 3 * pk(k) * tophat_j1(k * 8.0) ** 2)(math.exp(lnk))
    val, _ = integrate.quad(f, math.log(1e-5), math.log(1e2), limit=4000)
    assert abs(math.sqrt(val / (2 * math.pi ** 2)) - 0.8) < 1e-8


def test_sigma_v_independent_quadrature_and_magnitude():
    pk = O.PowerSpectrum(**COSMO)
    f = 0.3 ** 0.55
    val, _ = integrate.quad(lambda lnk: math.exp(lnk) * pk(math.exp(lnk)),
                            math.log(1e-5), math.log(1e2), limit=4000)
    ref = math.sqrt((100 * f) ** 2 * val / (6 * math.pi ** 2))
    sv = pk.sigma_v(f)
    assert abs(sv - ref) < 1e-8 * ref
    # linear-theory 1-D velocity dispersion of a sigma8 = 0.8 LCDM is ~300 km/s
    assert 250 < sv < 350


def test_transfer_function_limits():
    # T -> 1 on large scales, sound horizon ~147 Mpc for om h^2 = 0.147
    T = O.eh_nowiggle_transfer(np.array([1e-6]), 0.3, 0.05, 0.7, 2.7255)[0]
    assert abs(T - 1) < 1e-4
    s = O.sound_horizon_eh(0.3, 0.05, 0.7)
    assert 142 < s < 152
    # matter-radiation equality peak of P(k) near 0.015-0.025 h/Mpc
    pk = O.PowerSpectrum(**COSMO)
    k = np.logspace(-3, 0, 2000)
    kp = k[np.argmax(pk(k))]
    assert 0.01 < kp < 0.03


def _q_nobaryon(k, omega_m, h, T_cmb):
    # without baryons alpha_Gamma = 1 and Gamma_eff = omega_m h on every scale
    return k * (T_cmb / 2.7) ** 2 / (omega_m * h)


def test_transfer_without_baryons_depends_on_k_through_q_only():
    # EH98: with omega_b = 0 the shape parameter is omega_m h, so T is one
    # function of q = k theta^2 / (omega_m h) for any (omega_m, h, T_cmb)
    k = np.logspace(-4, 2, 61)
    Ta = O.eh_nowiggle_transfer(k, 0.3, 0.0, 0.7, 2.7255)
    for om, h, tc in ((0.2, 0.7, 2.7255), (0.3, 0.5, 2.7255), (0.45, 0.8, 2.9)):
        kb = k * (om * h) / (0.3 * 0.7) * (2.7255 / tc) ** 2
        Tb = O.eh_nowiggle_transfer(kb, om, 0.0, h, tc)
        assert np.max(np.abs(Tb / Ta - 1)) < 1e-12
    # baryons suppress small-scale power (alpha_Gamma < 1)
    assert O.eh_nowiggle_transfer(np.array([1.0]), 0.3, 0.05, 0.7, 2.7255)[0] < \
        O.eh_nowiggle_transfer(np.array([1.0]), 0.3, 0.0, 0.7, 2.7255)[0]


def test_transfer_small_and_large_q_asymptotes():
    om, h, tc = 0.3, 0.7, 2.7255
    # q -> infinity: T -> ln(1.8 q) / (14.2 q^2) (logarithmic CDM tail)
    for k in (1e5, 1e6):
        q = _q_nobaryon(k, om, h, tc)
        T = O.eh_nowiggle_transfer(np.array([k]), om, 0.0, h, tc)[0]
        assert abs(T * q * q * 14.2 / math.log(1.8 * q) - 1) < 2e-6
    # q -> 0: 1 - T = C0(0) q^2 / L0(0) with C0(0) = 14.2 + 731, L0(0) = ln(2e) = 1 + ln 2,
    # and d/dq ln[(1 - T)/q^2] -> -731*62.5/745.2 - (1.8/(2e))/(1 + ln 2)
    lead = 745.2 / (1.0 + math.log(2.0))
    slope = -731.0 * 62.5 / 745.2 - (1.8 / (2.0 * math.e)) / (1.0 + math.log(2.0))
    q1, q2 = 1e-6, 2e-6
    r = []
    for q in (q1, q2):
        k = q * om * h / (tc / 2.7) ** 2
        T = O.eh_nowiggle_transfer(np.array([k]), om, 0.0, h, tc)[0]
        r.append((1.0 - T) / (q * q))
    assert abs(r[0] / lead - 1) < 2e-4
    qa, qb = 1e-4, 2e-4
    ra = []
    for q in (qa, qb):
        k = q * om * h / (tc / 2.7) ** 2
        T = O.eh_nowiggle_transfer(np.array([k]), om, 0.0, h, tc)[0]
        ra.append(math.log((1.0 - T) / (q * q)))
    assert abs((ra[1] - ra[0]) / (qb - qa) / slope - 1) < 2e-2


# ---------------------------------------------------- point functions ----
def test_zbar_series_expansion():
    om = 0.3
    for d in [1.0, 5.0, 20.0]:
        x = 100 * d / O.C_KMS
        series = x + 0.75 * om * x ** 2 + 9 / 8 * om ** 2 * x ** 3
        assert abs(O.zbar(d, om) - series) < 10 * x ** 4 + 1e-15


def test_distance_modulus_zero_at_10pc():
    # d (1 + zbar) / h = 1e-5 Mpc  =>  mu = 0
    d = 1e-5 * 0.7
    zb = 100 * d / O.C_KMS       # zbar to first order at this distance
    assert abs(O.distance_modulus(d, 0.3, 0.7) - 5 * np.log10(1 + zb)) < 1e-12
    # and 5 mag per decade of distance (z -> 0)
    assert abs(O.distance_modulus(10 * d, 0.3, 0.7) - 5.0) < 1e-7


@pytest.mark.parametrize("d", [3.0, 47.0, 160.0])
def test_point_derivatives_complex_step(d):
    h = 1e-20
    om = 0.3
    dc = d + 1j * h
    assert abs(np.imag(O.zbar(dc, om)) / h - O.zbar_prime(d, om)) < 1e-12 * abs(O.zbar_prime(d, om))
    mu_cs = np.imag(5.0 * np.log10(dc * (1 + O.zbar(dc, om)) / 0.7)) / h
    assert abs(mu_cs - O.distance_modulus_prime(d, om)) < 1e-12 * abs(mu_cs)
    z = 0.03
    vo_cs = np.imag(O.C_KMS * (z - O.zbar(dc, om)) / (1 + O.zbar(dc, om))) / h
    assert abs(vo_cs - O.v_observed_prime(z, d, om)) < 1e-10 * abs(vo_cs)
    k_cs = np.imag(150.0 ** 2 + 80.0 ** 2 / (1 + O.zbar(dc, om)) ** 2) / h
    assert abs(k_cs - O.kappa2_prime(d, 80.0, om)) < 1e-10 * abs(k_cs)


def test_vobs_inverts_redshift_composition():
    # a point at distance d moving with v_r has 1+z = (1+zbar)(1+v_r/c);
    # the observed-velocity relation must return v_r exactly.
    om = 0.3
    d = np.array([10.0, 80.0, 150.0])
    vr = np.array([-400.0, 120.0, 900.0])
    zb = O.zbar(d, om)
    z = (1 + zb) * (1 + vr / O.C_KMS) - 1
    assert np.max(np.abs(O.v_observed(z, d, om) - vr)) < 1e-8


# --------------------------------------------------------------- CIC ----
def test_cic_node_linear_and_partition_of_unity():
    p, d = tiny_problem(N=8, L=80.0, n=60)
    N, D = p.N, p.delta
    cell, frac = O.cic_cells(p, d)
    const = np.full((N, N, N), 2.5)
    val, grad = O.cic_gather(p, const, cell, frac)
    assert np.max(np.abs(val - 2.5)) < 1e-13 and np.max(np.abs(grad)) < 1e-12
    # a linear field is reproduced inside a cell (away from the periodic seam)
    a = np.array([0.3, -1.1, 0.7])
    ix = np.arange(N) * D
    X, Y, Z = np.meshgrid(ix, ix, ix, indexing="ij")
    lin = a[0] * X + a[1] * Y + a[2] * Z
    inner = np.all(cell < N - 1, axis=1)
    val, grad = O.cic_gather(p, lin, cell, frac)
    x = p.observer + d[:, None] * p.rhat
    assert np.max(np.abs(val[inner] - x[inner] @ a)) < 1e-11
    assert np.max(np.abs(grad[inner] - a)) < 1e-11
    # node values are returned exactly
    pts = np.array([[2, 3, 4], [0, 0, 0], [7, 1, 5]]) * D
    obs = np.zeros(3)
    q = O.Problem(N, p.L, COSMO, 150.0, np.tile([1.0, 0, 0], (3, 1)), np.zeros(3), np.ones(3),
                  np.zeros(3), np.zeros(3), ("power", 0, 0, 1e9), observer=obs)
    rng = np.random.default_rng(1)
    g = rng.normal(size=(N, N, N))
    # point at node: d rhat = node (rhat along x, so use x-only nodes)
    dn = np.array([2.0, 5.0, 7.0]) * D
    c2, f2 = O.cic_cells(q, dn)
    v2, _ = O.cic_gather(q, g, c2, f2)
    assert np.array_equal(v2, g[[2, 5, 7], 0, 0])


def test_cic_adjoint_dot_product():
    p, d = tiny_problem(N=8, L=80.0, n=60)
    rng = np.random.default_rng(2)
    g = rng.normal(size=(8, 8, 8))
    r = rng.normal(size=p.n)
    cell, frac = O.cic_cells(p, d)
    val, _ = O.cic_gather(p, g, cell, frac)
    s = O.cic_scatter(p, r, cell, frac)
    assert abs(np.dot(val, r) - np.sum(g * s)) < 1e-13 * np.sum(np.abs(g * s)) * 10


def test_cell_sort_is_stable_brute_force():
    p, d = tiny_problem(N=4, L=40.0, n=200)
    lin, order = O.cell_sort_order(p, d)
    brute = sorted(range(p.n), key=lambda i: (lin[i], i))
    assert list(order) == brute


# ---------------------------------------------------- velocity field ----
def test_plane_wave_velocity_closed_form():
    p, _ = tiny_problem(N=16, L=160.0)
    N = p.N
    n0 = np.array([1, 2, -3])
    k0 = 2 * np.pi / p.L * n0
    x = np.arange(N) * p.delta
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    A = 0.37
    delta = A * np.cos(k0[0] * X + k0[1] * Y + k0[2] * Z)
    v = O.velocity_from_delta_k(p, np.fft.fftn(delta))
    s = np.sin(k0[0] * X + k0[1] * Y + k0[2] * Z)
    for j in range(3):
        ref = -p.aHf * A * k0[j] / np.dot(k0, k0) * s
        assert np.max(np.abs(v[j] - ref)) < 1e-10 * p.aHf


def test_linear_continuity_per_mode():
    # i k . v_k = -aHf delta_k for every mode off the Nyquist planes
    p, _ = tiny_problem(N=16, L=160.0)
    w = mock.white_field(16, 4)
    dk = O.delta_k(p, w)
    v = O.velocity_field(p, w)
    nx, ny, nz = p.mode_numbers()
    kf = 2 * np.pi / p.L
    div = sum(1j * kf * nj * np.fft.fftn(v[j]) for j, nj in enumerate((nx, ny, nz)))
    m = (np.abs(nx) != 8) & (np.abs(ny) != 8) & (np.abs(nz) != 8)
    err = np.max(np.abs(div[m] + p.aHf * dk[m]))
    assert err < 1e-9 * np.max(np.abs(p.aHf * dk))


def _mode_k(N, L):
    # |k| of every DFT mode, from integer mode numbers in (-N/2, N/2]
    n = np.array([i if i <= N // 2 else i - N for i in range(N)], dtype=np.float64)
    return 2.0 * np.pi / L * np.sqrt(n[:, None, None] ** 2 + n[None, :, None] ** 2 + n[None, None, :] ** 2)


def _impulse_response(p, window=None):
    # the colouring map is a convolution, so E_w[mean_x delta(x)^2] over white
    # fields w is the squared norm of its response to a unit impulse
    e0 = np.zeros((p.N,) * 3)
    e0[0, 0, 0] = 1.0
    dk = O.delta_k(p, e0)
    if window is not None:
        dk = dk * window
    return np.fft.ifftn(dk).real


def test_colouring_variance():
    # <delta(x)^2> = (1/V) sum_{k != 0} P(|k|), P taken from the power spectrum
    # itself at the mode wavenumbers (eq. prior-k with its variance per mode)
    for N, L in ((8, 200.0), (16, 500.0)):
        p, _ = tiny_problem(N=N, L=L)
        k = _mode_k(N, L)
        expect = np.sum(p.pk(k[k > 0])) / L ** 3
        got = np.sum(_impulse_response(p) ** 2)
        assert abs(got / expect - 1) < 1e-12
    # and the sample variance over white fields agrees within its MC error
    p, _ = tiny_problem(N=8, L=200.0)
    k = _mode_k(8, 200.0)
    expect = np.sum(p.pk(k[k > 0])) / 200.0 ** 3
    acc = np.mean([np.mean(np.fft.ifftn(O.delta_k(p, mock.white_field(8, 1000 + s))).real ** 2)
                   for s in range(300)])
    assert abs(acc / expect - 1) < 0.05


def test_colouring_reproduces_sigma8_on_a_resolved_grid():
    # a field coloured on a grid that resolves the 8 Mpc/h top-hat and holds
    # its large scales has, smoothed with that top-hat, the variance sigma8^2
    # of the continuum definition (0.9 % short at 64^3 in 400 Mpc/h: the
    # modes below the fundamental are missing)
    N, L = 64, 400.0
    p, _ = tiny_problem(N=N, L=L)
    var = np.sum(_impulse_response(p, tophat_j1(8.0 * _mode_k(N, L))) ** 2)
    assert abs(var / 0.8 ** 2 - 1) < 0.015


def test_velocity_field_is_real():
    p, _ = tiny_problem(N=8, L=80.0)
    w = mock.white_field(8, 9)
    dk = O.delta_k(p, w)
    for f in p.velocity_factors():
        im = np.fft.ifftn(f * dk).imag
        assert np.max(np.abs(im)) < 1e-10 * p.aHf


# ----------------------------------------------- posterior + gradient ----
def test_full_operator_adjoint():
    p, d = tiny_problem(N=8, L=80.0, n=50)
    rng = np.random.default_rng(7)
    w = rng.normal(size=(8, 8, 8))
    y = rng.normal(size=p.n)
    lhs = np.dot(O.forward_u(p, w, d), y)
    rhs = np.sum(w * O.data_gradient_w(p, d, y))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_likelihood_at_truth_is_chi2():
    # data drawn from the model itself: at the truth each point contributes
    # xi_mu^2/2 + xi_v^2/2 + ln kappa
    p, d = tiny_problem(N=8, L=80.0, n=64, sigma_cz=60.0)
    rng = np.random.default_rng(8)
    w = rng.normal(size=(8, 8, 8))
    u = O.forward_u(p, w, d)
    xm, xv = rng.normal(size=p.n), rng.normal(size=p.n)
    mu = O.distance_modulus(d, p.omega_m, p.h) + p.sigma_mu * xm
    k2 = O.kappa2(d, p.sigma_nl, p.sigma_cz, p.omega_m)
    vr = u + np.sqrt(k2) * xv
    zb = O.zbar(d, p.omega_m)
    z = zb + (1 + zb) * vr / O.C_KMS
    q = O.Problem(p.N, p.L, COSMO, p.sigma_nl, p.rhat, mu, p.sigma_mu, z * O.C_KMS,
                  p.sigma_cz, ("power", 0.0, 0.5, 1e3))
    psi = O.logpost(q, w, d)
    expect = 0.5 * np.sum(w * w) + np.sum(0.5 * xm ** 2 + 0.5 * xv ** 2 + 0.5 * np.log(k2))
    assert abs(psi - expect) < 1e-9 * abs(expect)


def _away_from_faces(p, d, h):
    t = (p.observer + d[:, None] * p.rhat) / p.delta
    f = t - np.floor(t)
    margin = 2 * h * 1.0 / p.delta + 1e-6
    return np.all((f > margin) & (f < 1 - margin), axis=1)


def test_gradient_central_differences():
    p, d = tiny_problem(N=8, L=80.0, n=40, sigma_cz=50.0)
    rng = np.random.default_rng(10)
    w = rng.normal(size=(8, 8, 8))
    psi, gw, gd = O.logpost_grad(p, w, d)
    h = 1e-4
    for _ in range(12):
        idx = tuple(rng.integers(0, 8, 3))
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (O.logpost(p, wp, d) - O.logpost(p, wm, d)) / (2 * h)
        assert abs(fd - gw[idx]) < 1e-5 * max(1.0, abs(gw[idx]))
    ok = np.nonzero(_away_from_faces(p, d, h))[0]
    assert ok.size > 10
    for i in ok[:15]:
        dp, dm = d.copy(), d.copy()
        dp[i] += h
        dm[i] -= h
        fd = (O.logpost(p, w, dp) - O.logpost(p, w, dm)) / (2 * h)
        assert abs(fd - gd[i]) < 1e-5 * max(1.0, abs(gd[i]))


def test_table_prior_interpolation():
    logdens = np.log(np.array([0.1, 0.3, 0.2, 0.4]))
    p, _ = tiny_problem(N=8, L=80.0, n=4, prior=("table", 5.0, 10.0, logdens))
    # bin centres return the table values exactly; outer half bins are flat
    c = 5.0 + 10.0 * (np.arange(4) + 0.5)
    lp, dl = O.log_prior_d(p, c)
    assert np.array_equal(lp, logdens)
    lp, dl = O.log_prior_d(p, np.array([5.0, 44.999]))
    assert lp[0] == logdens[0] and lp[1] == logdens[3] and np.all(dl == 0)
    # linear in between with the slope as derivative; continuous across centres
    x = np.array([12.5, 20.0, 27.5])
    lp, dl = O.log_prior_d(p, x)
    assert abs(lp[0] - 0.75 * logdens[0] - 0.25 * logdens[1]) < 1e-15
    assert abs(lp[1] - logdens[1]) < 1e-15
    assert abs(lp[2] - 0.25 * logdens[1] - 0.75 * logdens[2]) < 1e-15
    assert abs(dl[0] - (logdens[1] - logdens[0]) / 10.0) < 1e-15
    eps = 1e-9
    for cc in c[1:3]:
        a, _ = O.log_prior_d(p, np.array([cc - eps, cc + eps]))
        assert abs(a[1] - a[0]) < 1e-8
    lp2, _ = O.log_prior_d(p, np.array([4.9, 45.0]))
    assert np.all(np.isneginf(lp2))


def test_table_prior_gradient_central_differences():
    rng = np.random.default_rng(4)
    logdens = np.log(rng.uniform(0.1, 1.0, 12))
    p, _ = tiny_problem(N=8, L=80.0, n=6, prior=("table", 0.0, 4.0, logdens))
    d = np.array([3.1, 7.7, 13.3, 22.9, 31.7, 41.2])
    lp, dl = O.log_prior_d(p, d)
    h = 1e-6
    fd = (O.log_prior_d(p, d + h)[0] - O.log_prior_d(p, d - h)[0]) / (2 * h)
    assert np.max(np.abs(fd - dl)) < 1e-7


def test_out_of_domain_is_infinite():
    p, d = tiny_problem(N=8, L=80.0, n=5)
    w = np.zeros((8, 8, 8))
    d2 = d.copy()
    d2[0] = -1.0
    psi, gw, gd = O.logpost_grad(p, w, d2)
    assert np.isinf(psi) and psi > 0 and np.all(np.isfinite(gw))


# ------------------------------------------------------------ leapfrog ----
def _prior_only(N=8):
    return O.Problem(N, 80.0, COSMO, 150.0, np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                     np.zeros(0), np.zeros(0), ("power", 0.0, 0.0, 1.0))


def test_leapfrog_pure_prior_closed_form():
    p = _prior_only()
    rng = np.random.default_rng(12)
    q0, p0 = rng.normal(size=(8, 8, 8)), rng.normal(size=(8, 8, 8))
    eps, L = 0.3, 7
    w, _, pw, _, _, _, _ = O.leapfrog(p, q0, np.zeros(0), p0, np.zeros(0), eps, L)
    Mstep = np.array([[1 - eps ** 2 / 2, eps], [-eps * (1 - eps ** 2 / 4), 1 - eps ** 2 / 2]])
    ML = np.linalg.matrix_power(Mstep, L)
    assert np.max(np.abs(w - (ML[0, 0] * q0 + ML[0, 1] * p0))) < 1e-13
    assert np.max(np.abs(pw - (ML[1, 0] * q0 + ML[1, 1] * p0))) < 1e-13


def test_leapfrog_reversible():
    p, d = tiny_problem(N=8, L=80.0, n=30)
    rng = np.random.default_rng(13)
    w0 = 0.3 * rng.normal(size=(8, 8, 8))
    pw0 = rng.normal(size=(8, 8, 8))
    pd0 = rng.normal(size=p.n) / math.sqrt(p.minv_d)
    eps, L = 0.02, 6
    w1, d1, pw1, pd1, *_ = O.leapfrog(p, w0, d, pw0, pd0, eps, L)
    w2, d2, pw2, pd2, *_ = O.leapfrog(p, w1, d1, -pw1, -pd1, eps, L)
    assert np.max(np.abs(w2 - w0)) < 1e-12
    assert np.max(np.abs(d2 - d)) < 1e-10


def test_energy_error_second_order():
    p, d = tiny_problem(N=8, L=80.0, n=30)
    rng = np.random.default_rng(14)
    w0 = 0.3 * rng.normal(size=(8, 8, 8))
    pw0 = rng.normal(size=(8, 8, 8))
    tau = 0.4
    dH = []
    for eps in (0.04, 0.02):
        L = int(round(tau / eps))
        psi0 = O.logpost(p, w0, d)
        w1, _, pw1, _, psi1, _, _ = O.leapfrog(p, w0, d, pw0, np.zeros(p.n), eps, L, sample_d=False)
        dH.append(abs(psi1 + 0.5 * np.sum(pw1 ** 2) - psi0 - 0.5 * np.sum(pw0 ** 2)))
    assert 3.0 < dH[0] / dH[1] < 5.0


def test_prior_only_chain_samples_unit_normal():
    p = _prior_only(N=4)
    w = np.zeros((4, 4, 4))
    ws = []
    psi_grad = O.logpost_grad(p, w, np.zeros(0))
    for t in range(400):
        w, _, psi_grad, rec = O.hmc_trajectory(p, w, np.zeros(0), psi_grad, seed=5, traj=t,
                                               chain=0, eps=0.5, n_steps=3)
        ws.append(w.copy())
    ws = np.array(ws[50:])
    assert abs(ws.mean()) < 0.1
    assert abs(ws.var() - 1.0) < 0.15


# ------------------------------------------------------- dual averaging ----
def test_dual_averaging_fixed_point_and_direction():
    # acceptance exactly at the target leaves Hbar = 0: eps stays at 10 eps0
    da = O.DualAveraging(0.1, delta=0.65)
    for _ in range(20):
        e = da.update(0.65)
    assert abs(e - 1.0) < 1e-12 and abs(da.Hbar) < 1e-15
    # accepting more than the target makes the step grow, less makes it shrink
    hi, lo = O.DualAveraging(0.1), O.DualAveraging(0.1)
    for _ in range(30):
        hi.update(1.0)
        lo.update(0.0)
    assert hi.eps > 1.0 > lo.eps
    # the averaged step is a weighted mean of the iterates (log scale)
    assert lo.eps <= lo.eps_bar or abs(lo.eps - lo.eps_bar) < 1e-9


def test_dual_averaging_reaches_target_acceptance_on_a_gaussian():
    # pure prior (unit Gaussian in every coordinate): after adaptation the
    # chain's mean acceptance is near the target
    p = _prior_only(N=4)
    w = np.zeros((4, 4, 4))
    w, _, eps_bar, recs = O.adapt_step_size(p, w, np.zeros(0), seed=9, chain=0, traj0=0, n_warmup=300,
                                            eps0=0.05, n_steps=5, delta=0.65)
    psi_grad = O.logpost_grad(p, w, np.zeros(0))
    acc = []
    for t in range(400):
        w, _, psi_grad, rec = O.hmc_trajectory(p, w, np.zeros(0), psi_grad, seed=9, traj=1000 + t, chain=0,
                                               eps=eps_bar, n_steps=5)
        acc.append(O.accept_probability(rec["H_old"], rec["H_new"]))
    assert abs(np.mean(acc) - 0.65) < 0.1


# --------------------------------------------- redshift-distance prior ----
def test_redshift_distance_quadrature_and_expansion():
    om = 0.3
    z = np.array([1e-4, 0.01, 0.05, 0.1])
    got = O.redshift_distance(z, om)
    for zi, g in zip(z, got):
        ref, _ = integrate.quad(lambda x: 1.0 / np.sqrt(om * (1 + x) ** 3 + 1 - om), 0, zi, epsabs=0, epsrel=1e-13)
        assert abs(g - O.C_KMS / 100.0 * ref) < 1e-10 * g
        # d_z = (c/H0) (z - (3 Om/4) z^2 + O(z^3))
        series = O.C_KMS / 100.0 * (zi - 0.75 * om * zi ** 2)
        assert abs(g - series) < O.C_KMS / 100.0 * 2.0 * zi ** 3


def test_dz_prior_table_counts_and_normalisation():
    cz = np.array([1000.0, 1500.0, 2900.0, 3100.0, 12000.0])
    ld = O.dz_prior_table(cz, 0.3, 5.0, 10.0)
    dens = np.exp(ld)
    assert abs(np.sum(dens) * 5.0 - 1.0) < 1e-12
    dz = O.redshift_distance(cz / O.C_KMS, 0.3)
    assert len(ld) == int(np.ceil((dz.max() + 10.0) / 5.0))
    # bins with points have (count + 0.5) / (count' + 0.5) density ratios
    b = (dz / 5.0).astype(int)
    empty = [k for k in range(len(ld)) if k not in set(b)][0]
    assert abs(dens[b[0]] / dens[empty] - (np.sum(b == b[0]) + 0.5) / 0.5) < 1e-12


# ------------------------------------------------------ sampled sigma_NL ----
def test_dz_prior_kind_is_the_histogram_of_the_redshift_distances():
    # ("dz", bin, pad): eq. D from the catalogue's own cz (section "Priors");
    # default bin 5 Mpc/h and pad 3 sigma_v/H0
    p, _ = tiny_problem(N=8, L=400.0, n=300, prior=("dz", 0.0, 0.0))
    _, d0, bw, t = p.prior
    assert (d0, bw) == (0.0, 5.0)
    assert np.array_equal(t, O.dz_prior_table(p.cz, 0.3, 5.0, 3.0 * p.sigma_v / O.H0))
    q, _ = tiny_problem(N=8, L=400.0, n=300, prior=("dz", 4.0, 12.0))
    assert np.array_equal(q.prior[3], O.dz_prior_table(q.cz, 0.3, 4.0, 12.0))


@pytest.mark.parametrize("name", sorted(mock.PRESETS))
def test_preset_start_distances_inside_the_dz_prior_support(name):
    # the chains start at cz/H0, which is inside [0, max d_z + pad): d_z < cz/H0
    # by less than the pad at these redshifts
    spec = mock.PRESETS[name]
    cat = mock.make_catalog(spec)
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    lp, _ = O.log_prior_d(op, cat["d_init"])
    assert np.all(np.isfinite(lp))


def test_sigma_nl_gradient_central_differences_and_consistency():
    p, d = tiny_problem(N=8, L=80.0, n=40, sigma_cz=50.0)
    rng = np.random.default_rng(17)
    w = rng.normal(size=(8, 8, 8))
    s = 180.0
    psi, gw, gd, gs = O.logpost_grad_s(p, w, d, s)
    h = 1e-3
    fd = (O.logpost_grad_s(p, w, d, s + h)[0] - O.logpost_grad_s(p, w, d, s - h)[0]) / (2 * h)
    assert abs(fd - gs) < 1e-6 * max(1.0, abs(gs))
    # at the problem's own sigma_NL it is the ordinary posterior
    p.sigma_nl = s
    psi2, gw2, gd2 = O.logpost_grad(p, w, d)
    assert psi == psi2 and np.array_equal(gw, gw2) and np.array_equal(gd, gd2)
    assert np.isinf(O.logpost_grad_s(p, w, d, -1.0)[0])


def test_leapfrog_with_sigma_is_reversible():
    p, d = tiny_problem(N=8, L=80.0, n=30)
    rng = np.random.default_rng(18)
    w0 = 0.3 * rng.normal(size=(8, 8, 8))
    pw0 = rng.normal(size=(8, 8, 8))
    pd0 = rng.normal(size=p.n) / math.sqrt(p.minv_d)
    s0, ps0 = 200.0, 0.7
    w1, d1, s1, pw1, pd1, ps1, _ = O.leapfrog_s(p, w0, d, s0, pw0, pd0, ps0, 0.02, 6)
    w2, d2, s2, *_ = O.leapfrog_s(p, w1, d1, s1, -pw1, -pd1, -ps1, 0.02, 6)
    assert np.max(np.abs(w2 - w0)) < 1e-12 and abs(s2 - s0) < 1e-9
