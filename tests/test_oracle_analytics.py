"""Pins of the oracle's chain analytics (eq. int_mc, sections "Convergence" and
"Monopole and dipole") against closed forms and independent computations."""
import math

import numpy as np

from oracle import hamlet_oracle as O

COSMO = dict(omega_m=0.3, omega_b=0.05, h=0.7, n_s=0.96, sigma8=0.8, T_cmb=2.7255)


def problem(N=16, L=160.0):
    n = 4
    rhat = np.tile([1.0, 0.0, 0.0], (n, 1))
    return O.Problem(N, L, COSMO, 150.0, rhat, np.full(n, 35.0), np.full(n, 0.2), np.full(n, 3000.0),
                     np.zeros(n), ("power", 2.0, 0.5, 0.5 * L))


def test_density_field_of_a_cosine_is_its_coloured_cosine():
    # w = cos(2 pi n.i/N): DFT(w) is N^3/2 on modes +-n, so delta = sqrt(P(k_n)/Delta^3) cos(...)
    p = problem()
    N = p.N
    nvec = np.array([2, 1, 3])
    i = np.arange(N)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    phase = 2 * np.pi * (nvec[0] * gx + nvec[1] * gy + nvec[2] * gz) / N
    w = np.cos(phase)
    k = 2 * np.pi / p.L * math.sqrt(float(nvec @ nvec))
    expect = math.sqrt(p.pk(np.array([k]))[0] / p.delta ** 3) * np.cos(phase)
    assert np.max(np.abs(O.density_field(p, w) - expect)) < 1e-12 * np.max(np.abs(expect))


def test_radial_velocity_closed_forms():
    p = problem()
    off, r = O.node_offsets(p)
    # a uniform flow: v_r = rhat . V; along +x from the observer it is V_x
    V = np.array([120.0, -40.0, 75.0])
    v = np.broadcast_to(V[:, None, None, None], (3,) + r.shape)
    vr = O.radial_velocity(p, v)
    c = p.N // 2
    assert abs(vr[c + 3, c, c] - V[0]) < 1e-12
    assert abs(vr[c, c - 2, c] + V[1]) < 1e-12
    assert vr[c, c, c] == 0.0                      # the observer's own node
    # a purely radial field v = x - o has v_r = |x - o|
    vr2 = O.radial_velocity(p, off)
    assert np.max(np.abs(vr2 - r)) < 1e-12 * p.L


def test_sample_moments_two_states():
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(2, 5, 5))
    mean, var = O.sample_moments([a, b])
    assert np.allclose(mean, 0.5 * (a + b), rtol=0, atol=1e-15)
    assert np.allclose(var, 0.5 * (a - b) ** 2, rtol=0, atol=1e-15)
    m1, v1 = O.sample_moments([a])
    assert np.array_equal(m1, a) and not v1.any()


def test_convergence_metric_closed_forms():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(6, 6, 6))
    # identical states: the normalised running mean does not move
    assert np.all(O.convergence_metric([a, a, a]) < 1e-15)
    # states a, 2a: m_2/S_2 - m_1/S_1 = 1.5a/(2 s) - a/s = -a/(4 s), s = std(a)
    s = math.sqrt(np.mean(a * a) - np.mean(a) ** 2)
    got = O.convergence_metric([a, 2 * a])
    assert got.shape == (1,)
    assert abs(got[0] - 0.25 * math.sqrt(np.mean(a * a)) / s) < 1e-13


def test_sphere_moments_uniform_fields_and_brute_force():
    p = problem()
    _, r = O.node_offsets(p)
    delta = np.full(r.shape, 0.3)
    V = np.array([100.0, 20.0, -50.0])
    v = np.broadcast_to(V[:, None, None, None], (3,) + r.shape)
    out = O.sphere_moments(p, delta, v, [15.0, 40.0])
    for row in out:
        assert abs(row[0] - p.f * 0.3) < 1e-13
        assert np.allclose(row[1:4], V, atol=1e-12)
        assert abs(row[4] - math.sqrt(V @ V)) < 1e-10
    # R = 0 picks the observer's node alone
    rng = np.random.default_rng(2)
    dr = rng.normal(size=r.shape)
    vr = rng.normal(size=(3,) + r.shape)
    c = p.N // 2
    o = O.sphere_moments(p, dr, vr, [0.0])[0]
    assert abs(o[0] - p.f * dr[c, c, c]) < 1e-15
    assert np.allclose(o[1:4], vr[:, c, c, c], atol=1e-15)


def test_monopole_is_minus_divergence_over_H0():
    # divergence of the velocity taken spectrally (i k_j on every mode) by the
    # test itself, for a field without Nyquist components, averaged in a sphere
    p = problem()
    N = p.N
    rng = np.random.default_rng(3)
    wk = np.fft.fftn(rng.normal(size=(N, N, N)))
    n1 = np.fft.fftfreq(N, d=1.0 / N)
    nx, ny, nz = np.meshgrid(n1, n1, n1, indexing="ij")
    nyq = (np.abs(nx) == N // 2) | (np.abs(ny) == N // 2) | (np.abs(nz) == N // 2)
    wk[nyq] = 0.0
    w = np.fft.ifftn(wk).real
    v = O.velocity_field(p, w)
    kf = 2 * np.pi / p.L
    div = sum(np.fft.ifftn(1j * kf * n * np.fft.fftn(v[j])).real for j, n in enumerate((nx, ny, nz)))
    delta = O.density_field(p, w)
    _, r = O.node_offsets(p)
    for R in (20.0, 45.0, 70.0):
        m = r <= R
        mono = O.sphere_moments(p, delta, v, [R])[0, 0]
        assert abs(mono - (-div[m].mean() / O.H0)) < 1e-10 * max(1.0, abs(mono))
