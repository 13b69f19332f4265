"""HAMLET oracle -- plain, slow, FP64 CPU restatement of the paper's posterior,
its gradient and the HMC chain (Valade, Hoffman & Libeskind, "HAMLET: a
Hamiltonian Monte Carlo reconstruction of the local environment").

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers); both sides receive
the same seeded inputs from ``paper_2203_02369_gb300.mock`` and nothing else.

Everything is float64 numpy.  Library primitives used as single steps:
``numpy.fft.fftn/ifftn`` (the 3D DFT, cross-checked against a naive DFT in
the tests), ``numpy.linalg`` (dense Wiener-filter solve).  No blocking, fusion
or reordering beyond what the equations state.

Readings of points the paper leaves open (the CUDA path takes the same ones):
  * DFT forward is unnormalised with e^{-ik.x}; IDFT carries 1/N^3.  With this
    convention the linear velocity (eq. vel-field) is v_k = +i aHf k/k^2 delta_k,
    which is the sign that gives div v = -aHf delta (linear continuity).
  * The Fourier-mode prior (eq. prior-k) is sampled in whitened form:
    delta_k = sqrt(P(k)/Delta^3) DFT(w)_k with w ~ N(0,1) per grid node, so
    Psi_prior = |w|^2/2 and the identity mass matrix on w is eq. M_ab's choice
    (M^-1 = prior covariance) written in these variables.  P(0) = 0.
  * Odd factors k_j are zero on the Nyquist plane of axis j (keeps v real).
  * Interpolation is cloud-in-cell (trilinear) on nodes at i*Delta; the
    observer sits at the box centre; a point on a face belongs to the upper cell.
  * mu(d) = 5 log10(d (1+zbar)/h) + 25 with d in Mpc/h; zbar is the
    second-order relation of section "The Likelihood function: distances".
  * The distance prior (eq. D) is a caller-given histogram table or a power law;
    the table's ln pi is interpolated linearly between bin centres (a
    piecewise-constant histogram puts a jump in H at every bin crossing that
    the leapfrog cannot see).
  * Psi omits every additive constant independent of (w, d).
  * Leapfrog is kick-drift-kick with merged half kicks; Metropolis accepts iff
    ln U < H_old - H_new with U in (0, 1].
  * Random numbers: Philox-4x32-10 (Salmon et al., SC'11) with counter
    (pair index, trajectory, chain, stream tag) and key = seed; 53-bit
    uniforms; Box-Muller normals.
"""
from __future__ import annotations

import itertools
import math
import numpy as np

C_KMS = 299792.458           # speed of light, km/s
H0 = 100.0                   # km/s/(Mpc/h)

# ----------------------------------------------------------------------------
# Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11).
# ----------------------------------------------------------------------------
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF

TAG_FIELD = 0      # momenta of the whitened field
TAG_DIST = 1       # momenta of the distances
TAG_ACCEPT = 2     # Metropolis uniform


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds.  ctr: uint array (..., 4); key: 2 ints.

    One round maps (c0,c1,c2,c3) with key (k0,k1) to
    (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)); the key is
    bumped by the Weyl constants (W0, W1) before every round but the first.
    """
    ctr = np.asarray(ctr, dtype=np.uint64)
    c0, c1, c2, c3 = (ctr[..., i] & _MASK32 for i in range(4))
    k0 = np.uint64(int(key[0]) & _MASK32)
    k1 = np.uint64(int(key[1]) & _MASK32)
    m0 = np.uint64(_PHILOX_M0)
    m1 = np.uint64(_PHILOX_M1)
    mask = np.uint64(_MASK32)
    s32 = np.uint64(32)
    for r in range(10):
        if r > 0:
            k0 = np.uint64((int(k0) + _PHILOX_W0) & _MASK32)
            k1 = np.uint64((int(k1) + _PHILOX_W1) & _MASK32)
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniform53(a, b):
    """53-bit uniform in [0, 1) from two uint32 words: (a>>5, b>>6) / 2^53."""
    a = np.asarray(a, dtype=np.uint64) >> np.uint64(5)
    b = np.asarray(b, dtype=np.uint64) >> np.uint64(6)
    return (a.astype(np.float64) * 67108864.0 + b.astype(np.float64)) * (1.0 / 9007199254740992.0)


def seed_key(seed):
    seed = int(seed)
    return (seed & _MASK32, (seed >> 32) & _MASK32)


def philox_normals(n, seed, traj, chain, tag):
    """n standard normals for element indices 0..n-1.  Element i uses counter
    (i//2, traj, chain, tag); the pair (u1, u2) from words (0,1) and (2,3)
    gives r = sqrt(-2 ln(1-u1)), theta = 2 pi u2 and normals (r cos, r sin)."""
    npair = (n + 1) // 2
    ctr = np.zeros((npair, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(npair, dtype=np.uint64)
    ctr[:, 1] = traj
    ctr[:, 2] = chain
    ctr[:, 3] = tag
    x = philox4x32_10(ctr, seed_key(seed))
    u1 = uniform53(x[:, 0], x[:, 1])
    u2 = uniform53(x[:, 2], x[:, 3])
    r = np.sqrt(-2.0 * np.log(1.0 - u1))
    th = 2.0 * np.pi * u2
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:n]


def philox_accept_logu(seed, traj, chain):
    """ln U of the Metropolis test, U = 1 - u53 in (0, 1]."""
    x = philox4x32_10(np.array([[0, traj, chain, TAG_ACCEPT]], dtype=np.uint64), seed_key(seed))
    u = uniform53(x[0, 0], x[0, 1])
    return math.log(1.0 - float(u))


# ----------------------------------------------------------------------------
# Linear power spectrum: Eisenstein & Hu (1998) no-wiggle transfer function,
# normalised to sigma8 with a top-hat of radius 8 Mpc/h.
# ----------------------------------------------------------------------------
QUAD_KMIN = 1e-5      # h/Mpc
QUAD_KMAX = 1e2       # h/Mpc
QUAD_INTERVALS = 16384


def eh_nowiggle_transfer(k, omega_m, omega_b, h, T_cmb):
    """EH98 zero-baryon-oscillation transfer function, k in h/Mpc (EH98 eqs.
    26, 28-31: sound horizon s, alpha_Gamma, Gamma_eff(k), q, L0, C0)."""
    k = np.asarray(k, dtype=np.float64)
    omh2 = omega_m * h * h
    obh2 = omega_b * h * h
    fb = omega_b / omega_m
    theta = T_cmb / 2.7
    s = 44.5 * np.log(9.83 / omh2) / np.sqrt(1.0 + 10.0 * obh2 ** 0.75)
    alpha = 1.0 - 0.328 * np.log(431.0 * omh2) * fb + 0.38 * np.log(22.3 * omh2) * fb * fb
    gamma_eff = omega_m * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k * h * s) ** 4))
    q = k * theta * theta / gamma_eff
    L0 = np.log(2.0 * np.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def sound_horizon_eh(omega_m, omega_b, h):
    """EH98 eq. 26 approximation of the sound horizon, Mpc."""
    omh2 = omega_m * h * h
    obh2 = omega_b * h * h
    return 44.5 * math.log(9.83 / omh2) / math.sqrt(1.0 + 10.0 * obh2 ** 0.75)


def _simpson_lnk(f_of_k):
    """Composite Simpson rule in ln k on [QUAD_KMIN, QUAD_KMAX]."""
    n = QUAD_INTERVALS
    lnk = np.linspace(math.log(QUAD_KMIN), math.log(QUAD_KMAX), n + 1)
    k = np.exp(lnk)
    wts = np.ones(n + 1)
    wts[1:-1:2] = 4.0
    wts[2:-1:2] = 2.0
    hstep = (lnk[-1] - lnk[0]) / n
    return float(np.sum(wts * f_of_k(k)) * hstep / 3.0)


def tophat_window(x):
    return 3.0 * (np.sin(x) - x * np.cos(x)) / (x ** 3)


class PowerSpectrum:
    """P(k) = A k^n_s T(k)^2 in (Mpc/h)^3 with A fixed by sigma8."""

    def __init__(self, omega_m=0.3, omega_b=0.05, h=0.7, n_s=0.96, sigma8=0.8, T_cmb=2.7255):
        self.omega_m, self.omega_b, self.h = omega_m, omega_b, h
        self.n_s, self.sigma8, self.T_cmb = n_s, sigma8, T_cmb
        self.A = 1.0
        s2 = self.sigma2_R(8.0)
        self.A = sigma8 * sigma8 / s2

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        T = eh_nowiggle_transfer(k, self.omega_m, self.omega_b, self.h, self.T_cmb)
        return self.A * k ** self.n_s * T * T

    def sigma2_R(self, R):
        """sigma^2(R) = (1/2pi^2) int k^3 P(k) W(kR)^2 dln k."""
        return _simpson_lnk(lambda k: k ** 3 * self(k) * tophat_window(k * R) ** 2) / (2.0 * np.pi ** 2)

    def sigma_v(self, f_growth):
        """1-D linear velocity dispersion, km/s:
        sigma_v^2 = (H0 f)^2/(6 pi^2) int P(k) dk."""
        I = _simpson_lnk(lambda k: k * self(k))
        return math.sqrt((H0 * f_growth) ** 2 * I / (6.0 * np.pi ** 2))


def growth_rate(omega_m, f_growth=-1.0):
    return f_growth if f_growth > 0 else omega_m ** 0.55


# ----------------------------------------------------------------------------
# Point functions (section "The Likelihood function: distances/velocities").
# ----------------------------------------------------------------------------
def zbar(d, omega_m):
    """Second-order cosmological redshift of proper distance d (Mpc/h):
    zbar = 2/(3 Om) (1 - sqrt(1 - 3 Om H0 d / c))."""
    return 2.0 / (3.0 * omega_m) * (1.0 - np.sqrt(1.0 - 3.0 * omega_m * H0 * d / C_KMS))


def zbar_prime(d, omega_m):
    return (H0 / C_KMS) / np.sqrt(1.0 - 3.0 * omega_m * H0 * d / C_KMS)


def distance_modulus(d, omega_m, h):
    """mu = 5 log10(d_L / 10 pc), d_L = d (1 + zbar) in Mpc/h -> d_L/h Mpc."""
    return 5.0 * np.log10(d * (1.0 + zbar(d, omega_m)) / h) + 25.0


def distance_modulus_prime(d, omega_m):
    zb = zbar(d, omega_m)
    return 5.0 / np.log(10.0) * (1.0 / d + zbar_prime(d, omega_m) / (1.0 + zb))


def v_observed(z, d, omega_m):
    """Observed radial velocity (eq. vrobs): c (z - zbar)/(1 + zbar)."""
    zb = zbar(d, omega_m)
    return C_KMS * (z - zb) / (1.0 + zb)


def v_observed_prime(z, d, omega_m):
    zb = zbar(d, omega_m)
    return -C_KMS * zbar_prime(d, omega_m) * (1.0 + z) / (1.0 + zb) ** 2


def kappa2(d, sigma_nl, sigma_cz, omega_m):
    """eq. kappa: kappa^2 = sigma_NL^2 + sigma_cz^2/(1 + zbar)^2."""
    zb = zbar(d, omega_m)
    return sigma_nl * sigma_nl + sigma_cz * sigma_cz / (1.0 + zb) ** 2


def kappa2_prime(d, sigma_cz, omega_m):
    zb = zbar(d, omega_m)
    return -2.0 * sigma_cz * sigma_cz * zbar_prime(d, omega_m) / (1.0 + zb) ** 3


# ----------------------------------------------------------------------------
# The problem: grid, cosmology, catalogue, distance prior.
# ----------------------------------------------------------------------------
class Problem:
    """Everything the posterior depends on besides (w, d).

    prior: ("dz", bin_width, pad) -- eq. D built from the catalogue's observed
    redshifts by eq. e:dz (dz_prior_table; bin_width <= 0 means 5 Mpc/h,
    pad <= 0 means 3 sigma_v/H0), stored as the equivalent table;
    ("table", d0, bin_width, logdens array) or ("power", alpha, dmin, dmax).
    """

    def __init__(self, N, L, cosmo, sigma_nl, rhat, mu, sigma_mu, cz, sigma_cz,
                 prior, observer=None):
        self.N = int(N)
        self.L = float(L)
        self.delta = self.L / self.N
        self.observer = np.full(3, self.L / 2.0) if observer is None else np.asarray(observer, float)
        c = dict(cosmo)
        self.omega_m = c.get("omega_m", 0.3)
        self.h = c.get("h", 0.7)
        self.pk = PowerSpectrum(self.omega_m, c.get("omega_b", 0.05), self.h,
                                c.get("n_s", 0.96), c.get("sigma8", 0.8), c.get("T_cmb", 2.7255))
        self.f = growth_rate(self.omega_m, c.get("f_growth", -1.0))
        self.aHf = 1.0 * H0 * self.f          # a = 1 at z = 0
        self.sigma_v = self.pk.sigma_v(self.f)
        self.minv_d = (self.sigma_v / H0) ** 2  # eq. M_ab: sigma_v^2/H0^2 for distances
        self.sigma_nl = float(sigma_nl)
        self.rhat = np.asarray(rhat, float).reshape(-1, 3)
        self.mu = np.asarray(mu, float)
        self.sigma_mu = np.asarray(sigma_mu, float)
        self.cz = np.asarray(cz, float)
        self.z = self.cz / C_KMS
        self.sigma_cz = np.asarray(sigma_cz, float)
        if prior[0] == "dz":
            bw = prior[1] if prior[1] > 0 else 5.0
            pad = prior[2] if prior[2] > 0 else 3.0 * self.sigma_v / H0
            prior = ("table", 0.0, bw, dz_prior_table(self.cz, self.omega_m, bw, pad)) if self.cz.size else \
                ("table", 0.0, bw, np.zeros(1))
        self.prior = prior
        self.n = self.mu.shape[0]
        self._D = None

    # -- Fourier side -------------------------------------------------------
    def mode_numbers(self):
        """Signed integer mode numbers n_j on the full DFT grid (numpy order)."""
        N = self.N
        n1 = np.fft.fftfreq(N, d=1.0 / N)        # 0..N/2-1, -N/2..-1
        nx, ny, nz = np.meshgrid(n1, n1, n1, indexing="ij")
        return nx, ny, nz

    def colour_amplitude(self):
        """sqrt(P(|k|)/Delta^3) per mode, 0 at k = 0."""
        nx, ny, nz = self.mode_numbers()
        kmag = 2.0 * np.pi / self.L * np.sqrt(nx ** 2 + ny ** 2 + nz ** 2)
        amp = np.zeros_like(kmag)
        nz0 = kmag > 0
        amp[nz0] = np.sqrt(self.pk(kmag[nz0]) / self.delta ** 3)
        return amp

    def velocity_factors(self):
        """The three imaginary factors i aHf k_j^odd / k^2 of eq. vel-field
        (k_j^odd = 0 on the Nyquist plane of axis j), 0 at k = 0."""
        N = self.N
        nx, ny, nz = self.mode_numbers()
        k2 = (2.0 * np.pi / self.L) ** 2 * (nx ** 2 + ny ** 2 + nz ** 2)
        out = []
        for nj in (nx, ny, nz):
            kj = 2.0 * np.pi / self.L * np.where(np.abs(nj) == N // 2, 0.0, nj)
            fac = np.zeros(k2.shape, dtype=np.complex128)
            m = k2 > 0
            fac[m] = 1j * self.aHf * kj[m] / k2[m]
            out.append(fac)
        return out

    def operator_D(self):
        """D_j = velocity factor * colour amplitude (w-hat -> v_j-hat)."""
        if self._D is None:
            amp = self.colour_amplitude()
            self._D = [fj * amp for fj in self.velocity_factors()]
        return self._D


# ----------------------------------------------------------------------------
# Field maps.
# ----------------------------------------------------------------------------
def dft3_naive(x, sign=-1):
    """Plain O(N^6) 3D DFT sum_x x(r) e^{sign i 2pi n.r/N} (tiny grids only)."""
    N = x.shape[0]
    idx = np.arange(N)
    E = np.exp(sign * 2j * np.pi * np.outer(idx, idx) / N)
    out = np.zeros((N, N, N), dtype=np.complex128)
    for a in range(N):
        for b in range(N):
            for c in range(N):
                out[a, b, c] = np.sum(x * E[a][:, None, None] * E[b][None, :, None] * E[c][None, None, :])
    return out


def delta_k(prob, w):
    """Colouring: delta_k = sqrt(P/Delta^3) DFT(w)."""
    return prob.colour_amplitude() * np.fft.fftn(w)


def velocity_from_delta_k(prob, dk):
    """Linear velocity (eq. vel-field): v_j = IDFT(i aHf k_j/k^2 delta_k)."""
    return np.stack([np.fft.ifftn(f * dk).real for f in prob.velocity_factors()])


def velocity_field(prob, w):
    """v_j = IDFT(D_j DFT(w)) for j = x, y, z (shape (3, N, N, N))."""
    return velocity_from_delta_k(prob, delta_k(prob, w))


def velocity_adjoint(prob, s):
    """Adjoint of w -> v: sum_j IDFT(conj(D_j) DFT(s_j)) (real part)."""
    D = prob.operator_D()
    acc = np.zeros(s.shape[1:], dtype=np.complex128)
    for j in range(3):
        acc += np.conj(D[j]) * np.fft.fftn(s[j])
    return np.fft.ifftn(acc).real


# ----------------------------------------------------------------------------
# Cloud-in-cell interpolation.
# ----------------------------------------------------------------------------
def cic_cells(prob, d):
    """Lower-corner cell (n,3 int) and fractional offsets (n,3) of the points
    x_i = o + d_i rhat_i.  t = x/Delta is formed as (o + d*r)/Delta with one
    rounding per operation; cell = floor(t) mod N, frac = t - floor(t)."""
    x = prob.observer[None, :] + d[:, None] * prob.rhat
    t = x / prob.delta
    fl = np.floor(t)
    frac = t - fl
    cell = np.mod(fl.astype(np.int64), prob.N)
    return cell, frac


def cell_sort_order(prob, d):
    """Stable order of the points by linear cell index (ix*N + iy)*N + iz."""
    cell, _ = cic_cells(prob, d)
    N = prob.N
    lin = (cell[:, 0] * N + cell[:, 1]) * N + cell[:, 2]
    return lin, np.argsort(lin, kind="stable")


def _corners():
    return list(itertools.product((0, 1), repeat=3))


def cic_gather(prob, grid, cell, frac):
    """Trilinear value and spatial gradient of one grid at the points."""
    N = prob.N
    val = np.zeros(cell.shape[0])
    grad = np.zeros((cell.shape[0], 3))
    for a, b, c in _corners():
        w = [frac[:, 0] if a else 1.0 - frac[:, 0],
             frac[:, 1] if b else 1.0 - frac[:, 1],
             frac[:, 2] if c else 1.0 - frac[:, 2]]
        sgn = [1.0 if a else -1.0, 1.0 if b else -1.0, 1.0 if c else -1.0]
        g = grid[(cell[:, 0] + a) % N, (cell[:, 1] + b) % N, (cell[:, 2] + c) % N]
        val += w[0] * w[1] * w[2] * g
        grad[:, 0] += sgn[0] * w[1] * w[2] * g / prob.delta
        grad[:, 1] += sgn[1] * w[0] * w[2] * g / prob.delta
        grad[:, 2] += sgn[2] * w[0] * w[1] * g / prob.delta
    return val, grad


def cic_scatter(prob, values, cell, frac):
    """Adjoint of the gather: grid += value * W(corner) (np.add.at)."""
    N = prob.N
    grid = np.zeros((N, N, N))
    for a, b, c in _corners():
        w = ((frac[:, 0] if a else 1.0 - frac[:, 0]) *
             (frac[:, 1] if b else 1.0 - frac[:, 1]) *
             (frac[:, 2] if c else 1.0 - frac[:, 2]))
        np.add.at(grid, ((cell[:, 0] + a) % N, (cell[:, 1] + b) % N, (cell[:, 2] + c) % N), values * w)
    return grid


# ----------------------------------------------------------------------------
# Distance prior (eq. D).
# ----------------------------------------------------------------------------
def log_prior_d(prob, d):
    """ln pi_D(d) and its derivative; -inf outside the support.

    "table": the histogram of eq. D, read as ln pi given at the bin centres
    d0 + (b + 1/2) bin and interpolated linearly between them (flat in the
    outer half bins), so that the potential is continuous in d; the support
    is [d0, d0 + nbins * bin).  "power": ln pi = alpha ln d on [dmin, dmax].
    """
    kind = prob.prior[0]
    if kind == "table":
        _, d0, bw, logdens = prob.prior
        logdens = np.asarray(logdens, float)
        nb = logdens.shape[0]
        ok = (d >= d0) & (d < d0 + nb * bw)
        t = (d - d0) / bw - 0.5
        b = np.floor(t)
        f = t - b
        lo = np.clip(b, 0, nb - 1).astype(np.int64)
        hi = np.clip(b + 1, 0, nb - 1).astype(np.int64)
        inner = (b >= 0) & (b < nb - 1)
        lp = np.where(inner, (1.0 - f) * logdens[lo] + f * logdens[hi], logdens[np.where(b < 0, 0, nb - 1)])
        dl = np.where(inner, (logdens[hi] - logdens[lo]) / bw, 0.0)
        lp = np.where(ok, lp, -np.inf)
        dl = np.where(ok, dl, 0.0)
        return lp, dl
    if kind == "power":
        _, alpha, dmin, dmax = prob.prior
        ok = (d >= dmin) & (d <= dmax)
        lp = np.full(d.shape, -np.inf)
        dl = np.zeros(d.shape)
        lp[ok] = alpha * np.log(d[ok])
        dl[ok] = alpha / d[ok]
        return lp, dl
    raise ValueError(kind)


DZ_SIMPSON_INTERVALS = 64


def redshift_distance(z, omega_m):
    """eq. e:dz: d_z = (c/H0) int_0^z dz'/sqrt(Om (1+z')^3 + 1 - Om), Mpc/h;
    composite Simpson with DZ_SIMPSON_INTERVALS intervals on [0, z]."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    out = np.empty_like(z)
    n = DZ_SIMPSON_INTERVALS
    wts = np.ones(n + 1)
    wts[1:-1:2] = 4.0
    wts[2:-1:2] = 2.0
    for i, zi in enumerate(z):
        x = np.linspace(0.0, zi, n + 1)
        f = 1.0 / np.sqrt(omega_m * (1.0 + x) ** 3 + 1.0 - omega_m)
        out[i] = C_KMS / H0 * (zi / n) / 3.0 * float(np.sum(wts * f))
    return out


def dz_prior_table(cz, omega_m, bin_width, pad):
    """eq. D: histogram of the observed redshift distances on [0, max d_z +
    pad) in bins of bin_width, each count + 0.5, normalised to a density;
    returns ln density per bin (the table the distance prior interpolates)."""
    dz = redshift_distance(np.maximum(np.asarray(cz, float), 0.0) / C_KMS, omega_m)
    nb = int(np.ceil((dz.max() + pad) / bin_width))
    counts = np.zeros(nb)
    b = np.minimum((dz / bin_width).astype(np.int64), nb - 1)
    np.add.at(counts, b, 1.0)
    dens = (counts + 0.5) / ((counts + 0.5).sum() * bin_width)
    return np.log(dens)


def in_domain(prob, d):
    """d > 0 and 1 - 3 Om H0 d / c > 0 (zbar real)."""
    return (d > 0) & (1.0 - 3.0 * prob.omega_m * H0 * d / C_KMS > 0)


# ----------------------------------------------------------------------------
# Posterior: Psi = -ln Pi (eq. Psi) and its gradient.
# ----------------------------------------------------------------------------
def point_terms(prob, d, u, du, sigma_nl=None):
    """Per-point Psi_i, r_i = dPsi_i/du_i and dPsi_i/dd_i (u' = du given);
    sigma_nl overrides the problem's value (sampled sigma_NL)."""
    psi_i, r, gd, _ = point_terms_s(prob, d, u, du, sigma_nl)
    return psi_i, r, gd


def point_terms_s(prob, d, u, du, sigma_nl=None):
    """point_terms plus dPsi_i/dsigma_NL = (sigma/kappa^2)(1 - (v_obs-u)^2/kappa^2)."""
    snl = prob.sigma_nl if sigma_nl is None else float(sigma_nl)
    om = prob.omega_m
    ok = in_domain(prob, d)
    dd = np.where(ok, d, 1.0)
    mu_d = distance_modulus(dd, om, prob.h)
    mup = distance_modulus_prime(dd, om)
    vo = v_observed(prob.z, dd, om)
    vop = v_observed_prime(prob.z, dd, om)
    k2 = kappa2(dd, snl, prob.sigma_cz, om)
    k2p = kappa2_prime(dd, prob.sigma_cz, om)
    lp, dlp = log_prior_d(prob, dd)
    res_mu = prob.mu - mu_d
    res_v = vo - u
    psi_i = (res_mu ** 2 / (2.0 * prob.sigma_mu ** 2) + res_v ** 2 / (2.0 * k2)
             + 0.5 * np.log(k2) - lp)
    r = -res_v / k2
    gd = (-res_mu * mup / prob.sigma_mu ** 2 + res_v * (vop - du) / k2
          - res_v ** 2 * k2p / (2.0 * k2 * k2) + k2p / (2.0 * k2) - dlp)
    gs = snl / k2 * (1.0 - res_v ** 2 / k2)
    psi_i = np.where(ok, psi_i, np.inf)
    r = np.where(ok & np.isfinite(psi_i), r, 0.0)
    gd = np.where(ok & np.isfinite(psi_i), gd, 0.0)
    gs = np.where(ok & np.isfinite(psi_i), gs, 0.0)
    return psi_i, r, gd, gs


def predicted_u(prob, v, d):
    """u_i = rhat_i . v(o + d_i rhat_i) and its d-derivative."""
    cell, frac = cic_cells(prob, d)
    u = np.zeros(prob.n)
    du = np.zeros(prob.n)
    for j in range(3):
        val, grad = cic_gather(prob, v[j], cell, frac)
        u += prob.rhat[:, j] * val
        du += prob.rhat[:, j] * np.sum(grad * prob.rhat, axis=1)
    return u, du, cell, frac


def logpost(prob, w, d):
    psi, _, _ = logpost_grad(prob, w, d)
    return psi


def logpost_grad(prob, w, d):
    """Psi(w, d) = |w|^2/2 + sum_i [ (mu_i - mu(d_i))^2/(2 s_mu^2)
    + (v_obs(d_i) - u_i)^2/(2 kappa^2) + ln kappa - ln pi_D(d_i) ],
    with its gradient (dPsi/dw, dPsi/dd).  Follows eqs. covfefe:bay,
    likelihood, lmu, vrobs, vel-field, lvr, kappa, prior-k (whitened), D, Psi.
    """
    w = np.asarray(w, float)
    d = np.asarray(d, float)
    v = velocity_field(prob, w)
    u, du, cell, frac = predicted_u(prob, v, d)
    psi_i, r, gd = point_terms(prob, d, u, du)
    psi = 0.5 * float(np.sum(w * w)) + float(np.sum(psi_i))
    s = np.stack([cic_scatter(prob, r * prob.rhat[:, j], cell, frac) for j in range(3)])
    gw = w + velocity_adjoint(prob, s)
    return psi, gw, gd


def logpost_grad_s(prob, w, d, sigma_nl):
    """Psi and its gradient with sigma_NL as a parameter of q (eq. q): flat
    prior on sigma_NL > 0 (the paper gives none), Psi = +inf for sigma_NL <= 0.
    Returns (psi, dPsi/dw, dPsi/dd, dPsi/dsigma_NL)."""
    w = np.asarray(w, float)
    d = np.asarray(d, float)
    if not sigma_nl > 0:
        return np.inf, np.zeros_like(w), np.zeros_like(d), 0.0
    v = velocity_field(prob, w)
    u, du, cell, frac = predicted_u(prob, v, d)
    psi_i, r, gd, gs = point_terms_s(prob, d, u, du, sigma_nl)
    psi = 0.5 * float(np.sum(w * w)) + float(np.sum(psi_i))
    s = np.stack([cic_scatter(prob, r * prob.rhat[:, j], cell, frac) for j in range(3)])
    gw = w + velocity_adjoint(prob, s)
    return psi, gw, gd, float(np.sum(gs))


def leapfrog_s(prob, w, d, s, pw, pd, ps, eps, n_steps):
    """Kick-drift-kick leapfrog of (w, d, sigma_NL) with unit mass on
    sigma_NL (eq. M_ab).  Returns (w, d, s, pw, pd, ps, psi)."""
    w = np.array(w, float, copy=True)
    d = np.array(d, float, copy=True)
    pw = np.array(pw, float, copy=True)
    pd = np.array(pd, float, copy=True)
    psi, gw, gd, gs = logpost_grad_s(prob, w, d, s)
    pw -= 0.5 * eps * gw
    pd -= 0.5 * eps * gd
    ps -= 0.5 * eps * gs
    for l in range(n_steps):
        w += eps * pw
        d += eps * prob.minv_d * pd
        s += eps * ps
        psi, gw, gd, gs = logpost_grad_s(prob, w, d, s)
        c = eps if l < n_steps - 1 else 0.5 * eps
        pw -= c * gw
        pd -= c * gd
        ps -= c * gs
    return w, d, s, pw, pd, ps, psi


def data_gradient_w(prob, d, r):
    """A^T r: the field gradient produced by point residuals r (fixed d)."""
    cell, frac = cic_cells(prob, d)
    s = np.stack([cic_scatter(prob, r * prob.rhat[:, j], cell, frac) for j in range(3)])
    return velocity_adjoint(prob, s)


def forward_u(prob, w, d):
    """A w: predicted radial velocities for the field w at distances d."""
    v = velocity_field(prob, w)
    u, _, _, _ = predicted_u(prob, v, d)
    return u


# ----------------------------------------------------------------------------
# Hamiltonian Monte Carlo (sections "Hamiltonian trajectories", "Construction
# of HMC chains", "Integrating the HMC trajectories", "The Mass matrix").
# ----------------------------------------------------------------------------
def kinetic(prob, pw, pd):
    """p^T M^-1 p / 2 with M^-1 = I on w and (sigma_v/H0)^2 on d."""
    return 0.5 * float(np.sum(pw * pw)) + 0.5 * prob.minv_d * float(np.sum(pd * pd))


def leapfrog(prob, w, d, pw, pd, eps, n_steps, sample_d=True, grad0=None):
    """Kick-drift-kick leapfrog with consecutive half kicks merged.
    Returns (w, d, pw, pd, psi, gw, gd) at the end point."""
    w = np.array(w, float, copy=True)
    d = np.array(d, float, copy=True)
    pw = np.array(pw, float, copy=True)
    pd = np.array(pd, float, copy=True)
    if grad0 is None:
        psi, gw, gd = logpost_grad(prob, w, d)
    else:
        psi, gw, gd = grad0
    pw -= 0.5 * eps * gw
    if sample_d:
        pd -= 0.5 * eps * gd
    for l in range(n_steps):
        w += eps * pw
        if sample_d:
            d += eps * prob.minv_d * pd
        psi, gw, gd = logpost_grad(prob, w, d)
        c = eps if l < n_steps - 1 else 0.5 * eps
        pw -= c * gw
        if sample_d:
            pd -= c * gd
    return w, d, pw, pd, psi, gw, gd


def draw_momenta(prob, seed, traj, chain):
    """p_w ~ N(0, I), p_d ~ N(0, (H0/sigma_v)^2) from the Philox streams."""
    N = prob.N
    pw = philox_normals(N ** 3, seed, traj, chain, TAG_FIELD).reshape(N, N, N)
    pd = philox_normals(prob.n, seed, traj, chain, TAG_DIST) / math.sqrt(prob.minv_d)
    return pw, pd


def hmc_trajectory(prob, w, d, psi_grad, seed, traj, chain, eps, n_steps, sample_d=True):
    """One HMC transition: fresh momenta, leapfrog, Metropolis test.
    Returns (w, d, psi_grad, record dict)."""
    pw, pd = draw_momenta(prob, seed, traj, chain)
    if not sample_d:
        pd = np.zeros_like(pd)
    psi0 = psi_grad[0]
    H_old = psi0 + kinetic(prob, pw, pd)
    w1, d1, pw1, pd1, psi1, gw1, gd1 = leapfrog(prob, w, d, pw, pd, eps, n_steps,
                                                sample_d=sample_d, grad0=psi_grad)
    H_new = psi1 + kinetic(prob, pw1, pd1)
    logu = philox_accept_logu(seed, traj, chain)
    accept = bool(np.isfinite(H_new) and logu < H_old - H_new)
    rec = dict(H_old=H_old, H_new=H_new, logu=logu, accept=accept, psi=psi1 if accept else psi0)
    if accept:
        return w1, d1, (psi1, gw1, gd1), rec
    return w, d, psi_grad, rec


def run_chain(prob, w, d, seed, chain, traj0, n_traj, eps, n_steps, sample_d=True):
    """n_traj HMC transitions from (w, d); trajectory counters traj0.."""
    psi_grad = logpost_grad(prob, w, d)
    recs = []
    for t in range(n_traj):
        w, d, psi_grad, rec = hmc_trajectory(prob, w, d, psi_grad, seed, traj0 + t, chain,
                                             eps, n_steps, sample_d)
        recs.append(rec)
    return w, d, recs


# ----------------------------------------------------------------------------
# Step-size tuning by dual averaging (section "Integrating the HMC
# trajectories": the step size is tuned to a target acceptance of 0.65 with
# the dual-averaging scheme of Hoffman & Gelman).  After trajectory m with
# acceptance probability alpha_m = min(1, exp(H_old - H_new)):
#   Hbar_m = (1 - 1/(m + t0)) Hbar_{m-1} + (delta - alpha_m)/(m + t0)
#   log eps_m = mu - sqrt(m)/gamma * Hbar_m
#   log epsbar_m = m^-kappa log eps_m + (1 - m^-kappa) log epsbar_{m-1}
# with mu = log(10 eps_0), Hbar_0 = 0, log epsbar_0 = 0; the tuned step is
# epsbar at the end of the warm-up.
# ----------------------------------------------------------------------------
DA_GAMMA = 0.05
DA_T0 = 10.0
DA_KAPPA = 0.75


def accept_probability(H_old, H_new):
    if not np.isfinite(H_new):
        return 0.0
    return float(min(1.0, math.exp(min(0.0, H_old - H_new))))


class DualAveraging:
    def __init__(self, eps0, delta=0.65):
        self.mu = math.log(10.0 * eps0)
        self.delta = delta
        self.m = 0
        self.Hbar = 0.0
        self.log_eps = math.log(eps0)
        self.log_eps_bar = 0.0

    def update(self, alpha):
        self.m += 1
        m = float(self.m)
        w = 1.0 / (m + DA_T0)
        self.Hbar = (1.0 - w) * self.Hbar + w * (self.delta - alpha)
        self.log_eps = self.mu - math.sqrt(m) / DA_GAMMA * self.Hbar
        eta = m ** (-DA_KAPPA)
        self.log_eps_bar = eta * self.log_eps + (1.0 - eta) * self.log_eps_bar
        return math.exp(self.log_eps)

    @property
    def eps(self):
        return math.exp(self.log_eps)

    @property
    def eps_bar(self):
        return math.exp(self.log_eps_bar)


def adapt_step_size(prob, w, d, seed, chain, traj0, n_warmup, eps0, n_steps, delta=0.65, sample_d=True):
    """n_warmup HMC transitions with the step size adapted after each one;
    returns (w, d, eps_bar, records with the step used)."""
    da = DualAveraging(eps0, delta)
    psi_grad = logpost_grad(prob, w, d)
    recs = []
    eps = eps0
    for t in range(n_warmup):
        w, d, psi_grad, rec = hmc_trajectory(prob, w, d, psi_grad, seed, traj0 + t, chain, eps, n_steps,
                                             sample_d)
        rec["eps"] = eps
        recs.append(rec)
        eps = da.update(accept_probability(rec["H_old"], rec["H_new"]))
    return w, d, da.eps_bar, recs


# ----------------------------------------------------------------------------
# Dense Wiener filter for fixed distances (the posterior is then Gaussian).
# ----------------------------------------------------------------------------
def response_matrix(prob, d):
    """A (n x N^3): u = A w at fixed d, assembled column by column from the
    translation-invariant impulse response of w -> v (the response of the
    field e_0 shifted to every node)."""
    N = prob.N
    e0 = np.zeros((N, N, N))
    e0[0, 0, 0] = 1.0
    K = velocity_field(prob, e0)            # v_j response to a unit node at 0
    cell, frac = cic_cells(prob, d)
    A = np.zeros((prob.n, N ** 3))
    ar = np.arange(N)
    for a, b, c in _corners():
        wgt = ((frac[:, 0] if a else 1.0 - frac[:, 0]) *
               (frac[:, 1] if b else 1.0 - frac[:, 1]) *
               (frac[:, 2] if c else 1.0 - frac[:, 2]))
        gx = (cell[:, 0] + a) % N
        gy = (cell[:, 1] + b) % N
        gz = (cell[:, 2] + c) % N
        # v_j(g) from unit field at m equals K_j(g - m)
        for j in range(3):
            Kj = K[j]
            ix = (gx[:, None] - ar[None, :]) % N
            iy = (gy[:, None] - ar[None, :]) % N
            iz = (gz[:, None] - ar[None, :]) % N
            block = Kj[ix[:, :, None, None], iy[:, None, :, None], iz[:, None, None, :]]
            A += (wgt * prob.rhat[:, j])[:, None] * block.reshape(prob.n, N ** 3)
    return A


def wiener_filter(prob, d):
    """Posterior mean and marginal variances of w at fixed d:
    m = (I + A^T K^-1 A)^-1 A^T K^-1 v_obs, var = diag((I + A^T K^-1 A)^-1)."""
    A = response_matrix(prob, d)
    k2 = kappa2(d, prob.sigma_nl, prob.sigma_cz, prob.omega_m)
    vo = v_observed(prob.z, d, prob.omega_m)
    Aw = A / k2[:, None]
    P = np.eye(A.shape[1]) + A.T @ Aw
    Lc = np.linalg.cholesky(P)
    rhs = A.T @ (vo / k2)
    y = np.linalg.solve(Lc, rhs)
    mean = np.linalg.solve(Lc.T, y)
    Linv = np.linalg.inv(Lc)
    var = np.sum(Linv * Linv, axis=0)
    return mean, var


def problem_from_catalog(spec_N, spec_L, cosmo, sigma_nl, cat, prior=None):
    """Convenience: build a Problem from a mock catalogue dict; the distance
    prior defaults to eq. D from the catalogue's redshifts (section "Priors")."""
    if prior is None:
        prior = ("dz", 0.0, 0.0)
    return Problem(spec_N, spec_L, cosmo, sigma_nl, cat["rhat"], cat["mu"], cat["sigma_mu"],
                   cat["cz"], cat["sigma_cz"], prior)


# ----------------------------------------------------------------------------
# Chain analytics: Monte-Carlo means over chain states (eq. int_mc), the
# convergence monitor (section "Convergence") and the monopole and dipole of
# the velocity field in spheres about the observer (section "Monopole and
# dipole").
# ----------------------------------------------------------------------------
def density_field(prob, w):
    """delta(x) = IDFT(sqrt(P/Delta^3) DFT(w)): the coloured field."""
    return np.fft.ifftn(delta_k(prob, w)).real


def node_offsets(prob):
    """Offsets x - o of the grid nodes (positions i*Delta) from the observer,
    shape (3, N, N, N), and their lengths (no periodic wrap)."""
    i = np.arange(prob.N) * prob.delta
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    off = np.stack([gx - prob.observer[0], gy - prob.observer[1], gz - prob.observer[2]])
    r = np.sqrt(off[0] * off[0] + off[1] * off[1] + off[2] * off[2])
    return off, r


def radial_velocity(prob, v):
    """v_r = rhat . v at every node, rhat the unit vector from the observer
    (v_r = 0 at a node on the observer)."""
    off, r = node_offsets(prob)
    safe = np.where(r > 0, r, 1.0)
    return np.where(r > 0, (off[0] * v[0] + off[1] * v[1] + off[2] * v[2]) / safe, 0.0)


def sample_moments(samples):
    """eq. int_mc: mean of a functional over the n chain states, and the
    sample variance (divisor n - 1; zero for one state)."""
    a = np.stack([np.asarray(x, float) for x in samples])
    n = a.shape[0]
    mean = a.sum(axis=0) / n
    var = ((a - mean) ** 2).sum(axis=0) / (n - 1) if n > 1 else np.zeros_like(mean)
    return mean, var


def convergence_metric(delta_samples):
    """Section "Convergence": the change of <delta>/Sigma_delta between
    successive steps.  m_s = mean of the first s density fields (eq. int_mc),
    Sigma_s^2 = variance over the grid of the s-th field; the field
    m_s/Sigma_s - m_{s-1}/Sigma_{s-1} is summarised by its root mean square
    over the nodes.  Returns the values for s = 2..n (n - 1 of them)."""
    out = []
    m_prev = None
    s_prev = None
    acc = None
    for s, x in enumerate(delta_samples, start=1):
        x = np.asarray(x, float)
        acc = x.copy() if acc is None else acc + x
        m = acc / s
        sig = math.sqrt(float(np.mean(x * x)) - float(np.mean(x)) ** 2)
        if m_prev is not None:
            out.append(math.sqrt(float(np.mean((m / sig - m_prev / s_prev) ** 2))))
        m_prev, s_prev = m, sig
    return np.array(out)


def sphere_moments(prob, delta, v, radii):
    """Section "Monopole and dipole" in spheres |x - o| <= R about the
    observer, over the grid nodes inside: the monopole is the mean of
    -div v / H0, which by linear continuity (div v = -aHf delta, exact per mode
    away from the Nyquist planes) is a f <delta>; the dipole is the mean
    velocity (bulk flow) V.  Returns (R, 5): monopole, V_x, V_y, V_z, |V|."""
    _, r = node_offsets(prob)
    out = np.zeros((len(radii), 5))
    for k, R in enumerate(radii):
        m = r <= R
        cnt = int(m.sum())
        if cnt == 0:
            continue
        V = np.array([v[j][m].sum() / cnt for j in range(3)])
        out[k, 0] = 1.0 * prob.f * delta[m].sum() / cnt
        out[k, 1:4] = V
        out[k, 4] = math.sqrt(float(V @ V))
    return out
