"""Seeded synthetic peculiar-velocity catalogues shaped like the paper's mocks.

This module is the ONE input source shared by the CUDA path and the CPU oracle.
It holds none of the posterior's arithmetic: it only draws random numbers with
the shapes, sizes and distributions of the paper's mock surveys (section
"Mock Catalogue construction": observer at the box centre, isotropic
directions, a radial cut at 160 Mpc/h, 7.5k-30k points; the presets below
-- 16^3, 64^3 and 128^3 workloads and the batched catalogues -- fix the rest) and turns them into observables with first-order,
textbook relations (luminosity distance ~ distance, cz ~ H0 d + v_pec).  The
posterior absorbs that small mismatch with its own second-order relations.

Units: lengths in Mpc/h, velocities in km/s, H0 = 100 km/s/(Mpc/h).
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
import numpy as np

C_KMS = 299792.458
H0 = 100.0


@dataclass
class Cosmology:
    """LCDM parameters of the prior power spectrum (Eisenstein-Hu no-wiggle)."""
    omega_m: float = 0.3
    omega_b: float = 0.05
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    T_cmb: float = 2.7255
    f_growth: float = -1.0  # <= 0 means Omega_m**0.55


@dataclass
class MockSpec:
    """One synthetic catalogue plus the grid it is reconstructed on."""
    N: int
    L: float
    n_points: int
    r_max: float
    mask_deg: float          # |b| < mask_deg removed (0 = no mask)
    sigma_mu: tuple          # (lo, hi); lo == hi means fixed
    sigma_nl: float
    seed: int
    precision: str = "fp32"  # "fp32" (FP32 fields, FP64 energy) or "fp64"
    cosmo: Cosmology = field(default_factory=Cosmology)
    prior_bin: float = 5.0   # bin width (Mpc/h) of the distance prior's redshift-distance histogram


# Presets with the sizes of the paper's mocks (section "Mock Catalogue
# construction"), the rest fixed for these workloads.
PRESETS = {
    "grid16_500pts_fp64": MockSpec(N=16, L=200.0, n_points=500, r_max=80.0, mask_deg=0.0,
                        sigma_mu=(0.2, 0.2), sigma_nl=150.0, seed=0, precision="fp64"),
    "grid64_5000pts": MockSpec(N=64, L=500.0, n_points=5000, r_max=160.0, mask_deg=10.0,
                        sigma_mu=(0.2, 0.45), sigma_nl=250.0, seed=1),
    "grid128_30000pts": MockSpec(N=128, L=500.0, n_points=30000, r_max=160.0, mask_deg=10.0,
                         sigma_mu=(0.2, 0.45), sigma_nl=250.0, seed=2),
}


def batch_presets():
    """Eight catalogues, sizes log-spaced 2,000-30,000 points, seeds 100..107;
    even ones on 128^3, odd ones on 64^3 (box 500 Mpc/h)."""
    sizes = np.round(np.logspace(np.log10(2000), np.log10(30000), 8)).astype(int)
    out = []
    for i, n in enumerate(sizes):
        out.append(MockSpec(N=128 if i % 2 == 0 else 64, L=500.0, n_points=int(n),
                            r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                            sigma_nl=250.0, seed=100 + i))
    return out


def _directions(rng, n, mask_deg):
    """Unit vectors uniform on the sphere, rejecting |b| < mask_deg where the
    latitude b is measured from the grid's x-y plane (b = asin(z))."""
    out = np.empty((0, 3))
    smask = np.sin(np.deg2rad(mask_deg)) if mask_deg > 0 else -1.0
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        z = 2.0 * rng.random(m) - 1.0
        phi = 2.0 * np.pi * rng.random(m)
        s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        v = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
        if mask_deg > 0:
            v = v[np.abs(z) >= smask]
        out = np.concatenate([out, v], axis=0)
    out = out[:n]
    # renormalise so |rhat| == 1 to rounding
    out /= np.linalg.norm(out, axis=1, keepdims=True)
    return out


def _smooth_flow(rng, x, n_waves=8):
    """A random smooth peculiar-velocity field evaluated at positions x (n,3):
    a bulk flow plus longitudinal plane waves of wavelength 60-300 Mpc/h."""
    bulk = rng.normal(0.0, 200.0, size=3)
    v = np.broadcast_to(bulk, x.shape).copy()
    for _ in range(n_waves):
        khat = _directions(rng, 1, 0.0)[0]
        lam = rng.uniform(60.0, 300.0)
        k = 2.0 * np.pi / lam * khat
        amp = rng.normal(0.0, 150.0)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        v += amp * np.sin(x @ k + ph)[:, None] * khat[None, :]
    return v


def make_catalog(spec: MockSpec):
    """Draw one catalogue.  Returns a dict of float64 numpy arrays:

    rhat (n,3) unit directions, d_true (n,), mu (n,), sigma_mu (n,),
    cz (n,) km/s, sigma_cz (n,) (zeros), d_init (n,) starting distances.
    """
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    n = spec.n_points
    rhat = _directions(rng, n, spec.mask_deg)
    d_true = spec.r_max * rng.random(n) ** (1.0 / 3.0)     # density ~ r^2
    d_true = np.maximum(d_true, 1.0)
    lo, hi = spec.sigma_mu
    sigma_mu = np.full(n, lo) if lo == hi else rng.uniform(lo, hi, n)
    h = spec.cosmo.h
    # first-order observables: d_L ~ d, cz ~ H0 d + v_pec
    mu = 5.0 * np.log10(d_true / h) + 25.0 + sigma_mu * rng.normal(size=n)
    x = d_true[:, None] * rhat
    vr = np.sum(_smooth_flow(rng, x) * rhat, axis=1)
    cz = H0 * d_true + vr + spec.sigma_nl * rng.normal(size=n)
    sigma_cz = np.zeros(n)
    # chains start at the redshift-distance proxy cz/H0, kept off the observer
    d_init = np.maximum(cz / H0, 0.5 * spec.prior_bin)
    return dict(rhat=np.ascontiguousarray(rhat), d_true=d_true, mu=mu,
                sigma_mu=sigma_mu, cz=cz, sigma_cz=sigma_cz, d_init=d_init)


def white_field(N, seed):
    """A seeded N^3 white-noise field (float64), unit variance per node."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((N, N, N))


def spec_dict(spec: MockSpec):
    d = asdict(spec)
    return d
