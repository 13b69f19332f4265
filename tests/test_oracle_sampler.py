"""Sampler pin: with the distances held fixed the posterior of the whitened
field is Gaussian, so the oracle's HMC chain must reproduce the dense
Wiener-filter mean and marginal variances (section "Sampling by HMC chains",
eq. int_mc)."""
import numpy as np

from oracle import hamlet_oracle as O
from paper_2203_02369_gb300.ess import ess_columns

COSMO = dict(omega_m=0.3, omega_b=0.05, h=0.7, n_s=0.96, sigma8=0.8, T_cmb=2.7255)


def test_chain_mean_matches_wiener_filter():
    rng = np.random.default_rng(21)
    N, L, n = 8, 64.0, 60
    z = 2 * rng.random(n) - 1
    ph = 2 * np.pi * rng.random(n)
    s = np.sqrt(1 - z * z)
    rhat = np.stack([s * np.cos(ph), s * np.sin(ph), z], 1)
    d = 25 * (0.2 + 0.8 * rng.random(n))
    p = O.Problem(N, L, COSMO, 150.0, rhat, 5 * np.log10(d / 0.7) + 25, np.full(n, 0.2),
                  100 * d + 300 * rng.normal(size=n), np.zeros(n), ("power", 2.0, 0.5, 60))
    mean, var = O.wiener_filter(p, d)
    assert var.min() < 0.8          # the data constrain some modes
    w = np.zeros((N, N, N))
    pg = O.logpost_grad(p, w, d)
    S = []
    acc = 0
    for t in range(700):
        w, _, pg, rec = O.hmc_trajectory(p, w, d, pg, seed=1, traj=t, chain=0,
                                         eps=0.35, n_steps=6, sample_d=False)
        acc += rec["accept"]
        S.append(w.ravel().copy())
    S = np.array(S[100:])
    assert 0.3 < acc / 700 < 1.0
    cols = np.arange(0, N ** 3, 4)
    e = ess_columns(S[:, cols])
    zsc = (S[:, cols].mean(0) - mean[cols]) / np.sqrt(var[cols] / e)
    assert np.mean(np.abs(zsc) < 4) > 0.95
    ratio = S[:, cols].var(0) / var[cols]
    assert abs(np.median(ratio) - 1) < 0.15
