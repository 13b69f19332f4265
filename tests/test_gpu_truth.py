"""Recovery of a known truth by the GPU chain.

The shared input generator (mock.py) may hold none of the method's
arithmetic, so it cannot draw data from the model itself; here, in a test,
the oracle does: a whitened truth field w_true is coloured (eq. prior-k),
turned into the linear velocity field (eq. vel-field) and interpolated at the
true distances (CIC), and the catalogue's observables are drawn around the
model's own relations -- mu = mu(d_true) + sigma_mu N (eq. lmu) and
cz = c [zbar + (1 + zbar)(u_true + sigma_NL N)/c] (the inverse of eq. vrobs).
The GPU chain (FP32 fields, distances sampled, the distance prior of eq. D
from these redshifts) then runs from w = 0, d = cz/H0; its posterior-mean
radial velocity field (eq. int_mc, on the device) must follow the truth's
inside the surveyed sphere and not an unrelated field's.
"""
import numpy as np
import pytest
import torch

from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu


def _corr(a, b):
    a = a - a.mean()
    b = b - b.mean()
    return float(np.sum(a * b) / np.sqrt(np.sum(a * a) * np.sum(b * b)))


def test_chain_mean_velocity_follows_the_truth():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300.hamlet import Problem, State
    N, L, n, snl = 64, 500.0, 5000, 250.0
    spec = mock.MockSpec(N=N, L=L, n_points=n, r_max=160.0, mask_deg=10.0, sigma_mu=(0.2, 0.45), sigma_nl=snl,
                         seed=41)
    cat = mock.make_catalog(spec)           # directions, true distances and sigma_mu only
    cosmo = mock.spec_dict(spec)["cosmo"]
    rhat, d_true, smu = cat["rhat"], cat["d_true"], cat["sigma_mu"]
    base = O.Problem(N, L, cosmo, snl, rhat, np.zeros(n), smu, np.zeros(n), np.zeros(n), ("power", 2.0, 0.5, 240.0))
    w_true = mock.white_field(N, 4242)
    v_true = O.velocity_field(base, w_true)
    u_true, _, _, _ = O.predicted_u(base, v_true, d_true)
    rng = np.random.default_rng(7)
    mu = O.distance_modulus(d_true, base.omega_m, base.h) + smu * rng.normal(size=n)
    zb = O.zbar(d_true, base.omega_m)
    cz = O.C_KMS * (zb + (1.0 + zb) * (u_true + snl * rng.normal(size=n)) / O.C_KMS)

    p = Problem(N, L, spec.cosmo, snl, "fp32")
    p.set_catalog(rhat, mu, smu, cz, np.zeros(n))
    d0 = np.maximum(cz / 100.0, 2.5)
    st = State(p, [d0], seed=11)
    eps, _ = st.adapt_step_size(60, 20, 0.02, target=0.65)
    st.run_chain(100, 20, eps, use_graph=True, trace=False)           # burn-in
    st.analytics(True, [100.0], max_samples=4)
    tr = st.run_chain(300, 20, eps, use_graph=True, trace=True)
    assert 0.3 < tr["accept"].mean() < 0.98
    mean_vr = st.analytics_read(0)["mean_vr"].double().cpu().numpy()

    # compare over the nodes of the surveyed sphere outside the masked band
    off, r = O.node_offsets(base)
    inside = (r > 20.0) & (r < 120.0) & (np.abs(off[2]) > np.sin(np.radians(10.0)) * r)
    vr_true = O.radial_velocity(base, v_true)
    vr_other = O.radial_velocity(base, O.velocity_field(base, mock.white_field(N, 999)))
    c_true = _corr(mean_vr[inside], vr_true[inside])
    c_other = _corr(mean_vr[inside], vr_other[inside])
    print(f"posterior-mean v_r vs truth {c_true:.3f}, vs an unrelated field {c_other:.3f}")
    assert c_true > 0.5
    assert abs(c_other) < 0.25
