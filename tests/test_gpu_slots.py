"""Slotted states (continuous batching) on the GPU: every job loaded into a
slot draws the chain it draws alone in a one-chain state with the same seed
and chain word, while other jobs are loaded, run and released beside it
(FP64 path, 1e-12: the only difference allowed is the order of the atomic
scatter additions); the chain of a slot also matches the FP64 oracle's."""
import numpy as np
import pytest
import torch

from oracle import hamlet_oracle as O
from paper_2203_02369_gb300 import mock
from paper_2203_02369_gb300._lib import HamletError

pytestmark = pytest.mark.gpu

SEED = 17
EPS = 0.02
L_STEPS = 8


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import hamlet
    return hamlet


def _spec(k, N=16, n=400, prec="fp64"):
    L = 200.0 if N == 16 else 300.0
    return mock.MockSpec(N=N, L=L, n_points=n, r_max=0.3 * L, mask_deg=10.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=300 + k, precision=prec)


def _job(H, k, **kw):
    spec = _spec(k, **kw)
    cat = mock.make_catalog(spec)
    return spec, cat, H.Problem.from_mock(spec, cat)


def _alone(H, prob, cat, chain_id, n_traj, eps=EPS):
    st = H.State(prob, [cat["d_init"]], seed=SEED, chain_ids=[chain_id])
    tr = st.run_chain(n_traj, L_STEPS, eps, use_graph=True)[:, 0]
    g = st.get(0)
    out = (tr, g["w"].cpu().numpy(), g["d"].cpu().numpy())
    st.close()
    return out


def _same(tr_a, tr_b, rtol=1e-12):
    assert list(tr_a["accept"]) == list(tr_b["accept"])
    for f in ("H_old", "H_new", "psi"):
        a, b = np.asarray(tr_a[f]), np.asarray(tr_b[f])
        with np.errstate(invalid="ignore"):
            same = (a == b) | (np.abs(a - b) <= rtol * np.abs(b))   # an infinite H (rejected) on both sides
        assert np.all(same), (f, a, b)


def test_slots_jobs_match_their_alone_chains_through_loads_and_releases(H):
    jobs = [_job(H, k, n=300 + 100 * k) for k in range(4)]
    tmpl = H.Problem(16, 200.0, precision="fp64")
    sl = H.Slots(tmpl, n_slots=3, max_points=1000, seed=SEED)
    rec = {k: [] for k in range(4)}
    where = {}
    for k in (0, 1, 2):
        where[k] = sl.load(jobs[k][2], jobs[k][1]["d_init"], chain_id=k, eps0=EPS)
    with pytest.raises(HamletError, match="every slot is in use"):
        sl.load(jobs[3][2], jobs[3][1]["d_init"], chain_id=3, eps0=EPS)
    for _ in range(2):
        tr = sl.run(1, L_STEPS)[0]
        for k, i in where.items():
            rec[k].append(tr[i])
    # job 1 leaves from the middle: job 2 moves into its index
    fin1 = sl.get(where[1])
    moved = sl.release(where[1])
    assert moved == 2
    where[2] = where.pop(1)
    where[3] = sl.load(jobs[3][2], jobs[3][1]["d_init"], chain_id=3, eps0=EPS)
    assert sl.n_active == 3
    for _ in range(3):
        tr = sl.run(1, L_STEPS)[0]
        for k, i in where.items():
            rec[k].append(tr[i])
    finals = {k: sl.get(i) for k, i in where.items()}
    finals[1] = fin1
    torch.cuda.synchronize()
    for k in range(4):
        spec, cat, prob = jobs[k]
        got = np.array(rec[k])
        tr, w, d = _alone(H, prob, cat, k, len(got))
        _same(got, tr)
        assert np.linalg.norm(finals[k]["w"].cpu().numpy() - w) <= 1e-12 * np.linalg.norm(w)
        assert np.linalg.norm(finals[k]["d"].cpu().numpy() - d) <= 1e-12 * np.linalg.norm(d)
    sl.close()


def test_slot_chain_matches_the_oracle_chain(H):
    spec, cat, prob = _job(H, 7, n=500)
    other = _job(H, 8, n=350)
    tmpl = H.Problem(16, 200.0, precision="fp64")
    sl = H.Slots(tmpl, n_slots=2, max_points=600, seed=3)
    sl.load(other[2], other[1]["d_init"], chain_id=1, eps0=0.03)
    i = sl.load(prob, cat["d_init"], chain_id=0, eps0=0.03)
    got = sl.run(2, 10)[:, i]
    op = O.problem_from_catalog(spec.N, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    _, _, recs = O.run_chain(op, np.zeros((16, 16, 16)), cat["d_init"], seed=3, chain=0, traj0=0, n_traj=2,
                             eps=0.03, n_steps=10)
    for t in range(2):
        assert abs(got[t]["H_new"] - recs[t]["H_new"]) < 1e-9 * abs(recs[t]["H_new"])
    sl.close()


def test_slot_step_adaptation_matches_the_one_chain_adaptation(H):
    spec, cat, prob = _job(H, 9, n=400)
    other = _job(H, 10, n=300)
    st = H.State(prob, [cat["d_init"]], seed=SEED, chain_ids=[5])
    e_alone, tr_alone = st.adapt_step_size(6, L_STEPS, 0.05, target=0.7)
    st.close()
    tmpl = H.Problem(16, 200.0, precision="fp64")
    sl = H.Slots(tmpl, n_slots=2, max_points=500, seed=SEED)
    sl.load(other[2], other[1]["d_init"], chain_id=6, eps0=EPS)          # a neighbour that does not adapt
    i = sl.load(prob, cat["d_init"], chain_id=5, eps0=0.05, adapt_target=0.7)
    got = np.array([sl.run(1, L_STEPS)[0][i] for _ in range(6)])
    e = sl.adapt_end(i)
    # the step is a function of the acceptance probabilities exp(H_old -
    # H_new); their rounding-order noise (~1e-16 of H) is amplified by the
    # dual-averaging gain sqrt(m)/gamma = 20 sqrt(m), hence 1e-9 here
    assert abs(e - e_alone[0]) <= 1e-9 * e_alone[0]
    assert np.allclose(got["eps"], tr_alone[:, 0]["eps"], rtol=1e-9, atol=0)
    _same(got, tr_alone[:, 0], rtol=1e-10)
    sl.close()


def test_slot_job_sampling_sigma_nl_matches_its_alone_chain(H):
    """A job that samples sigma_NL (eq. q) beside one that holds it fixed
    draws the chain its one-chain state draws with sigma_NL sampled."""
    a = _job(H, 14, n=450)
    b = _job(H, 15, n=300)
    s0 = 230.0
    tmpl = H.Problem(16, 200.0, precision="fp64")
    sl = H.Slots(tmpl, n_slots=2, max_points=500, seed=SEED)
    sl.load(b[2], b[1]["d_init"], chain_id=8, eps0=EPS)
    i = sl.load(a[2], a[1]["d_init"], chain_id=7, eps0=EPS, sigma_nl0=s0)
    tr = sl.run(4, L_STEPS)
    got = tr[:, i]
    sig, gsig = sl.sigma_nl()
    # the fixed job reports its problem's value and no gradient, and draws its
    # one-chain (fixed sigma_NL) chain
    assert sig[1 - i] == b[0].sigma_nl
    assert gsig[1 - i] == 0.0
    ref_b, _, _ = _alone(H, b[2], b[1], 8, 4)
    _same(tr[:, 1 - i], ref_b)
    st = H.State(a[2], [a[1]["d_init"]], seed=SEED, chain_ids=[7])
    st.sample_sigma_nl(True, s0)
    ref = st.run_chain(4, L_STEPS, EPS, use_graph=True)[:, 0]
    rs, rg = st.sigma_nl()
    _same(got, ref)
    assert abs(sig[i] - rs[0]) <= 1e-12 * rs[0]
    assert sig[i] != s0                         # it moved
    st.close()
    sl.close()


def test_slots_reject_mismatched_and_oversize_jobs(H):
    tmpl = H.Problem(16, 200.0, precision="fp64")
    sl = H.Slots(tmpl, n_slots=2, max_points=100, seed=1)
    spec, cat, prob = _job(H, 11, n=400)
    with pytest.raises(HamletError, match="larger than the room"):
        sl.load(prob, cat["d_init"], chain_id=0, eps0=EPS)
    spec32, cat32, prob32 = _job(H, 12, N=32, n=50)
    with pytest.raises(HamletError, match="must be the state's"):
        sl.load(prob32, cat32["d_init"], chain_id=0, eps0=EPS)
    assert sl.n_active == 0
    assert sl.run(1, L_STEPS).shape == (1, 0)
    sl.close()


def test_batched_serving_job_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import serve

    def job(k, N, n, prec, arrival, n_traj):
        spec = mock.MockSpec(N=N, L=300.0 if N == 32 else 500.0, n_points=n, r_max=96.0 if N == 32 else 160.0,
                             mask_deg=10.0, sigma_mu=(0.2, 0.45), sigma_nl=250.0, seed=700 + k, precision=prec)
        return serve.Job(job_id=k, spec=spec, n_traj=n_traj, n_leapfrog=10, eps=0.01, arrival=arrival)

    alone = job(0, 32, 2000, "fp64", 0.0, 24)
    serve.BatchedServingLoop(max_slots=1, max_points=4000, keep_state=True, seed=SEED).run([alone])
    # the same job with FP64 neighbours that join and leave while it runs,
    # and an FP32 group of another grid overlapping on the device
    mix = ([job(0, 32, 2000, "fp64", 0.0, 24)] + [job(k, 32, 1000 + 500 * k, "fp64", 0.0, 2 + 3 * k)
                                                  for k in (1, 2, 3)]
           + [job(k, 64, 3000, "fp32", 0.0, 4) for k in (4, 5)])
    loop = serve.BatchedServingLoop(max_slots=3, max_points=4000, keep_state=True, seed=SEED, max_batch_traj=2)
    stats = loop.run(mix)
    assert not stats["errors"], stats["errors"]
    assert loop.max_active_seen >= 2
    x = mix[0]
    assert x.accept == alone.accept
    assert np.allclose(x.psi, alone.psi, rtol=1e-12, atol=0)
    w1, w0 = x.final_w.numpy(), alone.final_w.numpy()
    assert np.linalg.norm(w1 - w0) / np.linalg.norm(w0) < 1e-12
    d1, d0 = x.final_d.numpy(), alone.final_d.numpy()
    assert np.linalg.norm(d1 - d0) / np.linalg.norm(d0) < 1e-12
