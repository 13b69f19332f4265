"""Checkpoint / resume of a chain.  A chain written to a host file after K
trajectories and restored into a fresh state continues exactly as the
uninterrupted chain: its momenta and Metropolis uniforms are drawn from
Philox counters (element pair, trajectory, chain word, tag) under the
state's key, so position plus trajectory counter is the whole chain state
(FP64 path, 1e-12; the sum order of the scatter atomics is the only
difference between the two runs)."""
import numpy as np
import pytest
import torch

from _parity import check, check_scalar
from paper_2203_02369_gb300 import mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02369_gb300 import hamlet
    return hamlet


@pytest.mark.parametrize("sample_sigma", [False, True])
def test_resume_from_checkpoint_continues_the_chain(H, tmp_path, sample_sigma):
    spec = mock.PRESETS["grid16_500pts_fp64"]
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    K, L, eps = 4, 10, 0.03
    a = H.State(gp, [cat["d_init"]], seed=41, chain_ids=[3])
    if sample_sigma:
        a.sample_sigma_nl(True, 200.0)
    a.run_chain(K, L, eps)
    path = str(tmp_path / "chain.bin")
    a.save(path)
    ta = a.run_chain(K, L, eps)
    ga = a.get(0)
    # restore into chain 1 of a fresh two-chain state whose chain 1 has the same chain word
    b = H.State(gp, [cat["d_init"], cat["d_init"]], seed=41, chain_ids=[7, 3])
    if sample_sigma:
        b.sample_sigma_nl(True, 250.0)
    b.restore(path, chain=1)
    assert b.scalars(1)["traj"] == K
    tb = b.run_chain(K, L, eps)
    gb = b.get(1)
    assert np.array_equal(ta[:, 0]["traj"], tb[:, 1]["traj"])
    assert np.array_equal(ta[:, 0]["logu"], tb[:, 1]["logu"])
    assert np.array_equal(ta[:, 0]["accept"], tb[:, 1]["accept"])
    assert ta[:, 0]["accept"].sum() > 0
    for t in range(K):
        check_scalar(f"resume H_old {t}", tb[t, 1]["H_old"], ta[t, 0]["H_old"], 1e-12)
        check_scalar(f"resume H_new {t}", tb[t, 1]["H_new"], ta[t, 0]["H_new"], 1e-12)
    check("resume w", gb["w"], ga["w"], 1e-12)
    check("resume d", gb["d"], ga["d"], 1e-12)
    if sample_sigma:
        assert abs(b.sigma_nl()[0][1] - a.sigma_nl()[0][0]) <= 1e-12 * a.sigma_nl()[0][0]


def test_restore_rejects_another_stream_or_grid(H, tmp_path):
    spec = mock.PRESETS["grid16_500pts_fp64"]
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    a = H.State(gp, [cat["d_init"]], seed=41, chain_ids=[3])
    a.run_chain(1, 5, 0.03)
    path = str(tmp_path / "chain.bin")
    a.save(path)
    with pytest.raises(H.HamletError, match="Philox key"):
        H.State(gp, [cat["d_init"]], seed=42, chain_ids=[3]).restore(path)
    spec32 = mock.MockSpec(N=32, L=200.0, n_points=500, r_max=64.0, mask_deg=0.0, sigma_mu=(0.2, 0.45),
                           sigma_nl=250.0, seed=3, precision="fp64")
    cat32 = mock.make_catalog(spec32)
    with pytest.raises(H.HamletError, match="differ"):
        H.State(H.Problem.from_mock(spec32, cat32), [cat32["d_init"]], seed=41, chain_ids=[3]).restore(path)
    with open(path, "r+b") as fh:
        fh.truncate(100)
    with pytest.raises(H.HamletError):
        a.restore(path)


def test_state_io_with_host_buffers(H):
    """hm_state_set / hm_state_get take host memory as well as device
    memory: pinned and pageable host tensors give the same chain state as the
    device path, in both directions."""
    spec = mock.MockSpec(N=32, L=300.0, n_points=700, r_max=96.0, mask_deg=0.0, sigma_mu=(0.2, 0.45),
                         sigma_nl=250.0, seed=9, precision="fp32")
    cat = mock.make_catalog(spec)
    gp = H.Problem.from_mock(spec, cat)
    st = H.State(gp, [cat["d_init"]], seed=4)
    st.run_chain(2, 5, 0.02, use_graph=False, trace=False)
    ref = {k: v.cpu() for k, v in st.get(0).items()}
    for pin in (True, False):
        out = {k: (torch.empty_like(v).pin_memory() if pin else torch.empty_like(v)) for k, v in ref.items()}
        st.get(0, out=out)
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(out[k], ref[k]), k
        # write a modified state from host memory and read it back on the device
        w = ref["w"] * 0.5
        d = ref["d"] + 0.25
        st.set(0, w=w.pin_memory() if pin else w, d=d.pin_memory() if pin else d)
        g = st.get(0)
        torch.cuda.synchronize()
        assert torch.equal(g["w"].cpu(), w) and torch.equal(g["d"].cpu(), d)
        st.set(0, w=ref["w"].cuda(), d=ref["d"].cuda())
    with pytest.raises(ValueError):
        st.get(0, out={"w": torch.empty(5)})
