"""The C ABI from plain C: tests/c_client/hamlet_client.c includes only
include/hamlet.h and the CUDA runtime header, allocates its own device
buffers and calls libhamlet directly (no Python binding, no torch).  It
compiles and links here; on a GPU its Psi, gradient and chain agree with the
FP64 oracle and with the Python binding."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "hamlet_client.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def build_client(tmpdir):
    from paper_2203_02369_gb300 import build
    lib = build.build_library()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = os.path.join(str(tmpdir), "hamlet_client")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-O2", "-std=c11", "-Wall", "-Werror", SRC, "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), "-L", libdir, "-lhamlet", "-L", os.path.join(CUDA, "lib64"),
           "-lcudart", "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_client_compiles_and_links(tmp_path):
    exe = build_client(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_client_matches_oracle_and_binding(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from _parity import check, check_scalar
    from oracle import hamlet_oracle as O
    from paper_2203_02369_gb300 import mock
    from paper_2203_02369_gb300.hamlet import Problem
    exe = build_client(tmp_path)
    spec = mock.PRESETS["grid16_500pts_fp64"]          # 16^3, 200 Mpc/h, 500 points, FP64
    cat = mock.make_catalog(spec)
    w = mock.white_field(16, 5)
    d = cat["d_init"]
    n = d.shape[0]
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as fh:
        # nbins = 0: the default distance prior, eq. D from the redshifts
        fh.write(struct.pack("<iiqdddd", 16, 1, n, spec.L, spec.sigma_nl, 0.0, 0.0))
        fh.write(struct.pack("<ii", 0, 0))
        for a in (cat["rhat"], cat["mu"], cat["sigma_mu"], cat["cz"], w, d):
            fh.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    out = tmp_path / "out.bin"
    r = subprocess.run([exe, str(inp), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = out.read_bytes()
    psi = np.frombuffer(raw, np.float64, 1, 0)[0]
    gw = np.frombuffer(raw, np.float64, 16 ** 3, 8)
    gd = np.frombuffer(raw, np.float64, n, 8 + 8 * 16 ** 3)
    h = np.frombuffer(raw, np.float64, 2, 8 + 8 * 16 ** 3 + 8 * n)
    # the FP64 oracle
    op = O.problem_from_catalog(16, spec.L, mock.spec_dict(spec)["cosmo"], spec.sigma_nl, cat)
    rpsi, rgw, rgd = O.logpost_grad(op, w, d)
    check_scalar("C client psi", psi, rpsi, 1e-12)
    check("C client grad_w", gw, rgw, 1e-12)
    check("C client grad_d", gd, rgd, 1e-12)
    _, _, recs = O.run_chain(op, np.zeros((16, 16, 16)), d, seed=3, chain=0, traj0=0, n_traj=2, eps=0.03,
                             n_steps=10)
    for t in range(2):
        assert abs(h[t] - recs[t]["H_new"]) <= 1e-9 * abs(recs[t]["H_new"])
    # and the Python binding on the same inputs
    gp = Problem.from_mock(spec, cat)
    bpsi, bgw, bgd = gp.logpost_grad(torch.tensor(w, device="cuda"), torch.tensor(d, device="cuda"))
    assert abs(psi - bpsi.item()) <= 1e-12 * abs(rpsi)
    check("C client vs binding grad_w", gw, bgw, 1e-12)
    check("C client vs binding grad_d", gd, bgd, 1e-12)
