"""The C-ABI library builds, loads and exports every entry point that
include/hamlet.h declares (no GPU needed); host-side argument checks."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2203_02369_gb300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hamlet.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(hm_[a-z0-9_]+)\s*\(",
                                 text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(names) == bound


def test_supported_sizes():
    lib = _lib.load()
    for N in (8, 16, 32, 64, 128):
        assert lib.hm_supported(N, 0) == 1
    for N in (8, 16, 32, 64, 128):
        assert lib.hm_supported(N, 1) == 1
    assert lib.hm_supported(256, 0) == 1
    assert lib.hm_supported(256, 1) == 0
    assert lib.hm_supported(512, 0) == 0
    assert lib.hm_supported(48, 0) == 0


def test_invalid_problem_rejected_before_any_device_call():
    lib = _lib.load()
    d = _lib.hm_problem_desc()
    d.N = 48            # not a power of two
    d.L = 100.0
    h = ct.c_void_p()
    rc = lib.hm_init_problem(ct.byref(d), ct.byref(h))
    assert rc == _lib.HM_EINVAL
    assert b"unsupported grid" in lib.hm_last_error()
    d.N = 16
    d.omega_m = 0.3
    d.omega_b = 0.05
    d.h = 0.7
    d.sigma8 = 0.8
    d.T_cmb = 2.7255
    d.n_s = 0.96
    d.sigma_nl = 150.0
    d.prior_kind = _lib.HM_PRIOR_TABLE   # a table of 5 bins without its data
    d.prior_nbins = 5
    d.prior_bin = 5.0
    assert lib.hm_init_problem(ct.byref(d), ct.byref(h)) == _lib.HM_EINVAL
    d.prior_nbins = 0                    # the redshift-distance prior with a negative pad
    d.prior_kind = _lib.HM_PRIOR_DZ
    d.prior_pad = -1.0
    assert lib.hm_init_problem(ct.byref(d), ct.byref(h)) == _lib.HM_EINVAL
    assert b"prior_pad" in lib.hm_last_error()
    assert lib.hm_set_catalog(None, 0, None, None, None, None, None) == _lib.HM_EINVAL
    assert lib.hm_run_chain(None, 1, 1, None, 1, 0, None, None) == _lib.HM_EINVAL


def test_dz_prior_table_host_entry_matches_oracle():
    from oracle import hamlet_oracle as O
    from paper_2203_02369_gb300 import mock
    from paper_2203_02369_gb300.hamlet import dz_prior_table
    cat = mock.make_catalog(mock.PRESETS["grid64_5000pts"])
    got = dz_prior_table(cat["cz"], 0.3, 5.0, 12.0)
    ref = O.dz_prior_table(cat["cz"], 0.3, 5.0, 12.0)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 1e-12
