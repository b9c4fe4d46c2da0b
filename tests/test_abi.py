"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function that include/mf.h declares, and its host-built tables agree with
the oracle's (the Daubechies filters of Section 4's dictionary)."""

import os
import re
import subprocess

import numpy as np
import pytest

import paper_1504_06847_gb300 as mf
from oracle import daubechies

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1504_06847_gb300 import build

    build.build()
    yield


def _declared():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    return sorted(set(re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_function():
    declared = _declared()
    assert "mf_admm_iterate" in declared and "mf_plan_create" in declared
    out = subprocess.check_output(["nm", "-D", "--defined-only", mf.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (mf_[a-z0-9_]+)", out))
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    L = mf.lib()
    for d in declared:
        assert hasattr(L, d)


def test_binding_lists_the_exports():
    assert sorted(mf.EXPORTS) == _declared()


@pytest.mark.parametrize("K", range(1, 9))
def test_library_filters_match_oracle(K):
    lib_taps = np.array(mf.wavelet_filter(K))
    assert len(lib_taps) == 2 * K
    assert np.max(np.abs(lib_taps - daubechies.daubechies(K))) < 1e-14


def test_params_default_and_status_strings():
    p = mf.default_params()
    assert (p.mu_eps, p.mu_s, p.mu_nu) == (0.001, 0.05, 0.01)
    assert (p.rho_P, p.rho_T, p.rho_V, p.rho_S) == (1.0, 1.0, 1.0, 1.0)
    assert p.wavelet_levels == 3 and p.wavelet_mask == 0x1FF and p.precision == mf.MF_FP32
    assert mf.status_string(mf.MF_OK) == "ok"
    assert "invalid" in mf.status_string(mf.MF_ERR_INVALID)
    with pytest.raises(mf.MFError):
        mf.wavelet_filter(9)


def test_create_rejects_bad_sizes_without_touching_the_device():
    import ctypes

    h = ctypes.c_void_p()
    L = mf.lib()
    for N, Lb in [(24, 4), (8, 4), (4096, 4), (64, 1), (64, 129)]:
        assert L.mf_plan_create(N, Lb, ctypes.c_void_p(16), ctypes.byref(h)) == mf.MF_ERR_INVALID
    assert L.mf_plan_create(64, 4, None, ctypes.byref(h)) == mf.MF_ERR_INVALID
    assert L.mf_plan_create_f64(64, 65, ctypes.c_void_p(16), ctypes.byref(h)) == mf.MF_ERR_INVALID
    L.mf_plan_destroy(None)


def test_linear_and_visibility_entry_points_reject_bad_arguments_without_touching_the_device():
    import ctypes

    h = ctypes.c_void_p()
    L = mf.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks come first
    # linear convolution plans: N a power of two in [16, 1024]
    for N in (8, 24, 2048):
        assert L.mf_plan_create_linear(N, 4, fake, ctypes.byref(h)) == mf.MF_ERR_INVALID
    assert L.mf_plan_create_linear(64, 4, None, ctypes.byref(h)) == mf.MF_ERR_INVALID
    # visibility plans: N a power of two in [16, 512], counts >= 0, uv given when any count > 0
    counts = (ctypes.c_int * 3)(5, 0, 7)
    for N in (8, 48, 1024):
        assert L.mf_plan_create_vis(N, 3, counts, fake, None, ctypes.byref(h)) == mf.MF_ERR_INVALID
    assert L.mf_plan_create_vis(64, 3, None, fake, None, ctypes.byref(h)) == mf.MF_ERR_INVALID
    bad = (ctypes.c_int * 3)(5, -1, 7)
    assert L.mf_plan_create_vis(64, 3, bad, fake, None, ctypes.byref(h)) == mf.MF_ERR_INVALID
    assert L.mf_plan_create_vis(64, 3, counts, None, None, ctypes.byref(h)) == mf.MF_ERR_INVALID
    assert L.mf_plan_create_vis(64, 1, counts, fake, None, ctypes.byref(h)) == mf.MF_ERR_INVALID  # L >= 2
    assert L.mf_plan_create_vis(64, 3, counts, fake, None, None) == mf.MF_ERR_INVALID
    # model visibilities need a visibility plan and an output
    assert L.mf_vis_predict(None, None, fake, None) == mf.MF_ERR_INVALID
