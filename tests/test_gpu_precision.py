"""Precision form (FP32 cube, DCT as split-BF16 tcgen05 products with FP32
accumulation) against the FP64 oracle, through the C ABI.

Tolerance: 1e-4 relative after 50 iterations on the reconstructed cube X
(max |gpu - oracle| / max |oracle|); the state arrays on the error scale of
their own update (tests/_gpu.scales).  The split keeps 16 mantissa bits of
each operand and drops the lo x lo term, ~2^-16 relative per product.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1504_06847_gb300 as mf  # noqa: E402
from paper_1504_06847_gb300 import synth  # noqa: E402
from tests import _gpu  # noqa: E402

pytestmark = pytest.mark.gpu
PRM = synth.WORKLOAD_PARAMS


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _run(cube, n_iter, params=PRM, J=3, mask=0x1FF):
    plan = mf.Plan(torch.tensor(cube.psf, dtype=torch.float32, device="cuda"))
    plan.iterate(torch.tensor(cube.y, dtype=torch.float32, device="cuda"), n_iter, wavelet_levels=J,
                 wavelet_mask=mask, precision=mf.MF_FP32_DCT_SPLITBF16, **params)
    assert plan.report()["status"] == mf.MF_OK
    return plan


@pytest.mark.parametrize("n_iter", [1, 3])
def test_splitbf16_first_iterations(n_iter):
    c = synth.workload("64x64x8")
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, _ = pb.run(n_iter)
    errs = _gpu.compare(_gpu.gpu_state(_run(c, n_iter)), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-4, errs


def test_splitbf16_64x64x8_50_iterations():
    c = synth.workload("64x64x8")
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, _ = pb.run(50)
    errs = _gpu.compare(_gpu.gpu_state(_run(c, 50)), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert errs["X"] < 1e-4 and max(errs.values()) < 1e-4, errs


@pytest.mark.parametrize("L", [15, 32, 48])
def test_splitbf16_band_counts(L):
    c = synth.make_cube(64, L, n_sources=5, n_antennas=40, seed=L)
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, _ = pb.run(20)
    errs = _gpu.compare(_gpu.gpu_state(_run(c, 20)), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-4, errs


def test_splitbf16_256x256x32_50_iterations():
    c = synth.workload("256x256x32")
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, _ = pb.run(50)
    errs = _gpu.compare(_gpu.gpu_state(_run(c, 50)), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-4, errs


def test_splitbf16_rejected_beyond_64_bands():
    c = synth.make_cube(32, 80, n_sources=2, n_antennas=16, seed=1)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    with pytest.raises(mf.MFError) as e:
        plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), 1,
                     precision=mf.MF_FP32_DCT_SPLITBF16, **PRM)
    assert e.value.status == mf.MF_ERR_INVALID
