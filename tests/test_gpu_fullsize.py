"""The benchmarked configuration at full size against the FP64 oracle.

1024 x 1024 x 64 synthetic cube (300 sources, 20 % point sources, 512-antenna
disk array), Db1-Db8 + Haar, J = 3, split-BF16 tcgen05 DCTs, 64 x 64 wavelet
tiles: the launch configuration the benchmark times.  The oracle runs the same
iterations on the host cores (a few seconds per iteration), and every element
of the state is compared, on the scales of tests/_gpu.scales, with the
precision form's 1e-4 bound.  The FP64 residual and objective reductions are
compared with the oracle's history.
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
N_ITER = 3


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_splitbf16_1024x1024x64_full_state():
    c = synth.workload("1024x1024x64")
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, H = pb.run(N_ITER, hist=True)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    plan.set_option(mf.MF_OPT_WAV_TILE, 64)
    plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), N_ITER, precision=mf.MF_FP32_DCT_SPLITBF16,
                 resid_every=1, **PRM)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == N_ITER
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-4, errs
    red = {
        "objective": abs(rep["objective"] - H[-1, 3]) / H[-1, 3],
        "primal_res": abs(rep["primal_res"] - H[-1, 0]) / H[-1, 0],
        "dual_gamma": abs(rep["dual_gamma"] - H[-1, 6]) / H[-1, 6],
        "x_norm2": abs(rep["x_norm2"] - H[-1, 5]) / H[-1, 5],
    }
    _gpu.log_errors(red)
    assert max(red.values()) < 1e-4, red
    assert abs(rep["x_min"] - H[-1, 4]) <= 1e-4 * np.abs(st["X"]).max()
