"""The benchmarked configuration at full size against the FP64 oracle, at the
parity point of the workloads: 50 iterations.

1024 x 1024 x 64 synthetic cube (300 sources, 20 % point sources, 512-antenna
disk array), Db1-Db8 + Haar, J = 3, 64 x 64 wavelet tiles: the launch
configuration the benchmark times, with the spectral DCTs as split-BF16
tcgen05 products (bound 1e-4) and in FP32 (bound 1e-5).  One oracle run (a
few seconds per iteration on the host cores) serves both.  Every element of
the state is compared on the scales of tests/_gpu.scales.

The FP64 reductions of the last iteration are compared too.  The objective
and ||X||^2 are sums of the state itself: relative error, same bound.  The
primal residual, the multiplier change and the dual residual are squared
norms of CHANGES over one iteration, which after 50 iterations are small
beside the arrays they are differences of; an error of tol x (array scale) in
each state array then moves sqrt(residual) by up to a few tol x (2-norm of the
arrays differenced).  They are compared that way:
|sqrt(gpu) - sqrt(oracle)| <= tol * ||arrays||_2.
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
N_ITER = 50


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


@pytest.fixture(scope="module")
def reference():
    c = synth.workload("1024x1024x64")
    pb = oracle.Problem(c.psf, c.y, PRM)
    st = pb.zero_state()
    pb.iterate(st, N_ITER - 1)
    H = pb.iterate(st, 1, hist=True)  # the history of the last iteration only
    return c, pb, st, H


def _run(c, precision):
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    plan.set_option(mf.MF_OPT_WAV_TILE, 64)
    plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), N_ITER, precision=precision,
                 resid_every=N_ITER, **PRM)
    return plan


def _check(plan, pb, st, H, tol):
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == N_ITER
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < tol, errs
    plan.close()
    p = PRM
    h = H[-1]
    norm = lambda a: float(np.sqrt(np.sum(np.asarray(a, dtype=np.float64) ** 2)))
    b = pb.make_b(st) - pb.HtY
    gam = np.sqrt(sum(norm(st[g]) ** 2 for g in ("GP", "GT", "GV", "GS")))
    red = {
        "objective": abs(rep["objective"] - h[3]) / h[3],
        "x_norm2": abs(rep["x_norm2"] - h[5]) / h[5],
        "x_min": abs(rep["x_min"] - h[4]) / np.abs(st["X"]).max(),
        # changes over the last iteration, on the scale of the arrays differenced
        "primal_res": abs(np.sqrt(rep["primal_res"]) - np.sqrt(h[0])) / (gam / min(p["rho_P"], p["rho_T"],
                                                                                  p["rho_V"], p["rho_S"])),
        "dual_gamma": abs(np.sqrt(rep["dual_gamma"]) - np.sqrt(h[6])) / gam,
        "dual_res": abs(np.sqrt(rep["dual_res"]) - np.sqrt(h[1])) / norm(b),
    }
    _gpu.log_errors(red)
    assert max(red.values()) < tol, red


def test_splitbf16_1024x1024x64_50_iterations(reference):
    c, pb, st, H = reference
    _check(_run(c, mf.MF_FP32_DCT_SPLITBF16), pb, st, H, 1e-4)


def test_fp32_1024x1024x64_50_iterations(reference):
    c, pb, st, H = reference
    _check(_run(c, mf.MF_FP32), pb, st, H, 1e-5)
