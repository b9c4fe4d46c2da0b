"""Linear-convolution plans (mf_plan_create_linear): step I by conjugate
gradients through zero-padded 2N FFTs, against the oracle's linear mode.

The CUDA path runs the same recurrence as the oracle (same start, same number
of iterations per band), in FP32 with FP64 dot products.  Bounds: 1e-5 of
each array's scale (tests/_gpu.scales) after a few ADMM iterations; the
CG iterate is a continuous function of its inputs for a fixed iteration
count, so FP32 rounding moves it by a small multiple of FP32 epsilon times the
condition of the few Krylov steps taken.
"""

import types

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


def _run(c, n_iter, cg_iters, J=3, resid_every=0, precision=mf.MF_FP32):
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"), linear=True)
    plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), n_iter, wavelet_levels=J,
                 cg_iters=cg_iters, resid_every=resid_every, precision=precision, **PRM)
    return plan


@pytest.mark.parametrize("N,L,n_iter,cg_iters", [(32, 4, 1, 1), (64, 8, 5, 10), (128, 6, 10, 20)])
def test_linear_plan_matches_oracle(N, L, n_iter, cg_iters):
    c = synth.make_cube(N, L, n_sources=3 + N // 32, n_antennas=40, seed=60 + N)
    pb = oracle.Problem(c.psf, c.y, PRM, conv="linear", cg_iters=cg_iters)
    st, H = pb.run(n_iter, hist=True)
    plan = _run(c, n_iter, cg_iters, resid_every=n_iter)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == n_iter
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs
    assert abs(rep["objective"] - H[-1, 3]) < 1e-5 * H[-1, 3]


def test_asymmetric_psf():
    # H^T is applied with the conjugate transfer function (the mode-5 column
    # pass); with the recipe's point-symmetric PSFs H^T = H would hide a mistake
    c = synth.make_cube(64, 4, n_sources=4, n_antennas=32, seed=87)
    psf = synth.asymmetric_psf(c.psf, seed=87)
    pb = oracle.Problem(psf, c.y, PRM, conv="linear", cg_iters=10)
    st, _ = pb.run(3)
    plan = _run(types.SimpleNamespace(psf=psf, y=c.y), 3, 10)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


def test_first_step_is_the_cg_solve_of_hty():
    # from the zero state step I solves Q x = H^T y (b = 0) by cg_iters iterations from x = 0
    c = synth.make_cube(64, 4, n_sources=4, n_antennas=32, seed=71)
    pb = oracle.Problem(c.psf, c.y, PRM, conv="linear", cg_iters=30)
    x_ref = pb.solve(pb.HtY, cg_iters=30)
    plan = _run(c, 1, 30)
    assert _gpu.rel_err(plan.x().double().cpu().numpy(), x_ref) < 1e-5


def test_linear_plan_rejects_bad_use():
    c = synth.make_cube(32, 4, n_sources=2, n_antennas=16, seed=3)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"), linear=True)
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    with pytest.raises(mf.MFError) as e:
        plan.iterate(y, 1, cg_iters=0, **PRM)
    assert e.value.status == mf.MF_ERR_INVALID
    with pytest.raises(mf.MFError) as e:
        plan.backward(y, 2, torch.zeros_like(y), rho=1.0)
    assert e.value.status == mf.MF_ERR_INVALID
    with pytest.raises(ValueError):
        mf.Plan(torch.tensor(c.psf, dtype=torch.float64, device="cuda"), linear=True)


def test_largest_image():
    # N = 1024, the largest a linear-convolution plan takes (its transforms run at 2N = 2048)
    c = synth.make_cube(1024, 2, n_sources=6, n_antennas=40, seed=96)
    pb = oracle.Problem(c.psf, c.y, PRM, conv="linear", cg_iters=2)
    st, _ = pb.run(1)
    plan = _run(c, 1, 2)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs
