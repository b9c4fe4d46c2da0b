"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI.

- The largest image the library takes (N = 2048) and the most bands (L = 128),
  element by element on the scales of tests/_gpu.scales, bound 1e-5 as for
  every FP32 case.  The cubes use the workloads' array density (256
  antennas).  With very sparse uv coverage the FP32 path loses digits in
  step I (measured with 32 antennas after 3 iterations: 6e-7 at 512^2,
  8e-6 at 1024^2, 5e-4 at 2048^2, while 256 antennas give 4e-7 at 2048^2); the
  FP64 plan is the form for such cubes.
- The degenerate cube y = 0: the optimum is X = 0 and Algorithm 1 from the
  zero state never leaves it, so every state array stays exactly zero (all
  three arithmetic forms).
(Sizes outside the documented range are refused on the host: tests/test_abi.py.)
"""

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


@pytest.mark.parametrize("N,L,n_iter", [(2048, 2, 3), (32, 128, 8)])
def test_largest_sizes(N, L, n_iter):
    # 256 antennas, the density of the workloads: with far sparser uv coverage
    # (e.g. 32 antennas on a 2048^2 grid) FP32 step I loses digits, see the
    # module docstring
    c = synth.make_cube(N, L, n_sources=max(2, int(40 * (N / 256) ** 2) // 8), n_antennas=256, seed=N + L)
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, _ = pb.run(n_iter)
    plan = _gpu.run_gpu(c, PRM, n_iter)
    assert plan.report()["status"] == mf.MF_OK
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


@pytest.mark.parametrize("precision,dtype", [(mf.MF_FP32, torch.float32), (mf.MF_FP32_DCT_SPLITBF16, torch.float32),
                                             (mf.MF_FP64, torch.float64)])
def test_zero_cube_stays_zero(precision, dtype):
    c = synth.make_cube(64, 8, n_sources=3, n_antennas=32, seed=5)
    plan = mf.Plan(torch.tensor(c.psf, dtype=dtype, device="cuda"))
    y = torch.zeros(8, 64, 64, dtype=dtype, device="cuda")
    plan.iterate(y, 6, precision=precision, resid_every=1, **PRM)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK
    for a in (mf.ARR_X, mf.ARR_GAMMA_P, mf.ARR_S_DCT, mf.ARR_GAMMA_V, mf.ARR_GAMMA_S_DCT, mf.ARR_B, mf.ARR_GAMMA_T):
        assert torch.count_nonzero(plan.get(a)).item() == 0, a
    assert rep["primal_res"] == 0.0 and rep["objective"] == 0.0 and rep["x_norm2"] == 0.0

