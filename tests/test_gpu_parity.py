"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: the reconstructed cube X within 1e-5 relative (max |gpu - oracle| /
max |oracle|) of the FP64 oracle after 50 iterations for the FP32 path, 1e-10
for the FP64 instantiation.  The other state arrays are held to the same bounds
on the error scale of their own update (see tests/_gpu.scales: a multiplier is
compared on rho_c times the primal quantity of its constraint).
Sizes span several tiles of every kernel and the ragged cases (N = 16 with a
2 x 2 coarsest band, L not a power of two, masks without Db1, J = 1).
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


_cache = {}


def _oracle(name, n_iter, params=PRM, J=3, mask=0x1FF, cube=None):
    key = (name, n_iter, tuple(sorted(params.items())), J, mask)
    if key not in _cache:
        c = cube if cube is not None else synth.workload(name)
        pb = oracle.Problem(c.psf, c.y, params, J=J, mask=mask)
        st, H = pb.run(n_iter, hist=True)
        _cache[key] = (c, pb, st, H)
    return _cache[key]


def test_step_I_first_iteration():
    # From the zero state, X_1 = (H^T H + rho I)^-1 H^T Y (Eq. linsystemX with b = H^T Y).
    c, pb, st, _ = _oracle("64x64x8", 1)
    plan = _gpu.run_gpu(c, PRM, 1)
    x = plan.x().double().cpu().numpy()
    ref = pb.solve(pb.HtY)
    assert _gpu.rel_err(x, ref) < 2e-6
    assert _gpu.rel_err(x, st["X"]) < 2e-6


@pytest.mark.parametrize("n_iter", [1, 2, 5])
def test_full_state_early_iterations(n_iter):
    c, pb, st, _ = _oracle("64x64x8", n_iter)
    plan = _gpu.run_gpu(c, PRM, n_iter)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 5e-6, errs


def test_fp32_64x64x8_50_iterations():
    c, pb, st, _ = _oracle("64x64x8", 50)
    plan = _gpu.run_gpu(c, PRM, 50)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert errs["X"] < 1e-5, errs
    assert max(errs.values()) < 1e-5, errs


def test_fp64_64x64x8_50_iterations():
    c, pb, st, _ = _oracle("64x64x8", 50)
    plan = _gpu.run_gpu(c, PRM, 50, dtype=torch.float64)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-10, errs


def test_fp32_256x256x32_100_iterations():
    c, pb, st, _ = _oracle("256x256x32", 100)
    plan = _gpu.run_gpu(c, PRM, 100)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


@pytest.mark.parametrize("N,L,J,mask", [
    (16, 2, 3, 0x1FF),      # smallest cube: 2 x 2 coarsest band, filters longer than the level
    (32, 15, 2, 0x1FF),     # L not a power of two (padded DCT tile), paper's band count
    (64, 8, 1, 0x1FF),      # single level: the coarsest low-low band is level 1's
    (64, 5, 4, 0x100),      # Haar alone (K = 1 slot without Db1)
    (128, 3, 3, 0b010100110),  # a subset without Db1 and Haar
    (32, 4, 4, 0x1FF),      # deepest J for N = 32
])
def test_shapes_and_dictionaries(N, L, J, mask):
    c = synth.make_cube(N, L, n_sources=4, n_antennas=24, seed=N + L + J)
    n_iter = 12
    _, pb, st, _ = _oracle(f"custom{N},{L},{J},{mask}", n_iter, J=J, mask=mask, cube=c)
    plan = _gpu.run_gpu(c, PRM, n_iter, J=J, mask=mask)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


def test_paper_parameters():
    c = synth.make_cube(64, 15, n_sources=6, n_antennas=48, seed=15)
    _, pb, st, _ = _oracle("paper64x15", 30, params=synth.PAPER_PARAMS, cube=c)
    plan = _gpu.run_gpu(c, synth.PAPER_PARAMS, 30)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


def test_residual_report_matches_oracle():
    c, pb, st, H = _oracle("64x64x8", 20)
    plan = _gpu.run_gpu(c, PRM, 20, dtype=torch.float64, resid_every=5)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == 20
    p = PRM
    # primal residual = sum_c ||dGamma_c||^2 / rho_c^2 (all rho equal here)
    assert abs(rep["primal_res"] - H[-1, 0]) < 1e-9 * H[-1, 0]
    assert abs(rep["dual_gamma"] - H[-1, 6]) < 1e-9 * H[-1, 6]
    assert abs(rep["x_min"] - H[-1, 4]) < 1e-12
    assert abs(rep["x_norm2"] - H[-1, 5]) < 1e-10 * H[-1, 5]
    assert abs(rep["objective"] - H[-1, 3]) < 1e-9 * H[-1, 3], (rep, H[-1])
    # Boyd dual residual of the (X, V) | (P, T, S) split
    assert abs(rep["dual_res"] - H[-1, 1]) < 1e-9 * H[-1, 1], (rep["dual_res"], H[-1, 1])
    assert p["rho_P"] == 1.0


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 1e-3)])
def test_dual_residual_distinct_penalties(dtype, tol):
    # distinct rho_c, so a penalty applied to the wrong term shows; the first
    # iterations, where every term of the change is large
    prm = dict(mu_eps=0.003, mu_s=0.04, mu_nu=0.015, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)
    c = synth.make_cube(32, 6, n_sources=3, n_antennas=24, seed=17)
    pb = oracle.Problem(c.psf, c.y, prm, J=2)
    _, H = pb.run(3, hist=True)
    plan = _gpu.run_gpu(c, prm, 3, J=2, dtype=dtype, resid_every=1)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == 3
    err = abs(rep["dual_res"] - H[-1, 1]) / H[-1, 1]
    _gpu.log_errors({"dual_res": err})
    assert err < tol, err


@pytest.mark.parametrize("L", [100, 128])
def test_dual_residual_many_bands(L):
    # more than 64 bands (FP32 only: FP64 plans take at most 64): the spectral
    # part of the dual residual then gives each thread 16 bands of a pixel
    # spectrum instead of 8 (100 leaves a ragged last group)
    dtype, tol = torch.float32, 1e-3
    prm = dict(mu_eps=0.003, mu_s=0.04, mu_nu=0.015, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)
    c = synth.make_cube(32, L, n_sources=3, n_antennas=24, seed=L)
    pb = oracle.Problem(c.psf, c.y, prm, J=2)
    _, H = pb.run(3, hist=True)
    plan = _gpu.run_gpu(c, prm, 3, J=2, dtype=dtype, resid_every=1)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == 3
    errs = {"dual_res": abs(rep["dual_res"] - H[-1, 1]) / H[-1, 1],
            "primal_res": abs(rep["primal_res"] - H[-1, 0]) / H[-1, 0]}
    _gpu.log_errors(errs)
    assert max(errs.values()) < tol, errs


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-10)])
def test_asymmetric_psf(dtype, tol):
    # the recipe's PSFs are point-symmetric (H^T = H); this one is not, so the
    # conjugate filter of step I and H^T y are exercised
    c = synth.make_cube(32, 4, n_sources=4, n_antennas=32, seed=55)
    psf = synth.asymmetric_psf(c.psf, seed=55)
    pb = oracle.Problem(psf, c.y, PRM)
    st, _ = pb.run(10)
    plan = _gpu.run_gpu(types.SimpleNamespace(psf=psf, y=c.y), PRM, 10, dtype=dtype)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < tol, errs


def test_deterministic():
    c = synth.workload("64x64x8")
    a = _gpu.gpu_state(_gpu.run_gpu(c, PRM, 7))
    b = _gpu.gpu_state(_gpu.run_gpu(c, PRM, 7))
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_warm_start_continues():
    c = synth.workload("64x64x8")
    one = _gpu.run_gpu(c, PRM, 10)
    two = _gpu.run_gpu(c, PRM, 4)
    two.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), 6, warm_start=1, **PRM)
    assert np.array_equal(one.x().cpu().numpy(), two.x().cpu().numpy())
    # checkpoint / restore
    buf = two.get_state().clone()
    x_before = two.x().clone()
    two.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), 3, warm_start=1, **PRM)
    two.set_state(buf)
    assert torch.equal(two.x(), x_before)


def test_nonfinite_input_is_reported():
    c = synth.make_cube(32, 4, n_sources=2, n_antennas=16, seed=3)
    y = c.y.copy()
    y[1, 5, 7] = np.nan
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    plan.iterate(torch.tensor(y, dtype=torch.float32, device="cuda"), 3, resid_every=1, **PRM)
    assert plan.report()["status"] == mf.MF_ERR_NONFINITE


def test_invalid_parameters_rejected():
    c = synth.make_cube(32, 4, n_sources=2, n_antennas=16, seed=3)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    bad = [dict(rho_T=0.0), dict(mu_s=-1.0), dict(wavelet_levels=5), dict(wavelet_mask=0),
           dict(wavelet_mask=0x200), dict(precision=mf.MF_FP64)]
    for kw in bad:
        args = dict(PRM)
        args.update(kw)
        with pytest.raises(mf.MFError) as e:
            plan.iterate(y, 1, **args)
        assert e.value.status == mf.MF_ERR_INVALID
    plan.iterate(y, 1, **PRM)  # still usable
    assert plan.report()["status"] == mf.MF_OK
