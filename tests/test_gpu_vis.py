"""Visibility-domain plans (mf_plan_create_vis): the measurement model of
Section 2's last paragraph, step I by conjugate gradients on the Toeplitz form
of Re(Phi^H W Phi), against the oracle's exact non-uniform DFT.

The inputs follow the synthetic recipe (weights summing to 1 per band, so that
the dirty beam peaks at 1): Re(Phi^H W Phi) + rho I then has a condition number
of a few units and FP32 conjugate gradients stay within FP32 rounding of the
FP64 iterates (with raw unit weights the condition number is ~2.6e3 at 64^2 and
32 antennas, and FP32 CG drifts 3e-5 from FP64 after 30 iterations: a property
of the arithmetic, not of the kernels).

The CUDA path computes the Toeplitz kernel and the dirty image Re(Phi^H W y)
by gridding (type-1 non-uniform FFT, exponential-of-semicircle kernel of width
8 at oversampling 2, whose approximation error is about 1e-7 of
sum w |c|) and FP32 FFTs; both are compared with the oracle's direct sums at
1e-5 of their maximum (the FP32 parity bound).  The ADMM state after a few
iterations is compared like the linear-convolution plans' (1e-5 of each
array's scale).  The data-fit term of the report is formed as
1/2 x.(A x) - x.d + 1/2 sum w |y|^2, whose FP32 rounding is relative to the
largest of those terms, so the objective is compared at 1e-5 of
objective + 1/2 sum w |y|^2.  Inputs are rounded to FP32 before both sides see
them.
"""

import ctypes

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


def _f32(c):
    """The observation as both sides see it: visibilities and weights rounded to FP32."""
    vis = [v.astype(np.complex64).astype(np.complex128) for v in c.vis]
    w = [a.astype(np.float32).astype(np.float64) for a in c.weights]
    return vis, w


def _plan(N, c, weights=True):
    uv = [torch.tensor(q, dtype=torch.float32, device="cuda") for q in c.uv]
    w = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in c.weights] if weights else None
    return mf.Plan.from_visibilities(N, uv, w)


def _y(c):
    return torch.tensor(np.concatenate(c.vis).astype(np.complex64), device="cuda")


def _problem(N, c, cg_iters, J=3, weights=True):
    vis, w = _f32(c)
    return oracle.Problem.visibilities(N, c.uv, vis, PRM, weights=w if weights else None, J=J, cg_iters=cg_iters)


CASES = [(32, 3, 16, 1, 1), (64, 4, 24, 5, 10), (128, 3, 40, 8, 12)]


@pytest.mark.parametrize("N,L,ants,n_iter,cg_iters", CASES)
def test_vis_plan_matches_oracle(N, L, ants, n_iter, cg_iters):
    c = synth.make_visibilities(N, L, n_sources=3 + N // 32, n_antennas=ants, seed=80 + N, random_weights=True)
    pb = _problem(N, c, cg_iters)
    st, H = pb.run(n_iter, hist=True)
    plan = _plan(N, c)
    plan.iterate(_y(c), n_iter, cg_iters=cg_iters, resid_every=n_iter, **PRM)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK and rep["resid_iter"] == n_iter
    d = plan.get(mf.ARR_HTY).double().cpu().numpy()
    errs = {"HtY": _gpu.rel_err(d, pb.HtY)}
    errs.update(_gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st)))
    assert max(errs.values()) < 1e-5, errs
    c0 = 0.5 * sum(np.sum(w * np.abs(v) ** 2) for v, w in zip(*_f32(c)))
    red = {"objective": abs(rep["objective"] - H[-1, 3]) / (H[-1, 3] + c0),
           "x_norm2": abs(rep["x_norm2"] - H[-1, 5]) / H[-1, 5]}
    _gpu.log_errors(red)
    assert max(red.values()) < 1e-5, red


def test_first_step_is_the_cg_solve_of_the_dirty_image():
    # from the zero state step I solves Q x = Re(Phi^H W y) by cg_iters iterations from x = 0
    c = synth.make_visibilities(64, 3, n_sources=4, n_antennas=32, seed=91)
    pb = _problem(64, c, 30)
    x_ref = pb.solve(pb.HtY, cg_iters=30)
    plan = _plan(64, c)
    plan.iterate(_y(c), 1, cg_iters=30, **PRM)
    assert _gpu.rel_err(plan.x().double().cpu().numpy(), x_ref) < 1e-5


def test_band_without_visibilities():
    # an empty band has A = 0 and d = 0: step I gives X = b / rho_bar there
    c = synth.make_visibilities(32, 3, n_sources=3, n_antennas=12, seed=92, random_weights=True)
    c.uv[1], c.vis[1], c.weights[1] = c.uv[1][:0], c.vis[1][:0], c.weights[1][:0]
    pb = _problem(32, c, 6)
    st, _ = pb.run(4)
    plan = _plan(32, c)
    plan.iterate(_y(c), 4, cg_iters=6, **PRM)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs
    assert np.all(plan.get(mf.ARR_HTY)[1].cpu().numpy() == 0.0)


def test_vis_plan_rejects_bad_input():
    c = synth.make_visibilities(32, 2, n_sources=2, n_antennas=8, seed=93)
    uv = [torch.tensor(q, dtype=torch.float32, device="cuda") for q in c.uv]
    for bad in (16.0, -16.0, float("nan")):  # |u| must stay below N/2
        uvb = [t.clone() for t in uv]
        uvb[1][3, 0] = bad
        with pytest.raises(mf.MFError) as e:
            mf.Plan.from_visibilities(32, uvb)
        assert e.value.status == mf.MF_ERR_INVALID
    w = [torch.ones(t.shape[0], device="cuda") for t in uv]
    w[0][0] = -1.0
    with pytest.raises(mf.MFError) as e:
        mf.Plan.from_visibilities(32, uv, w)
    assert e.value.status == mf.MF_ERR_INVALID
    with pytest.raises(mf.MFError) as e:
        mf.Plan.from_visibilities(1024, [t * 32 for t in uv])  # N above 512
    assert e.value.status == mf.MF_ERR_INVALID
    plan = mf.Plan.from_visibilities(32, uv)
    y = _y(c)
    with pytest.raises(ValueError):
        plan.iterate(y[:-1], 1, cg_iters=2, **PRM)
    with pytest.raises(mf.MFError) as e:
        plan.iterate(y, 1, cg_iters=0, **PRM)
    assert e.value.status == mf.MF_ERR_INVALID
    with pytest.raises(mf.MFError):
        plan.set(mf.ARR_HTY, torch.zeros(2, 32, 32, device="cuda"))


def test_unit_weights_without_a_weight_array():
    # weights NULL: every w_m = 1 (one CG iteration: no amplification by the conditioning)
    c = synth.make_visibilities(32, 3, n_sources=3, n_antennas=10, seed=94)
    c.weights = [np.ones(len(v)) for v in c.vis]
    pb = _problem(32, c, 1, weights=False)
    st, _ = pb.run(1)
    plan = _plan(32, c, weights=False)
    plan.iterate(_y(c), 1, cg_iters=1, **PRM)
    assert _gpu.rel_err(plan.get(mf.ARR_HTY).double().cpu().numpy(), pb.HtY) < 1e-5
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


def test_largest_image():
    # N = 512, the largest a visibility plan takes (its Toeplitz kernels are gridded at 4N)
    c = synth.make_visibilities(512, 2, n_sources=8, n_antennas=20, seed=95, random_weights=True)
    pb = _problem(512, c, 3)
    st, _ = pb.run(2)
    plan = _plan(512, c)
    plan.iterate(_y(c), 2, cg_iters=3, **PRM)
    errs = {"HtY": _gpu.rel_err(plan.get(mf.ARR_HTY).double().cpu().numpy(), pb.HtY)}
    errs.update(_gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st)))
    assert max(errs.values()) < 1e-5, errs


def test_all_visibilities_at_the_origin():
    # degenerate coverage: every uv point at (0, 0), so k is the constant sum of the
    # weights and Re(Phi^H W Phi) = (sum w) 1 1^T has rank one, with the eigenvalue
    # N^2 sum w.  The weights are scaled to sum 1/N^2 so that this eigenvalue is 1 and
    # Q stays well conditioned (with sum w = 1 its condition number is about 94 at
    # N = 32 and FP32 conjugate gradients drift about 6e-5 from the FP64 ones)
    c = synth.make_visibilities(32, 3, n_sources=2, n_antennas=8, seed=97, random_weights=True)
    # one ADMM iteration: with such weak data the regularisers shrink X about 70-fold
    # by the third, which leaves X a small difference of right-hand-side terms (its
    # relative error there, ~3e-5, is the FP32 rounding of those terms, ~3e-10)
    c.uv = [np.zeros_like(q) for q in c.uv]
    c.weights = [a / 32 ** 2 for a in c.weights]
    pb = _problem(32, c, 4)
    st, _ = pb.run(1)
    plan = _plan(32, c)
    plan.iterate(_y(c), 1, cg_iters=4, **PRM)
    d = plan.get(mf.ARR_HTY).double().cpu().numpy()
    errs = {"HtY": _gpu.rel_err(d, pb.HtY)}
    errs.update(_gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st)))
    assert max(errs.values()) < 1e-5, errs
    for l in range(3):  # the dirty image of band l is the constant Re(sum_m w_m y_m)
        assert np.ptp(d[l]) <= 1e-5 * np.abs(d[l]).max()


@pytest.mark.parametrize("N,L,ants", [(64, 3, 24), (512, 2, 20)])
def test_predict_matches_the_oracle_operator(N, L, ants):
    # mf_vis_predict (type-2 non-uniform FFT, about 1e-7 of sum |x|) against the exact sum
    c = synth.make_visibilities(N, L, n_sources=4, n_antennas=ants, seed=99 + N, random_weights=True)
    pb = _problem(N, c, 1)
    x = np.random.default_rng(N).uniform(0.0, 1.0, size=(L, N, N)).astype(np.float32)
    ref = pb.apply_H(x.astype(np.float64))
    plan = _plan(N, c)
    got = plan.predict(torch.tensor(x, device="cuda")).cpu().numpy().astype(np.complex128)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    _gpu.log_errors({"predict": float(err)})
    assert err < 1e-5, err


def test_predicted_residual_gives_the_data_fit():
    # 1/2 sum w |y - Phi X|^2 from the model visibilities of the plan's X equals the
    # oracle's data-fit term for its X (X agrees to ~1e-6; the fit is a difference
    # ten times smaller than y at 20 dB, hence the 1e-4 bound)
    c = synth.make_visibilities(64, 3, n_sources=4, n_antennas=24, seed=100, random_weights=True)
    pb = _problem(64, c, 6)
    st, _ = pb.run(4)
    plan = _plan(64, c)
    plan.iterate(_y(c), 4, cg_iters=6, **PRM)
    vis, w = _f32(c)
    y = np.concatenate(vis)
    wc = np.concatenate(w)
    model = plan.predict().cpu().numpy().astype(np.complex128)
    fit_gpu = 0.5 * np.sum(wc * np.abs(y - model) ** 2)
    fit_ref = 0.5 * np.sum(wc * np.abs(y - pb.apply_H(st["X"])) ** 2)
    _gpu.log_errors({"fit": float(abs(fit_gpu - fit_ref) / fit_ref)})
    assert abs(fit_gpu - fit_ref) < 1e-4 * fit_ref, (fit_gpu, fit_ref)


def test_predict_rejects_other_plans():
    c = synth.make_cube(32, 4, n_sources=2, n_antennas=16, seed=3)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        plan.predict()
    out = torch.empty(8, device="cuda")
    assert mf.lib().mf_vis_predict(plan._h, None, ctypes.c_void_p(out.data_ptr()), None) == mf.MF_ERR_INVALID
