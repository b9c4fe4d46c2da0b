"""Spectral dictionary with the Chebyshev basis (spectral_mask bit 1): the CUDA
path against the oracle's union-of-bases steps IV-VI (Section 3, step V with
m_nu bases; Section 4's Chebyshev suggestion), and the library's Chebyshev
matrix against the oracle's.

The library builds the orthonormal Chebyshev basis as the eigenvectors of the
discrete Chebyshev difference equation (long double Jacobi rotations); the
oracle by the Stieltjes procedure: two constructions of one matrix, compared
to 1e-13 for L <= 64.  Parity bounds as everywhere: 1e-5 (FP32 plans) and
1e-10 (FP64 plans) of each array's scale; Gamma_V2 on rho_V max |S W_2|.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1504_06847_gb300 as mf  # noqa: E402
from paper_1504_06847_gb300 import synth  # noqa: E402
from tests import _gpu  # noqa: E402

PRM = synth.WORKLOAD_PARAMS


@pytest.mark.parametrize("L", [2, 3, 8, 15, 32, 64])
def test_library_chebyshev_matrix_equals_the_oracles(L):
    from paper_1504_06847_gb300 import build

    build.build()
    C2 = np.array(mf.spectral_basis(mf.SPECTRAL_CHEBYSHEV, L))
    assert np.max(np.abs(C2 - oracle.chebyshev_matrix(L))) < 1e-13
    assert np.max(np.abs(np.array(mf.spectral_basis(mf.SPECTRAL_DCT, L)) - oracle.dct_matrix(L))) < 1e-14


@pytest.fixture(scope="module")
def gpu():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _views(plan, pb, st, mask):
    g = _gpu.gpu_state(plan)
    o = _gpu.oracle_view(pb, st)
    sc = _gpu.scales(pb, st)
    C2 = oracle.chebyshev_matrix(pb.L)
    GV = st["GV"] if pb.mnu > 1 else st["GV"][None]
    S2 = np.abs(np.einsum("kl,lij->kij", C2, st["S"])).max()
    if mask & 2:
        g["GV2"] = plan.get(mf.ARR_GAMMA_V2).double().cpu().numpy()
        o["GV2"] = GV[-1]
        sc["GV2"] = pb.params["rho_V"] * S2
    if mask & 1:
        o["GV"] = GV[0]
    else:
        g.pop("GV")
        o.pop("GV")
    return g, o, sc


@pytest.mark.gpu
@pytest.mark.parametrize("mask,dtype,tol", [(3, torch.float32, 1e-5), (2, torch.float32, 1e-5),
                                            (3, torch.float64, 1e-10)])
def test_dictionary_matches_oracle(gpu, mask, dtype, tol):
    c = synth.workload("64x64x8")
    spectral = tuple(name for bit, name in ((1, "dct"), (2, "cheb")) if mask & bit)
    n_iter = 30
    pb = oracle.Problem(c.psf, c.y, PRM, spectral=spectral)
    st, H = pb.run(n_iter, hist=True)
    prec = mf.MF_FP32 if dtype == torch.float32 else mf.MF_FP64
    plan = mf.Plan(torch.tensor(c.psf, dtype=dtype, device="cuda"))
    plan.iterate(torch.tensor(c.y, dtype=dtype, device="cuda"), n_iter, spectral_mask=mask, precision=prec,
                 resid_every=n_iter, **PRM)
    rep = plan.report()
    assert rep["status"] == mf.MF_OK
    g, o, sc = _views(plan, pb, st, mask)
    errs = _gpu.compare(g, o, sc, keys=tuple(g))
    assert max(errs.values()) < tol, errs
    red = {"objective": abs(rep["objective"] - H[-1, 3]) / H[-1, 3],
           "primal_res": abs(rep["primal_res"] - H[-1, 0]) / H[-1, 0],
           "dual_res": abs(rep["dual_res"] - H[-1, 1]) / H[-1, 1]}
    _gpu.log_errors(red)
    assert red["objective"] < tol and (dtype == torch.float32 or max(red.values()) < tol), red


@pytest.mark.gpu
def test_dictionary_rejections(gpu):
    c = synth.make_cube(32, 4, n_sources=2, n_antennas=16, seed=3)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    for kw in (dict(spectral_mask=0), dict(spectral_mask=4),
               dict(spectral_mask=3, precision=mf.MF_FP32_DCT_SPLITBF16)):
        with pytest.raises(mf.MFError) as e:
            plan.iterate(y, 1, **dict(PRM, **kw))
        assert e.value.status == mf.MF_ERR_INVALID
    with pytest.raises(mf.MFError):
        plan.backward(y, 2, torch.zeros_like(y), rho=1.0, spectral_mask=3)


@pytest.mark.gpu
def test_most_bands(gpu):
    # L = 64, the most bands the Chebyshev basis is offered for
    c = synth.make_cube(32, 64, n_sources=3, n_antennas=16, seed=98)
    pb = oracle.Problem(c.psf, c.y, PRM, spectral=("dct", "cheb"))
    st, _ = pb.run(8)
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), 8, spectral_mask=3, **PRM)
    g, o, sc = _views(plan, pb, st, 3)
    errs = _gpu.compare(g, o, sc, keys=tuple(g))
    assert max(errs.values()) < 1e-5, errs


@pytest.mark.gpu
def test_warm_restart_from_a_saved_state(gpu):
    # the plan keeps S in the Chebyshev basis (M S^) beside S^; a state set from
    # outside makes it rebuild that array before the next iteration, so that
    # 3 + (save, restore into a new plan) + 3 iterations equal 6 in one plan
    c = synth.workload("64x64x8")
    psf = torch.tensor(c.psf, dtype=torch.float32, device="cuda")
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    a = mf.Plan(psf)
    a.iterate(y, 6, spectral_mask=3, **PRM)
    b = mf.Plan(psf)
    b.iterate(y, 3, spectral_mask=3, **PRM)
    state = b.get_state().clone()
    cont = mf.Plan(psf)
    cont.set_state(state)
    cont.iterate(y, 3, spectral_mask=3, warm_start=1, **PRM)
    ga, gc = _gpu.gpu_state(a), _gpu.gpu_state(cont)
    ga["GV2"] = a.get(mf.ARR_GAMMA_V2).double().cpu().numpy()
    gc["GV2"] = cont.get(mf.ARR_GAMMA_V2).double().cpu().numpy()
    errs = {k: _gpu.rel_err(gc[k], ga[k]) for k in ga}
    assert max(errs.values()) < 1e-5, errs
