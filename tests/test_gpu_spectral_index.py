"""The CUDA spectral-index fit (mf_spectral_index) against the oracle's.

Per pixel the kernel forms log S(nu_l) and three dot products with the rows of
the fit's pseudo-inverse P in FP32.  Its error is bounded by the FP32 rounding
of each log and of each product-sum: |d coef_k| <= 4 eps32 sum_l |P_kl| (|log S_l| + 1),
which the test evaluates per pixel.  Pixels with a value <= floor must be NaN
on both sides.  Shapes: L = 3 (the fewest bands that determine the fit), 15
(the paper's bands) and 64, N not a multiple of the block size.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1504_06847_gb300 as mf  # noqa: E402

EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module")
def gpu():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


@pytest.mark.gpu
@pytest.mark.parametrize("N,L", [(37, 3), (64, 15), (45, 64)])
def test_fit_matches_oracle(gpu, N, L):
    rng = np.random.default_rng(N + L)
    nu = 1.0 + np.sort(rng.uniform(0, 1, size=L)) + 0.01 * np.arange(L)
    u = np.log(nu / nu[0])[:, None, None]
    cube = (rng.uniform(0.05, 2.0, size=(N, N)) * np.exp((rng.uniform(-1, 1, size=(N, N))
                                                          + rng.uniform(-0.3, 0.3, size=(N, N)) * u) * u))
    cube *= np.exp(0.01 * rng.normal(size=cube.shape))  # not exactly of the model's form
    cube[:, 3, 4] = 0.0          # no log-scale fit
    cube[L // 2, 7, 1] = -0.5
    c32 = cube.astype(np.float32)
    outs = mf.spectral_index(torch.tensor(c32, device="cuda"), nu)
    torch.cuda.synchronize()
    ref = oracle.spectral_index(c32.astype(np.float64), nu)
    A = np.stack([np.ones(L), u.ravel(), u.ravel() ** 2], axis=1)
    P = np.linalg.pinv(A)
    logs = np.log(np.where(c32 > 0, c32, 1.0).astype(np.float64))
    for k in range(3):
        g = outs[k].double().cpu().numpy()
        assert np.array_equal(np.isnan(g), np.isnan(ref[k])), k
        assert np.isnan(g[3, 4]) and np.isnan(g[7, 1])
        bound = 4 * EPS32 * np.einsum("l,lij->ij", np.abs(P[k]), np.abs(logs) + 1.0)
        ok = ~np.isnan(ref[k])
        assert np.all(np.abs(g - ref[k])[ok] <= bound[ok]), (k, np.max((np.abs(g - ref[k]) / bound)[ok]))


def test_rejects_bad_input_without_touching_the_device():
    import ctypes

    from paper_1504_06847_gb300 import build

    build.build()
    L = mf.lib()

    nu = (ctypes.c_double * 3)(1.0, 1.0, 1.0)  # one distinct frequency: no fit
    fake = ctypes.c_void_p(256)  # never dereferenced: checks come first
    assert L.mf_spectral_index(8, 3, fake, nu, 1.0, 0.0, fake, fake, fake, None) == mf.MF_ERR_INVALID
    nu2 = (ctypes.c_double * 2)(1.0, 2.0)
    assert L.mf_spectral_index(8, 2, fake, nu2, 1.0, 0.0, fake, fake, fake, None) == mf.MF_ERR_INVALID
