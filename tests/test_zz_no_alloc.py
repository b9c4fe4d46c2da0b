"""The allocation-free step I entry point (mf_xstep_noalloc) against the plan path.

Callers that cannot allocate device memory (no cudaMalloc where they run) use
mf_xstep_noalloc: its scratch is a static device array of the library.  Its
result must equal the step I of mf_admm_iterate for the same right-hand side
b, on consecutive calls (the shared static scratch keeps the previous call's
contents, which must not leak into the next result).  This file is collected
last on purpose.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1504_06847_gb300 as mf  # noqa: E402
from paper_1504_06847_gb300 import synth  # noqa: E402

PRM = synth.WORKLOAD_PARAMS


def test_rejects_cubes_beyond_the_static_scratch():
    from paper_1504_06847_gb300 import build

    build.build()
    p = mf.default_params(**PRM)
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    L = mf.lib()
    assert L.mf_xstep_noalloc(1024, 64, fake, fake, fake, ctypes.byref(p), fake) == mf.MF_ERR_TOO_LARGE
    assert L.mf_xstep_noalloc(256, 16, fake, fake, fake, ctypes.byref(p), fake) == mf.MF_ERR_TOO_LARGE
    assert L.mf_xstep_noalloc(24, 4, fake, fake, fake, ctypes.byref(p), fake) == mf.MF_ERR_INVALID
    assert "static scratch" in mf.status_string(mf.MF_ERR_TOO_LARGE)


def _plan_step_one(cube, b):
    """Step I of the plan path with right-hand side b: run one iteration to set the
    state up, overwrite b, run one warm iteration and read its X."""
    plan = mf.Plan(torch.tensor(cube.psf, dtype=torch.float32, device="cuda"))
    y = torch.tensor(cube.y, dtype=torch.float32, device="cuda")
    plan.iterate(y, 1, **PRM)
    plan.set(mf.ARR_B, b)
    plan.iterate(y, 1, warm_start=1, **PRM)
    x = plan.x().clone()
    plan.close()
    return x


@pytest.mark.gpu
def test_noalloc_xstep_matches_plan_path_on_two_calls():
    """Consecutive calls with different shapes and PSFs (so the second cannot
    reuse the first one's transfer function, Nyquist columns or twiddles left
    in the static array), each against the plan path's step I; the smaller
    case also against the oracle's step I (Eq. linsystemX, solved with the
    Fourier filter of Section 3), and an in-place call (x_out aliasing b)."""
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(5)
    cases = [synth.make_cube(128, 16, n_sources=8, n_antennas=64, seed=11),   # 2^18 voxels
             synth.make_cube(64, 8, n_sources=4, n_antennas=40, seed=12)]
    for call, cube in enumerate(cases):
        L, N = cube.y.shape[0], cube.y.shape[-1]
        assert N * N * L <= mf.XSTEP_NOALLOC_MAX_VOXELS
        psf = torch.tensor(cube.psf, dtype=torch.float32, device="cuda")
        y = torch.tensor(cube.y, dtype=torch.float32, device="cuda")
        b = torch.tensor(0.3 * rng.normal(size=cube.y.shape), dtype=torch.float32, device="cuda")
        ref = _plan_step_one(cube, b)
        x_out = torch.full_like(y, float("nan"))
        mf.xstep_noalloc(psf, y, b, x_out, **PRM)
        torch.cuda.synchronize()
        err = (x_out - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-6, (call, err)
        if call == 1:
            pb = oracle.Problem(cube.psf, cube.y, PRM)
            xo = pb.solve(pb.HtY + b.double().cpu().numpy())
            x = x_out.double().cpu().numpy()
            assert np.abs(x - xo).max() / np.abs(xo).max() < 1e-5
            # in place: the result replaces b
            bb = b.clone()
            mf.xstep_noalloc(psf, y, bb, bb, **PRM)
            torch.cuda.synchronize()
            assert torch.equal(bb, x_out)
