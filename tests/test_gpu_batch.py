"""Batched form: several cubes of uneven N and L in one CUDA-graph launch.

Each cube's result must equal its own mf_admm_iterate run bit for bit (the
batch changes the launch structure, not the arithmetic), and one cube is
checked against the FP64 oracle.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1504_06847_gb300 as mf  # noqa: E402
from paper_1504_06847_gb300 import autotune, synth  # noqa: E402
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


def _cubes(shapes, seed0=400):
    out = []
    for i, (N, L) in enumerate(shapes):
        out.append(synth.make_cube(N, L, n_sources=max(2, int(40 * (N / 256) ** 2)), n_antennas=64, seed=seed0 + i))
    return out


def _plans(cubes):
    return [mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda")) for c in cubes]


def _ys(cubes):
    return [torch.tensor(c.y, dtype=torch.float32, device="cuda") for c in cubes]


@pytest.mark.parametrize("precision", [mf.MF_FP32, mf.MF_FP32_DCT_SPLITBF16])
def test_batch_equals_solo_runs(precision):
    shapes = [(64, 8), (128, 16), (32, 4), (256, 32), (64, 15)]
    cubes = _cubes(shapes)
    plans, ys = _plans(cubes), _ys(cubes)
    mf.batch_iterate(plans, ys, 12, precision=precision, **PRM)
    for c, p, y in zip(cubes, plans, ys):
        solo = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
        solo.iterate(y, 12, precision=precision, **PRM)
        a, b = _gpu.gpu_state(p), _gpu.gpu_state(solo)
        for k in a:
            assert np.array_equal(a[k], b[k]), (c.y.shape, k)
        assert p.report()["status"] == mf.MF_OK


def test_batch_cube_matches_oracle():
    cubes = _cubes([(64, 8), (128, 16)], seed0=7)
    plans, ys = _plans(cubes), _ys(cubes)
    mf.batch_iterate(plans, ys, 20, **PRM)
    pb = oracle.Problem(cubes[0].psf, cubes[0].y, PRM)
    st, _ = pb.run(20)
    errs = _gpu.compare(_gpu.gpu_state(plans[0]), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-5, errs


def test_batch_sixteen_uneven_cubes_warm_continuation():
    # 16 cubes, N in {128, 256, 512}, L in {16, 32, 64}; two batch calls equal one longer solo run
    rng = np.random.default_rng(400)
    shapes = [(int(rng.choice([128, 256, 512])), int(rng.choice([16, 32, 64]))) for _ in range(16)]
    cubes = _cubes(shapes)
    plans, ys = _plans(cubes), _ys(cubes)
    mf.batch_iterate(plans, ys, 6, **PRM)
    mf.batch_iterate(plans, ys, 4, warm_start=1, **PRM)
    for i in (0, 7, 15):
        solo = mf.Plan(torch.tensor(cubes[i].psf, dtype=torch.float32, device="cuda"))
        solo.iterate(ys[i], 10, **PRM)
        assert torch.equal(plans[i].x(), solo.x()), shapes[i]


def test_batch_rejects_bad_input():
    cubes = _cubes([(32, 4), (32, 4)])
    plans, ys = _plans(cubes), _ys(cubes)
    with pytest.raises(mf.MFError) as e:
        mf.batch_iterate([plans[0], plans[0]], [ys[0], ys[1]], 2, **PRM)
    assert e.value.status == mf.MF_ERR_INVALID
    p64 = mf.Plan(torch.tensor(cubes[0].psf, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        mf.batch_iterate([p64], [ys[0]], 2, **PRM)


def test_autotuner_keeps_results_identical(tmp_path):
    c = synth.make_cube(256, 16, n_sources=10, n_antennas=64, seed=3)
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    ref = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    ref.iterate(y, 5, **PRM)
    p = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    rec = autotune.tune(p, y, cache=str(tmp_path / "tune.json"), **PRM)
    assert rec["wav_tile"] in (32, 64)
    p.iterate(y, 5, **PRM)
    assert torch.equal(p.x(), ref.x())
    rec2 = autotune.tune(p, y, cache=str(tmp_path / "tune.json"), **PRM)  # cached
    assert rec2["wav_tile"] == rec["wav_tile"]
    # the other tile gives bitwise the same iterate
    other = 32 if rec["wav_tile"] == 64 else 64
    p.set_option(mf.MF_OPT_WAV_TILE, other)
    p.iterate(y, 5, **PRM)
    assert torch.equal(p.x(), ref.x())


@pytest.mark.parametrize("n_iter", [4, 3])
def test_repeated_calls_relaunch_the_graph_exactly(n_iter):
    # identical consecutive calls relaunch the captured graph (even n_iter); an odd
    # n_iter swaps the Gamma_T double buffer, so each call captures anew: both must
    # equal one solo run of all the iterations, bit for bit
    shapes = [(64, 8), (32, 4), (128, 16)]
    cubes = _cubes(shapes, seed0=31)
    plans, ys = _plans(cubes), _ys(cubes)
    mf.batch_iterate(plans, ys, n_iter, **PRM)
    for _ in range(3):
        mf.batch_iterate(plans, ys, n_iter, warm_start=1, resid_every=2, **PRM)
    for c, p, y in zip(cubes, plans, ys):
        solo = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
        solo.iterate(y, n_iter, **PRM)
        for _ in range(3):
            solo.iterate(y, n_iter, warm_start=1, resid_every=2, **PRM)
        a, b = _gpu.gpu_state(p), _gpu.gpu_state(solo)
        for k in a:
            assert np.array_equal(a[k], b[k]), (c.y.shape, k)
        ra, rb = p.report(), solo.report()
        assert ra["iters_done"] == rb["iters_done"] == 4 * n_iter
        assert ra["resid_iter"] == rb["resid_iter"] and ra["objective"] == rb["objective"]
