"""Failure path of the bounded device waits, exercised without a GPU fault.

The split-BF16 spectral kernel waits on an mbarrier for its tensor-core
products, with an SM-cycle limit.  The test-only plan option
MF_OPT_TEST_TC_STALL makes CTA 0 skip its product and the commit that would
complete that wait, and shortens its limit: the wait runs out with nothing in
flight, the CTA records the expiry in the plan's device error word, frees its
tensor memory and returns.  The host must see MF_ERR_TIMEOUT, the latched
status must block further work until cleared, and the plan must then iterate
to the oracle's result again.  Few stalled launches are made (each CTA holds
64 of an SM's 512 tensor-memory columns), so even a lost allocation could not
exhaust an SM.
"""

import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1504_06847_gb300 as mf  # noqa: E402
from paper_1504_06847_gb300 import synth  # noqa: E402
from tests import _gpu  # noqa: E402

pytestmark = pytest.mark.gpu
PRM = synth.WORKLOAD_PARAMS
SPLIT = mf.MF_FP32_DCT_SPLITBF16


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_expired_tensor_core_wait_is_reported_and_the_plan_recovers():
    c = synth.workload("64x64x8")
    plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    plan.set_option(mf.MF_OPT_TEST_TC_STALL, 100000)  # ~50 us at 2 GHz
    plan.iterate(y, 2, precision=SPLIT, **PRM)
    assert plan.report()["status"] == mf.MF_ERR_TIMEOUT
    with pytest.raises(mf.MFError) as e:  # latched until cleared
        plan.iterate(y, 1, precision=SPLIT, **PRM)
    assert e.value.status == mf.MF_ERR_TIMEOUT
    plan.set_option(mf.MF_OPT_TEST_TC_STALL, 0)
    plan.clear_status()
    assert plan.report()["status"] == mf.MF_OK
    n_iter = 50
    plan.iterate(y, n_iter, precision=SPLIT, **PRM)
    assert plan.report()["status"] == mf.MF_OK
    pb = oracle.Problem(c.psf, c.y, PRM)
    st, _ = pb.run(n_iter)
    errs = _gpu.compare(_gpu.gpu_state(plan), _gpu.oracle_view(pb, st), _gpu.scales(pb, st))
    assert max(errs.values()) < 1e-4, errs


def test_clear_status_rejects_null():
    assert mf.lib().mf_plan_clear_status(None) == mf.MF_ERR_INVALID
