"""Host-side contracts of the C ABI on a GPU:

* a pinned host field may be overwritten as soon as ftk_plan_execute
  returns (the call waits for its copy), and the results still match the
  oracle;
* ftk_plan_download_into fills a caller-owned (pinned) record buffer and
  reports a short buffer with FTK_ERR_NOMEM and the true count;
* a stream's device state that grows past its server's budget is refused
  with FTK_ERR_BUSY before anything is allocated, and the server's count
  never exceeds the budget.
"""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

from parity_util import compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2011_08697_gb300 import build, ftk
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ftk


def _pinned_records(F, n):
    t = torch.empty(max(1, n) * F.CP_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    return t.numpy().view(F.CP_DTYPE), t


@pytest.mark.parametrize("make", [
    lambda: synth.spiral_woven(256, 16, sigma=1e-3, seed=0),
    lambda: synth.gaussian_blobs((40, 36, 32), 5, nblobs=12, seed=7, sigma_range=(2.0, 6.0)),
    lambda: synth.random_levels((5, 23, 37), seed=1),
])
def test_pinned_input_reusable_after_execute(F, make):
    f = make()
    ref = cp.track(f)
    host = torch.from_numpy(f.copy()).pin_memory()
    side = torch.cuda.Stream()
    with F.Plan(f.shape) as plan:
        for _ in range(2):
            host.copy_(torch.from_numpy(f))
            plan.execute(host, side)
            host.zero_()               # the copy has completed: overwriting is safe
            compare_full(plan.download(), ref)
        host.copy_(torch.from_numpy(f))
        plan.execute(host, side)
        host.fill_(0.5)
        buf, _keep = _pinned_records(F, len(ref["face_id"]) + 7)
        got = plan.download_into(buf)
        compare_full(got, ref)
        if len(ref["face_id"]) > 1:
            short, _k2 = _pinned_records(F, len(ref["face_id"]) - 1)
            with pytest.raises(F.FtkError) as e:
                plan.download_into(short)
            assert e.value.status == 3


def test_stream_growth_is_charged_to_the_budget(F):
    shape = (64, 64)
    big = F.Server(1 << 40)
    s = F.Stream(shape, server=big)
    fp = big.used()
    s.close(False)
    assert big.used() == 0
    big.close()
    tight = F.Server(fp)                 # room for the stream as opened, no more
    s = F.Stream(shape, server=tight)
    assert tight.used() == fp
    f = synth.random_levels((80, 64, 64), seed=3)
    pushed = 0
    with pytest.raises(F.FtkError) as e:
        for k in range(f.shape[0]):
            s.push(torch.from_numpy(np.ascontiguousarray(f[k])).cuda())
            pushed += 1
            assert tight.used() <= fp
    assert e.value.status == 6, e.value
    # the footprint charged at open covers the first push; the union-find
    # slots of the punctures kept from it make the next one grow
    assert pushed >= 1
    assert tight.used() <= fp
    s.close(False)
    assert tight.used() == 0
    tight.close()


def test_bounded_device_loops_report_timeout(F):
    """With the union-find bound set to one step, a run whose trajectories
    need deeper finds gives up and reports FTK_ERR_TIMEOUT (no fault, no
    hang); with the defaults restored the same plan matches the oracle."""
    L = F.lib()
    cases = [synth.spiral_woven(32, 10), synth.random_levels((4, 7, 9, 8), seed=21)]
    for f in cases:
        ref = cp.track(f)
        assert len(np.unique(ref["label"])) < len(ref["face_id"])   # some trajectory has >= 2 faces
        with F.Plan(f.shape) as plan:
            x = torch.from_numpy(f).cuda()
            try:
                assert L.ftk_debug_set_wait_limits(1, 1) == 0
                plan.execute(x)
                with pytest.raises(F.FtkError) as e:
                    plan.count()
                assert e.value.status == 5
            finally:
                assert L.ftk_debug_set_wait_limits(0, 0) == 0
            plan.execute(x)
            compare_full(plan.download(), ref)
