"""The allocation-free entry point ftk_track_cp2d_noalloc, called through the
C ABI, must return exactly what the allocating entry point ftk_track_cp2d
returns, and (on the small odd-shaped fields) what the CPU oracle returns.  It exists for callers that cannot allocate device memory (a host
application that has reserved the GPU's memory for its own pool, code that
must not trigger the device synchronisation cudaMalloc/cudaFree can cause);
its scratch is one static device array shared by every call, so the test
calls it twice in a row to show that stale contents from the previous call do
not leak into the next.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth
from parity_util import compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OFF_TOL = 1e-5   # the tolerance the parity tests use for locations


def _noalloc(F, x, cap, dims=None):
    L = F.lib()
    nt, ny, nx = dims if dims is not None else x.shape
    out = torch.empty(max(cap, 1) * F.CP_DTYPE.itemsize, dtype=torch.uint8, device=x.device)
    cnt = ctypes.c_int64(-1)
    p = F.make_params()
    st = L.ftk_track_cp2d_noalloc(ctypes.c_void_p(x.data_ptr()), nx, ny, nt, ctypes.byref(p),
                                  ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    n = cnt.value
    rec = None
    if st == 0:
        rec = np.frombuffer(out[: n * F.CP_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=F.CP_DTYPE)
    return st, n, rec


def _same(a, b):
    assert len(a) == len(b)
    for k in ("face_id", "label", "base", "morse_index", "ordinal", "ndim"):
        assert np.array_equal(a[k], b[k]), k
    if len(a):
        assert float(np.max(np.abs(a["off"] - b["off"]))) <= OFF_TOL


def test_noalloc_matches_allocating_entry_point():
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    fields = [synth.spiral_woven(256, 16, sigma=1e-3, seed=4),
              synth.spiral_woven(32, 10)]
    for f in fields:
        x = torch.from_numpy(f).cuda()
        ref = F.ftk_track_cp2d(x)
        assert len(ref) > 0
        for _ in range(2):       # two calls in a row share the scratch array
            st, n, got = _noalloc(F, x, cap=len(ref) + 100)
            assert st == 0, F.lib().ftk_last_error()
            assert n == len(ref)
            _same(got, ref)


def test_noalloc_reports_short_output_buffer():
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    x = torch.from_numpy(synth.spiral_woven(32, 10)).cuda()
    ref = F.ftk_track_cp2d(x)
    st, n, _ = _noalloc(F, x, cap=len(ref) // 2)
    assert st == 3 and n == len(ref)          # FTK_ERR_NOMEM with the true count
    st, n, got = _noalloc(F, x, cap=len(ref))
    assert st == 0
    _same(got, ref)


def test_noalloc_odd_shapes_and_no_device_allocation():
    """Odd widths and heights (the tiled kernel reads them in place), and
    device free memory unchanged across calls once the kernels are loaded."""
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    for f in (synth.random_levels((5, 17, 33), seed=5),
              synth.spiral_woven(37, 6, sigma=0.02, seed=1, ny=29)):
        x = torch.from_numpy(f).cuda()
        ref = F.ftk_track_cp2d(x)
        st, n, got = _noalloc(F, x, cap=len(ref) + 3)
        assert st == 0, F.lib().ftk_last_error()
        _same(got, ref)
        compare_full(got, cp.track(f))        # and the oracle itself
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            st, n, got = _noalloc(F, x, cap=len(ref) + 3)
            assert st == 0
            _same(got, ref)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_grids_beyond_its_limits():
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    # more segments (nt * ceil(ny / rows per tile)) than FTK_NOALLOC_MAX_SEGMENTS
    x = torch.zeros((300_000, 2, 4), dtype=torch.float32, device="cuda")
    st, n, _ = _noalloc(F, x, cap=16)
    assert st == 1 and n == 0
    # rows too wide for the detect tile
    x = torch.zeros((1, 2, 4000), dtype=torch.float32, device="cuda")
    st, n, _ = _noalloc(F, x, cap=16)
    assert st == 1 and n == 0
