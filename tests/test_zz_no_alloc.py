"""gs_bin_noalloc, the binning entry point for callers that cannot allocate
device memory (a fixed memory budget owned by a host application's allocator,
loops that cannot afford the device synchronisation of cudaMalloc/cudaFree,
callers without a gs_ctx).  Its results must equal gs_bin's bit for bit
(integer keys, indices and ranges), on two calls in a row, since every call
reuses the same static scratch array; the second call must not change the
device's free memory.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2406_18533_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2406_18533_gb300 import build
    build.build()
    from paper_2406_18533_gb300 import engine
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return engine


def _upload(eng, pjs):
    t = lambda k, dt: torch.from_numpy(np.stack([p[k] for p in pjs]).astype(dt)).cuda()
    return eng.Proj(t("xy", np.float32), t("conic_o", np.float32), t("rgb_d", np.float32), t("radius", np.int32))


def _noalloc(eng, proj, cams, tile, bins, with_needed=True):
    from paper_2406_18533_gb300 import binding as b
    needed = ctypes.c_uint64(0)
    ps, bs = proj.struct(), bins.struct()
    st = b.lib().gs_bin_noalloc(ctypes.byref(ps), b.camera_array(cams), len(cams), tile, ctypes.byref(bs),
                                ctypes.byref(needed) if with_needed else None,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, int(needed.value)


def test_noalloc_binning_equals_gs_bin_on_two_calls(eng):
    W, H, tile = 150, 90, 16
    cams = [synth.test_camera(W, H), synth.test_camera(W, H)]
    ctx = eng.Context(tile=tile)
    for call, seed in enumerate((21, 22)):
        pjs = [synth.synthetic_proj(5000, W, H, seed=seed + 7 * v, ties=200) for v in range(len(cams))]
        proj = _upload(eng, pjs)
        ref = ctx.bin(proj, cams)                       # the existing entry point
        F = ref.F
        tiles = eng.total_tiles(cams, tile)
        out = eng.Bins.empty(F + 1000, tiles)
        out.ranges.fill_(-1)                            # stale values must be overwritten
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st, needed = _noalloc(eng, proj, cams, tile, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0 and needed == F
        if call == 1:
            assert free1 == free0, "the allocation-free binning changed the device's free memory"
        assert int(out.count.item()) == F
        assert torch.equal(out.keys[:F], ref.keys[:F])
        assert torch.equal(out.vals[:F], ref.vals[:F])
        assert torch.equal(out.ranges, ref.ranges)


def test_noalloc_binning_reports_capacity_and_limits(eng):
    from paper_2406_18533_gb300 import binding as b
    W, H, tile = 64, 48, 16
    cams = [synth.test_camera(W, H)]
    pj = synth.synthetic_proj(800, W, H, seed=5)
    proj = _upload(eng, [pj])
    ref = eng.Context(tile=tile).bin(proj, cams)
    small = eng.Bins.empty(16, eng.total_tiles(cams, tile))
    st, needed = _noalloc(eng, proj, cams, tile, small)
    assert st == b.GS_ERR_CAPACITY and needed == ref.F
    # without needed_host the overflow is only visible as *count == 0 (documented):
    # the call returns GS_OK and writes nothing past the capacity
    small.count.fill_(12345)
    st, _ = _noalloc(eng, proj, cams, tile, small, with_needed=False)
    torch.cuda.synchronize()
    assert st == b.GS_OK and int(small.count.item()) == 0
    # beyond the fixed scratch: rejected on the host before any work
    big = eng.Bins.empty(16, eng.total_tiles(cams, tile))
    big.keys = torch.empty(b.NOALLOC_MAX_FRAGS + 1, dtype=torch.int64, device="cuda")
    big.vals = torch.empty(b.NOALLOC_MAX_FRAGS + 1, dtype=torch.int32, device="cuda")
    assert _noalloc(eng, proj, cams, tile, big)[0] == b.GS_ERR_INVALID_ARG
    many = eng.Proj.empty(2, b.NOALLOC_MAX_PAIRS // 2 + 1)
    assert _noalloc(eng, many, cams * 2, tile, small)[0] == b.GS_ERR_INVALID_ARG
    assert _noalloc(eng, proj, cams, 12, small)[0] == b.GS_ERR_INVALID_ARG
