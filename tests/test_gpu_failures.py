"""Failure paths on the GPU, produced without faulting, trapping or hanging it.

* A bounded device wait that runs out: tile 0 of every radix-sort pass
  withholds its look-back counts (a flag nothing sets) and the waits of the
  later tiles are limited to 64 polls.  The binning must report
  GS_ERR_TIMEOUT, every kernel after it must stay inside its buffers (the
  compositing runs on the broken lists and the stream stays healthy), a
  training step must leave the parameters untouched, and the next call with
  the default limit must give the correct result.
* Non-finite parameters in strict mode report GS_ERR_NONFINITE.
* An injected allocation failure returns GS_ERR_OOM and leaves the context
  usable.
* Corrupt caller tile ranges are refused on the device (GS_ERR_INVALID_ARG),
  with no read outside the fragment list.
"""
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


def _proj(eng, pj):
    t = lambda k, dt: torch.from_numpy(pj[k][None].astype(dt)).cuda()
    return eng.Proj(t("xy", np.float32), t("conic_o", np.float32), t("rgb_d", np.float32), t("radius", np.int32))


def test_lookback_wait_runs_out_reports_timeout_and_recovers(eng):
    from paper_2406_18533_gb300 import binding as b
    W, H = 320, 240
    pj = synth.synthetic_proj(12000, W, H, seed=21)
    cam = synth.test_camera(W, H)
    proj = _proj(eng, pj)
    ctx = eng.Context()
    good = ctx.bin(proj, [cam])
    assert good.F > 3 * 4096                         # several sort tiles per pass
    ref = [t[:good.F].clone() for t in (good.keys, good.vals)] + [good.ranges.clone()]
    assert ctx.status()[0] == b.GS_OK
    lib = b.lib()
    try:
        assert lib.gs_debug_set_lookback(64, 1) == b.GS_OK
        bad = ctx.bin(proj, [cam], capacity=good.capacity)
        code, _ = ctx.status()
        assert code == b.GS_ERR_TIMEOUT
        # the kernels after the failed sort stay in bounds: composite on the broken lists
        img, T, nc = ctx.render_fwd(proj, bad, [cam])
        torch.cuda.synchronize()
        assert bool(torch.isfinite(img).all()) and bool(torch.isfinite(T).all())
        r = bad.ranges.cpu().numpy().view(np.uint32)
        assert int(r.max()) <= good.capacity
    finally:
        lib.gs_debug_set_lookback(0, 0)
    again = ctx.bin(proj, [cam], capacity=good.capacity)
    assert ctx.status()[0] == b.GS_OK
    assert torch.equal(again.keys[:good.F], ref[0]) and torch.equal(again.vals[:good.F], ref[1])
    assert torch.equal(again.ranges, ref[2])


def test_training_step_with_a_failed_sort_changes_nothing(eng):
    from paper_2406_18533_gb300 import binding as b
    sc, rng = synth.aerial_scene(60_000, n_clusters=8, seed=3)
    cams = synth.ring_cameras(rng, 2, (30.0, 90.0), W=256, H=144)
    tg = torch.from_numpy(np.stack([synth.blurred_noise_target(rng, 144, 256) for _ in cams])).cuda()
    ctx = eng.Context()
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    ctx.train_step(P, G, M, V, 0, cams, tg, check=True)      # sizes the scratch, step 1
    before = P.flat().clone()
    lib = b.lib()
    try:
        lib.gs_debug_set_lookback(64, 1)
        ctx.train_step(P, G, M, V, 0, cams, tg)
        torch.cuda.synchronize()
        code, _ = ctx.status()
    finally:
        lib.gs_debug_set_lookback(0, 0)
    assert code == b.GS_ERR_TIMEOUT
    assert torch.equal(P.flat(), before)                      # update and step counter skipped
    ctx.train_step(P, G, M, V, 0, cams, tg, check=True)      # step 2 now
    ref_ctx = eng.Context()
    P2 = eng.DeviceScene.from_host(sc)
    G2, M2, V2 = P2.zeros_like(), P2.zeros_like(), P2.zeros_like()
    for _ in range(2):
        ref_ctx.train_step(P2, G2, M2, V2, 0, cams, tg, check=True)
    a, r = P.flat().cpu().numpy().astype(np.float64), P2.flat().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r)


def test_strict_nonfinite_reports(eng):
    from paper_2406_18533_gb300 import binding as b
    sc = synth.tiny_scene(300, seed=2)
    sc.mo[7, 1] = np.nan
    sc.q[9, 2] = np.inf
    cam = synth.test_camera(64, 48)
    P = eng.DeviceScene.from_host(sc)
    lax = eng.Context()
    lax.preprocess(P, [cam])
    assert lax.status()[0] == b.GS_OK and lax.counters()["culled_nonfinite"] == 2
    strict = eng.Context(strict_nonfinite=1)
    strict.preprocess(P, [cam])
    assert strict.status()[0] == b.GS_ERR_NONFINITE
    assert strict.status()[0] == b.GS_OK                      # read once, then cleared


def test_injected_allocation_failure_leaves_the_context_usable(eng):
    from paper_2406_18533_gb300 import binding as b
    sc, rng = synth.aerial_scene(30_000, n_clusters=8, seed=4)
    cams = synth.ring_cameras(rng, 2, (30.0, 90.0), W=192, H=108)
    tg = torch.from_numpy(np.stack([synth.blurred_noise_target(rng, 108, 192) for _ in cams])).cuda()
    ctx = eng.Context()
    lib = b.lib()
    try:
        assert lib.gs_debug_fail_alloc(3) == b.GS_OK
        with pytest.raises(b.GSError) as ei:
            ctx.reserve(sc.N, cams, 200_000)
        assert ei.value.status == b.GS_ERR_OOM
    finally:
        lib.gs_debug_fail_alloc(-1)
    ctx.reserve(sc.N, cams, 200_000)
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    loss = ctx.train_step(P, G, M, V, 1, cams, tg, check=True)
    ref = eng.Context()
    P2 = eng.DeviceScene.from_host(sc)
    G2, M2, V2 = P2.zeros_like(), P2.zeros_like(), P2.zeros_like()
    loss2 = ref.train_step(P2, G2, M2, V2, 1, cams, tg, check=True)
    assert torch.allclose(loss, loss2, rtol=1e-6)


def test_corrupt_tile_ranges_are_refused(eng):
    """Caller-supplied tile ranges that end past the fragment list, or are
    reversed, make gs_render_fwd and gs_render_bwd blend nothing on those
    tiles instead of reading outside the list (the first kind also reports
    GS_ERR_INVALID_ARG; reversed ranges also come from a sort that failed,
    which is reported already); every other tile renders as before."""
    from paper_2406_18533_gb300 import binding as b
    W, H, tile = 160, 96, 16
    pj = synth.synthetic_proj(4000, W, H, seed=23)
    cam = synth.test_camera(W, H)
    proj = _proj(eng, pj)
    ctx = eng.Context(tile=tile)
    bins = ctx.bin(proj, [cam])
    img0, T0, nc0 = ctx.render_fwd(proj, bins, [cam])
    torch.cuda.synchronize()
    assert ctx.status()[0] == b.GS_OK
    cap = bins.capacity
    assert int(bins.ranges[3, 1] - bins.ranges[3, 0]) > 0 and int(bins.ranges[7, 1] - bins.ranges[7, 0]) > 0
    bins.ranges[3, 0], bins.ranges[3, 1] = cap - 2, cap + 4096        # ends past the list
    bins.ranges[7, 0], bins.ranges[7, 1] = 9, 4                       # reversed
    img, T, nc = ctx.render_fwd(proj, bins, [cam])
    torch.cuda.synchronize()
    assert ctx.status()[0] == b.GS_ERR_INVALID_ARG
    bad = torch.zeros(H, W, dtype=torch.bool, device="cuda")
    bad[0:16, 48:64] = True                                           # tile 3 of a 10-tile row
    bad[0:16, 112:128] = True                                         # tile 7
    assert bool((T[0][bad] == 1).all()) and bool((nc[0][bad] == 0).all())
    assert torch.equal(img[0][:, ~bad], img0[0][:, ~bad]) and torch.equal(T[0][~bad], T0[0][~bad])
    dimg = torch.ones_like(img)
    g = ctx.render_bwd(proj, bins, [cam], T, nc, dimg)
    torch.cuda.synchronize()
    assert ctx.status()[0] == b.GS_ERR_INVALID_ARG
    assert all(bool(torch.isfinite(getattr(g, k)).all()) for k in ("d_xy_o", "d_conic", "d_rgb"))
