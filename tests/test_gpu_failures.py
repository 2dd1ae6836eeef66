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
