"""Densification on the GPU (gs_densify, gs_set_densify_stats,
gs_reset_opacity) against the oracle.  The integer structure of a
densification (which Gaussians are pruned, kept, cloned or split, and where
each output row lands) is decided by float32 comparisons that both sides make
the same way, so it must match bit for bit; copied rows must be bit-exact, and
split children's means (float32 on the GPU, FP64 in the oracle) match to
float32 rounding."""
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


def _scene(flat):
    N = flat.shape[0]
    f = np.ascontiguousarray(flat, np.float32)
    return synth.Scene(f[:, 0:4].copy(), f[:, 4:8].copy(), f[:, 8:12].copy(),
                       f[:, 12:60].reshape(N, 12, 4).transpose(1, 0, 2).copy())


def _case(N=50_000, seed=3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((N, 60)).astype(np.float32)
    p[:, 7] = 0
    p[:, 3] = rng.normal(0.0, 3.0, N).astype(np.float32)         # some below logit(0.005) = -5.29
    p[:, 4:7] = rng.normal(np.log(0.05), 0.8, (N, 3)).astype(np.float32)
    m = (rng.standard_normal((N, 60)) * 0.1).astype(np.float32)
    v = (rng.random((N, 60)) * 0.1).astype(np.float32)
    cnt = rng.integers(0, 9, N).astype(np.uint32)
    thr = np.float32(0.3)
    acc = (rng.random(N) * 0.6 * cnt).astype(np.float32)
    exact = rng.random(N) < 0.05                                   # exactly at the threshold
    acc[exact] = (thr * cnt[exact].astype(np.float32)).astype(np.float32)
    normals = rng.standard_normal((N, 2, 3)).astype(np.float32)
    return p, m, v, acc, cnt, normals, float(thr)


def test_densify_matches_oracle(eng, oracle):
    p, m, v, acc, cnt, normals, thr = _case()
    ref_p, ref_m, ref_v, src, kind = oracle.densify(p, m, v, acc, cnt, normals.astype(np.float64), thr, 0.1)
    assert {1, 2, 3, 4} <= set(kind.tolist()) and len(ref_p) != len(p)
    ctx = eng.Context()
    P, M, V = (eng.DeviceScene.from_host(_scene(a)) for a in (p, m, v))
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    Po, Mo, Vo = ctx.densify(P, M, V, t(acc, np.float32), t(cnt.view(np.int32), np.int32),
                             t(normals.reshape(-1), np.float32), thr, 0.1)
    assert Po.N == len(ref_p)
    gp, gm, gv = (x.flat().cpu().numpy() for x in (Po, Mo, Vo))
    copy = kind != 3
    assert np.array_equal(gp[copy], ref_p[copy].astype(np.float32))
    assert np.array_equal(gm, ref_m.astype(np.float32)) and np.array_equal(gv, ref_v.astype(np.float32))
    child = kind == 3
    assert np.array_equal(gp[child][:, 3:60], ref_p[child][:, 3:60].astype(np.float32))
    err = np.abs(gp[child][:, 0:3] - ref_p[child][:, 0:3])
    scale = np.abs(ref_p[child][:, 0:3]) + np.exp(p[src[child], 4:7].astype(np.float64)).max(1, keepdims=True) * 4
    assert (err <= 4e-6 * scale).all()


def test_densify_capacity_overflow_reports_needed(eng, oracle):
    from paper_2406_18533_gb300 import binding as b
    p, m, v, acc, cnt, normals, thr = _case(N=4000, seed=5)
    need = len(oracle.densify(p, m, v, acc, cnt, normals.astype(np.float64), thr, 0.1)[0])
    ctx = eng.Context()
    P, M, V = (eng.DeviceScene.from_host(_scene(a)) for a in (p, m, v))
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    with pytest.raises(b.GSError) as ei:
        ctx.densify(P, M, V, t(acc, np.float32), t(cnt.view(np.int32), np.int32), t(normals.reshape(-1), np.float32),
                    thr, 0.1, capacity=need - 1)
    assert ei.value.status == b.GS_ERR_CAPACITY


def test_opacity_reset_matches_oracle(eng, oracle):
    p, m, v, *_ = _case(N=3000, seed=7)
    ctx = eng.Context()
    P, M, V = (eng.DeviceScene.from_host(_scene(a)) for a in (p, m, v))
    ctx.reset_opacity(P, M, V, 0.01)
    rp, rm, rv = oracle.reset_opacity(p, m, v, 0.01)
    assert np.array_equal(P.flat().cpu().numpy(), rp) and np.array_equal(M.flat().cpu().numpy(), rm)
    assert np.array_equal(V.flat().cpu().numpy(), rv)


def test_training_statistics_match_oracle(eng, oracle):
    """Two training steps with the statistics on: per Gaussian the number of
    views that saw it (exact wherever float32 cannot decide the visibility
    the other way) and the summed lengths of its per-view position gradients
    (relative L2 1e-3) against the oracle's two steps."""
    sc, rng = synth.aerial_scene(30_000, n_clusters=6, seed=8)
    cams = synth.ring_cameras(rng, 2, (30.0, 70.0), W=192, H=108)
    tg = np.stack([synth.blurred_noise_target(rng, 108, 192) for _ in cams])
    lr6 = (1.6e-4 * 70, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-4)
    ctx = eng.Context(lr=lr6)
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    acc = torch.zeros(sc.N, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(sc.N, dtype=torch.int32, device="cuda")
    ctx.set_densify_stats(acc, cnt)
    ctx.train_step(P, G, M, V, 1, cams, torch.from_numpy(tg).cuda(), check=True)
    torch.cuda.synchronize()
    ctx.set_densify_stats(None, None)
    st = dict(acc=np.zeros(sc.N), cnt=np.zeros(sc.N, np.int64))
    z = np.zeros((sc.N, 60))
    oracle.train_step(sc, cams, tg, z, z, 1, lr6, stats=st)
    sure = np.ones(sc.N, bool)
    for cam in cams:
        bd = oracle.fp32_bounds(sc, cam)
        inner = (bd["rect_in"][:, 0] <= bd["rect_in"][:, 1]) & (bd["rect_in"][:, 2] <= bd["rect_in"][:, 3])
        sure &= inner | (bd["vis_out"] == 0)
    c = cnt.cpu().numpy().astype(np.int64)
    assert np.array_equal(c[sure], st["cnt"][sure]) and st["cnt"].sum() > 10000
    a = acc.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a[sure] - st["acc"][sure]) <= 1e-3 * np.linalg.norm(st["acc"][sure])
