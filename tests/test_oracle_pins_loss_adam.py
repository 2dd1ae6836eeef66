"""More oracle pins: finite differences under a general camera pose (with the
off-axis Jacobian clamp active), the L1 + SSIM loss (Sec. 2.1 step 3) and Adam
with the batch scaling of Eq. 1-2 (Sec. 4).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from paper_2406_18533_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _set_param(sc, g, j, val):
    if j < 4:
        sc.mo[g, j] = val
    elif j < 8:
        sc.ls[g, j - 4] = val
    elif j < 12:
        sc.q[g, j - 8] = val
    else:
        k = j - 12
        sc.sh[k // 4, g, k % 4] = val


def _fd_check(oracle, sc, cam, dimg, gauss, params=None, tol=2e-6):
    grad, fw, _ = oracle.grad_view(sc, cam, dimg)
    flat = sc.flat()
    for g in gauss:
        scale = max(1e-3, np.abs(grad[g]).max())
        for j in (params if params is not None else [j for j in range(60) if j != 7]):
            th = float(flat[g, j])
            h = 2.0 ** -18 * max(1.0, abs(th))
            tp, tm = float(np.float32(th + h)), float(np.float32(th - h))
            _set_param(sc, g, j, tp)
            lp = float((oracle.render(sc, cam)["img"] * dimg).sum())
            _set_param(sc, g, j, tm)
            lm = float((oracle.render(sc, cam)["img"] * dimg).sum())
            _set_param(sc, g, j, th)
            fd = (lp - lm) / (tp - tm)
            assert abs(fd - grad[g, j]) <= tol * scale + tol * abs(grad[g, j]), (g, j, fd, grad[g, j])
    return grad, fw


def test_fd_general_pose_and_offaxis_clamp(oracle):
    """A camera with a non-trivial rotation and translation, and one Gaussian
    whose centre lies beyond 1.3 tan(fov/2) (so the Jacobian uses the clamped
    x/z) while its footprint still reaches the image."""
    W, H = 40, 32
    cam = synth.camera_look_at((0.4, -0.3, -0.5), (0.1, 0.05, 2.8), (0.1, -1.0, 0.05), W, H, 60.0)
    Rw = cam.R.astype(np.float64)
    C = cam.center
    for seed in range(300):
        sc = synth.tiny_scene(5, seed=seed, spread=0.3, depth=(2.3, 3.0), log_s=(-2.8, 0.3), logit=(-0.3, 0.5))
        # Gaussian 0: off-axis, large, in front of the camera
        pc = np.array([1.05 * 2.6, 0.1, 2.6])            # camera-space: x/z = 1.05
        xw = Rw.T @ pc + C
        sc.mo[0, 0:3] = xw
        sc.ls[0, 0:3] = math.log(0.45)
        out = oracle.render(sc, cam)
        pr = out["proj"]
        if out["margin"].min() < 2e-3 or pr["vis"].sum() < 5:
            continue
        e = pr["ext3"]
        if np.any(np.abs(e - np.round(e)) < 1e-3):
            continue
        edges = np.concatenate([pr["xy"][:, 0] - pr["radius"], pr["xy"][:, 0] + pr["radius"],
                                pr["xy"][:, 1] - pr["radius"], pr["xy"][:, 1] + pr["radius"]]) / 16
        if np.any(np.abs(edges - np.round(edges)) * 16 < 1e-3):
            continue
        break
    else:
        raise RuntimeError("no clean scene")
    lim = 1.3 * (W / 2) / cam.fx
    pcs = (Rw @ (sc.mo[:, 0:3].astype(np.float64) - C).T).T
    assert pcs[0, 0] / pcs[0, 2] > lim                    # the clamp is active for Gaussian 0
    assert pr["xy"][0, 0] > W                              # its centre is off-screen
    rng = np.random.default_rng(2)
    dimg = rng.standard_normal((3, H, W))
    grad, _ = _fd_check(oracle, sc, cam, dimg, gauss=range(5))
    assert np.abs(grad[0, 0:3]).max() > 0


def test_fd_sh_degree_lower(oracle):
    """Degrees below 3 use only the first (d+1)^2 coefficients; the rest get no gradient."""
    W, H = 32, 32
    cam = synth.test_camera(W=W, H=H)
    sc = synth.tiny_scene(3, seed=9, spread=0.2, depth=(2.0, 2.5), log_s=(-2.6, 0.2))
    sc.sh_degree = 1
    rng = np.random.default_rng(4)
    dimg = rng.standard_normal((3, H, W))
    grad, _, _ = oracle.grad_view(sc, cam, dimg)
    assert np.all(grad[:, 12 + 12:] == 0) and np.abs(grad[:, 12:24]).max() > 0


# ---------------------------------------------------------------- loss

def _ssim_brute(x, y):
    """Per-pixel SSIM with explicit window loops (zero padding), mean over all."""
    w = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    w /= w.sum()
    w2 = np.outer(w, w)
    C, H, W = x.shape
    tot = 0.0
    for c in range(C):
        for i in range(H):
            for j in range(W):
                mx = my = exx = eyy = exy = 0.0
                for di in range(-5, 6):
                    for dj in range(-5, 6):
                        ii, jj = i + di, j + dj
                        if 0 <= ii < H and 0 <= jj < W:
                            ww = w2[di + 5, dj + 5]
                            a, b = x[c, ii, jj], y[c, ii, jj]
                            mx += ww * a
                            my += ww * b
                            exx += ww * a * a
                            eyy += ww * b * b
                            exy += ww * a * b
                sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
                C1, C2 = 0.01 ** 2, 0.03 ** 2
                tot += (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return tot / x.size


def test_ssim_brute_force(oracle):
    rng = np.random.default_rng(0)
    x = rng.random((3, 9, 13))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    L, _, l1, s = oracle.ssim_loss(x, y)
    sb = _ssim_brute(x, y)
    assert s == pytest.approx(sb, abs=1e-13)
    assert l1 == pytest.approx(np.abs(x - y).mean(), abs=1e-15)
    assert L == pytest.approx(0.8 * np.abs(x - y).mean() + 0.2 * (1 - sb), abs=1e-13)


def test_ssim_identity_and_gradient_zero(oracle):
    rng = np.random.default_rng(1)
    x = rng.random((3, 20, 17))
    L, dx, l1, s = oracle.ssim_loss(x, x)
    assert s == pytest.approx(1.0, abs=1e-14) and L == pytest.approx(0.0, abs=1e-14)
    assert np.abs(dx).max() < 1e-14                # L1 term: sign(0) = 0, SSIM term: stationary


def test_l1_gradient_is_sign(oracle):
    """With y = x except a tiny bump at one pixel the SSIM term is stationary
    (its gradient is O(bump)), so the gradient there is the L1 term
    0.8 sign(x - y) / n = -0.8 / n, and 0 elsewhere (sign(0) = 0)."""
    rng = np.random.default_rng(2)
    x = rng.random((3, 16, 16))
    y = x.copy()
    i = (1, 5, 7)
    y[i] += 1e-9
    _, d, _, _ = oracle.ssim_loss(x, y)
    n = x.size
    assert d[i] == pytest.approx(-0.8 / n, rel=1e-6)
    mask = np.ones_like(d, bool)
    mask[i] = False
    assert np.abs(d[mask]).max() < 1e-9


def test_loss_finite_differences(oracle):
    rng = np.random.default_rng(3)
    x = rng.random((3, 14, 12))
    y = rng.random((3, 14, 12))
    L, dx, _, _ = oracle.ssim_loss(x, y)
    for idx in [(0, 0, 0), (1, 7, 5), (2, 13, 11), (0, 3, 10), (2, 0, 6)]:
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.ssim_loss(xp, y)[0] - oracle.ssim_loss(xm, y)[0]) / (2 * h)
        assert fd == pytest.approx(dx[idx], rel=1e-6, abs=1e-11)


# ---------------------------------------------------------------- Adam (Eq. 1-2)

def test_adam_batch_scaling_matches_paper_equations(oracle):
    gold = json.load(open(os.path.join(GOLDEN, "eq1_eq2_batch_scaling.json")))
    lr6 = (1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3)
    N = 4
    rng = np.random.default_rng(0)
    p = rng.standard_normal((N, 60))
    g = rng.standard_normal((N, 60))
    m = rng.standard_normal((N, 60)) * 0.1
    v = rng.random((N, 60)) * 0.1
    for case in gold["cases"]:
        B = case["batch"]
        b1, b2, f = case["beta1"], case["beta2"], case["lr_factor"]
        p2, m2, v2 = oracle.adam(p, g, m, v, step=3, lr6=lr6, beta1=gold["beta1"], beta2=gold["beta2"], batch=B)
        assert np.allclose(m2, b1 * m + (1 - b1) * g, rtol=1e-14, atol=1e-15)
        assert np.allclose(v2, b2 * v + (1 - b2) * g * g, rtol=1e-14, atol=1e-15)
        lr = oracle.lane_lr(lr6) * f
        mh, vh = m2 / (1 - b1 ** 3), v2 / (1 - b2 ** 3)
        assert np.allclose(p2, p - lr * mh / (np.sqrt(vh) + 1e-15), rtol=1e-13, atol=1e-15)


def test_adam_first_step_moves_by_lr(oracle):
    """At step 1 m_hat = g and v_hat = g^2, so |dp| = lr' wherever |g| >> eps."""
    lr6 = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-4)
    rng = np.random.default_rng(1)
    p = rng.standard_normal((10, 60))
    g = rng.standard_normal((10, 60))
    for B in (1, 4, 16):
        p2, _, _ = oracle.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr6, batch=B)
        expect = oracle.lane_lr(lr6) * math.sqrt(B)
        assert np.allclose(np.abs(p2 - p), np.broadcast_to(expect, p.shape), rtol=1e-9, atol=0)
    p2, _, _ = oracle.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr6, batch=4,
                           scale_lr_sqrt_b=False, scale_beta_pow_b=False)
    assert np.allclose(np.abs(p2 - p), np.broadcast_to(oracle.lane_lr(lr6), p.shape), rtol=1e-9)


def test_lane_groups_cover_59_parameters(oracle):
    v = oracle.lane_lr((1, 2, 3, 4, 5, 6))
    assert list(v[0:3]) == [1, 1, 1] and v[3] == 4 and list(v[4:7]) == [2, 2, 2] and v[7] == 0
    assert list(v[8:12]) == [3] * 4 and list(v[12:15]) == [5] * 3 and np.all(v[15:] == 6)


# ---------------------------------------------------------------- batch mean (Sec. 4 derivation)

def test_train_step_gradient_is_mean_over_views(oracle):
    """The batch gradient is the mean of the per-view gradients (g = sum_k g_k / b)."""
    sc = synth.tiny_scene(30, seed=5, spread=0.5)
    cams = [synth.test_camera(W=32, H=24), synth.camera_look_at((0.2, 0.1, -0.3), (0, 0, 3), (0, -1, 0), 32, 24, 60)]
    rng = np.random.default_rng(0)
    tg = rng.random((2, 3, 24, 32))
    N = sc.N
    z = np.zeros((N, 60))
    _, _, _, losses, grad = oracle.train_step(sc, cams, tg, z, z, 1, (1e-3,) * 6)
    per = []
    for b in range(2):
        fw = oracle.render(sc, cams[b])
        L, dimg, _, _ = oracle.ssim_loss(fw["img"], tg[b])
        assert L == pytest.approx(losses[b], abs=1e-15)
        per.append(oracle.grad_view(sc, cams[b], dimg)[0])
    assert np.allclose(grad, (per[0] + per[1]) / 2, rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- visible-only Adam

def test_visible_only_adam_rows(oracle):
    """Visible-only Adam takes dense Adam's step (pinned above to Eq. 1-2) on
    the visible rows and leaves p, m and v of the others exactly as they were;
    with every row visible it is dense Adam."""
    lr6 = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-4)
    rng = np.random.default_rng(3)
    N = 50
    p, g = rng.standard_normal((N, 60)), rng.standard_normal((N, 60))
    m, v = rng.standard_normal((N, 60)) * 0.1, rng.random((N, 60)) * 0.1
    vis = rng.random(N) < 0.4
    g[~vis] = 0.0                                  # an unseen Gaussian has no gradient
    for B, step in ((1, 1), (16, 7)):
        dp, dm, dv = oracle.adam(p, g, m, v, step, lr6, batch=B)
        sp, sm, sv = oracle.adam(p, g, m, v, step, lr6, batch=B, visible=vis)
        assert np.array_equal(sp[vis], dp[vis]) and np.array_equal(sm[vis], dm[vis]) and np.array_equal(sv[vis], dv[vis])
        assert np.array_equal(sp[~vis], p[~vis]) and np.array_equal(sm[~vis], m[~vis]) and np.array_equal(sv[~vis], v[~vis])
        # dense Adam moves the unseen rows (stale moments), visible-only does not
        assert np.abs(dp[~vis] - p[~vis]).max() > 0
        ap, am, av = oracle.adam(p, g, m, v, step, lr6, batch=B, visible=np.ones(N, bool))
        assert np.array_equal(ap, dp) and np.array_equal(am, dm) and np.array_equal(av, dv)


def test_train_step_visible_only_skips_unseen_gaussians(oracle):
    """In a training step, visible means some view of the batch gives the
    Gaussian a tile rectangle; Gaussians behind both cameras keep p, m, v,
    the others take the dense step."""
    sc = synth.tiny_scene(40, seed=6, spread=0.5)
    sc.mo[:8, 2] = -2.0                            # behind both cameras
    cams = [synth.test_camera(W=32, H=24), synth.camera_look_at((0.2, 0.1, -0.3), (0, 0, 3), (0, -1, 0), 32, 24, 60)]
    rng = np.random.default_rng(1)
    tg = rng.random((2, 3, 24, 32))
    N = sc.N
    m, v = rng.standard_normal((N, 60)) * 1e-3, rng.random((N, 60)) * 1e-6
    lr6 = (1e-3,) * 6
    dp, dm, dv, _, grad = oracle.train_step(sc, cams, tg, m, v, 2, lr6)
    sp, sm, sv, _, grad2 = oracle.train_step(sc, cams, tg, m, v, 2, lr6, sparse=True)
    seen = np.zeros(N, bool)
    for cam in cams:
        seen |= oracle.project(sc, cam)["radius"] > 0
    assert not seen[:8].any() and seen[8:].sum() > 10
    # (the oracle's backward adds with OpenMP atomics: equal up to summation order)
    assert np.allclose(grad, grad2, rtol=1e-10, atol=1e-18) and np.all(grad[~seen] == 0)
    p0 = sc.flat().astype(np.float64)
    assert np.array_equal(sp[~seen], p0[~seen]) and np.array_equal(sm[~seen], m[~seen]) and np.array_equal(sv[~seen], v[~seen])
    assert np.allclose(sp[seen], dp[seen], rtol=1e-10, atol=1e-15) and np.allclose(sm[seen], dm[seen], rtol=1e-8, atol=1e-18)
    assert np.abs(dp[~seen] - p0[~seen]).max() > 0


# ---------------------------------------------------------------- densification (App. A.1)

def _densify_case():
    """Eight Gaussians, one per case: pruned (opacity below 0.005), kept (no
    view, low gradient), cloned (gradient test passes exactly at the
    threshold, small scale), split (large scale), and others."""
    rng = np.random.default_rng(9)
    N = 8
    p = rng.standard_normal((N, 60)).astype(np.float32)
    p[:, 7] = 0
    p[:, 3] = 1.0                                           # opacity 0.73
    p[0, 3] = -6.0                                          # opacity 0.0025: pruned
    p[:, 4:7] = np.log(0.05)                                # small scales
    p[3, 4:7] = (np.log(0.05), np.log(0.5), np.log(0.02))   # one axis large: split
    p[6, 4:7] = np.log(0.3)
    m = rng.standard_normal((N, 60)).astype(np.float32) * 0.1
    v = rng.random((N, 60)).astype(np.float32) * 0.1
    cnt = np.array([5, 0, 4, 4, 3, 2, 7, 4], np.uint32)
    thr = np.float32(0.25)
    acc = (thr * cnt.astype(np.float32)).astype(np.float32)  # exactly at the threshold: grows
    acc[1] = 9.0                                            # no view: kept whatever acc says
    acc[4] = np.nextafter(acc[4], np.float32(0))            # one ulp below: kept
    acc[5] *= 3
    normals = rng.standard_normal((N, 2, 3))
    return p, m, v, acc, cnt, normals, float(thr)


def test_densify_actions_and_rows(oracle):
    p, m, v, acc, cnt, normals, thr = _densify_case()
    act = oracle.densify_actions(p, acc, cnt, thr, 0.1)
    assert list(act) == [0, 1, 2, 3, 1, 2, 3, 2]
    po, mo, vo, src, kind = oracle.densify(p, m, v, acc, cnt, normals, thr, 0.1)
    assert len(po) == 7 - 0 + 3 * 1 + 2 * 1 - 2 + 2          # 1 pruned, 2 kept, 3 clones (+3), 2 splits (+2)
    assert list(src) == [1, 2, 2, 3, 3, 4, 5, 5, 6, 6, 7, 7]
    assert list(kind) == [1, 2, 4, 3, 3, 1, 2, 4, 3, 3, 2, 4]
    for r, (g, k) in enumerate(zip(src, kind)):
        if k in (1, 2, 4):
            assert np.array_equal(po[r], p[g].astype(np.float64))
            if k == 4:
                assert not po[r].any() or (mo[r] == 0).all() and (vo[r] == 0).all()
            else:
                assert np.array_equal(mo[r], m[g].astype(np.float64)) and np.array_equal(vo[r], v[g].astype(np.float64))
        else:
            # a child: R^T (x_child - x) / s recovers its normal draw exactly
            q = p[g, 8:12].astype(np.float64)
            R = np.zeros(9)
            oracle.lib().or_quat_rot(oracle._i64(1), oracle._p(np.ascontiguousarray(q[None])), oracle._p(R))
            s = np.exp(p[g, 4:7].astype(np.float64))
            xi = (R.reshape(3, 3).T @ (po[r, 0:3] - p[g, 0:3])) / s
            c = r - int(np.nonzero(src == g)[0][0])
            assert np.allclose(xi, normals[g, c], atol=1e-12)
            assert np.array_equal(po[r, 4:7].astype(np.float32),
                                  (p[g, 4:7] - np.float32(math.log(1.6))).astype(np.float32))
            assert np.array_equal(po[r, 8:60], p[g, 8:60].astype(np.float64)) and po[r, 3] == p[g, 3]
            assert (mo[r] == 0).all() and (vo[r] == 0).all()


def test_split_children_follow_the_gaussian(oracle):
    """Split children drawn from standard normals lie at N(mean, R S^2 R^T):
    over 20,000 draws the offsets' covariance matches the Gaussian's (3%)."""
    rng = np.random.default_rng(2)
    n = 20000
    p = np.zeros((n, 60), np.float32)
    p[:, 3] = 2.0
    p[:, 4:7] = np.log([0.3, 0.1, 0.05])
    p[:, 8:12] = [0.9, 0.3, -0.2, 0.25]
    acc = np.ones(n, np.float32)
    cnt = np.ones(n, np.uint32)
    normals = rng.standard_normal((n, 2, 3))
    po, _, _, src, kind = oracle.densify(p, p * 0, p * 0, acc, cnt, normals, 0.5, 0.01)
    assert (kind == 3).all() and len(po) == 2 * n
    d = po[:, 0:3]
    C = np.cov(d.T)
    q = p[0, 8:12].astype(np.float64)
    R = np.zeros(9)
    oracle.lib().or_quat_rot(oracle._i64(1), oracle._p(np.ascontiguousarray(q[None])), oracle._p(R))
    R = R.reshape(3, 3)
    S = np.diag(np.exp(p[0, 4:7].astype(np.float64)) ** 2)
    ref = R @ S @ R.T
    assert np.abs(C - ref).max() < 0.03 * np.abs(ref).max()


def test_opacity_reset(oracle):
    rng = np.random.default_rng(4)
    p = rng.standard_normal((20, 60)).astype(np.float32) * 4
    m = rng.standard_normal((20, 60)).astype(np.float32)
    v = rng.random((20, 60)).astype(np.float32)
    p2, m2, v2 = oracle.reset_opacity(p, m, v, 0.01)
    o2 = 1 / (1 + np.exp(-p2[:, 3].astype(np.float64)))
    o = 1 / (1 + np.exp(-p[:, 3].astype(np.float64)))
    assert np.allclose(o2, np.minimum(o, 0.01), rtol=1e-6)
    assert (m2[:, 3] == 0).all() and (v2[:, 3] == 0).all()
    keep = np.ones(60, bool)
    keep[3] = False
    assert np.array_equal(p2[:, keep], p[:, keep]) and np.array_equal(m2[:, keep], m[:, keep])


def test_densify_statistics_count_visible_views(oracle):
    """Statistics of one step: each Gaussian's count is the number of views
    of the batch that see it (a Gaussian behind one camera counts once), and
    its sum is the sum of the lengths of its per-view position gradients."""
    sc = synth.tiny_scene(30, seed=5, spread=0.5)
    cams = [synth.test_camera(W=32, H=24), synth.camera_look_at((0.0, 0.0, 8.0), (0, 0, 3), (0, -1, 0), 32, 24, 60)]
    sc.mo[0, 2] = 9.0                                # behind the second camera: only the first sees it
    rng = np.random.default_rng(0)
    tg = rng.random((2, 3, 24, 32))
    st = dict(acc=np.zeros(30), cnt=np.zeros(30, np.int64))
    z = np.zeros((30, 60))
    oracle.train_step(sc, cams, tg, z, z, 1, (1e-3,) * 6, stats=st)
    vis = np.stack([oracle.project(sc, c)["vis"] > 0 for c in cams])
    assert np.array_equal(st["cnt"], vis.sum(0)) and vis[0, 0] and not vis[1, 0]
    ref = np.zeros(30)
    for b, cam in enumerate(cams):
        fw = oracle.render(sc, cam)
        _, dimg, _, _ = oracle.ssim_loss(fw["img"], tg[b])
        pr = fw["proj"]
        g2d = oracle.render_bwd(cam.W, cam.H, 16, fw["toff"], fw["gidx"], pr["xy"], pr["conic_o"], pr["rgb"], dimg)
        ref += np.where(vis[b], np.sqrt(g2d[:, 0] ** 2 + g2d[:, 1] ** 2), 0.0)
    assert np.allclose(st["acc"], ref, rtol=1e-9, atol=1e-15)
