"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, invariants, brute force, finite differences, quadrature, and the
paper's Eq. 1-2.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from paper_2406_18533_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- SH, quaternions

def test_sh_orthonormal_by_quadrature(oracle):
    """Real SH (degree <= 3) are orthonormal on the sphere: Gauss-Legendre in
    cos(theta) x uniform phi quadrature is exact for these polynomial degrees."""
    nt, nphi = 12, 24
    ct, wt = np.polynomial.legendre.leggauss(nt)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    st = np.sqrt(1 - ct ** 2)
    d = np.stack(np.broadcast_arrays(st[:, None] * np.cos(phi)[None], st[:, None] * np.sin(phi)[None],
                                     ct[:, None] * np.ones_like(phi)[None]), -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).reshape(-1)
    Y = np.zeros((d.shape[0], 16))
    oracle.lib().or_sh_eval(oracle._i64(d.shape[0]), oracle._p(np.ascontiguousarray(d)), oracle._p(Y))
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_condon_shortley_signs(oracle):
    """Degree-1 functions follow the Condon-Shortley phase: Y_1^{-1} ~ -y,
    Y_1^0 ~ +z, Y_1^1 ~ -x (the convention of the 3DGS colour model)."""
    d = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    Y = np.zeros((3, 16))
    oracle.lib().or_sh_eval(oracle._i64(3), oracle._p(d), oracle._p(Y))
    c1 = math.sqrt(3 / (4 * math.pi))
    assert Y[0, 3] == pytest.approx(-c1) and Y[1, 1] == pytest.approx(-c1) and Y[2, 2] == pytest.approx(c1)
    assert Y[0, 0] == pytest.approx(0.5 / math.sqrt(math.pi))


def test_quaternion_rotation(oracle):
    rng = np.random.default_rng(3)
    q = rng.standard_normal((50, 4)) * 3
    R = np.zeros((50, 9))
    oracle.lib().or_quat_rot(oracle._i64(50), oracle._p(q), oracle._p(R))
    R = R.reshape(50, 3, 3)
    assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-12
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-12
    # (cos t/2, 0, 0, sin t/2) is a right-handed rotation by t about +z
    t = 0.7
    qz = np.array([[math.cos(t / 2), 0, 0, math.sin(t / 2)]])
    Rz = np.zeros(9)
    oracle.lib().or_quat_rot(oracle._i64(1), oracle._p(qz), oracle._p(Rz))
    ref = np.array([[math.cos(t), -math.sin(t), 0], [math.sin(t), math.cos(t), 0], [0, 0, 1]])
    assert np.abs(Rz.reshape(3, 3) - ref).max() < 1e-15


# ---------------------------------------------------------------- closed form, one isotropic Gaussian

def _iso_scene(z, sigma, logit, dc, scale_xyz=None):
    """One Gaussian on the optical axis.  Returns the scene and the float32-stored
    values (scales, logit, DC) the closed forms must use."""
    sc = synth._empty_scene(1)
    sc.mo[0] = (0, 0, z, logit)
    s = scale_xyz if scale_xyz is not None else (sigma, sigma, sigma)
    sc.ls[0] = (math.log(s[0]), math.log(s[1]), math.log(s[2]), 0)
    sc.q[0] = (1, 0, 0, 0)
    sc.sh[:] = 0
    sc.sh[0, 0, 0:3] = dc
    eff = dict(s=np.exp(sc.ls[0, :3].astype(np.float64)), logit=float(sc.mo[0, 3]),
               dc=sc.sh[0, 0, 0:3].astype(np.float64))
    return sc, eff


def _iso_closed_form(cam, z, sx, sy, o, rgb):
    f = cam.fx
    s2x = (f * sx / z) ** 2 + 0.3
    s2y = (f * sy / z) ** 2 + 0.3
    px = np.arange(cam.W) + 0.5 - cam.cx
    py = np.arange(cam.H) + 0.5 - cam.cy
    DX, DY = np.meshgrid(px, py)
    G = np.exp(-0.5 * (DX ** 2 / s2x + DY ** 2 / s2y))
    a_raw = o * G
    alpha = np.minimum(0.99, a_raw)
    alpha = np.where(alpha < 1 / 255, 0.0, alpha)
    return dict(alpha=alpha, G=G, DX=DX, DY=DY, s2x=s2x, s2y=s2y, clamped=a_raw >= 0.99)


def test_closed_form_isotropic_image(oracle):
    cam = synth.test_camera(W=64, H=48)
    z, sigma, logit = 3.0, 0.02, 0.3
    dc = np.array([0.4, -0.2, 1.1])
    sc, eff = _iso_scene(z, sigma, logit, dc)
    sigma, logit, dc = eff["s"][0], eff["logit"], eff["dc"]
    pr = oracle.project(sc, cam)
    f = cam.fx
    s2 = (f * sigma / z) ** 2 + 0.3
    assert pr["xy"][0] == pytest.approx([cam.cx, cam.cy], abs=1e-12)
    assert pr["conic_o"][0, :3] == pytest.approx([1 / s2, 0, 1 / s2], rel=1e-12, abs=1e-15)
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(s2))
    rgb = dc * 0.5 / math.sqrt(math.pi) + 0.5
    assert pr["rgb"][0] == pytest.approx(np.maximum(rgb, 0), abs=1e-14)
    out = oracle.render(sc, cam)
    o = 1 / (1 + math.exp(-logit))
    cf = _iso_closed_form(cam, z, sigma, sigma, o, rgb)
    # pixels outside the footprint rectangle see nothing
    r = pr["radius"][0]
    inside = (np.abs(cf["DX"]) <= 16 * 8) & (np.abs(cf["DY"]) <= 16 * 8)  # whole 64x48 image is within r's tiles here
    expect = np.maximum(rgb, 0)[:, None, None] * cf["alpha"][None]
    assert r > 0 and inside.all()
    assert np.abs(out["img"] - expect).max() < 1e-12
    assert np.abs(out["T_final"] - (1 - cf["alpha"])).max() < 1e-12


def test_closed_form_clamp_and_cut(oracle):
    """o -> 1 saturates alpha at 0.99 near the centre; pixels where o G < 1/255
    get exactly nothing (bg = 0)."""
    cam = synth.test_camera(W=64, H=48)
    z, sigma = 3.0, 0.5
    sc, eff = _iso_scene(z, sigma, 9.0, np.array([1.0, 1.0, 1.0]))
    sigma = eff["s"][0]
    out = oracle.render(sc, cam)
    o = 1 / (1 + math.exp(-9.0))
    rgb = 0.5 / math.sqrt(math.pi) + 0.5
    cf = _iso_closed_form(cam, z, sigma, sigma, o, rgb)
    c = out["img"][0]
    assert cf["clamped"].sum() > 0
    assert np.all(np.abs(c[cf["clamped"]] - 0.99 * rgb) < 1e-14)
    cut = o * cf["G"] < 1 / 255
    assert cut.sum() > 0 and np.all(c[cut] == 0.0) and np.all(c[~cut] > 0)


def test_closed_form_isotropic_gradients(oracle):
    """dC/du = rgb alpha dx / s^2, du/dx = f/z (the Jacobian's x-terms vanish on
    the axis), dC/dlog(sx) = rgb alpha dx^2/(2 s^4) * 2 (f sx/z)^2, and
    dC/dlogit = rgb G o (1 - o) on unclamped pixels."""
    cam = synth.test_camera(W=64, H=48)
    z, sx, sy = 3.0, 0.03, 0.02
    logit = -0.4
    dc = np.array([0.6, 0.1, 0.2])
    sc, eff = _iso_scene(z, None, logit, dc, scale_xyz=(sx, sy, 0.05))
    (sx, sy, _), logit, dc = eff["s"], eff["logit"], eff["dc"]
    rng = np.random.default_rng(0)
    dimg = rng.standard_normal((3, cam.H, cam.W))
    grad, fw, g2d = oracle.grad_view(sc, cam, dimg)
    o = 1 / (1 + math.exp(-logit))
    rgb = dc * 0.5 / math.sqrt(math.pi) + 0.5
    cf = _iso_closed_form(cam, z, sx, sy, o, rgb)
    A = cf["alpha"]
    w = (dimg * rgb[:, None, None]).sum(0)     # sum_ch dL/dC_ch rgb_ch
    du = (w * A * cf["DX"] / cf["s2x"]).sum()
    dv = (w * A * cf["DY"] / cf["s2y"]).sum()
    assert g2d[0, 0] == pytest.approx(du, rel=1e-10)
    assert g2d[0, 1] == pytest.approx(dv, rel=1e-10)
    f = cam.fx
    assert grad[0, 0] == pytest.approx(f / z * du, rel=1e-10)
    assert grad[0, 1] == pytest.approx(f / z * dv, rel=1e-10)
    dlsx = (w * A * cf["DX"] ** 2 / (2 * cf["s2x"] ** 2)).sum() * 2 * (f * sx / z) ** 2
    dlsy = (w * A * cf["DY"] ** 2 / (2 * cf["s2y"] ** 2)).sum() * 2 * (f * sy / z) ** 2
    assert grad[0, 4] == pytest.approx(dlsx, rel=1e-10)
    assert grad[0, 5] == pytest.approx(dlsy, rel=1e-10)
    assert abs(grad[0, 6]) < 1e-12 * max(1, abs(dlsx))        # sz does not reach the image on the axis
    dlogit = (w * (A > 0) * cf["G"]).sum() * o * (1 - o)
    assert grad[0, 3] == pytest.approx(dlogit, rel=1e-10)
    # colour: dC/dsh_dc = Y0 alpha summed
    Y0 = 0.5 / math.sqrt(math.pi)
    for ch in range(3):
        assert grad[0, 12 + ch] == pytest.approx(Y0 * (dimg[ch] * A).sum(), rel=1e-10)


# ---------------------------------------------------------------- invariant

def test_weights_plus_transmittance_is_one(oracle):
    W, H = 96, 80
    pj = synth.synthetic_proj(400, W, H, seed=5)
    rect, vis = oracle.rect_f32(pj["xy"][:, 0], pj["xy"][:, 1], pj["radius"], W, H)
    toff, gidx = oracle.bin_view(rect, vis, pj["rgb_d"][:, 3], W, H)
    ones = np.ones((400, 3))
    out = oracle.render_fwd(W, H, 16, toff, gidx, pj["xy"], pj["conic_o"], ones)
    assert np.abs(out["img"][0] + out["T_final"] - 1).max() < 1e-12
    assert out["n_contrib"].max() > 10 and (out["T_final"] < 0.5).mean() > 0.2


# ---------------------------------------------------------------- rectangles and lists

def test_rect_is_tile_interval_overlap(oracle):
    """Tile tx is in the rectangle iff [tx T, (tx+1) T) meets [u - r, u + r]
    (and likewise for y), clipped to the image; checked tile by tile."""
    W, H, T = 100, 70, 16
    pj = synth.synthetic_proj(300, W, H, seed=2)
    u, v, r = pj["xy"][:, 0], pj["xy"][:, 1], pj["radius"]
    rect, vis = oracle.rect_f32(u, v, r, W, H, T)
    TX, TY = -(-W // T), -(-H // T)
    for g in range(300):
        uu, vv, rr = float(u[g]), float(v[g]), int(r[g])
        xs = [tx for tx in range(TX) if rr > 0 and tx * T <= uu + rr and uu - rr < (tx + 1) * T]
        ys = [ty for ty in range(TY) if rr > 0 and ty * T <= vv + rr and vv - rr < (ty + 1) * T]
        if xs and ys:
            assert vis[g] == 1 and list(rect[g]) == [xs[0], xs[-1], ys[0], ys[-1]]
        else:
            assert vis[g] == 0


def test_bin_lists_match_lexsort(oracle):
    W, H, T = 80, 64, 16
    pj = synth.synthetic_proj(500, W, H, seed=7, ties=60)
    rect, vis = oracle.rect_f32(pj["xy"][:, 0], pj["xy"][:, 1], pj["radius"], W, H, T)
    depth = pj["rgb_d"][:, 3]
    toff, gidx = oracle.bin_view(rect, vis, depth, W, H, T)
    TX = -(-W // T)
    for t in range(len(toff) - 1):
        tx, ty = t % TX, t // TX
        mem = [g for g in range(500) if vis[g] and rect[g, 0] <= tx <= rect[g, 1] and rect[g, 2] <= ty <= rect[g, 3]]
        mem = np.array(mem, np.int64)
        order = mem[np.lexsort((mem, depth[mem]))] if len(mem) else mem
        assert np.array_equal(gidx[toff[t]:toff[t + 1]], order)


# ---------------------------------------------------------------- brute force

def _brute_render(W, H, T, u, v, conic_o, rgb, rect, vis, depth32):
    u, v = np.asarray(u, np.float64), np.asarray(v, np.float64)
    conic_o, rgb = np.asarray(conic_o, np.float64), np.asarray(rgb, np.float64)
    img = np.zeros((3, H, W))
    Tf = np.ones((H, W))
    nc = np.zeros((H, W), np.int64)
    n = len(u)
    for py in range(H):
        for px in range(W):
            tx, ty = px // T, py // T
            S = [g for g in range(n) if vis[g] and rect[g][0] <= tx <= rect[g][1] and rect[g][2] <= ty <= rect[g][3]]
            S.sort(key=lambda g: (float(depth32[g]), g))
            Tt, C, last = 1.0, [0.0, 0.0, 0.0], 0
            for k, g in enumerate(S):
                dx, dy = px + 0.5 - u[g], py + 0.5 - v[g]
                a, b, c, o = conic_o[g]
                power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if power > 0:
                    continue
                alpha = min(0.99, o * math.exp(power))
                if alpha < 1 / 255:
                    continue
                Tn = Tt * (1 - alpha)
                if Tn < 1e-4:
                    break
                for ch in range(3):
                    C[ch] += rgb[g][ch] * alpha * Tt
                Tt, last = Tn, k + 1
            img[:, py, px] = C
            Tf[py, px] = Tt
            nc[py, px] = last
    return img, Tf, nc


@pytest.mark.parametrize("seed", [0, 1])
def test_brute_force_tiny_scene(oracle, seed):
    W, H = 32, 32
    sc = synth.tiny_scene(48, seed=seed, spread=0.5, log_s=(-2.6, 0.4))
    cam = synth.test_camera(W=W, H=H)
    out = oracle.render(sc, cam)
    pr = out["proj"]
    img, Tf, nc = _brute_render(W, H, 16, pr["xy"][:, 0], pr["xy"][:, 1], pr["conic_o"], pr["rgb"], pr["rect"],
                                pr["vis"], pr["depth"].astype(np.float32))
    assert np.abs(out["img"] - img).max() < 1e-13
    assert np.abs(out["T_final"] - Tf).max() < 1e-13
    assert np.array_equal(out["n_contrib"], nc)
    assert nc.max() > 3


def test_depth_ties_follow_index(oracle):
    """Two Gaussians at exactly the same float32 depth: the lower index composites
    first, so swapping their colours changes the image the way brute force says."""
    W, H = 32, 32
    pj = synth.synthetic_proj(2, W, H, seed=0)
    pj["xy"][:] = [[16.2, 15.7], [15.1, 16.6]]
    pj["conic_o"][:] = [[0.02, 0.001, 0.03, 0.8], [0.03, -0.002, 0.02, 0.7]]
    pj["radius"][:] = [14, 14]
    pj["rgb_d"][:, 3] = 5.0
    rgb = np.array([[1.0, 0, 0], [0, 0, 1.0]])
    rect, vis = oracle.rect_f32(pj["xy"][:, 0], pj["xy"][:, 1], pj["radius"], W, H)
    toff, gidx = oracle.bin_view(rect, vis, pj["rgb_d"][:, 3], W, H)
    out = oracle.render_fwd(W, H, 16, toff, gidx, pj["xy"], pj["conic_o"], rgb)
    img, _, _ = _brute_render(W, H, 16, pj["xy"][:, 0], pj["xy"][:, 1], pj["conic_o"], rgb, rect, vis,
                              pj["rgb_d"][:, 3])
    assert np.abs(out["img"] - img).max() < 1e-14
    # front one (index 0) is red: at the shared centre red dominates blue
    assert out["img"][0, 16, 16] > out["img"][2, 16, 16]


def test_permutation_invariance(oracle):
    sc = synth.tiny_scene(200, seed=4, spread=0.5)
    cam = synth.test_camera(W=48, H=40)
    a = oracle.render(sc, cam)["img"]
    perm = np.random.default_rng(1).permutation(200)
    sp = synth.Scene(sc.mo[perm].copy(), sc.ls[perm].copy(), sc.q[perm].copy(), sc.sh[:, perm].copy())
    b = oracle.render(sp, cam)["img"]
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("tile,window", [(16, (32, 16, 48, 32)), (8, (8, 40, 40, 24)), (32, (64, 0, 32, 64))])
def test_window_render_equals_whole_view(oracle, tile, window):
    """A window of a view composited alone equals the same pixels of the whole
    view, including Gaussians outside the window whose Jacobian is clamped at
    the whole view's field of view; a camera cut down to the window would clamp
    them at its own narrower field of view and give another image."""
    sc = synth.tiny_scene(400, seed=3, spread=1.6, log_s=(-2.5, -0.3))
    cam = synth.test_camera(W=128, H=96)
    x0, y0, w, h = window
    full = oracle.render(sc, cam, tile)
    win = oracle.render_window(sc, cam, window, tile)
    ref = full["img"][:, y0:y0 + h, x0:x0 + w]
    assert np.abs(win["img"] - ref).max() < 1e-12
    assert np.array_equal(win["n_contrib"], full["n_contrib"][y0:y0 + h, x0:x0 + w])
    assert np.allclose(win["margin"], full["margin"][y0:y0 + h, x0:x0 + w], rtol=1e-9, atol=1e-12)
    assert win["n_contrib"].max() > 3
    cut = synth.Camera(R=cam.R, t=cam.t, fx=cam.fx, fy=cam.fy, cx=np.float32(cam.cx - x0),
                       cy=np.float32(cam.cy - y0), W=w, H=h, near=cam.near)
    assert np.abs(oracle.render(sc, cut, tile)["img"] - ref).max() > 1e-6


def test_window_must_start_on_the_tile_grid(oracle):
    sc = synth.tiny_scene(10, seed=0)
    cam = synth.test_camera(W=64, H=48)
    with pytest.raises(ValueError):
        oracle.render_window(sc, cam, (8, 0, 32, 32), 16)
    with pytest.raises(ValueError):
        oracle.render_window(sc, cam, (48, 0, 32, 32), 16)


# ---------------------------------------------------------------- finite differences

def _fd_ok_scene(oracle, seed, N, cam, dimg):
    """Resample until no threshold decision or rectangle sits near a discontinuity."""
    for s in range(seed, seed + 200):
        sc = synth.tiny_scene(N, seed=s, spread=0.35, depth=(2.0, 3.0), log_s=(-2.8, 0.3), logit=(-0.5, 0.8))
        out = oracle.render(sc, cam)
        pr = out["proj"]
        if out["margin"].min() < 2e-3:
            continue
        e = pr["ext3"][pr["vis"] > 0]
        if np.any(np.abs(e - np.round(e)) < 1e-3):
            continue
        T = 16
        edges = np.concatenate([(pr["xy"][:, 0] - pr["radius"]) / T, (pr["xy"][:, 0] + pr["radius"]) / T,
                                (pr["xy"][:, 1] - pr["radius"]) / T, (pr["xy"][:, 1] + pr["radius"]) / T])
        if np.any(np.abs(edges - np.round(edges)) * T < 1e-3):
            continue
        if np.any(pr["rgb_raw"].min(1) < 1e-3) or pr["vis"].sum() < N - 1:
            continue
        return sc
    raise RuntimeError("no clean scene found")


def _loss_of(oracle, sc, cam, dimg):
    return float((oracle.render(sc, cam)["img"] * dimg).sum())


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


def _get_param(sc, g, j):
    return float(sc.flat()[g, j])


def test_finite_differences_all_parameters(oracle):
    """Central differences of <dimg, img> in FP64 against the analytic gradient
    for all 59 parameters of every Gaussian of a small clean scene.  The
    parameters are float32 inputs, so the step is taken between two float32
    values and the difference quotient divides by that exact step."""
    cam = synth.test_camera(W=40, H=32)
    rng = np.random.default_rng(11)
    dimg = rng.standard_normal((3, 32, 40))
    sc = _fd_ok_scene(oracle, 0, 6, cam, dimg)
    grad, _, _ = oracle.grad_view(sc, cam, dimg)
    checked = 0
    for g in range(sc.N):
        for j in range(60):
            if j == 7:
                continue
            th = _get_param(sc, g, j)
            h = 2.0 ** -18 * max(1.0, abs(th))
            tp, tm = float(np.float32(th + h)), float(np.float32(th - h))
            _set_param(sc, g, j, tp)
            lp = _loss_of(oracle, sc, cam, dimg)
            _set_param(sc, g, j, tm)
            lm = _loss_of(oracle, sc, cam, dimg)
            _set_param(sc, g, j, th)
            fd = (lp - lm) / (tp - tm)
            an = grad[g, j]
            scale = max(1e-3, np.abs(grad[g]).max())
            assert abs(fd - an) <= 1e-6 * scale + 1e-6 * abs(an), (g, j, fd, an)
            checked += 1
    assert checked == sc.N * 59
