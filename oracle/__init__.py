"""FP64 CPU oracle for the 3DGS training hot path (arXiv 2406.18533, Sec. 2.1 and Sec. 4).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package; the library under
``paper_2406_18533_gb300`` never does, and this package never imports it.

Parts:

* ``gs_oracle.c`` (plain C, double precision): Gaussian transformation
  (Sec. 2.1 step 1), per-tile lists, per-pixel front-to-back compositing
  (Sec. 2.1 step 2) and the analytic backward of both.
* ``ssim_loss`` (numpy + scipy correlation, double precision): the L1 + SSIM
  loss of Sec. 2.1 step 3 and its gradient.
* ``adam`` (numpy, double precision): Adam with the batch-size scaling of
  Eq. 1 (learning rate times sqrt(batch)) and Eq. 2 (betas to the power batch).

Parity pins live in ``tests/test_oracle_*.py``; none of them compares the
oracle with itself.  Every function here is pinned (closed forms, invariants,
brute force, finite differences, quadrature); nothing is "parity unpinned"
apart from the conventions the paper leaves open (camera axes, dilation, the
colour offset, the stop rule, the background), which no test can fix.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_gs_oracle.so")
_lib = None
_lock = threading.Lock()

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.or_bin_count.restype = ctypes.c_int64
            _lib.or_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i64(x):
    return ctypes.c_int64(int(x))


def cam16(cam) -> np.ndarray:
    c = np.empty(16, np.float64)
    c[0:9] = np.asarray(cam.R, np.float32).astype(np.float64).reshape(9)
    c[9:12] = np.asarray(cam.t, np.float32).astype(np.float64)
    c[12:16] = [cam.fx, cam.fy, cam.cx, cam.cy]
    return c


def _scene_arrays(scene):
    return (np.ascontiguousarray(scene.mo, np.float32), np.ascontiguousarray(scene.ls, np.float32),
            np.ascontiguousarray(scene.q, np.float32), np.ascontiguousarray(scene.sh, np.float32))


def num_threads() -> int:
    return int(lib().or_num_threads())


# ----------------------------------------------------------------------------
# Sec. 2.1 step 1: Gaussian transformation
# ----------------------------------------------------------------------------

def project(scene, cam, tile=16):
    """Per-Gaussian projected state of one view, FP64."""
    mo, ls, q, sh = _scene_arrays(scene)
    N = mo.shape[0]
    out = dict(xy=np.zeros((N, 2)), conic_o=np.zeros((N, 4)), rgb=np.zeros((N, 3)), rgb_raw=np.zeros((N, 3)),
               depth=np.zeros(N), ext3=np.zeros(N), radius=np.zeros(N, np.int32), rect=np.zeros((N, 4), np.int32))
    c = cam16(cam)
    lib().or_preprocess(_i64(N), _p(mo), _p(ls), _p(q), _p(sh), ctypes.c_int(scene.sh_degree), _p(c),
                        ctypes.c_int(cam.W), ctypes.c_int(cam.H), ctypes.c_double(cam.near), ctypes.c_int(tile),
                        _p(out["xy"]), _p(out["conic_o"]), _p(out["rgb"]), _p(out["rgb_raw"]), _p(out["depth"]),
                        _p(out["ext3"]), _p(out["radius"]), _p(out["rect"]))
    out["vis"] = (out["radius"] > 0).astype(np.int32)
    return out


def rect_f32(u, v, radius, W, H, tile=16):
    """Tile rectangles from float32 centres and integer radii, IEEE single ops."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    r = np.ascontiguousarray(radius, np.int32)
    n = u.shape[0]
    rect = np.zeros((n, 4), np.int32)
    vis = np.zeros(n, np.int32)
    lib().or_rect_f32(_i64(n), _p(u), _p(v), _p(r), ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile),
                      _p(rect), _p(vis))
    return rect, vis


def bin_view(rect, vis, depth_f32, W, H, tile=16):
    """Per-tile lists (CSR) ordered by (float32 depth, index)."""
    rect = np.ascontiguousarray(rect, np.int32)
    vis = np.ascontiguousarray(vis, np.int32)
    d = np.ascontiguousarray(depth_f32, np.float32)
    n = rect.shape[0]
    F = int(lib().or_bin_count(_i64(n), _p(rect), _p(vis)))
    nt = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    toff = np.zeros(nt + 1, np.int64)
    gidx = np.zeros(max(F, 1), np.int32)
    lib().or_bin(_i64(n), _p(rect), _p(vis), _p(d), ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile),
                 _p(toff), _p(gidx))
    return toff, gidx[:F]


# ----------------------------------------------------------------------------
# Sec. 2.1 step 2: rendering, forward and backward
# ----------------------------------------------------------------------------

def _blend_params(bg, alpha_min, alpha_max, T_min):
    return np.array([alpha_min, alpha_max, T_min, bg[0], bg[1], bg[2]], np.float64)


def render_fwd(W, H, tile, toff, gidx, xy, conic_o, rgb, bg=(0.0, 0.0, 0.0),
               alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN):
    xy = np.ascontiguousarray(xy, np.float64)
    conic_o = np.ascontiguousarray(conic_o, np.float64)
    rgb = np.ascontiguousarray(rgb, np.float64)
    toff = np.ascontiguousarray(toff, np.int64)
    gidx = np.ascontiguousarray(gidx, np.int32)
    img = np.zeros((3, H, W))
    Tf = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    marg = np.zeros((H, W))
    ne = np.zeros((H, W), np.int32)
    prm = _blend_params(bg, alpha_min, alpha_max, T_min)
    lib().or_render_fwd(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile), _p(toff), _p(gidx), _p(xy),
                        _p(conic_o), _p(rgb), _p(prm), _p(img), _p(Tf), _p(nc), _p(marg), _p(ne))
    return dict(img=img, T_final=Tf, n_contrib=nc, margin=marg, n_eval=ne)


def render_bwd(W, H, tile, toff, gidx, xy, conic_o, rgb, dimg, bg=(0.0, 0.0, 0.0),
               alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN):
    """Gradient of <dimg, img> w.r.t. (u, v, a, b, c, o, r, g, b) per Gaussian: [n, 9]."""
    xy = np.ascontiguousarray(xy, np.float64)
    conic_o = np.ascontiguousarray(conic_o, np.float64)
    rgb = np.ascontiguousarray(rgb, np.float64)
    toff = np.ascontiguousarray(toff, np.int64)
    gidx = np.ascontiguousarray(gidx, np.int32)
    dimg = np.ascontiguousarray(dimg, np.float64)
    n = xy.shape[0]
    g2d = np.zeros((n, 9))
    prm = _blend_params(bg, alpha_min, alpha_max, T_min)
    lib().or_render_bwd(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile), _p(toff), _p(gidx), _p(xy),
                        _p(conic_o), _p(rgb), _p(prm), _p(dimg), _p(g2d))
    return g2d


def preprocess_bwd(scene, cam, g2d, tile=16):
    """dL/dparams [N, 60] of one view from the per-Gaussian screen-space gradients."""
    mo, ls, q, sh = _scene_arrays(scene)
    N = mo.shape[0]
    g2d = np.ascontiguousarray(g2d, np.float64)
    grad = np.zeros((N, 60))
    c = cam16(cam)
    lib().or_preprocess_bwd(_i64(N), _p(mo), _p(ls), _p(q), _p(sh), ctypes.c_int(scene.sh_degree), _p(c),
                            ctypes.c_int(cam.W), ctypes.c_int(cam.H), ctypes.c_double(cam.near),
                            ctypes.c_int(tile), _p(g2d), _p(grad))
    return grad


def render(scene, cam, tile=16, **kw):
    """Full forward of one view in FP64: project, bin by FP64 rectangles and
    depth rounded to float32, composite."""
    pr = project(scene, cam, tile)
    toff, gidx = bin_view(pr["rect"], pr["vis"], pr["depth"].astype(np.float32), cam.W, cam.H, tile)
    out = render_fwd(cam.W, cam.H, tile, toff, gidx, pr["xy"], pr["conic_o"], pr["rgb"], **kw)
    out.update(proj=pr, toff=toff, gidx=gidx)
    return out


def render_window(scene, cam, window, tile=16, **kw):
    """Forward of one view over a tile-aligned pixel window (x0, y0, w, h):
    the same image as ``render`` on those pixels, for views too large to
    composite whole.

    The transformation runs with the view's own camera, so that the off-axis
    clamp of the EWA Jacobian (1.3 times the half field of view of the whole
    view) is the view's; a smaller camera covering only the window would clamp
    differently.  Lists hold the Gaussians whose tile rectangle meets the
    window's tiles, in the order ``render`` gives them (float32 depth, then
    index).  The returned ``proj`` is restricted to those Gaussians (``index``
    gives their positions in the scene) with centres in window coordinates."""
    x0, y0, w, h = (int(a) for a in window)
    if x0 % tile or y0 % tile or w < 1 or h < 1 or x0 + w > cam.W or y0 + h > cam.H:
        raise ValueError("window must start on the tile grid and lie inside the view")
    pr = project(scene, cam, tile)
    tx0, ty0 = x0 // tile, y0 // tile
    TXw, TYw = (w + tile - 1) // tile, (h + tile - 1) // tile
    r = pr["rect"]
    keep = (pr["vis"] > 0) & (r[:, 1] >= tx0) & (r[:, 0] < tx0 + TXw) & (r[:, 3] >= ty0) & (r[:, 2] < ty0 + TYw)
    idx = np.nonzero(keep)[0]
    sub = {k: v[idx].copy() for k, v in pr.items()}
    rect = sub["rect"]
    rect[:, 0] = np.maximum(rect[:, 0] - tx0, 0)
    rect[:, 1] = np.minimum(rect[:, 1] - tx0, TXw - 1)
    rect[:, 2] = np.maximum(rect[:, 2] - ty0, 0)
    rect[:, 3] = np.minimum(rect[:, 3] - ty0, TYw - 1)
    sub["xy"] = sub["xy"] - np.array([x0, y0], np.float64)
    toff, gidx = bin_view(rect, sub["vis"], sub["depth"].astype(np.float32), w, h, tile)
    out = render_fwd(w, h, tile, toff, gidx, sub["xy"], sub["conic_o"], sub["rgb"], **kw)
    out.update(proj=sub, toff=toff, gidx=gidx, index=idx)
    return out


def fp32_flags(fw, W, H, tile=16, margin=1e-3):
    """Pixels of a forward (``render`` or ``render_window`` output) whose value
    float32 arithmetic may legitimately decide otherwise: pixels within the
    relative ``margin`` of an alpha, opacity-clamp or transmittance threshold
    (the compositor's own record), and pixels that a Gaussian with borderline
    tile membership (its 3-sigma radius within rounding of an integer, or a
    rectangle edge within rounding of a tile line) could reach at half the
    alpha cut, in the outermost tile rows and columns of its rectangle.
    Returns (flag [H, W] bool, number of borderline Gaussians)."""
    pr = fw["proj"]
    bad = fw["margin"] <= margin
    e = pr["ext3"]
    border = (pr["radius"] > 0) & (np.abs(e - np.round(e)) < 1e-4)
    for k in range(2):
        for sgn in (-1, 1):
            edge = (pr["xy"][:, k] + sgn * np.maximum(pr["radius"], np.ceil(e))) / tile
            border |= (np.abs(edge - np.round(edge)) * tile < 1e-3) & (e > 0)
    TX = (W + tile - 1) // tile
    TY = (H + tile - 1) // tile
    tiles_px = np.zeros((H, W), bool)
    for g in np.nonzero(border)[0]:
        r = max(int(math.ceil(e[g])), 0)
        x0, x1 = int((pr["xy"][g, 0] - r) // tile), int((pr["xy"][g, 0] + r) // tile)
        y0, y1 = int((pr["xy"][g, 1] - r) // tile), int((pr["xy"][g, 1] + r) // tile)
        for ty in range(max(0, y0 - 1), min(TY - 1, y1 + 1) + 1):
            for tx in range(max(0, x0 - 1), min(TX - 1, x1 + 1) + 1):
                if tx <= x0 or tx >= x1 or ty <= y0 or ty >= y1:
                    ys = np.arange(ty * tile, min(H, (ty + 1) * tile)) + 0.5 - pr["xy"][g, 1]
                    xs = np.arange(tx * tile, min(W, (tx + 1) * tile)) + 0.5 - pr["xy"][g, 0]
                    DX, DY = np.meshgrid(xs, ys)
                    a, b, c, o = pr["conic_o"][g]
                    reach = o * np.exp(-0.5 * (a * DX * DX + c * DY * DY) - b * DX * DY) >= 0.5 / 255
                    view = tiles_px[ty * tile:ty * tile + DX.shape[0], tx * tile:tx * tile + DX.shape[1]]
                    view |= reach
    return bad | tiles_px, int(border.sum())


def grad_view(scene, cam, dimg, tile=16, **kw):
    """dL/dparams [N, 60] of one view for an upstream image gradient."""
    fw = render(scene, cam, tile, **kw)
    pr = fw["proj"]
    g2d = render_bwd(cam.W, cam.H, tile, fw["toff"], fw["gidx"], pr["xy"], pr["conic_o"], pr["rgb"], dimg, **kw)
    return preprocess_bwd(scene, cam, g2d, tile), fw, g2d


# ----------------------------------------------------------------------------
# Sec. 2.1 step 3: L1 + SSIM loss
# ----------------------------------------------------------------------------

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
LAMBDA_DSSIM = 0.2


def ssim_window(size=11, sigma=1.5):
    ax = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-ax ** 2 / (2 * sigma ** 2))
    g /= g.sum()
    return np.outer(g, g)


def _corr(x, w):
    from scipy.ndimage import correlate
    return correlate(x, w, mode="constant", cval=0.0)


def ssim_loss(img, tgt):
    """L = 0.8 mean|I - T| + 0.2 (1 - mean SSIM(I, T)) over one [3, H, W] image,
    SSIM with an 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2,
    C2 = 0.03^2.  Returns (L, dL/dI, l1, ssim_mean)."""
    x = np.asarray(img, np.float64)
    y = np.asarray(tgt, np.float64)
    n = x.size
    w = ssim_window()
    dx = np.zeros_like(x)
    S_sum = 0.0
    for ch in range(x.shape[0]):
        X, Y = x[ch], y[ch]
        mx, my = _corr(X, w), _corr(Y, w)
        sxx = _corr(X * X, w) - mx * mx
        syy = _corr(Y * Y, w) - my * my
        sxy = _corr(X * Y, w) - mx * my
        n1, n2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2
        d1, d2 = mx * mx + my * my + SSIM_C1, sxx + syy + SSIM_C2
        S = n1 * n2 / (d1 * d2)
        S_sum += S.sum()
        A = 2 * my * n2 / (d1 * d2) - S * 2 * mx / d1        # dS/dmu_x
        Bm = -S / d2                                         # dS/dsigma_xx
        Cm = 2 * n1 / (d1 * d2)                              # dS/dsigma_xy
        dS = _corr(A - 2 * mx * Bm - my * Cm, w) + 2 * X * _corr(Bm, w) + Y * _corr(Cm, w)
        dx[ch] = -LAMBDA_DSSIM * dS / n
    l1 = np.abs(x - y).mean()
    ssim_mean = S_sum / n
    dx += (1 - LAMBDA_DSSIM) * np.sign(x - y) / n
    L = (1 - LAMBDA_DSSIM) * l1 + LAMBDA_DSSIM * (1 - ssim_mean)
    return L, dx, l1, ssim_mean


# ----------------------------------------------------------------------------
# Sec. 4: Adam with the batch-size scaling rules (Eq. 1 and Eq. 2)
# ----------------------------------------------------------------------------

def lane_lr(lr6):
    """Per-float learning rate in the 60-float layout from the six groups
    (mean, scale, quat, opacity, sh_dc, sh_rest)."""
    lm, lsc, lq, lo, ldc, lrest = lr6
    v = np.zeros(60)
    v[0:3] = lm
    v[3] = lo
    v[4:7] = lsc
    v[8:12] = lq
    v[12:15] = ldc
    v[15:60] = lrest
    return v


def adam(p, g, m, v, step, lr6, beta1=0.9, beta2=0.999, eps=1e-15, batch=1,
         scale_lr_sqrt_b=True, scale_beta_pow_b=True):
    """One Adam step on [N, 60] arrays (FP64).  lr' = lr sqrt(B) (Eq. 1),
    beta' = beta^B (Eq. 2), bias correction with the betas actually used.
    Returns (p, m, v) as new arrays."""
    b1 = beta1 ** batch if scale_beta_pow_b else beta1
    b2 = beta2 ** batch if scale_beta_pow_b else beta2
    lr = lane_lr(lr6) * (math.sqrt(batch) if scale_lr_sqrt_b else 1.0)
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train_step(scene, cams, targets, m, v, step, lr6, tile=16, **adam_kw):
    """One batched training step: per view render + loss + backward, mean of
    the per-view parameter gradients over the batch, Adam.  Returns
    (new_flat_params [N,60], m, v, losses[B], grad [N,60])."""
    B = len(cams)
    N = scene.N
    grad = np.zeros((N, 60))
    losses = []
    for b, cam in enumerate(cams):
        fw = render(scene, cam, tile)
        L, dimg, _, _ = ssim_loss(fw["img"], targets[b])
        losses.append(L)
        pr = fw["proj"]
        g2d = render_bwd(cam.W, cam.H, tile, fw["toff"], fw["gidx"], pr["xy"], pr["conic_o"], pr["rgb"], dimg)
        grad += preprocess_bwd(scene, cam, g2d, tile)
    grad /= B
    p = scene.flat().astype(np.float64)
    p2, m2, v2 = adam(p, grad, m, v, step, lr6, batch=B, **adam_kw)
    return p2, m2, v2, np.array(losses), grad
