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


# ----------------------------------------------------------------------------
# Every result a float32 evaluation may legitimately give (Sec. 2.1 step 2
# decided in single precision)
# ----------------------------------------------------------------------------

EVAL_M0 = 4e-6   # relative alpha error of the float32 exponential and of the
                 # float32 constants 1/255, 0.99, 1e-4 (see or_render_fwd_set)


def rect_f64(u, v, radius, W, H, tile=16):
    """The transformation's double-precision tile rectangles for given centres
    and integer radii (the routine ``project`` uses)."""
    u = np.ascontiguousarray(u, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    r = np.ascontiguousarray(radius, np.int32)
    n = u.shape[0]
    rect = np.zeros((n, 4), np.int32)
    vis = np.zeros(n, np.int32)
    lib().or_rect_f64(_i64(n), _p(u), _p(v), _p(r), ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile),
                      _p(rect), _p(vis))
    return rect, vis


def fp32_bounds(scene, cam, tile=16):
    """Per Gaussian of one view, bounds on a float32 transformation's error
    (``or_fp32_bounds``): err [N, 6] = (du, dv, dA, dB, dC, rinv), de [N]
    (error of the 3-sigma extent), rect_in / rect_out [N, 4] (tiles covered by
    every / by some such evaluation; empty when x0 > x1), vis_out [N]."""
    mo, ls, q, sh = _scene_arrays(scene)
    N = mo.shape[0]
    out = dict(err=np.zeros((N, 6)), de=np.zeros(N), rect_in=np.zeros((N, 4), np.int32),
               rect_out=np.zeros((N, 4), np.int32), vis_out=np.zeros(N, np.int32))
    c = cam16(cam)
    lib().or_fp32_bounds(_i64(N), _p(mo), _p(ls), _p(q), _p(sh), ctypes.c_int(scene.sh_degree), _p(c),
                         ctypes.c_int(cam.W), ctypes.c_int(cam.H), ctypes.c_double(cam.near), ctypes.c_int(tile),
                         _p(out["err"]), _p(out["de"]), _p(out["rect_in"]), _p(out["rect_out"]), _p(out["vis_out"]))
    return out


def render_set(W, H, tile, toff, gidx, xy, conic_o, rgb, err=None, rect=None, rect_in=None,
               bg=(0.0, 0.0, 0.0), alpha_min=ALPHA_MIN, alpha_max=ALPHA_MAX, T_min=T_MIN, m0=EVAL_M0, cap=256):
    """Compositing (``or_render_fwd_set``): the exact result of every pixel
    (``img``, ``T_final``, ``n_contrib``, equal to ``render_fwd``) and every
    other result a float32 evaluation may give (``alt_off`` [H*W+1] offsets
    into ``alt`` [n, 5] = r, g, b, T, n_contrib), with ``flags`` [H, W]
    (1: other results exist; 2: alpha near its clamp at a blended entry;
    4: more than ``cap`` results, the set is incomplete).  ``err`` = None:
    exact screen-space inputs; ``rect`` = None: exact tile membership."""
    xy = np.ascontiguousarray(xy, np.float64)
    conic_o = np.ascontiguousarray(conic_o, np.float64)
    rgb = np.ascontiguousarray(rgb, np.float64)
    toff = np.ascontiguousarray(toff, np.int64)
    gidx = np.ascontiguousarray(gidx, np.int32)
    e = None if err is None else np.ascontiguousarray(err, np.float64)
    r = None if rect is None else np.ascontiguousarray(rect, np.int32)
    ri = None if rect_in is None else np.ascontiguousarray(rect_in, np.int32)
    img = np.zeros((3, H, W))
    Tf = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    flags = np.zeros((H, W), np.int32)
    n_alt = np.zeros((H, W), np.int32)
    prm = _blend_params(bg, alpha_min, alpha_max, T_min)
    pe = None if e is None else _p(e)
    pr_ = None if r is None else _p(r)
    pri = None if ri is None else _p(ri)
    args = (ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile), _p(toff), _p(gidx), _p(xy), _p(conic_o), _p(rgb),
            _p(prm), pe, pr_, pri, ctypes.c_double(m0), ctypes.c_int(cap))
    lib().or_render_fwd_set(*args, _p(img), _p(Tf), _p(nc), _p(flags), _p(n_alt), None, None)
    alt_off = np.zeros(H * W + 1, np.int64)
    np.cumsum(n_alt.reshape(-1), out=alt_off[1:])
    alt = np.zeros((max(int(alt_off[-1]), 1), 5))
    if alt_off[-1] > 0:
        lib().or_render_fwd_set(*args, _p(img), _p(Tf), _p(nc), _p(flags), _p(n_alt), _p(alt_off), _p(alt))
    return dict(img=img, T_final=Tf, n_contrib=nc, flags=flags, alt_off=alt_off, alt=alt[:int(alt_off[-1])])


def _primary_rects(pr):
    """Exact rectangles with invisible Gaussians as empty ones (x0 > x1)."""
    r = pr["rect"].copy()
    r[pr["vis"] == 0] = (1, 0, 1, 0)
    return r


def render_admissible(scene, cam, tile=16, **kw):
    """Every result a float32 pipeline (float32 transformation within
    ``fp32_bounds``, float32 compositing) may give for one view: the exact
    result (``render``'s image) plus the alternatives of ``render_set``, with
    tile lists that hold every Gaussian some such evaluation may place in a
    tile."""
    pr = project(scene, cam, tile)
    bd = fp32_bounds(scene, cam, tile)
    toff, gidx = bin_view(bd["rect_out"], bd["vis_out"], pr["depth"].astype(np.float32), cam.W, cam.H, tile)
    out = render_set(cam.W, cam.H, tile, toff, gidx, pr["xy"], pr["conic_o"], pr["rgb"], err=bd["err"],
                     rect=_primary_rects(pr), rect_in=bd["rect_in"], **kw)
    out.update(proj=pr, bounds=bd)
    return out


def render_window_admissible(scene, cam, window, tile=16, **kw):
    """``render_admissible`` on a tile-aligned window (x0, y0, w, h) of a view
    (the transformation runs with the view's own camera, as in
    ``render_window``); ``index`` lists the Gaussians some evaluation may
    place in the window's tiles."""
    x0, y0, w, h = (int(a) for a in window)
    if x0 % tile or y0 % tile or w < 1 or h < 1 or x0 + w > cam.W or y0 + h > cam.H:
        raise ValueError("window must start on the tile grid and lie inside the view")
    pr = project(scene, cam, tile)
    bd = fp32_bounds(scene, cam, tile)
    tx0, ty0 = x0 // tile, y0 // tile
    TXw, TYw = (w + tile - 1) // tile, (h + tile - 1) // tile

    def clip(r):
        r = r.copy()
        r[:, 0] = np.maximum(r[:, 0] - tx0, 0)
        r[:, 1] = np.minimum(r[:, 1] - tx0, TXw - 1)
        r[:, 2] = np.maximum(r[:, 2] - ty0, 0)
        r[:, 3] = np.minimum(r[:, 3] - ty0, TYw - 1)
        empty = (r[:, 0] > r[:, 1]) | (r[:, 2] > r[:, 3])
        r[empty] = (1, 0, 1, 0)
        return r, ~empty

    ro = bd["rect_out"].copy()
    ro[bd["vis_out"] == 0] = (1, 0, 1, 0)
    ro_w, keep = clip(ro)
    idx = np.nonzero(keep)[0]
    rect_w, _ = clip(_primary_rects(pr)[idx])
    rin_w, _ = clip(bd["rect_in"][idx])
    xy = pr["xy"][idx] - np.array([x0, y0], np.float64)
    toff, gidx = bin_view(ro_w[idx], np.ones(len(idx), np.int32), pr["depth"][idx].astype(np.float32), w, h, tile)
    out = render_set(w, h, tile, toff, gidx, xy, pr["conic_o"][idx], pr["rgb"][idx], err=bd["err"][idx],
                     rect=rect_w, rect_in=rin_w, **kw)
    out.update(index=idx)
    return out


def grad_view(scene, cam, dimg, tile=16, **kw):
    """dL/dparams [N, 60] of one view for an upstream image gradient."""
    fw = render(scene, cam, tile, **kw)
    pr = fw["proj"]
    g2d = render_bwd(cam.W, cam.H, tile, fw["toff"], fw["gidx"], pr["xy"], pr["conic_o"], pr["rgb"], dimg, **kw)
    return preprocess_bwd(scene, cam, g2d, tile), fw, g2d


# ----------------------------------------------------------------------------
# Algorithm 1: division points of a sequence of blocks by their costs
# ----------------------------------------------------------------------------

def division_points(cost, P):
    """Algorithm 1 ("Calculation of Division Points") for integer block costs
    and P parts: CT = cumsum(cost), ET = CT[-1] / P, thresholds arange(0, P)
    * ET, DP = searchsorted(CT, thresholds) (first index reaching each
    threshold), with the comparison CT[i] >= k CT[-1] / P taken exactly as
    P CT[i] >= k CT[-1].  Part k covers [DP[k], DP[k + 1]), the last ends at
    len(cost)."""
    CT = np.cumsum(np.asarray(cost, np.int64))
    thr = np.arange(P, dtype=np.int64) * CT[-1]
    return np.searchsorted(CT * P, thr, side="left").astype(np.int64)


# ----------------------------------------------------------------------------
# Densification (App. A.1): clone / split by the mean position-gradient length
# and the scale, prune by opacity, opacity reset
# ----------------------------------------------------------------------------

def _f32_log(x):
    """log of a float32 value, in double, rounded once to float32."""
    return np.float32(math.log(float(np.float32(x))))


def densify_thresholds(grad_threshold, scale_threshold, min_opacity, split_div):
    """The float32 thresholds the decisions compare against: (grad, log scale,
    opacity logit, log split divisor)."""
    mo = float(np.float32(min_opacity))
    return (np.float32(grad_threshold), _f32_log(scale_threshold), np.float32(math.log(mo / (1.0 - mo))),
            _f32_log(split_div))


def densify_actions(p, acc, cnt, grad_threshold, scale_threshold, min_opacity=0.005, split_div=1.6):
    """Action per Gaussian of the flat parameters p [N, 60] (float32 values):
    0 prune (opacity logit below logit(min_opacity)), 1 keep, 2 clone (the
    mean gradient test acc >= thr * cnt passes, float32, and the largest
    log-scale <= log(scale_threshold)), 3 split (the test passes, larger)."""
    g, lst, lmin, _ = densify_thresholds(grad_threshold, scale_threshold, min_opacity, split_div)
    p = np.asarray(p, np.float32)
    acc = np.asarray(acc, np.float32)
    cnt = np.asarray(cnt, np.int64)
    prune = ~(p[:, 3] >= lmin)
    grow = (cnt > 0) & (acc >= (g * cnt.astype(np.float32)).astype(np.float32))
    smax = np.fmax(p[:, 4], np.fmax(p[:, 5], p[:, 6]))
    act = np.where(grow, np.where(smax <= lst, 2, 3), 1)
    return np.where(prune, 0, act)


def densify(p, m, v, acc, cnt, normals, grad_threshold, scale_threshold, min_opacity=0.005, split_div=1.6):
    """One densification of flat [N, 60] parameters and moments.  Outputs keep
    the input order, each Gaussian's rows together: keep -> the row with its
    moments; clone -> the row with its moments, then a copy with zero moments;
    split -> two children at mean + R(q) diag(exp(log s)) xi_k (xi =
    normals[g, k], FP64), log-scale - log(split_div) (float32), the rest
    copied, zero moments; prune -> nothing.  Returns (p, m, v, src, kind):
    src the source index of each output row, kind its action (1, 2, 3, and
    4 for a clone's copy)."""
    p = np.asarray(p, np.float32)
    m = np.asarray(m, np.float32)
    v = np.asarray(v, np.float32)
    normals = np.asarray(normals, np.float64).reshape(-1, 2, 3)
    act = densify_actions(p, acc, cnt, grad_threshold, scale_threshold, min_opacity, split_div)
    _, _, _, ldiv = densify_thresholds(grad_threshold, scale_threshold, min_opacity, split_div)
    rows_p, rows_m, rows_v, src, kind = [], [], [], [], []
    zero = np.zeros(60)
    R = np.zeros((len(p), 9))
    lib().or_quat_rot(_i64(len(p)), _p(np.ascontiguousarray(p[:, 8:12], np.float64)), _p(R))
    for g in range(len(p)):
        a = int(act[g])
        if a == 0:
            continue
        if a in (1, 2):
            rows_p.append(p[g].astype(np.float64)); rows_m.append(m[g].astype(np.float64))
            rows_v.append(v[g].astype(np.float64)); src.append(g); kind.append(a)
            if a == 2:
                rows_p.append(p[g].astype(np.float64)); rows_m.append(zero); rows_v.append(zero)
                src.append(g); kind.append(4)
            continue
        s = np.exp(p[g, 4:7].astype(np.float64))
        for k in range(2):
            child = p[g].astype(np.float64).copy()
            child[0:3] = p[g, 0:3].astype(np.float64) + R[g].reshape(3, 3) @ (s * normals[g, k])
            child[4:7] = (p[g, 4:7] - ldiv).astype(np.float32)
            child[7] = 0.0
            rows_p.append(child); rows_m.append(zero); rows_v.append(zero); src.append(g); kind.append(3)
    shape = (len(rows_p), 60)
    mk = lambda rows: np.array(rows).reshape(shape) if rows else np.zeros((0, 60))
    return mk(rows_p), mk(rows_m), mk(rows_v), np.array(src, np.int64), np.array(kind, np.int64)


def reset_opacity(p, m, v, max_opacity=0.01):
    """Opacity reset: logit = min(logit, logit(max_opacity)) (float32), and
    the opacity lane of both moments set to 0.  Returns new arrays."""
    mx = float(np.float32(max_opacity))
    lmax = np.float32(math.log(mx / (1.0 - mx)))
    p, m, v = (np.array(a, np.float32) for a in (p, m, v))
    p[:, 3] = np.minimum(p[:, 3], lmax)
    m[:, 3] = 0.0
    v[:, 3] = 0.0
    return p, m, v


# ----------------------------------------------------------------------------
# Storage order of the Gaussians (Morton code of the position)
# ----------------------------------------------------------------------------

def morton_cells(xyz):
    """10-bit cell per axis of float32 positions [N, 3]: floor((x - lo) *
    (1024 / (hi - lo))) with each float32 operation rounded separately
    (numpy float32 arithmetic), clamped to [0, 1023]; lo / hi over the rows
    whose three coordinates are finite; a non-finite row or a flat axis gives 0."""
    x = np.asarray(xyz, np.float32)
    ok = np.all(np.isfinite(x), axis=1)
    cells = np.zeros(x.shape, np.int64)
    if not ok.any():
        return cells
    lo, hi = x[ok].min(0), x[ok].max(0)
    for a in range(3):
        if not hi[a] > lo[a]:
            continue
        scale = np.float32(1024.0) / np.float32(hi[a] - lo[a])
        with np.errstate(invalid="ignore"):
            q = np.floor((x[:, a] - lo[a]).astype(np.float32) * scale)
        q = np.where(ok, q, 0)
        cells[:, a] = np.clip(q, 0, 1023).astype(np.int64)
    return cells


def morton_code(cells):
    """Interleave three 10-bit cells into a 30-bit code: bit b of x to bit 3b,
    of y to 3b + 1, of z to 3b + 2."""
    c = np.asarray(cells, np.int64)
    code = np.zeros(c.shape[0], np.int64)
    for b in range(10):
        for a in range(3):
            code |= ((c[:, a] >> b) & 1) << (3 * b + a)
    return code


def morton_order(scene):
    """The storage permutation: Gaussian indices sorted stably by Morton code."""
    return np.argsort(morton_code(morton_cells(scene.mo[:, :3])), kind="stable").astype(np.int64)


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
         scale_lr_sqrt_b=True, scale_beta_pow_b=True, visible=None):
    """One Adam step on [N, 60] arrays (FP64).  lr' = lr sqrt(B) (Eq. 1),
    beta' = beta^B (Eq. 2), bias correction with the betas actually used.
    ``visible`` [N] (optional): visible-only Adam -- rows with visible False
    keep p, m and v unchanged (no update, no decay of the moments); the
    others take the step above.  Returns (p, m, v) as new arrays."""
    b1 = beta1 ** batch if scale_beta_pow_b else beta1
    b2 = beta2 ** batch if scale_beta_pow_b else beta2
    lr = lane_lr(lr6) * (math.sqrt(batch) if scale_lr_sqrt_b else 1.0)
    p0 = np.asarray(p, np.float64)
    m0 = np.asarray(m, np.float64)
    v0 = np.asarray(v, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * m0 + (1 - b1) * g
    v = b2 * v0 + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = p0 - lr * mh / (np.sqrt(vh) + eps)
    if visible is not None:
        keep = ~np.asarray(visible, bool)
        p[keep], m[keep], v[keep] = p0[keep], m0[keep], v0[keep]
    return p, m, v


def train_step(scene, cams, targets, m, v, step, lr6, tile=16, sparse=False, stats=None, **adam_kw):
    """One batched training step: per view render + loss + backward, mean of
    the per-view parameter gradients over the batch, Adam.  sparse=True:
    visible-only Adam, a Gaussian being visible when some view of the batch
    gives it a tile rectangle (radius > 0).  stats (a dict with arrays "acc"
    [N] and "cnt" [N]): densification statistics, |dL_v/d(u, v)| of each view
    in which the Gaussian is visible added to acc, 1 to cnt.  Returns
    (new_flat_params [N,60], m, v, losses[B], grad [N,60])."""
    B = len(cams)
    N = scene.N
    grad = np.zeros((N, 60))
    losses = []
    visible = np.zeros(N, bool)
    for b, cam in enumerate(cams):
        fw = render(scene, cam, tile)
        visible |= fw["proj"]["vis"] > 0
        L, dimg, _, _ = ssim_loss(fw["img"], targets[b])
        losses.append(L)
        pr = fw["proj"]
        g2d = render_bwd(cam.W, cam.H, tile, fw["toff"], fw["gidx"], pr["xy"], pr["conic_o"], pr["rgb"], dimg)
        grad += preprocess_bwd(scene, cam, g2d, tile)
        if stats is not None:
            seen = pr["vis"] > 0
            stats["acc"][seen] += np.hypot(g2d[seen, 0], g2d[seen, 1])
            stats["cnt"][seen] += 1
    grad /= B
    p = scene.flat().astype(np.float64)
    p2, m2, v2 = adam(p, grad, m, v, step, lr6, batch=B, visible=visible if sparse else None, **adam_kw)
    return p2, m2, v2, np.array(losses), grad
