"""Pins of the oracle's admissible-set renderer (``render_set``) and of its
float32 error model (``fp32_bounds``), and of the double-precision tile
rectangle (``rect_f64``).  CPU only.

The set renderer must (a) give the definition's own result as its primary
result, (b) contain the other outcome of every decision within its bound of
the threshold -- the alpha cut, the transmittance stop, tile membership --
each checked against the definition evaluated with that decision forced,
and (c) contain every result of the definition evaluated from inputs moved
within the declared error bounds (sampled).  The error model must bound the
error of float32 evaluations of the transformation."""
import math

import numpy as np
import pytest

from paper_2406_18533_gb300 import synth


# ---------------------------------------------------------------- rect_f64

def test_rect_f64_is_tile_interval_overlap(oracle):
    """Tile tx is in the double-precision rectangle iff [tx T, (tx+1) T) meets
    [u - r, u + r] (likewise y), clipped to the image; centres inside, just
    outside and far outside the image, radii that end exactly on a tile line."""
    W, H, T = 100, 70, 16
    rng = np.random.default_rng(4)
    n = 400
    u = rng.random(n) * (W + 60) - 30
    v = rng.random(n) * (H + 60) - 30
    r = rng.integers(0, 40, n).astype(np.int32)
    # radii reaching exactly to a tile line, on either side
    k = np.arange(0, n, 5)
    u[k] = np.round(u[k]) + 0.0
    r[k] = np.maximum(1, np.abs(((np.round(u[k]) // T) + 1) * T - u[k])).astype(np.int32)
    k2 = np.arange(1, n, 5)
    v[k2] = 48.0 - r[k2]                     # v + r = 48 exactly: the tile row starting at 48 is met
    # centres just outside the image
    u[2::7] = -r[2::7] - 1e-9
    v[3::7] = H + r[3::7] - 1e-9
    rect, vis = oracle.rect_f64(u, v, r, W, H, T)
    TX, TY = -(-W // T), -(-H // T)
    for g in range(n):
        uu, vv, rr = float(u[g]), float(v[g]), int(r[g])
        xs = [tx for tx in range(TX) if rr > 0 and tx * T <= uu + rr and uu - rr < (tx + 1) * T]
        ys = [ty for ty in range(TY) if rr > 0 and ty * T <= vv + rr and vv - rr < (ty + 1) * T]
        if xs and ys:
            assert vis[g] == 1 and list(rect[g]) == [xs[0], xs[-1], ys[0], ys[-1]], g
        else:
            assert vis[g] == 0, g
    assert vis.sum() > 100 and (vis == 0).sum() > 20


def test_project_uses_rect_f64(oracle):
    """The transformation's rectangles are rect_f64 of its own centres and radii."""
    sc, cams, _ = synth.workload_c0(N=3000)
    pr = oracle.project(sc, cams[0])
    rect, vis = oracle.rect_f64(pr["xy"][:, 0], pr["xy"][:, 1], pr["radius"], 256, 256, 16)
    assert np.array_equal(vis, pr["vis"]) and np.array_equal(rect[vis > 0], pr["rect"][vis > 0])


# ---------------------------------------------------------------- helpers

def _lists(oracle, pj, W, H, tile=16):
    rect, vis = oracle.rect_f32(pj["xy"][:, 0], pj["xy"][:, 1], pj["radius"], W, H, tile)
    toff, gidx = oracle.bin_view(rect, vis, pj["rgb_d"][:, 3], W, H, tile)
    return rect, vis, toff, gidx


def _results_at(ref, py, px):
    """All results of the set at one pixel: rows (r, g, b, T, n_contrib)."""
    W = ref["img"].shape[2]
    p = py * W + px
    prim = np.array([*ref["img"][:, py, px], ref["T_final"][py, px], ref["n_contrib"][py, px]])
    return np.vstack([prim, ref["alt"][ref["alt_off"][p]:ref["alt_off"][p + 1]]])


def _contains(rows, img_px, T=None, tol=1e-12):
    d = np.abs(rows[:, :3] - np.asarray(img_px)[None]).max(1)
    if T is not None:
        d = np.maximum(d, np.abs(rows[:, 3] - T))
    return bool((d <= tol).any())


# ---------------------------------------------------------------- (a) primary = definition

@pytest.mark.parametrize("seed", [1, 5])
def test_primary_equals_definition(oracle, seed):
    W, H = 100, 70
    pj = synth.synthetic_proj(3000, W, H, seed=seed, ties=50)
    _, _, toff, gidx = _lists(oracle, pj, W, H)
    ref = oracle.render_fwd(W, H, 16, toff, gidx, pj["xy"], pj["conic_o"], pj["rgb_d"][:, :3])
    s = oracle.render_set(W, H, 16, toff, gidx, pj["xy"], pj["conic_o"], pj["rgb_d"][:, :3])
    assert np.array_equal(s["img"], ref["img"]) and np.array_equal(s["T_final"], ref["T_final"])
    assert np.array_equal(s["n_contrib"], ref["n_contrib"])
    # a pixel has other results only where some decision is within a relative
    # 1e-3 of its threshold (or_render_fwd's own margin record)
    assert np.all(ref["margin"][(s["flags"] & 1) > 0] < 1e-3)
    assert (s["flags"] & 4).sum() == 0


# ---------------------------------------------------------------- (b) forced decisions

def _two_gaussian_proj(o1, rgb1=(0.2, 0.9, 0.4)):
    """A wide Gaussian behind and a small one in front, both centred near
    (16.3, 15.8) of a 32 x 32 view."""
    pj = dict(xy=np.array([[16.3, 15.8], [16.3, 15.8]], np.float32),
              conic_o=np.array([[0.01, 0.0, 0.01, 0.6], [0.2, 0.03, 0.15, o1]], np.float32),
              rgb_d=np.array([[0.8, 0.1, 0.3, 9.0], [*rgb1, 2.0]], np.float32),
              radius=np.array([40, 12], np.int32))
    return pj


def test_alpha_cut_alternative(oracle):
    """The front Gaussian's alpha at one pixel is put a few float32 rounding
    errors above 1/255: the set there holds the result with it blended (the
    definition) and the result without it (the definition on the scene
    without the front Gaussian); pixels where its alpha is far from the cut
    get no other result."""
    W = H = 32
    pj = _two_gaussian_proj(0.5)
    py, px = 16 + 6, 16 + 5
    a, b, c = (float(x) for x in pj["conic_o"][1, :3])
    dx, dy = px + 0.5 - float(pj["xy"][1, 0]), py + 0.5 - float(pj["xy"][1, 1])
    G = math.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
    pj["conic_o"][1, 3] = np.float32((1 / 255) * (1 + 3e-7) / G)
    rect, vis, toff, gidx = _lists(oracle, pj, W, H)
    args = (pj["xy"], pj["conic_o"], pj["rgb_d"][:, :3])
    s = oracle.render_set(W, H, 16, toff, gidx, *args)
    full = oracle.render_fwd(W, H, 16, toff, gidx, *args)
    rows = _results_at(s, py, px)
    assert len(rows) == 2
    one = {k: v[:1] for k, v in pj.items()}
    _, _, t1, g1 = _lists(oracle, one, W, H)
    back = oracle.render_fwd(W, H, 16, t1, g1, one["xy"], one["conic_o"], one["rgb_d"][:, :3])
    assert _contains(rows, full["img"][:, py, px], full["T_final"][py, px])
    assert _contains(rows, back["img"][:, py, px], back["T_final"][py, px])
    assert abs(full["img"][1, py, px] - back["img"][1, py, px]) > 1e-3      # the decision matters
    assert int((s["flags"] & 1).sum()) <= 4                                  # only pixels at the cut


def test_transmittance_stop_alternative(oracle):
    """Two saturated Gaussians (alpha clamped at 0.99) over a pixel take T
    to (1 - 0.99)^2, within rounding of T_min = 1e-4: the set holds the
    result that blends both (T_min just below) and the one that stops before
    the second (T_min just above), each the definition with that T_min."""
    W = H = 32
    pj = _two_gaussian_proj(0.999)
    pj["conic_o"][0, 3] = 0.999
    pj["conic_o"][0, :3] = [0.2, 0.03, 0.15]
    pj["rgb_d"][0, 3] = 1.5
    rect, vis, toff, gidx = _lists(oracle, pj, W, H)
    args = (pj["xy"], pj["conic_o"], pj["rgb_d"][:, :3])
    s = oracle.render_set(W, H, 16, toff, gidx, *args)
    py, px = 15, 16
    rows = _results_at(s, py, px)
    lo = oracle.render_fwd(W, H, 16, toff, gidx, *args, T_min=1e-4 * (1 - 1e-9))
    hi = oracle.render_fwd(W, H, 16, toff, gidx, *args, T_min=1e-4 * (1 + 1e-9))
    assert lo["n_contrib"][py, px] == 2 and hi["n_contrib"][py, px] == 1
    for r in (lo, hi):
        assert _contains(rows, r["img"][:, py, px], r["T_final"][py, px])
    # and the n_contrib of each result is the definition's
    assert sorted(rows[:, 4].astype(int).tolist()) == [1, 2]


def test_membership_alternative(oracle):
    """A Gaussian whose rectangle may or may not cover a tile (the tile lies
    outside its certain rectangle): on that tile the set holds the results
    with and without it in the list; on tiles of its certain rectangle it has
    no other result."""
    W, H = 48, 32
    pj = dict(xy=np.array([[30.0, 12.0], [14.5, 15.2]], np.float32),
              conic_o=np.array([[0.01, 0.0, 0.01, 0.5], [0.05, 0.0, 0.05, 0.8]], np.float32),
              rgb_d=np.array([[0.3, 0.3, 0.9, 9.0], [0.9, 0.2, 0.1, 3.0]], np.float32),
              radius=np.array([40, 10], np.int32))
    rect_big = np.array([[0, 2, 0, 1], [0, 1, 0, 1]], np.int32)      # G1 possibly: columns 0 and 1
    vis = np.ones(2, np.int32)
    d = pj["rgb_d"][:, 3]
    args = (pj["xy"], pj["conic_o"], pj["rgb_d"][:, :3])
    t_out, g_out = oracle.bin_view(rect_big, vis, d, W, H)
    rect_in = np.array([[0, 2, 0, 1], [0, 0, 0, 1]], np.int32)
    rect_prim = np.array([[0, 2, 0, 1], [0, 0, 0, 1]], np.int32)
    s = oracle.render_set(W, H, 16, t_out, g_out, *args, rect=rect_prim, rect_in=rect_in)
    t_p, g_p = oracle.bin_view(rect_prim, vis, d, W, H)
    without = oracle.render_fwd(W, H, 16, t_p, g_p, *args)
    with_ = oracle.render_fwd(W, H, 16, t_out, g_out, *args)
    assert np.array_equal(s["img"], without["img"])             # primary: the exact rectangle
    py, px = 15, 17                                             # tile column 1, near G1's centre
    rows = _results_at(s, py, px)
    assert _contains(rows, with_["img"][:, py, px], with_["T_final"][py, px])
    assert abs(with_["img"][0, py, px] - without["img"][0, py, px]) > 1e-2
    assert not np.any(s["flags"][:, :16] & 1)                  # tile column 0: certain


# ---------------------------------------------------------------- (c) perturbed inputs stay in the set

def test_inputs_within_bounds_give_results_in_the_set(oracle):
    """Opacities are tuned so that many (pixel, Gaussian) alphas sit within
    1e-7 of the cut.  With centres declared exact to 1e-6 px, the definition
    evaluated at centres moved by up to 5e-7 px gives, on every pixel, a
    result of the set (to 1e-5, far below the 2e-3 jump a flipped decision
    makes), and some of those moves flip decisions."""
    W = H = 32
    n = 40
    pj = synth.synthetic_proj(n, W, H, seed=3, max_sigma=3.0)
    rng = np.random.default_rng(0)
    u, v = pj["xy"][:, 0].astype(np.float64), pj["xy"][:, 1].astype(np.float64)
    for g in range(n):
        px, py = int(np.clip(u[g] + rng.integers(-3, 4), 0, W - 1)), int(np.clip(v[g] + rng.integers(-3, 4), 0, H - 1))
        a, b, c = (float(x) for x in pj["conic_o"][g, :3])
        dx, dy = px + 0.5 - u[g], py + 0.5 - v[g]
        G = math.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
        o = (1 / 255) * (1 + rng.uniform(-1e-7, 1e-7)) / G
        if o < 0.95:
            pj["conic_o"][g, 3] = np.float32(o)
    rect, vis, toff, gidx = _lists(oracle, pj, W, H)
    err = np.zeros((n, 6))
    err[:, 0:2] = 1e-6
    s = oracle.render_set(W, H, 16, toff, gidx, pj["xy"], pj["conic_o"], pj["rgb_d"][:, :3], err=err)
    assert (s["flags"] & 1).sum() >= 10 and (s["flags"] & 4).sum() == 0
    W_, H_ = np.meshgrid(np.arange(W), np.arange(H))
    flips = 0
    for k in range(20):
        xy = pj["xy"].astype(np.float64) + rng.uniform(-5e-7, 5e-7, (n, 2))
        r = oracle.render_fwd(W, H, 16, toff, gidx, xy, pj["conic_o"], pj["rgb_d"][:, :3])
        flips += int((np.abs(r["img"] - s["img"]).max(0) > 1e-4).sum())
        for py, px in zip(H_.reshape(-1), W_.reshape(-1)):
            assert _contains(_results_at(s, py, px), r["img"][:, py, px], r["T_final"][py, px], 1e-5), (k, py, px)
    assert flips > 0


# ---------------------------------------------------------------- the float32 error model

def _f32_transform(sc, cam, tile=16):
    """One float32 evaluation of the transformation (numpy single precision,
    no fused operations; the depth through double and rounded once)."""
    f = np.float32
    x = sc.mo[:, :3].astype(f)
    R = np.asarray(cam.R, f)
    t = np.asarray(cam.t, f)
    px = R[0, 0] * x[:, 0] + R[0, 1] * x[:, 1] + R[0, 2] * x[:, 2] + t[0]
    py = R[1, 0] * x[:, 0] + R[1, 1] * x[:, 1] + R[1, 2] * x[:, 2] + t[1]
    x64 = x.astype(np.float64)
    pz = (float(t[2]) + R[2, 0].astype(np.float64) * x64[:, 0] + R[2, 1].astype(np.float64) * x64[:, 1]
          + R[2, 2].astype(np.float64) * x64[:, 2]).astype(f)
    iz = f(1) / pz
    u = f(cam.fx) * px * iz + f(cam.cx)
    v = f(cam.fy) * py * iz + f(cam.cy)
    limx = f(1.3) * (f(0.5) * f(cam.W) / f(cam.fx))
    limy = f(1.3) * (f(0.5) * f(cam.H) / f(cam.fy))
    tx = np.clip(px * iz, -limx, limx)
    ty = np.clip(py * iz, -limy, limy)
    J00, J02 = f(cam.fx) * iz, -f(cam.fx) * tx * iz
    J11, J12 = f(cam.fy) * iz, -f(cam.fy) * ty * iz
    T0 = np.stack([J00 * R[0, j] + J02 * R[2, j] for j in range(3)], 1)
    T1 = np.stack([J11 * R[1, j] + J12 * R[2, j] for j in range(3)], 1)
    s = np.exp(sc.ls[:, :3].astype(f))
    q = sc.q.astype(f)
    qn = q / np.sqrt((q * q).sum(1, dtype=f))[:, None]
    w, qx, qy, qz = qn[:, 0], qn[:, 1], qn[:, 2], qn[:, 3]
    one, two = f(1), f(2)
    Rq = np.stack([one - two * (qy * qy + qz * qz), two * (qx * qy - w * qz), two * (qx * qz + w * qy),
                   two * (qx * qy + w * qz), one - two * (qx * qx + qz * qz), two * (qy * qz - w * qx),
                   two * (qx * qz - w * qy), two * (qy * qz + w * qx), one - two * (qx * qx + qy * qy)], 1)
    M = (Rq.reshape(-1, 3, 3) * s[:, None, :]).astype(f)
    S = np.einsum("nik,njk->nij", M, M).astype(f)
    TS0 = np.einsum("nj,njk->nk", T0, S).astype(f)
    TS1 = np.einsum("nj,njk->nk", T1, S).astype(f)
    A = (TS0 * T0).sum(1, dtype=f) + f(0.3)
    B = (TS0 * T1).sum(1, dtype=f)
    C = (TS1 * T1).sum(1, dtype=f) + f(0.3)
    det = A * C - B * B
    m = f(0.5) * (A + C)
    lam = m + np.sqrt(np.maximum(f(0), m * m - det))
    e3 = f(3) * np.sqrt(lam)
    conic = np.stack([C / det, -B / det, A / det], 1)
    return u, v, e3, conic


@pytest.mark.parametrize("which", ["c0", "aerial"])
def test_fp32_bounds_hold_for_a_float32_transformation(oracle, which):
    """The centre, 3-sigma extent, rectangle and (through the power at the
    alpha cut) the conic of a float32 transformation stay within the bounds."""
    if which == "c0":
        sc, cams, _ = synth.workload_c0(N=20000)
        cam = cams[0]
    else:
        sc, rng = synth.aerial_scene(20000, n_clusters=16, seed=2, log_s=(-2.5, 1.2))
        cam = synth.ring_cameras(rng, 1, (25.0, 25.0))[0]
    pr = oracle.project(sc, cam)
    bd = oracle.fp32_bounds(sc, cam)
    u, v, e3, conic = _f32_transform(sc, cam)
    vis = pr["vis"] > 0
    err = bd["err"]
    ratios = {}
    ratios["u"] = (np.abs(u.astype(np.float64) - pr["xy"][:, 0]) / err[:, 0])[vis].max()
    ratios["v"] = (np.abs(v.astype(np.float64) - pr["xy"][:, 1]) / err[:, 1])[vis].max()
    ratios["ext3"] = (np.abs(e3.astype(np.float64) - pr["ext3"]) / bd["de"])[vis].max()
    # rectangles of the float32 values lie between rect_in and rect_out
    r32 = np.ceil(e3.astype(np.float64)).astype(np.int32)
    rect32, vis32 = oracle.rect_f32(u, v, r32, cam.W, cam.H, 16)
    ro, ri = bd["rect_out"], bd["rect_in"]
    k = vis32 > 0
    assert np.all(bd["vis_out"][k] > 0)
    assert np.all((ro[k, 0] <= rect32[k, 0]) & (rect32[k, 1] <= ro[k, 1]) & (ro[k, 2] <= rect32[k, 2])
                  & (rect32[k, 3] <= ro[k, 3]))
    kin = k & (ri[:, 0] <= ri[:, 1]) & (ri[:, 2] <= ri[:, 3])
    assert np.all((rect32[kin, 0] <= ri[kin, 0]) & (ri[kin, 1] <= rect32[kin, 1]) & (rect32[kin, 2] <= ri[kin, 2])
                  & (ri[kin, 3] <= rect32[kin, 3]))
    # the power at offsets on the alpha-cut ellipse, from the float32 conic
    rng = np.random.default_rng(1)
    idx = np.nonzero(vis & (pr["conic_o"][:, 3] > 1 / 255))[0]
    a, b, c, o = (pr["conic_o"][idx, j] for j in range(4))
    L = 2 * np.log(o * 255)
    th = rng.random(len(idx)) * 2 * np.pi
    ex, ey = np.cos(th), np.sin(th)
    q = a * ex * ex + 2 * b * ex * ey + c * ey * ey
    dx, dy = ex * np.sqrt(L / q), ey * np.sqrt(L / q)
    p64 = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    cf = conic[idx].astype(np.float64)
    p32c = -0.5 * (cf[:, 0] * dx * dx + cf[:, 2] * dy * dy) - cf[:, 1] * dx * dy
    gx, gy = np.abs(a * dx + b * dy), np.abs(b * dx + c * dy)
    e = err[idx]
    bound = 0.5 * (gx * gx * e[:, 2] + 2 * gx * gy * e[:, 3] + gy * gy * e[:, 4]) + np.abs(p64) * e[:, 5]
    ratios["power"] = (np.abs(p32c - p64) / bound).max()
    print({k_: float(r) for k_, r in ratios.items()})
    for name, r in ratios.items():
        assert r <= 1.0, (name, r)


# ---------------------------------------------------------------- storage order

def test_morton_code_interleaves_bits(oracle):
    c = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [1023, 1023, 1023], [5, 3, 6]])
    code = oracle.morton_code(c)
    assert list(code[:5]) == [1, 2, 4, 8, 2 ** 30 - 1]
    # 5 = 101b, 3 = 011b, 6 = 110b: bits (x,y,z) per level 0: (1,1,0), 1: (0,1,1), 2: (1,0,1)
    assert code[5] == (1 | 2) | ((2 | 4) << 3) | ((1 | 4) << 6)


def test_morton_order_is_z_order_of_a_grid(oracle):
    """A shuffled 8 x 8 x 8 lattice of spacing 8 plus one corner point at 64
    spans a box of edge 64, so the cells are exactly 128 x the lattice
    coordinates (the corner clamps to 1023).  The order then visits the
    lattice in Z-order: it equals the brute-force sort of the lattice indices'
    interleaved bits, and every aligned 2 x 2 x 2 block is contiguous."""
    g = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(0)
    g = g[rng.permutation(len(g))]
    xyz = np.concatenate([g * 8.0, [[64.0, 64.0, 64.0]]]).astype(np.float32)
    cells = oracle.morton_cells(xyz)
    assert np.array_equal(cells[:-1], g * 128) and np.array_equal(cells[-1], [1023, 1023, 1023])
    sc = synth._empty_scene(len(xyz))
    sc.mo[:, :3] = xyz
    order = oracle.morton_order(sc)
    assert order[-1] == len(g)
    brute = sorted(range(len(g)), key=lambda i: sum(((int(g[i, a]) >> b) & 1) << (3 * b + a)
                                                    for b in range(3) for a in range(3)))
    assert list(order[:-1]) == brute
    blocks = g[order[:-1]] // 2
    for k in range(0, len(g), 8):
        assert len({tuple(r) for r in blocks[k:k + 8]}) == 1


def test_morton_order_ties_and_nonfinite(oracle):
    """Equal positions keep index order; non-finite positions take cell 0 and
    do not widen the box."""
    sc = synth._empty_scene(6)
    sc.mo[:, :3] = [[1, 1, 1], [0, 0, 0], [1, 1, 1], [np.nan, 0, 0], [0, 0, 0], [1, 1, 1]]
    cells = oracle.morton_cells(sc.mo[:, :3])
    assert np.array_equal(cells[3], [0, 0, 0]) and np.array_equal(cells[0], [1023, 1023, 1023])
    assert list(oracle.morton_order(sc)) == [1, 3, 4, 0, 2, 5]


# ---------------------------------------------------------------- Algorithm 1

def test_division_points_closed_forms(oracle):
    """Uniform costs: with CT = 1..8 and 4 parts the thresholds are 0, 2, 4, 6
    and the first blocks reaching them are 0, 1, 3, 5.  One heavy block takes
    a part of its own.  Against the printed float form
    searchsorted(CT, arange(P) * CT[-1] / P) wherever CT[-1] / P is exact."""
    assert list(oracle.division_points([1] * 8, 4)) == [0, 1, 3, 5]
    assert list(oracle.division_points([1, 1, 100, 1, 1], 3)) == [0, 2, 2]
    rng = np.random.default_rng(0)
    for _ in range(50):
        T, P = int(rng.integers(1, 400)), int(rng.integers(1, 40))
        c = rng.integers(0, 50, T)
        c[-1] += P - (c.sum() % P)                 # CT[-1] divisible by P: the float form is exact
        CT = np.cumsum(c)
        ref = np.searchsorted(CT, np.arange(P) * (CT[-1] // P), side="left")
        assert np.array_equal(oracle.division_points(c, P), ref)
    d = oracle.division_points(rng.integers(0, 9, 1000), 37)
    assert d[0] == 0 and np.all(np.diff(d) >= 0) and d[-1] <= 1000
