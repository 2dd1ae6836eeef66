"""The training path's tile culling rule (bin.cu, row_interval_mask), restated
in float32 numpy, never drops a tile that holds a pixel centre inside the
alpha >= 1/255 ellipse (brute force over the pixel centres in float64).

The rule: per tile row, the ellipse f(d) = a dx^2 + 2 b dx dy + c dy^2 <= L
meets the row's band of pixel-centre dy in an x-interval whose ends sit at
the band's dy closest to the ellipse's rightmost and leftmost points, widened
by 1e-3 relative plus 0.01 pixel.  The GPU tests check the kernel itself
(culled images bit-identical to the rectangle rule); this pins the geometry
on many random ellipses, tile sizes and offsets."""
import numpy as np

f32 = np.float32


def row_interval_mask(a, b, c, L, u, v, x0, x1, y0, y1, T):
    a, b, c, L, u, v, T = map(f32, (a, b, c, L, u, v, T))
    det = f32(a * c - b * b)
    rel, ab = f32(1e-3), f32(1e-2)
    aL = f32(a * L)
    Y = f32(np.sqrt(f32(aL / det)) * f32(1 + rel) + ab)
    dyr = f32(-b * np.sqrt(f32(L * f32(1 / c) / det)))
    ia = f32(1 / a)
    w = x1 - x0 + 1
    m = 0
    for ty in range(y0, y1 + 1):
        py0 = f32(f32(ty) * T + f32(0.5) - v)
        lo, hi = max(f32(py0 - ab), -Y), min(f32(py0 + (T - 1) + ab), Y)
        if not lo <= hi:
            continue
        dr, dl = min(max(dyr, lo), hi), min(max(-dyr, lo), hi)
        sr = f32(np.sqrt(max(f32(aL - det * dr * dr), f32(0))))
        sl = f32(np.sqrt(max(f32(aL - det * dl * dl), f32(0))))
        xr, xl = f32((sr - b * dr) * ia), f32(-(sl + b * dl) * ia)
        mm = f32((xr - xl) * rel + ab)
        XR, XL = f32(u + xr + mm), f32(u + xl - mm)
        tl = int(max(np.ceil(f32((XL - (T - f32(0.5))) / T)), x0))
        th = int(min(np.floor(f32((XR - f32(0.5)) / T)), x1))
        for tx in range(tl, th + 1):
            m |= 1 << ((ty - y0) * w + (tx - x0))
    return m


def brute_force(a, b, c, L, u, v, x0, x1, y0, y1, T):
    w, m = x1 - x0 + 1, 0
    for ty in range(y0, y1 + 1):
        for tx in range(x0, x1 + 1):
            X, Y = np.meshgrid(tx * T + 0.5 + np.arange(T) - u, ty * T + 0.5 + np.arange(T) - v)
            if ((a * X * X + 2 * b * X * Y + c * Y * Y) <= L).any():
                m |= 1 << ((ty - y0) * w + (tx - x0))
    return m


def test_row_interval_rule_keeps_every_tile_with_a_pixel_inside():
    rng = np.random.default_rng(0)
    cases = extra = 0
    while cases < 600:
        T = int(rng.choice([8, 16, 32]))
        s1, s2 = np.exp(rng.uniform(np.log(0.3), np.log(40), 2))
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        S = R @ np.diag([s1 * s1, s2 * s2]) @ R.T + 0.3 * np.eye(2)
        C = np.linalg.inv(S)
        o = rng.uniform(0.01, 1.0)
        L = 2 * np.log(o * 255)
        if L <= 0:
            continue
        u, v = rng.uniform(0, 200, 2)
        r = int(np.ceil(3 * np.sqrt(np.linalg.eigvalsh(S).max())))
        x0, x1 = max(int((u - r) // T), 0), int((u + r) // T)
        y0, y1 = max(int((v - r) // T), 0), int((v + r) // T)
        if (x1 - x0 + 1) * (y1 - y0 + 1) > 64:
            continue
        # the kernel's threshold carries ellipse_terms' margin (0.1% + 1e-4; the
        # condition-number term only widens further)
        mk = row_interval_mask(C[0, 0], C[0, 1], C[1, 1], L * 1.001 + 1e-4, u, v, x0, x1, y0, y1, T)
        bf = brute_force(C[0, 0], C[0, 1], C[1, 1], L, u, v, x0, x1, y0, y1, T)
        assert bf & ~mk == 0, (cases, T, u, v, bin(bf), bin(mk))
        extra += bin(mk & ~bf).count("1")
        cases += 1
    assert extra < 0.1 * cases        # conservative, but not far from exact
