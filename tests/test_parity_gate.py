"""The bench's parity gate (host logic) on CPU: a stand-in context whose
render is the oracle's own whole-view image (rounded to float32) passes; an
error of 1e-3 planted at any pixel of the compared window fails it, an
ambiguous pixel (one with several admissible results) included; the same
error outside the window does not count."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_18533_gb300 import synth  # noqa: E402


class _Params:
    def __init__(self, sc):
        self.mo, self.ls = torch.from_numpy(sc.mo.copy()), torch.from_numpy(sc.ls.copy())
        self.q, self.sh = torch.from_numpy(sc.q.copy()), torch.from_numpy(sc.sh.copy())


class _Ctx:
    tile = 16

    def __init__(self, img):
        self.img = img

    def render(self, P, cams, check=False):
        return torch.from_numpy(self.img.astype(np.float32))[None]


@pytest.fixture(scope="module")
def setup():
    import bench
    import oracle
    sc = synth.tiny_scene(600, seed=5, spread=1.2, log_s=(-3.0, -0.8))
    cam = synth.test_camera(W=320, H=288)
    full = oracle.render(sc, cam)
    return bench, oracle, sc, cam, full


def test_gate_passes_on_the_oracle_image(setup):
    bench, oracle, sc, cam, full = setup
    r = bench.parity_gate(_Ctx(full["img"]), _Params(sc), [cam])
    assert r["pass"] and r["max_abs_err"] < 1e-6
    assert r["pixels"] == 256 * 256 and "(32,16)" in r["window"]


@pytest.mark.parametrize("ambiguous", [False, True])
def test_gate_fails_on_an_error_inside_the_window(setup, ambiguous):
    bench, oracle, sc, cam, full = setup
    x0, y0 = 32, 16
    win = oracle.render_window_admissible(sc, cam, (x0, y0, 256, 256))
    ys, xs = np.nonzero(((win["flags"] & 1) > 0) == ambiguous)
    assert len(ys) > 0
    img = full["img"].copy()
    py, px = ys[len(ys) // 2], xs[len(xs) // 2]
    p = py * 256 + px
    alts = win["alt"][win["alt_off"][p]:win["alt_off"][p + 1], 1]
    # 1e-3 away from the exact result and from every other admissible one
    step = 1e-3
    while np.any(np.abs(full["img"][1, y0 + py, x0 + px] + step - alts) < 1e-3):
        step += 1e-3
    img[1, y0 + py, x0 + px] += step
    r = bench.parity_gate(_Ctx(img), _Params(sc), [cam])
    assert not r["pass"] and r["max_abs_err"] >= 1e-3 - 1e-6 and r["unchecked_px"] == 0
    out = full["img"].copy()
    out[1, 5, 5] += 1e-3                                 # outside the window (x < 32)
    assert bench.parity_gate(_Ctx(out), _Params(sc), [cam])["pass"]
