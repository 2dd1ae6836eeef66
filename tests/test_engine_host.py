"""Host-side pieces of the torch glue, on CPU tensors: the parameter planes'
layout (the 60-float record of each Gaussian, the same on the host scene and
the device planes, and in the ABI struct) and the tile count of a batch."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_18533_gb300 import engine, synth  # noqa: E402


def test_planes_flatten_like_the_host_scene():
    sc = synth.tiny_scene(37, seed=2)
    ds = engine.DeviceScene.from_host(sc, device="cpu")
    assert ds.N == 37 and tuple(ds.sh.shape) == (12, 37, 4)
    assert np.array_equal(ds.flat().numpy(), sc.flat())
    # record layout: mean + logit, log-scales + pad, quaternion, 48 SH floats
    f = sc.flat()
    assert np.array_equal(f[:, 0:3], sc.mo[:, :3]) and np.array_equal(f[:, 3], sc.mo[:, 3])
    assert np.array_equal(f[:, 12:15], sc.sh[0, :, 0:3])          # the DC coefficient's RGB


def test_host_tensors_never_reach_the_library():
    """The ABI takes device pointers only: host planes are refused before any
    call (there is no CPU path to fall back to)."""
    ds = engine.DeviceScene.from_host(synth.tiny_scene(5, seed=1), device="cpu")
    with pytest.raises(ValueError, match="CUDA"):
        ds.struct()
    z = ds.zeros_like()
    assert z.N == 5 and float(z.flat().abs().sum()) == 0.0
    c = ds.clone()
    c.mo += 1
    assert not torch.equal(c.mo, ds.mo)


def test_total_tiles_of_a_mixed_batch():
    cams = [synth.test_camera(W=1920, H=1080), synth.test_camera(W=97, H=61)]
    assert engine.total_tiles(cams, 16) == 120 * 68 + 7 * 4
    assert engine.total_tiles(cams, 32) == 60 * 34 + 4 * 2


def test_autograd_function_refuses_views_of_different_sizes():
    """The autograd Function renders views of one size per call (one image
    tensor [B, 3, H, W]); a mixed batch is refused before any library call."""
    ds = engine.DeviceScene.from_host(synth.tiny_scene(5, seed=1), device="cpu")
    params = [t.clone().requires_grad_(True) for t in (ds.mo, ds.ls, ds.q, ds.sh)]
    cams = [synth.test_camera(W=64, H=48), synth.test_camera(W=32, H=48)]
    with pytest.raises(ValueError, match="one size"):
        engine.rasterize(params, None, cams)
    with pytest.raises(ValueError, match="one size"):
        engine.rasterize(params, None, [])
