"""Caller workspace (gs_set_workspace, gs_workspace_size): a context that
takes all of its scratch from one caller-owned device buffer.  Training in a
workspace of exactly gs_workspace_size bytes gives the same steps as a
context that allocates for itself (the first step's losses bit for bit: the
same kernels on the same inputs) and changes the device's free memory by
nothing; a workspace one buffer too small is refused with GS_ERR_OOM before
anything runs, and the context then trains in a big enough one."""
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


def _case(seed=31):
    sc, rng = synth.aerial_scene(40_000, n_clusters=6, seed=seed)
    cams = synth.ring_cameras(rng, 3, (25.0, 80.0), W=256, H=144)
    tg = torch.from_numpy(np.stack([synth.blurred_noise_target(rng, 144, 256) for _ in cams])).cuda()
    return sc, cams, tg


def _capacity(eng, sc, cams, tg):
    """A fragment capacity that the steps below stay within: 1.5 x the
    fragments of a first step on a context that sizes itself."""
    ctx = eng.Context()
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    first = ctx.train_step(P, G, M, V, 0, cams, tg, check=True).clone()
    F = ctx.counters()["F"]
    ctx.train_step(P, G, M, V, 0, cams, tg, check=True)
    torch.cuda.synchronize()
    ctx.close()
    return int(F * 1.5) + 4096, first


def test_training_in_a_caller_workspace_matches_and_allocates_nothing(eng):
    from paper_2406_18533_gb300 import binding as b
    sc, cams, tg = _case()
    cap, first_ref = _capacity(eng, sc, cams, tg)
    ctx = eng.Context()
    need = ctx.workspace_size(sc.N, cams, cap)
    assert need > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    ctx.set_workspace(ws)
    ctx.reserve(sc.N, cams, cap)
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    loss = torch.empty(len(cams), dtype=torch.float32, device="cuda")
    out = torch.empty(3, len(cams), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(3):
        ctx.train_step(P, G, M, V, 0, cams, tg, loss_out=loss, check=True)
        out[k].copy_(loss)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert ctx.status()[0] == b.GS_OK
    assert free1 == free0, (free0, free1)
    assert torch.equal(out[0], first_ref)
    assert torch.isfinite(out).all() and (out[2] < out[0]).all()


def test_a_workspace_too_small_is_refused(eng):
    from paper_2406_18533_gb300 import binding as b
    sc, cams, tg = _case(seed=32)
    cap, first_ref = _capacity(eng, sc, cams, tg)
    ctx = eng.Context()
    need = ctx.workspace_size(sc.N, cams, cap)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    ctx.set_workspace(small)
    with pytest.raises(b.GSError) as ei:
        ctx.reserve(sc.N, cams, cap)
    assert ei.value.status == b.GS_ERR_OOM
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    ctx.set_workspace(ws)
    ctx.reserve(sc.N, cams, cap)
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    first = ctx.train_step(P, G, M, V, 0, cams, tg, check=True)
    torch.cuda.synchronize()
    assert torch.equal(first, first_ref)
    ctx.set_workspace(None)                       # back to cudaMalloc: still trains
    ctx.train_step(P, G, M, V, 0, cams, tg, check=True)
    torch.cuda.synchronize()
    assert ctx.status()[0] == b.GS_OK
