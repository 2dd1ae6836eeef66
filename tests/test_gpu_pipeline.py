"""engine.train_from_host: training steps fed from pinned host memory with
the next step's upload overlapping the current step and each step's losses
read back one step later.  It must train exactly as direct gs_train_step
calls on device targets: the first step's losses bit for bit, later ones up
to the order of the gradient atomics, with every step's losses delivered in
order, for one reused target tensor and for a different one per step."""
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


@pytest.mark.parametrize("per_step", [False, True])
def test_train_from_host_matches_direct_steps(eng, per_step):
    sc, rng = synth.aerial_scene(30_000, n_clusters=6, seed=51)
    cams = synth.ring_cameras(rng, 3, (25.0, 80.0), W=256, H=144)
    tgs = [np.stack([synth.blurred_noise_target(rng, 144, 256) for _ in cams]) for _ in range(2)]
    steps = 4
    order = [k % 2 if per_step else 0 for k in range(steps)]
    ref_ctx = eng.Context()
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    ref = []
    for k in range(steps):
        t = torch.from_numpy(tgs[order[k]]).cuda()
        ref.append(ref_ctx.train_step(P, G, M, V, 0, cams, t, check=True).cpu().numpy())
    ctx = eng.Context()
    ctx.reserve(sc.N, cams, int(ref_ctx.counters()["F"] * 1.5) + 4096)
    P2 = eng.DeviceScene.from_host(sc)
    G2, M2, V2 = P2.zeros_like(), P2.zeros_like(), P2.zeros_like()
    hosts = [torch.from_numpy(t).pin_memory() for t in tgs]
    seen = []
    last = eng.train_from_host(ctx, P2, G2, M2, V2, cams, [hosts[i] for i in order] if per_step else hosts[0],
                               steps, on_loss=lambda k, l: seen.append((k, l)))
    assert ctx.status()[0] == 0
    assert [k for k, _ in seen] == list(range(steps))
    assert np.array_equal(seen[0][1], ref[0])
    for k in range(1, steps):
        assert np.allclose(seen[k][1], ref[k], rtol=1e-5, atol=0), k
    assert np.array_equal(last, seen[-1][1])
    a = P.flat().cpu().numpy().astype(np.float64)
    b = P2.flat().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    with pytest.raises(ValueError):
        eng.train_from_host(ctx, P2, G2, M2, V2, cams, torch.from_numpy(tgs[0]), 1)
