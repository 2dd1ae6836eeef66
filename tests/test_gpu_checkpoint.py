"""Checkpoint and resume on the GPU: a training run saved after its first
step and resumed in a new context continues exactly where it stopped.  The
resumed context starts from the saved bits (parameters, Adam moments, step
counter, hyperparameters), so its first loss equals the uninterrupted run's
second loss bit for bit (a forward pass of identical inputs); the updates
after that agree up to the order of the gradient atomics."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_resume_continues_the_run(eng, tmp_path):
    from paper_2406_18533_gb300 import checkpoint as ck
    sc, rng = synth.aerial_scene(30_000, n_clusters=6, seed=41)
    cams = synth.ring_cameras(rng, 2, (25.0, 80.0), W=256, H=144)
    tg = torch.from_numpy(np.stack([synth.blurred_noise_target(rng, 144, 256) for _ in cams])).cuda()
    lr6 = (1.6e-4 * 60, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-4)
    ctx = eng.Context(lr=lr6, px_per_thread=2)
    P = eng.DeviceScene.from_host(sc)
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    ctx.train_step(P, G, M, V, 0, cams, tg, check=True)
    path = str(tmp_path / "run.ckpt")
    assert ck.save(path, ctx, P, M, V) == 1
    saved = [x.flat().cpu().numpy() for x in (P, M, V)]
    later = [ctx.train_step(P, G, M, V, 0, cams, tg, check=True).clone() for _ in range(2)]
    torch.cuda.synchronize()
    final = [x.flat().cpu().numpy().astype(np.float64) for x in (P, M, V)]

    ctx2, P2, M2, V2 = ck.load(path)
    assert ctx2.get_step() == 1
    assert ctx2.hp.px_per_thread == 2 and abs(ctx2.hp.lr[0] - lr6[0]) < 1e-9
    for a, b in zip(saved, (P2, M2, V2)):
        assert np.array_equal(a.view(np.uint32), b.flat().cpu().numpy().view(np.uint32))
    G2 = P2.zeros_like()
    resumed = [ctx2.train_step(P2, G2, M2, V2, 0, cams, tg, check=True).clone() for _ in range(2)]
    torch.cuda.synchronize()
    assert ctx2.get_step() == 3
    assert torch.equal(resumed[0], later[0])
    assert torch.allclose(resumed[1], later[1], rtol=1e-5, atol=0)
    for a, b in zip(final, (P2, M2, V2)):
        assert _rel(b.flat().cpu().numpy().astype(np.float64), a) < 1e-5


def test_step_counter_accessors(eng):
    from paper_2406_18533_gb300 import binding as b
    ctx = eng.Context()
    assert ctx.get_step() == 0
    ctx.set_step(41)
    assert ctx.get_step() == 41
    with pytest.raises(b.GSError) as ei:
        ctx.set_step(-1)
    assert ei.value.status == b.GS_ERR_INVALID_ARG
