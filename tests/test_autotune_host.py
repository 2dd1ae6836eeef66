"""Host logic of the launch-shape autotuner, on CPU: the candidate set and
the rule that shapes the library rejects (GS_ERR_INVALID_ARG at context
creation) are skipped, while any other error propagates."""
import pytest

torch = pytest.importorskip("torch")

from paper_2406_18533_gb300 import autotune, binding, synth  # noqa: E402


def test_candidates_cover_every_shape_once():
    c = autotune.candidates()
    assert len(c) == len(set(c)) == 27
    assert {t for t, _, _ in c} == {8, 16, 32}
    assert {b for _, b, _ in c} == {32, 64, 128}
    assert {p for _, _, p in c} == {1, 2, 4}


def _cams():
    return [synth.test_camera(W=32, H=32)]


def test_rejected_shapes_are_skipped(monkeypatch):
    seen = []

    def reject(**hp):
        seen.append((hp["tile"], hp["smem_batch"], hp["px_per_thread"]))
        raise binding.GSError("gs_create", binding.GS_ERR_INVALID_ARG, "unbuilt shape")

    monkeypatch.setattr(autotune, "Context", reject)
    with pytest.raises(RuntimeError, match="no supported launch shape"):
        autotune.tune(None, _cams(), torch.zeros(1, 3, 32, 32), shapes=[(8, 32, 1), (32, 128, 1)])
    assert seen == [(8, 32, 1), (32, 128, 1)]


def test_other_errors_propagate(monkeypatch):
    def fail(**hp):
        raise binding.GSError("gs_create", binding.GS_ERR_CUDA, "device")

    monkeypatch.setattr(autotune, "Context", fail)
    with pytest.raises(binding.GSError):
        autotune.tune(None, _cams(), torch.zeros(1, 3, 32, 32), shapes=[(16, 64, 1)])
