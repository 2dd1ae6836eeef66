"""Host logic of the continuous-batching render server, on CPU: batch
admission (arrival order, view and pixel budgets, free device memory) and the
latency report."""
import collections
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2406_18533_gb300 import serve  # noqa: E402


def _req(rid, arrival, W, H):
    return serve.Request(rid, arrival, types.SimpleNamespace(W=W, H=H))


def _server(max_batch, max_pixels, reserve=0):
    s = object.__new__(serve.RenderServer)           # no device state needed for admission
    s.max_batch, s.max_pixels, s.hbm_reserve = max_batch, max_pixels, reserve
    return s


def test_admission_keeps_arrival_order_and_budgets(monkeypatch):
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (1 << 40, 1 << 40))
    q = collections.deque([_req(0, 0.0, 640, 360), _req(1, 0.1, 1280, 720), _req(2, 0.2, 640, 360),
                           _req(3, 0.3, 3840, 2160), _req(4, 0.4, 640, 360)])
    s = _server(max_batch=8, max_pixels=640 * 360 * 2 + 1280 * 720)
    b = s._admit(q)
    assert [r.rid for r in b] == [0, 1, 2]              # the 4K request would exceed the pixel budget
    assert [r.rid for r in q] == [3, 4]                  # no overtaking: it waits at the head
    s2 = _server(max_batch=1, max_pixels=1 << 30)
    assert [r.rid for r in s2._admit(q)] == [3]


def test_admission_respects_free_device_memory(monkeypatch):
    img = 3 * 4 * 640 * 360                              # bytes of one 360p float image
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (2 * img + 100, 1 << 40))
    q = collections.deque([_req(i, 0.01 * i, 640, 360) for i in range(5)])
    s = _server(max_batch=8, max_pixels=1 << 30, reserve=100)
    assert [r.rid for r in s._admit(q)] == [0, 1]
    assert len(q) == 3


def test_latency_report():
    rs = []
    for i in range(10):
        r = _req(i, 0.1 * i, 100, 10)
        r.done = 0.1 * i + 0.002 * (i + 1)               # latencies 2, 4, ..., 20 ms
        rs.append(r)
    rep = serve.latency_report(rs, skip=2)              # drops the two earliest arrivals
    assert rep["requests"] == 8
    assert rep["p50_ms"] == pytest.approx(13.0)                # median of 6, 8, ..., 20 ms
    assert rep["max_ms"] == pytest.approx(20.0)
    span = rs[-1].done - rs[2].arrival
    assert rep["frames_per_s"] == pytest.approx(8 / span)
    assert rep["mpix_per_s"] == pytest.approx(8 * 1000 / span / 1e6)


def test_a_request_that_can_never_fit_is_rejected_on_arrival(monkeypatch):
    """A request above the batch pixel budget (or above the device memory
    minus the reserve) is rejected when it arrives instead of blocking the
    queue: the requests behind it are still served."""
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (1 << 30, 1 << 30))
    s = _server(max_batch=4, max_pixels=640 * 360 * 2, reserve=0)
    launched = []

    class _Slot:
        busy = []

    s.slots = [_Slot()]
    s.batches = 0

    def launch(slot, batch):
        launched.append([r.rid for r in batch])
        for r in batch:
            r.done = 0.0
        s.batches += 1

    s._launch = launch
    reqs = [_req(0, 0.0, 3840, 2160), _req(1, 0.0, 640, 360), _req(2, 0.0, 640, 360)]
    done = s.run(reqs)
    assert [r.rid for r in done if r.rejected] == [0] and "exceeds" in done[0].rejected
    assert launched == [[1, 2]]
    big = _server(max_batch=4, max_pixels=1 << 40, reserve=(1 << 30) - 2000)
    assert big._never_fits(_req(3, 0.0, 640, 360), 1 << 30)
    assert big._never_fits(_req(4, 0.0, 10, 10), 1 << 30) is None
    for r in reqs[1:]:
        r.done = 0.001
    rep = serve.latency_report(reqs)
    assert rep["rejected"] == 1 and rep["requests"] == 2
