"""Checkpoint file format (paper_2406_18533_gb300.checkpoint) on the host:
an exact round trip of every plane, the step and the hyperparameter bytes,
and refusal of a file that is truncated, of another kind or of another
version, before anything is allocated."""
import os
import struct

import numpy as np
import pytest

from paper_2406_18533_gb300 import checkpoint as ck


def _sets(N, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(3):
        out.append({"mo": rng.standard_normal((N, 4)).astype(np.float32),
                    "ls": rng.standard_normal((N, 4)).astype(np.float32),
                    "q": rng.standard_normal((N, 4)).astype(np.float32),
                    "sh": rng.standard_normal((12, N, 4)).astype(np.float32)})
    out[0]["mo"][3, 1] = np.nan                        # bits, not values, must survive
    out[2]["sh"][5, 7, 2] = -0.0
    return out


def test_round_trip_is_exact(tmp_path):
    N = 1234
    sets = _sets(N)
    hp = bytes(range(200))
    path = str(tmp_path / "a.ckpt")
    ck.write(path, 77, hp, 3, sets)
    assert os.path.getsize(path) == ck._HEAD.size + len(hp) + ck.state_bytes(N)
    step, hp2, deg, back = ck.read(path)
    assert (step, hp2, deg) == (77, hp, 3)
    for a, b in zip(sets, back):
        for k in ("mo", "ls", "q", "sh"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


def test_planes_may_come_one_at_a_time(tmp_path):
    N = 10
    sets = _sets(N, seed=1)
    calls = []
    lazy = [{k: (lambda a=a, k=k: calls.append(k) or a[k]) for k in a} for a in sets]
    path = str(tmp_path / "b.ckpt")
    ck.write(path, 1, b"x", 3, lazy)
    assert calls == ["mo", "ls", "q", "sh"] * 3
    assert np.array_equal(ck.read(path)[3][1]["sh"], sets[1]["sh"])


def test_bad_files_are_refused(tmp_path):
    N = 50
    path = str(tmp_path / "c.ckpt")
    ck.write(path, 3, b"hp", 3, _sets(N))
    raw = open(path, "rb").read()
    short = str(tmp_path / "short.ckpt")
    open(short, "wb").write(raw[:-4])
    with pytest.raises(ValueError, match="bytes"):
        ck.read(short)
    other = str(tmp_path / "other.ckpt")
    open(other, "wb").write(b"NOTACKPT" + raw[8:])
    with pytest.raises(ValueError, match="magic"):
        ck.read(other)
    newer = str(tmp_path / "newer.ckpt")
    open(newer, "wb").write(raw[:8] + struct.pack("<I", 2) + raw[12:])
    with pytest.raises(ValueError, match="version"):
        ck.read(newer)
    with pytest.raises(ValueError, match="shape"):
        bad = _sets(N)
        bad[1]["q"] = bad[1]["q"][:-1]
        ck.write(str(tmp_path / "d.ckpt"), 0, b"", 3, bad)
    assert not any(n.startswith("d.ckpt") for n in os.listdir(tmp_path))   # the partial file is removed
