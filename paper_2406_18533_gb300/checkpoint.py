"""Checkpoint and resume of a training state.

A training state is the Gaussians' parameters, the Adam moments m and v (the
same 60 floats per Gaussian), the context's device-side Adam step counter
(gs_get_step / gs_set_step) and the hyperparameters (gs_hparams, which hold
the learning rates and the batch rules of Eq. 1-2).  The library draws no
random numbers during training (cameras and targets are the caller's), so
there is no generator state to keep; a caller's view sampler is its own.

File layout (little-endian):

    magic    8 bytes  b"GSCKPT\\0\\1"
    version  uint32   1
    degree   uint32   SH degree
    N        uint64   Gaussians
    step     int64    device step counter
    hp_size  uint32   bytes of the gs_hparams struct that follow
    hp       hp_size bytes
    then three parameter sets (p, m, v), each the planes mo [N,4], ls [N,4],
    q [N,4], sh [12,N,4] as float32, in that order.

The file is written to a temporary name and renamed, so a crash while saving
leaves the previous checkpoint intact.  Reading checks the magic, the
version, the struct size and the file length before it allocates anything.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

MAGIC = b"GSCKPT\x00\x01"
VERSION = 1
_HEAD = struct.Struct("<8sIIQqI")
PLANES = (("mo", (4,)), ("ls", (4,)), ("q", (4,)), ("sh", (12, 4)))


def _plane_shape(name, N):
    return (12, N, 4) if name == "sh" else (N, 4)


def state_bytes(N: int) -> int:
    """Bytes of the three parameter sets of N Gaussians."""
    return 3 * 60 * 4 * int(N)


def write(path: str, step: int, hp_bytes: bytes, sh_degree: int, sets) -> None:
    """sets: three mappings (p, m, v) from plane name to a float32 array of
    the plane's shape, or a callable returning it (called once, in file
    order, so a caller can copy one plane at a time from the device)."""
    N = None
    tmp = f"{path}.tmp{os.getpid()}"
    try:
        with open(tmp, "wb") as f:
            for k, planes in enumerate(sets):
                for name, _ in PLANES:
                    a = planes[name]
                    a = a() if callable(a) else a
                    a = np.ascontiguousarray(a, dtype=np.float32)
                    if N is None:
                        N = a.shape[0] if name != "sh" else a.shape[1]
                        f.write(_HEAD.pack(MAGIC, VERSION, int(sh_degree), int(N), int(step), len(hp_bytes)))
                        f.write(hp_bytes)
                    if a.shape != _plane_shape(name, N):
                        raise ValueError(f"set {k} plane {name}: shape {a.shape}, expected {_plane_shape(name, N)}")
                    f.write(memoryview(a).cast("B"))
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise


def read(path: str):
    """Returns (step, hp_bytes, sh_degree, [p, m, v]) with each set a dict of
    float32 arrays; raises ValueError on a file that is not a complete
    checkpoint of this version."""
    size = os.path.getsize(path)
    with open(path, "rb") as f:
        head = f.read(_HEAD.size)
        if len(head) != _HEAD.size:
            raise ValueError("not a checkpoint: file too short")
        magic, version, degree, N, step, hp_size = _HEAD.unpack(head)
        if magic != MAGIC:
            raise ValueError("not a checkpoint: bad magic")
        if version != VERSION:
            raise ValueError(f"checkpoint version {version}, expected {VERSION}")
        if size != _HEAD.size + hp_size + state_bytes(N):
            raise ValueError(f"checkpoint of {N} Gaussians should be {_HEAD.size + hp_size + state_bytes(N)} "
                             f"bytes, file has {size}")
        hp = f.read(hp_size)
        sets = []
        for _ in range(3):
            planes = {}
            for name, _ in PLANES:
                shape = _plane_shape(name, N)
                planes[name] = np.fromfile(f, dtype="<f4", count=int(np.prod(shape))).reshape(shape)
            sets.append(planes)
    return int(step), hp, int(degree), sets


def save(path: str, ctx, p, m, v) -> int:
    """Writes the state of a training context and its device parameter sets
    (engine.DeviceScene); returns the step saved.  Synchronises."""
    step = ctx.get_step()
    hp = bytes(ctx.hp)
    sets = [{name: (lambda s=s, name=name: getattr(s, name).cpu().numpy()) for name, _ in PLANES}
            for s in (p, m, v)]
    write(path, step, hp, p.sh_degree, sets)
    return step


def load(path: str, device="cuda"):
    """Reads a checkpoint into a new training context: returns (ctx, p, m, v)
    with the saved hyperparameters and step counter, ready for the next
    gs_train_step (step == 0)."""
    import torch
    from . import binding as B
    from .engine import Context, DeviceScene
    step, hp, degree, sets = read(path)
    if len(hp) != ctypes.sizeof(B.gs_hparams):
        raise ValueError(f"hyperparameters of {len(hp)} bytes, this library's are {ctypes.sizeof(B.gs_hparams)}")
    ctx = Context()
    ctx.hp = B.gs_hparams.from_buffer_copy(hp)
    ctx._c("gs_set_hparams", ctx.h, ctypes.byref(ctx.hp))
    ctx.set_step(step)
    scenes = []
    for planes in sets:
        t = {k: torch.from_numpy(planes[k]).to(device) for k, _ in PLANES}
        scenes.append(DeviceScene(t["mo"], t["ls"], t["q"], t["sh"], degree))
    return (ctx, *scenes)
