"""PyTorch glue around libgs: device memory (torch tensors), streams, and a
``torch.autograd.Function`` whose backward is the library's hand-written
backward kernels.  No arithmetic of the method happens here; every step runs
in libgs's CUDA kernels through the C ABI (``binding``).
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import binding as B


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_f32(t: torch.Tensor, name: str):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")


@dataclasses.dataclass
class DeviceScene:
    """Parameter planes (or gradients / Adam moments) on the GPU."""
    mo: torch.Tensor      # [N, 4]
    ls: torch.Tensor      # [N, 4]
    q: torch.Tensor       # [N, 4]
    sh: torch.Tensor      # [12, N, 4]
    sh_degree: int = 3

    @property
    def N(self) -> int:
        return int(self.mo.shape[0])

    @classmethod
    def from_host(cls, sc, device="cuda", pin=False):
        f = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device, non_blocking=pin))
        return cls(f(sc.mo), f(sc.ls), f(sc.q), f(sc.sh), sc.sh_degree)

    @classmethod
    def zeros(cls, N, device="cuda", sh_degree=3):
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=device)
        return cls(z(N, 4), z(N, 4), z(N, 4), z(12, N, 4), sh_degree)

    def zeros_like(self):
        return DeviceScene.zeros(self.N, self.mo.device, self.sh_degree)

    def struct(self) -> B.gs_scene:
        for n in ("mo", "ls", "q", "sh"):
            _check_f32(getattr(self, n), n)
        return B.gs_scene(_ptr(self.mo), _ptr(self.ls), _ptr(self.q), _ptr(self.sh), self.N, self.sh_degree, 0)

    def flat(self) -> torch.Tensor:
        """[N, 60] copy in the (mo, ls, q, sh) float order."""
        return torch.cat([self.mo, self.ls, self.q, self.sh.permute(1, 0, 2).reshape(self.N, 48)], 1)

    def clone(self):
        return DeviceScene(self.mo.clone(), self.ls.clone(), self.q.clone(), self.sh.clone(), self.sh_degree)


@dataclasses.dataclass
class Proj:
    xy: torch.Tensor       # [B, N, 2]
    conic_o: torch.Tensor  # [B, N, 4]
    rgb_d: torch.Tensor    # [B, N, 4]
    radius: torch.Tensor   # [B, N] int32

    @classmethod
    def empty(cls, Bv, N, device="cuda"):
        e = lambda *s, dt=torch.float32: torch.empty(*s, dtype=dt, device=device)
        return cls(e(Bv, N, 2), e(Bv, N, 4), e(Bv, N, 4), e(Bv, N, dt=torch.int32))

    def struct(self) -> B.gs_proj:
        Bv, N = self.radius.shape
        return B.gs_proj(_ptr(self.xy), _ptr(self.conic_o), _ptr(self.rgb_d), _ptr(self.radius), N, Bv, 0)


@dataclasses.dataclass
class ProjGrad:
    d_xy_o: torch.Tensor   # [B, N, 4]
    d_conic: torch.Tensor
    d_rgb: torch.Tensor

    @classmethod
    def empty(cls, Bv, N, device="cuda"):
        e = lambda: torch.empty(Bv, N, 4, dtype=torch.float32, device=device)
        return cls(e(), e(), e())

    def struct(self) -> B.gs_proj_grad:
        return B.gs_proj_grad(_ptr(self.d_xy_o), _ptr(self.d_conic), _ptr(self.d_rgb))


@dataclasses.dataclass
class Bins:
    keys: torch.Tensor     # [cap] int64 (uint64 bits)
    vals: torch.Tensor     # [cap] int32 (uint32 bits)
    ranges: torch.Tensor   # [tiles, 2] int32 (uint32 bits)
    count: torch.Tensor    # [1] int32
    F: int = 0

    @classmethod
    def empty(cls, cap, tiles, device="cuda"):
        return cls(torch.empty(max(cap, 1), dtype=torch.int64, device=device),
                   torch.empty(max(cap, 1), dtype=torch.int32, device=device),
                   torch.zeros(max(tiles, 1), 2, dtype=torch.int32, device=device),
                   torch.zeros(1, dtype=torch.int32, device=device))

    @property
    def capacity(self) -> int:
        return int(self.keys.shape[0])

    def struct(self) -> B.gs_bins:
        return B.gs_bins(_ptr(self.keys), _ptr(self.vals), _ptr(self.ranges), _ptr(self.count), self.capacity)


def total_tiles(cams, tile):
    return sum(((c.W + tile - 1) // tile) * ((c.H + tile - 1) // tile) for c in cams)


class Context:
    """One libgs context (hyperparameters + scratch), used from one stream."""

    def __init__(self, **hparams):
        self.hp = B.default_hparams(**hparams)
        h = ctypes.c_void_p()
        B.call("gs_create", ctypes.byref(h), ctypes.byref(self.hp))
        self.h = h
        self._bins_cap = 0

    def close(self):
        if self.h:
            B.lib().gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def tile(self) -> int:
        return int(self.hp.tile)

    def set_hparams(self, **kw):
        for k, v in kw.items():
            if k in ("bg", "lr"):
                arr = getattr(self.hp, k)
                for i, x in enumerate(v):
                    arr[i] = float(x)
            else:
                setattr(self.hp, k, v)
        B.call("gs_set_hparams", self.h, ctypes.byref(self.hp), ctx=self.h)

    def _c(self, name, *args):
        return B.call(name, *args, ctx=self.h)

    # ---------------------------------------------------------------- steps
    def preprocess(self, scene: DeviceScene, cams, out: Proj | None = None) -> Proj:
        out = out or Proj.empty(len(cams), scene.N, scene.mo.device)
        cs = B.camera_array(cams)
        s, p = scene.struct(), out.struct()
        self._c("gs_preprocess", self.h, ctypes.byref(s), cs, len(cams), ctypes.byref(p), _stream())
        return out

    def bin(self, proj: Proj, cams, capacity: int | None = None) -> Bins:
        tiles = total_tiles(cams, self.tile)
        cap = capacity if capacity is not None else max(self._bins_cap, 1 << 16)
        while True:
            bins = Bins.empty(cap, tiles, proj.xy.device)
            needed = ctypes.c_uint64(0)
            ps, bs = proj.struct(), bins.struct()
            st = B.lib().gs_bin(self.h, ctypes.byref(ps), B.camera_array(cams), len(cams), ctypes.byref(bs),
                                ctypes.byref(needed), _stream())
            if st == B.GS_ERR_CAPACITY and capacity is None:
                self.status()      # clear the device status word
                cap = int(needed.value * 1.25) + 1024
                continue
            if st != B.GS_OK:
                raise B.GSError("gs_bin", st, B.lib().gs_last_error(self.h).decode())
            bins.F = int(needed.value)
            self._bins_cap = max(self._bins_cap, cap)
            return bins

    def render_fwd(self, proj: Proj, bins: Bins, cams):
        Bv = len(cams)
        H, W = cams[0].H, cams[0].W
        dev = proj.xy.device
        img = torch.empty(Bv, 3, H, W, dtype=torch.float32, device=dev)
        T = torch.empty(Bv, H, W, dtype=torch.float32, device=dev)
        nc = torch.empty(Bv, H, W, dtype=torch.int32, device=dev)
        ps, bs = proj.struct(), bins.struct()
        self._c("gs_render_fwd", self.h, ctypes.byref(ps), ctypes.byref(bs), B.camera_array(cams), Bv, _ptr(img),
                _ptr(T), _ptr(nc), _stream())
        return img, T, nc

    def render_bwd(self, proj: Proj, bins: Bins, cams, T, nc, dimg) -> ProjGrad:
        _check_f32(dimg, "d_img")
        Bv, N = proj.radius.shape
        g = ProjGrad.empty(Bv, N, proj.xy.device)
        ps, bs, gs = proj.struct(), bins.struct(), g.struct()
        self._c("gs_render_bwd", self.h, ctypes.byref(ps), ctypes.byref(bs), B.camera_array(cams), Bv, _ptr(T),
                _ptr(nc), _ptr(dimg), ctypes.byref(gs), _stream())
        return g

    def preprocess_bwd(self, scene: DeviceScene, cams, proj: Proj, pg: ProjGrad, out: DeviceScene | None = None,
                       scale: float | None = None):
        """Gradients of the parameters; the views' contributions are averaged
        (the paper's batch gradient) unless ``scale`` is given, which then
        multiplies their sum (scale=1: the sum)."""
        out = out or scene.zeros_like()
        s, p, g, o = scene.struct(), proj.struct(), pg.struct(), out.struct()
        if scale is None:
            self._c("gs_preprocess_bwd", self.h, ctypes.byref(s), B.camera_array(cams), len(cams), ctypes.byref(p),
                    ctypes.byref(g), ctypes.byref(o), _stream())
        else:
            self._c("gs_preprocess_bwd_scaled", self.h, ctypes.byref(s), B.camera_array(cams), len(cams),
                    ctypes.byref(p), ctypes.byref(g), ctypes.byref(o), float(scale), _stream())
        return out

    def loss(self, img: torch.Tensor, target: torch.Tensor):
        _check_f32(img, "img")
        _check_f32(target, "target")
        Bv, _, H, W = img.shape
        loss = torch.empty(Bv, dtype=torch.float32, device=img.device)
        dimg = torch.empty_like(img)
        self._c("gs_loss", self.h, _ptr(img), _ptr(target), Bv, W, H, _ptr(loss), _ptr(dimg), _stream())
        return loss, dimg

    def adam_step(self, p: DeviceScene, g: DeviceScene, m: DeviceScene, v: DeviceScene, step: int, batch: int):
        sp, sg, sm, sv = p.struct(), g.struct(), m.struct(), v.struct()
        self._c("gs_adam_step", self.h, ctypes.byref(sp), ctypes.byref(sg), ctypes.byref(sm), ctypes.byref(sv),
                int(step), int(batch), _stream())

    def adam_step_sparse(self, p: DeviceScene, g: DeviceScene, m: DeviceScene, v: DeviceScene,
                         visible: torch.Tensor, step: int, batch: int):
        if visible.dtype != torch.uint8 or not visible.is_cuda or visible.numel() != p.N:
            raise ValueError("visible must be a CUDA uint8 tensor with one entry per Gaussian")
        sp, sg, sm, sv = p.struct(), g.struct(), m.struct(), v.struct()
        self._c("gs_adam_step_sparse", self.h, ctypes.byref(sp), ctypes.byref(sg), ctypes.byref(sm),
                ctypes.byref(sv), _ptr(visible), int(step), int(batch), _stream())

    def set_densify_stats(self, acc: torch.Tensor | None, cnt: torch.Tensor | None):
        """gs_set_densify_stats: training steps accumulate |dL_v/d(u, v)| per
        visible (view, Gaussian) into acc (float32 [N]) and count into cnt
        (int32 [N], uint32 bits); None stops it."""
        if acc is None:
            self._c("gs_set_densify_stats", self.h, None, None, 0)
            self._dstats = None
            return
        if acc.dtype != torch.float32 or cnt.dtype != torch.int32 or acc.numel() != cnt.numel():
            raise ValueError("acc must be float32 and cnt int32, one entry per Gaussian each")
        self._c("gs_set_densify_stats", self.h, _ptr(acc), _ptr(cnt), int(acc.numel()))
        self._dstats = (acc, cnt)        # keep them alive while the library holds their addresses

    def densify(self, p: DeviceScene, m: DeviceScene, v: DeviceScene, acc, cnt, normals, grad_threshold,
                scale_threshold, min_opacity=0.005, split_div=1.6, capacity=None):
        """gs_densify: returns (p, m, v) of the densified scene (new tensors)."""
        cap = capacity if capacity is not None else 2 * p.N
        po, mo, vo = (DeviceScene.zeros(cap, p.mo.device, p.sh_degree) for _ in range(3))
        dp = B.gs_densify_params(float(grad_threshold), float(scale_threshold), float(min_opacity), float(split_div))
        n_out = ctypes.c_int64(0)
        sp, sm, sv, so, smo, svo = p.struct(), m.struct(), v.struct(), po.struct(), mo.struct(), vo.struct()
        self._c("gs_densify", self.h, ctypes.byref(sp), ctypes.byref(sm), ctypes.byref(sv), _ptr(acc), _ptr(cnt),
                _ptr(normals), ctypes.byref(dp), ctypes.byref(so), ctypes.byref(smo), ctypes.byref(svo), int(cap),
                ctypes.byref(n_out), _stream())
        n = int(n_out.value)
        cut = lambda s: DeviceScene(s.mo[:n].clone(), s.ls[:n].clone(), s.q[:n].clone(),
                                    s.sh[:, :n].contiguous(), s.sh_degree)
        return cut(po), cut(mo), cut(vo)

    def reset_opacity(self, p: DeviceScene, m: DeviceScene, v: DeviceScene, max_opacity=0.01):
        sp, sm, sv = p.struct(), m.struct(), v.struct()
        self._c("gs_reset_opacity", self.h, ctypes.byref(sp), ctypes.byref(sm), ctypes.byref(sv),
                ctypes.c_float(max_opacity), _stream())

    def division_points(self, cost: torch.Tensor, parts: int) -> torch.Tensor:
        """gs_division_points (Algorithm 1) of int32 (uint32 bits) costs."""
        div = torch.empty(parts, dtype=torch.int32, device=cost.device)
        self._c("gs_division_points", self.h, _ptr(cost), int(cost.numel()), int(parts), _ptr(div), _stream())
        return div

    def spatial_order(self, scene: DeviceScene) -> torch.Tensor:
        """gs_spatial_order: the Morton-order permutation of the Gaussians (int32 view of uint32)."""
        perm = torch.empty(max(scene.N, 1), dtype=torch.int32, device=scene.mo.device)
        s = scene.struct()
        self._c("gs_spatial_order", self.h, ctypes.byref(s), _ptr(perm), _stream())
        return perm[:scene.N]

    def permute(self, scene: DeviceScene, perm: torch.Tensor) -> DeviceScene:
        """gs_permute: a new scene with entry i = scene's entry perm[i]."""
        out = scene.zeros_like()
        s, d = scene.struct(), out.struct()
        self._c("gs_permute", self.h, ctypes.byref(s), _ptr(perm), ctypes.byref(d), _stream())
        return out

    def train_step(self, p, g, m, v, step, cams, targets, loss_out=None, cam_arr=None, check=False):
        """One gs_train_step.  check=True synchronises, and when the fragment
        buffer overflowed (the library then skipped the update) grows it and
        runs the same step again."""
        Bv = len(cams)
        loss_out = loss_out if loss_out is not None else torch.empty(Bv, dtype=torch.float32, device=targets.device)
        sp, sg, sm, sv = p.struct(), g.struct(), m.struct(), v.struct()
        self._c("gs_train_step", self.h, ctypes.byref(sp), ctypes.byref(sg), ctypes.byref(sm), ctypes.byref(sv),
                int(step), cam_arr if cam_arr is not None else B.camera_array(cams), Bv, _ptr(targets),
                _ptr(loss_out), _stream())
        if check and self._grew(p.N, cams):
            return self.train_step(p, g, m, v, step, cams, targets, loss_out, cam_arr, check=True)
        return loss_out

    def render(self, scene: DeviceScene, cams, imgs=None, cam_arr=None, check=False):
        """gs_render of a batch of views (sizes may differ).  check=True as in
        train_step: synchronise, grow the fragment buffer on overflow, render again."""
        if imgs is None:
            imgs = [torch.empty(3, c.H, c.W, dtype=torch.float32, device=scene.mo.device) for c in cams]
        arr = (ctypes.c_void_p * len(cams))(*[t.data_ptr() for t in imgs])
        s = scene.struct()
        self._c("gs_render", self.h, ctypes.byref(s), cam_arr if cam_arr is not None else B.camera_array(cams),
                len(cams), arr, _stream())
        if check and self._grew(scene.N, cams):
            return self.render(scene, cams, imgs, cam_arr, check=True)
        return imgs

    def _grew(self, N, cams) -> bool:
        code, needed = self.status()
        if code == B.GS_ERR_CAPACITY:
            self.reserve(N, cams, int(needed * 1.25) + 4096)
            return True
        if code != B.GS_OK:
            raise B.GSError("device status", code, B.lib().gs_last_error(self.h).decode())
        return False

    def reserve(self, N, cams, frag_capacity):
        self._c("gs_reserve", self.h, int(N), B.camera_array(cams), len(cams), int(frag_capacity))

    def get_step(self) -> int:
        """The device-side Adam step counter (synchronises)."""
        out = ctypes.c_int64(0)
        self._c("gs_get_step", self.h, ctypes.byref(out), _stream())
        return int(out.value)

    def set_step(self, step: int):
        self._c("gs_set_step", self.h, int(step), _stream())

    def workspace_size(self, N, cams, frag_capacity):
        """Bytes of caller workspace gs_reserve(N, cams, frag_capacity) takes."""
        n = ctypes.c_size_t(0)
        st = B.lib().gs_workspace_size(ctypes.byref(self.hp), int(N), B.camera_array(cams), len(cams),
                                       int(frag_capacity), ctypes.byref(n))
        if st != B.GS_OK:
            raise B.GSError("gs_workspace_size", st, "")
        return int(n.value)

    def set_workspace(self, ws):
        """Take all scratch from `ws` (a caller-owned uint8 CUDA tensor, kept
        alive here) instead of cudaMalloc; None returns to cudaMalloc."""
        if ws is None:
            self._c("gs_set_workspace", self.h, None, 0, _stream())
        else:
            self._c("gs_set_workspace", self.h, ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(),
                    _stream())
        self._ws = ws

    # ---------------------------------------------------------------- status
    def status(self):
        code = ctypes.c_int32(0)
        needed = ctypes.c_uint64(0)
        self._c("gs_get_status", self.h, _stream(), ctypes.byref(code), ctypes.byref(needed))
        return int(code.value), int(needed.value)

    def count_work(self, on: bool = True):
        """Counts the blending kernels' work (forward evaluations and
        contributing positions, backward walked and blended pairs) from the
        next step on (off by default: counting costs issue slots)."""
        self._c("gs_count_work", self.h, int(bool(on)))

    def counters(self):
        out = (ctypes.c_uint64 * 6)()
        self._c("gs_get_counters", self.h, _stream(), out)
        return dict(F=int(out[0]), evals_fwd=int(out[1]), evals_bwd=int(out[2]), walked_bwd=int(out[3]),
                    culled_nonfinite=int(out[4]), contrib_positions=int(out[5]))


def train_from_host(ctx: Context, p: DeviceScene, g: DeviceScene, m: DeviceScene, v: DeviceScene, cams,
                    host_targets, steps: int, cam_arr=None, on_loss=None):
    """`steps` training steps (gs_train_step, step counter on the device) whose
    targets come from pinned host memory, pipelined: the upload of step k+1's
    targets runs on a copy stream into the second of two device buffers
    while step k computes, and step k's losses come back to the host (pinned,
    on the compute stream) and are handed to on_loss(k, losses) while step
    k+1 runs.  host_targets: one pinned [B, 3, H, W] float32 tensor used by
    every step, or a sequence of `steps` of them.  Returns the last step's
    losses (numpy).  Synchronises at the end."""
    seq = isinstance(host_targets, (list, tuple))
    first = host_targets[0] if seq else host_targets
    if not first.is_pinned():
        raise ValueError("host targets must be in pinned memory")
    Bv = len(cams)
    arr = cam_arr if cam_arr is not None else B.camera_array(cams)
    dev = p.mo.device
    main = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(dev)
    bufs = [torch.empty(first.shape, dtype=torch.float32, device=dev) for _ in range(2)]
    uploaded = [torch.cuda.Event() for _ in range(2)]
    released = [torch.cuda.Event() for _ in range(2)]
    loss_dev = torch.empty(Bv, dtype=torch.float32, device=dev)
    loss_host = [torch.empty(Bv, dtype=torch.float32).pin_memory() for _ in range(2)]
    loss_ready = [torch.cuda.Event() for _ in range(2)]

    def upload(k):
        b = k % 2
        with torch.cuda.stream(copy):
            if k >= 2:
                copy.wait_event(released[b])          # step k - 2 is done with this buffer
            bufs[b].copy_(host_targets[k] if seq else host_targets, non_blocking=True)
            uploaded[b].record(copy)

    last = None
    if steps > 0:
        upload(0)
    for k in range(steps):
        b = k % 2
        if k + 1 < steps:
            upload(k + 1)
        main.wait_event(uploaded[b])
        ctx.train_step(p, g, m, v, 0, cams, bufs[b], loss_out=loss_dev, cam_arr=arr)
        released[b].record(main)
        loss_host[b].copy_(loss_dev, non_blocking=True)
        loss_ready[b].record(main)
        if k > 0:                                    # the previous step's losses, one step behind
            loss_ready[1 - b].synchronize()
            last = loss_host[1 - b].numpy().copy()
            if on_loss:
                on_loss(k - 1, last)
    if steps > 0:
        b = (steps - 1) % 2
        loss_ready[b].synchronize()
        last = loss_host[b].numpy().copy()
        if on_loss:
            on_loss(steps - 1, last)
    torch.cuda.synchronize(dev)
    return last


class RasterizeGaussians(torch.autograd.Function):
    """image[B,3,H,W] = render(params) with a hand-written backward, for B
    views of one size.

    Forward: gs_preprocess -> gs_bin -> gs_render_fwd.  Saved for backward:
    the per-(view, Gaussian) screen-space state, the sorted fragments and the
    per-pixel T_final / n_contrib; no per-fragment state.  Backward:
    gs_render_bwd -> gs_preprocess_bwd_scaled with scale 1, so the parameter
    gradient is the sum of the views' contributions (the autograd contract
    for a function with B outputs stacked); Context.train_step applies the
    paper's batch mean instead."""

    @staticmethod
    def forward(ctx, mo, ls, q, sh, gsctx: Context, cams, sh_degree: int):
        if len(cams) < 1 or any((c.W, c.H) != (cams[0].W, cams[0].H) for c in cams):
            raise ValueError("the autograd path renders one or more views of one size")
        scene = DeviceScene(mo.detach().contiguous(), ls.detach().contiguous(), q.detach().contiguous(),
                            sh.detach().contiguous(), sh_degree)
        proj = gsctx.preprocess(scene, cams)
        bins = gsctx.bin(proj, cams)
        img, T, nc = gsctx.render_fwd(proj, bins, cams)
        ctx.gsctx, ctx.cams, ctx.scene, ctx.proj, ctx.bins = gsctx, cams, scene, proj, bins
        ctx.save_for_backward(T, nc)
        return img

    @staticmethod
    def backward(ctx, dimg):
        T, nc = ctx.saved_tensors
        pg = ctx.gsctx.render_bwd(ctx.proj, ctx.bins, ctx.cams, T, nc, dimg.contiguous())
        g = ctx.gsctx.preprocess_bwd(ctx.scene, ctx.cams, ctx.proj, pg, scale=1.0)
        return g.mo, g.ls, g.q, g.sh, None, None, None


def rasterize(scene_tensors, gsctx: Context, cams, sh_degree=3):
    mo, ls, q, sh = scene_tensors
    return RasterizeGaussians.apply(mo, ls, q, sh, gsctx, tuple(cams), sh_degree)
