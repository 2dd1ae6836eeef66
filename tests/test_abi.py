"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gs.h declares; the ctypes mirror of every struct has the C size.
No compute call is made (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgs():
    from paper_2406_18533_gb300 import build, binding
    build.build()
    return binding.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gs_status|const char \*|int32_t|uint64_t)\s*\*?\s*(gs_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(libgs):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(libgs, n), n


def test_binding_covers_every_entry_point(libgs):
    from paper_2406_18533_gb300 import binding
    assert set(_declared()) == set(binding.SIGNATURES)


def test_abi_version_and_defaults(libgs):
    from paper_2406_18533_gb300 import binding
    assert libgs.gs_abi_version() == 5
    hp = binding.default_hparams()
    assert hp.tile == 16 and hp.smem_batch == 64 and hp.px_per_thread == 1
    assert abs(hp.alpha_min - 1 / 255) < 1e-9 and abs(hp.alpha_max - 0.99) < 1e-7 and abs(hp.T_min - 1e-4) < 1e-10
    assert hp.scale_lr_sqrt_b == 1 and hp.scale_beta_pow_b == 1 and abs(hp.lambda_dssim - 0.2) < 1e-7


def test_struct_layout_matches_c(tmp_path):
    """sizeof and every field offset of the ctypes mirrors equal what gcc
    computes from include/gs.h."""
    from paper_2406_18533_gb300 import binding as b
    structs = [b.gs_camera, b.gs_scene, b.gs_hparams, b.gs_proj, b.gs_proj_grad, b.gs_bins, b.gs_densify_params]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', 'int main(void) {']
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for st in structs:
        n = st.__name__
        assert int(out[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(out[f"{n}.{f}"]) == getattr(st, f).offset, (n, f)
    assert ctypes.sizeof(b.gs_camera) == 80


def test_invalid_arguments_rejected_on_host(libgs):
    """Host-side checks return GS_ERR_INVALID_ARG before any CUDA call."""
    from paper_2406_18533_gb300 import binding as b
    hp = b.default_hparams(tile=12)
    h = ctypes.c_void_p()
    assert libgs.gs_create(ctypes.byref(h), ctypes.byref(hp)) == b.GS_ERR_INVALID_ARG
    hp = b.default_hparams(smem_batch=100)
    assert libgs.gs_create(ctypes.byref(h), ctypes.byref(hp)) == b.GS_ERR_INVALID_ARG
    hp = b.default_hparams(tile=32, smem_batch=128)
    assert libgs.gs_create(ctypes.byref(h), ctypes.byref(hp)) == b.GS_ERR_INVALID_ARG
    for ppt, tile in ((0, 16), (3, 16), (4, 8)):   # 1, 2 or 4 pixels per thread; 4 needs tile >= 16
        hp = b.default_hparams(px_per_thread=ppt, tile=tile)
        assert libgs.gs_create(ctypes.byref(h), ctypes.byref(hp)) == b.GS_ERR_INVALID_ARG
    assert libgs.gs_create(None, None) == b.GS_ERR_INVALID_ARG
    assert libgs.gs_destroy(None) == b.GS_ERR_INVALID_ARG
    size = ctypes.c_size_t(0)
    assert libgs.gs_workspace_size(None, 10, None, 1, 0, ctypes.byref(size)) == b.GS_ERR_INVALID_ARG


def test_workspace_size_grows_with_problem(libgs):
    from paper_2406_18533_gb300 import binding as b, synth
    cams = b.camera_array([synth.test_camera(64, 48)])
    s1, s2 = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert libgs.gs_workspace_size(None, 1000, cams, 1, 10000, ctypes.byref(s1)) == 0
    assert libgs.gs_workspace_size(None, 100000, cams, 1, 10000, ctypes.byref(s2)) == 0
    assert s2.value > s1.value > 0


def test_workspace_size_counts_every_buffer_of_the_configuration(libgs):
    """gs_workspace_size is a host-side dry run of gs_reserve: deterministic,
    a whole number of 256-byte regions, larger by at least the visibility
    mask with visible-only Adam and by the cost and range arrays with the
    measured-cost schedules, and it validates the hyperparameters."""
    from paper_2406_18533_gb300 import binding as b, synth
    cams = b.camera_array([synth.test_camera(640, 360)] * 3)
    N, cap = 50000, 400000

    def size(**kw):
        hp = b.default_hparams(**kw)
        out = ctypes.c_size_t(0)
        assert libgs.gs_workspace_size(ctypes.byref(hp), N, cams, 3, cap, ctypes.byref(out)) == 0
        return out.value

    base = size()
    assert base == size() and base % 256 == 0
    assert size(sparse_adam=1) >= base + N
    assert size(schedule=1) > base and size(schedule=2) > base
    assert size(tile=8) > base                       # more tiles: longer range and order arrays
    hp = b.default_hparams(schedule=3)
    out = ctypes.c_size_t(0)
    assert libgs.gs_workspace_size(ctypes.byref(hp), N, cams, 3, cap, ctypes.byref(out)) == b.GS_ERR_INVALID_ARG


def test_bin_noalloc_rejects_bad_arguments_on_host(libgs):
    """gs_bin_noalloc checks its sizes before touching the device: views,
    tile edge, null outputs, and the fixed scratch's limits (2^18 pairs,
    2^20 fragments)."""
    from paper_2406_18533_gb300 import binding as b, synth
    fake = 256                                          # never dereferenced: every case fails first
    cams = b.camera_array([synth.test_camera(64, 48)] * 2)
    needed = ctypes.c_uint64(0)

    def call(B=1, N=100, tile=16, cap=1000, ranges=fake, count=fake, keys=fake, vals=fake, W=None):
        proj = b.gs_proj(fake, fake, fake, fake, N, B, 0)
        out = b.gs_bins(keys, vals, ranges, count, cap)
        cs = cams
        if W is not None:
            cs = b.camera_array([synth.test_camera(64, 48)] * B)
            cs[0].W = W
        return libgs.gs_bin_noalloc(ctypes.byref(proj), cs, B, tile, ctypes.byref(out), ctypes.byref(needed), None)

    bad = b.GS_ERR_INVALID_ARG
    assert call(B=0) == bad
    assert call(B=b.GS_MAX_VIEWS + 1) == bad
    assert call(tile=12) == bad
    assert call(ranges=None) == bad
    assert call(count=None) == bad
    assert call(keys=None) == bad                       # capacity > 0 needs key and value arrays
    assert call(N=(1 << 18) + 1) == bad                 # B * N above the scratch's pair limit
    assert call(B=2, N=1 << 17 | 1) == bad
    assert call(cap=(1 << 20) + 1) == bad               # fragment capacity above the limit
    assert call(W=0) == bad                             # camera sizes checked on the host
    assert libgs.gs_bin_noalloc(None, cams, 1, 16, None, ctypes.byref(needed), None) == bad


def test_injected_allocation_failure_gives_oom(libgs):
    """The allocation-failure hook makes gs_create fail with GS_ERR_OOM before
    any device call (so this runs without a GPU), returns no context, and
    fires once."""
    import ctypes
    from paper_2406_18533_gb300 import binding as b
    assert libgs.gs_debug_fail_alloc(-2) == b.GS_ERR_INVALID_ARG
    assert libgs.gs_debug_fail_alloc(0) == b.GS_OK
    h = ctypes.c_void_p(1)
    assert libgs.gs_create(ctypes.byref(h), None) == b.GS_ERR_OOM
    assert not h.value
    st = libgs.gs_create(ctypes.byref(h), None)         # injection spent: reaches the device
    assert st in (b.GS_OK, b.GS_ERR_CUDA)
    if st == b.GS_OK:
        libgs.gs_destroy(h)
    assert libgs.gs_debug_set_lookback(0, 0) == b.GS_OK
