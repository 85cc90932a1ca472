"""The C-ABI library loads and exports every function include/hivc.h declares;
host-only entry points (no GPU work) behave as documented."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "hivc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(hivc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def hv():
    from paper_2008_10273_gb300 import build, hivc

    build.build()
    hivc.lib()
    return hivc


def test_every_declared_symbol_is_exported(hv):
    names = _declared_functions()
    assert len(names) >= 15
    L = hv.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in hivc.h but not exported"
    bound = {p[0] for p in hv.PROTOTYPES}
    assert set(names) == bound, f"binding/header mismatch: {set(names) ^ bound}"


def test_host_only_entry_points(hv):
    L = hv.lib()
    c = hv.config_default()
    assert (c.chroma, c.block, c.op, c.precision, c.max_cycles) == (1, 16, 0, 0, 40)
    assert c.iframe_tol == 1e-8
    assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0  # width/height unset
    c.width, c.height = 1920, 1080
    b = L.hivc_decoder_bytes(ctypes.byref(c))
    assert 100e6 < b < 400e6
    # a batch pool sized at creation for 8 inter frames is counted in
    c.batch_frames = 8
    assert L.hivc_decoder_bytes(ctypes.byref(c)) > b + 8 * 1920 * 1080 * 4
    for bad in (-1, 4097):
        c.batch_frames = bad
        assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0
    c.batch_frames = 0
    c.layout_groups = 2
    assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0
    c.layout_groups = 0
    c.fused_residual = 2
    assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0
    c.fused_residual = 0
    c.flat_start = 2
    assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0
    c.flat_start = 0
    for bad in (0, 1001):  # the correction loop runs on the device: its cycle cap is bounded
        c.max_cycles = bad
        assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0
    c.max_cycles = 40
    c.block = 17
    assert L.hivc_decoder_bytes(ctypes.byref(c)) == 0
    h = ctypes.c_void_p()
    assert L.hivc_decoder_create(ctypes.byref(c), ctypes.byref(h)) == hv.HIVC_E_INVALID
    assert h.value is None
    assert L.hivc_status_str(hv.HIVC_E_NO_REFERENCE).decode().startswith("inter frame")
    assert L.hivc_block_residual_workspace_bytes(1920, 1080, 16, 70000) > 70000 * 4
    assert L.hivc_block_residual_workspace_bytes(0, 1080, 16, 10) == 0
    # struct layouts the binding relies on
    assert ctypes.sizeof(hv.Config) == 72 and hv.Config.flat_start.offset == 68
    assert ctypes.sizeof(hv.Residual) == 32
    # hivc_stats: the per-family int64 pixel counts follow the launch counts
    assert hv.Stats.kernel_pixels.offset == 120 and ctypes.sizeof(hv.Stats) == 192


def test_oracle_is_not_reachable_from_the_product():
    """The product package never imports the oracle (the oracle is test
    infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2008_10273_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("oracles", ""), f"{f} mentions the oracle"
