"""The C ABI library builds, loads and exports every function that
include/tdgs.h declares (no GPU needed: only host-side helpers are called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdgs.h")


@pytest.fixture(scope="module")
def libtdgs():
    from paper_2511_16298_gb300 import build
    return ctypes.CDLL(build.build())


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdgs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_steps():
    names = declared_functions()
    for step in ("tdgs_count_tiles", "tdgs_scan", "tdgs_duplicate_keys", "tdgs_sort_pairs",
                 "tdgs_tile_ranges", "tdgs_sort_frame", "tdgs_context_create",
                 "tdgs_context_destroy", "tdgs_context_sync"):
        assert step in names


def test_every_declared_symbol_is_exported(libtdgs):
    missing = [n for n in declared_functions() if not hasattr(libtdgs, n)]
    assert not missing, missing


def test_host_helpers(libtdgs):
    from paper_2511_16298_gb300 import tdgs
    assert tdgs.num_tiles(1280, 720) == 80 * 45
    assert tdgs.num_tiles(1920, 1080) == 120 * 68
    assert tdgs.num_tiles(640, 360) == 40 * 23
    assert tdgs.tile_bits(256, 256) == 8
    assert tdgs.tile_bits(1280, 720) == 12
    assert tdgs.tile_bits(1920, 1080) == 13
    assert tdgs.tile_bits(16, 16) == 0
    assert tdgs.tile_bits(17, 16) == 1
    L = tdgs.lib()
    assert L.tdgs_status_string(0) == b"ok"
    assert L.tdgs_status_string(5) == b"cross-block wait timed out"
    assert L.tdgs_sort_variant_count() >= 3
    for bits, threads, items, occ in tdgs.sort_variants():
        assert 8 <= bits <= 11 and threads % 32 == 0 and items >= 1 and 1 <= occ <= 4


def test_context_create_rejects_bad_device(libtdgs):
    from paper_2511_16298_gb300 import tdgs
    h = ctypes.c_void_p()
    assert tdgs.lib().tdgs_context_create(ctypes.byref(h), -1) == tdgs.INVALID_ARGUMENT
    assert not h.value
    assert tdgs.lib().tdgs_context_create(None, 0) == tdgs.INVALID_ARGUMENT
    tdgs.lib().tdgs_context_destroy(None)  # no-op


def test_preprocess_host_checks(libtdgs):
    """Layouts of the preprocessing structs and the host-side argument
    checks that need no device."""
    from paper_2511_16298_gb300 import synth, tdgs
    assert synth.GAUSSIAN3D.itemsize == 16 and synth.COV3D.itemsize == 32
    assert synth.CAMERA.itemsize == 76
    L = tdgs.lib()
    cam = synth.camera((0.0, 0.0, -10.0), (0.0, 0.0, 0.0), 640, 360)
    buf = ctypes.create_string_buffer(cam.tobytes(), 76)
    assert L.tdgs_preprocess(None, None, None, 0, ctypes.cast(buf, ctypes.c_void_p), None, None,
                             None) == tdgs.INVALID_ARGUMENT
