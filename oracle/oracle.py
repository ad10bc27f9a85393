"""Python view of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Loads ``oracle/_build/libtdgs_oracle.so`` (built from ``tdgs_oracle.cpp``
with g++, no CUDA) and wraps each step of the 3DGS tile depth sort
(Sec. II-A: tile count, PrefixSum, DuplicateWithTile, Sorting, Identify
Range) as a numpy function.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg import this module; the library product never
does.  It shares no code with the CUDA path; the two meet only in the
seeded inputs of ``paper_2511_16298_gb300.synth``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdgs_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libtdgs_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, OVERFLOW = 0, 1, 3


def compile_oracle(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library (portable flags:
    no -march, no fast-math, no floating-point contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_oracle(_SRC, _LIB_PATH)


def load(path: str):
    """Load an oracle library from ``path`` and declare its signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    u32 = ctypes.c_uint32
    L.oracle_count_tiles.argtypes = [P, u32, u32, u32, P]
    L.oracle_scan.argtypes = [P, u32, P, P]
    L.oracle_duplicate.argtypes = [P, P, u32, u32, u32, P, P, u32]
    L.oracle_sort_pairs.argtypes = [P, P, u32]
    L.oracle_tile_ranges.argtypes = [P, u32, u32, P]
    L.oracle_sort_frame_normalized.argtypes = [P, u32, u32, u32, P, P, u32, P, P]
    L.oracle_sort_frame_normalized.restype = ctypes.c_int
    L.oracle_render.argtypes = [P, P, P, P, P, u32, u32, P, P]
    L.oracle_render.restype = ctypes.c_int
    L.oracle_preprocess.argtypes = [P, P, u32, P, P, P]
    L.oracle_preprocess.restype = ctypes.c_int
    L.oracle_num_tiles.argtypes = [u32, u32]
    L.oracle_num_tiles.restype = u32
    for f in ("oracle_count_tiles", "oracle_scan", "oracle_duplicate",
              "oracle_sort_pairs", "oracle_tile_ranges"):
        getattr(L, f).restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


class Oracle:
    """The five steps bound to one oracle library (the default build, or a
    variant compiled from edited source in the oracle's own tests)."""

    def __init__(self, library=None):
        self._L = library

    def _lib(self):
        return self._L if self._L is not None else lib()

    def count_tiles(self, g, width, height):
        return count_tiles(g, width, height, L=self._lib())

    def scan(self, counts):
        return scan(counts, L=self._lib())

    def duplicate(self, g, offsets, m, width, height):
        return duplicate(g, offsets, m, width, height, L=self._lib())

    def sort_pairs(self, keys, values):
        return sort_pairs(keys, values, L=self._lib())

    def tile_ranges(self, sorted_keys, num_tiles):
        return tile_ranges(sorted_keys, num_tiles, L=self._lib())

    def sort_frame(self, g, width, height):
        return sort_frame(g, width, height, L=self._lib())

    def preprocess(self, g3, cov, cam):
        return preprocess(g3, cov, cam, L=self._lib())

    def sort_frame_normalized(self, g, width, height):
        return sort_frame_normalized(g, width, height, L=self._lib())

    def render(self, rec, conic, rgb, sorted_values, ranges, width, height, background):
        return render(rec, conic, rgb, sorted_values, ranges, width, height, background, L=self._lib())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _records(g: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(g)
    assert g.dtype.itemsize == 16
    return g


def count_tiles(g: np.ndarray, width: int, height: int, L=None):
    g = _records(g)
    counts = np.zeros(len(g), dtype=np.uint32)
    st = (L or lib()).oracle_count_tiles(_ptr(g), len(g), width, height, _ptr(counts))
    return st, counts


def scan(counts: np.ndarray, L=None):
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    offsets = np.zeros(len(counts), dtype=np.uint32)
    total = np.zeros(1, dtype=np.uint64)
    st = (L or lib()).oracle_scan(_ptr(counts), len(counts), _ptr(offsets), _ptr(total))
    return st, offsets, int(total[0])


def duplicate(g: np.ndarray, offsets: np.ndarray, m: int, width: int, height: int, L=None):
    g = _records(g)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    keys = np.zeros(m, dtype=np.uint64)
    values = np.zeros(m, dtype=np.uint32)
    st = (L or lib()).oracle_duplicate(_ptr(g), _ptr(offsets), len(g), width, height,
                                       _ptr(keys), _ptr(values), m)
    return st, keys, values


def sort_pairs(keys: np.ndarray, values: np.ndarray, L=None):
    keys = np.array(keys, dtype=np.uint64, copy=True)
    values = np.array(values, dtype=np.uint32, copy=True)
    st = (L or lib()).oracle_sort_pairs(_ptr(keys), _ptr(values), len(keys))
    return st, keys, values


def tile_ranges(sorted_keys: np.ndarray, num_tiles: int, L=None):
    sorted_keys = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    ranges = np.zeros((num_tiles, 2), dtype=np.uint32)
    st = (L or lib()).oracle_tile_ranges(_ptr(sorted_keys), len(sorted_keys), num_tiles, _ptr(ranges))
    return st, ranges


_REC = np.dtype([("x", "<f4"), ("y", "<f4"), ("depth", "<f4"), ("radius", "<i4")])


def preprocess(g3: np.ndarray, cov: np.ndarray, cam: np.ndarray, L=None):
    """Preprocessing of 3D Gaussians for one camera: returns (status,
    records, conic_opacity) with records as 16-byte (x, y, depth, radius)
    and conic_opacity as (n, 4) float32.  g3: 16-byte records (mean,
    opacity); cov: 32-byte records (xx, xy, xz, yy, yz, zz, pad, pad);
    cam: one 76-byte camera block."""
    g3 = np.ascontiguousarray(g3)
    cov = np.ascontiguousarray(cov)
    cam = np.ascontiguousarray(cam)
    assert g3.dtype.itemsize == 16 and cov.dtype.itemsize == 32 and cam.dtype.itemsize == 76
    assert cam.size == 1 and len(cov) == len(g3)
    n = len(g3)
    rec = np.zeros(n, dtype=_REC)
    conic = np.zeros((n, 4), dtype=np.float32)
    st = (L or lib()).oracle_preprocess(_ptr(g3), _ptr(cov), n, _ptr(cam.reshape(1)), _ptr(rec), _ptr(conic))
    return st, rec, conic


def sort_frame_normalized(g: np.ndarray, width: int, height: int, L=None):
    """The 32-bit normalised-key frame (tile << 10 | 10-bit normalised
    depth): returns (status, keys uint32, values uint32, ranges (T, 2))."""
    g = _records(g)
    st, counts = count_tiles(g, width, height, L)
    m_cap = int(counts.astype(np.uint64).sum()) if st == OK else 0
    keys = np.zeros(m_cap, dtype=np.uint32)
    values = np.zeros(m_cap, dtype=np.uint32)
    T = num_tiles(width, height, L)
    ranges = np.zeros((T, 2), dtype=np.uint32)
    m = np.zeros(1, dtype=np.uint32)
    st = (L or lib()).oracle_sort_frame_normalized(_ptr(g), len(g), width, height, _ptr(keys), _ptr(values),
                                                   m_cap, _ptr(m), _ptr(ranges))
    return st, keys[:int(m[0])], values[:int(m[0])], ranges


def render(rec, conic, rgb, sorted_values, ranges, width: int, height: int, background, L=None):
    """Front-to-back blend of each tile's sorted Gaussians: returns (status,
    image (height, width, 3) float32).  rec: 16-byte records; conic: (n, 4)
    float32 (a, b, c, opacity); rgb: (n, 3) float32; sorted_values: the
    sorted Gaussian indices; ranges: (tiles, 2) uint32."""
    rec = np.ascontiguousarray(rec)
    conic = np.ascontiguousarray(conic, dtype=np.float32)
    rgb = np.ascontiguousarray(rgb, dtype=np.float32)
    sv = np.ascontiguousarray(sorted_values, dtype=np.uint32)
    rg = np.ascontiguousarray(ranges, dtype=np.uint32)
    bg = np.ascontiguousarray(background, dtype=np.float32)
    img = np.zeros((height, width, 3), dtype=np.float32)
    st = (L or lib()).oracle_render(_ptr(rec), _ptr(conic), _ptr(rgb), _ptr(sv), _ptr(rg), width, height,
                                    _ptr(bg), _ptr(img))
    return st, img


def num_tiles(width: int, height: int, L=None) -> int:
    return int((L or lib()).oracle_num_tiles(width, height))


def sort_frame(g: np.ndarray, width: int, height: int, L=None) -> dict:
    """All five steps in order; returns every intermediate and the status
    of the first step that failed (later steps are then skipped)."""
    out = {"status": OK, "m": 0}
    st, counts = count_tiles(g, width, height, L)
    out["counts"] = counts
    if st != OK:
        out["status"] = st
        return out
    st, offsets, m = scan(counts, L)
    out.update(offsets=offsets, m=m)
    if st != OK:
        out["status"] = st
        return out
    st, keys, values = duplicate(g, offsets, m, width, height, L)
    out.update(unsorted_keys=keys, unsorted_values=values)
    if st != OK:
        out["status"] = st
        return out
    _, skeys, svalues = sort_pairs(keys, values, L)
    out.update(keys=skeys, values=svalues)
    st, ranges = tile_ranges(skeys, num_tiles(width, height, L), L)
    out.update(ranges=ranges, status=st)
    return out
