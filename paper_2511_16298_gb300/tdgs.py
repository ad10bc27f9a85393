"""Python binding of libtdgs (the C ABI in ``include/tdgs.h``).

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are torch CUDA tensors; their device pointers and the current
torch stream are handed to the C calls.  If the shared library has not been
built, importing works but the first call raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

OK = 0
INVALID_ARGUMENT = 1
OUT_OF_MEMORY = 2
OVERFLOW = 3
CUDA_ERROR = 4
TIMEOUT = 5
CAPACITY = 6
SORT_DEPTH_POSITIVE = 1
TUNE_SORT_VARIANT, TUNE_TILE_DIGIT_BITS, TUNE_CTAS_PER_SM, TUNE_DEPTH_DIGIT_BITS = 0, 1, 3, 4

_lock = threading.Lock()
_lib = None


class TdgsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = lib().tdgs_status_string(status).decode() if _lib else str(status)
        super().__init__(f"{where}: {name} ({status}){': ' + detail if detail else ''}")


class _Range(ctypes.Structure):
    _fields_ = [("start", ctypes.c_uint32), ("end", ctypes.c_uint32)]


class _Frame(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32)]


class _View(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("n", ctypes.c_uint32), ("f", _Frame)]


class _ViewResult(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("values", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("m", ctypes.c_uint32), ("num_tiles", ctypes.c_uint32)]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64),
                ("items", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libtdgs.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(path)
            P, u32, i32, st = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int
            F = _Frame
            sig = {
                "tdgs_context_create": ([ctypes.POINTER(P), i32], st),
                "tdgs_context_destroy": ([P], None),
                "tdgs_context_sync": ([P, P], st),
                "tdgs_status_string": ([i32], ctypes.c_char_p),
                "tdgs_last_error": ([P], ctypes.c_char_p),
                "tdgs_num_tiles": ([F], u32),
                "tdgs_tile_bits": ([F], u32),
                "tdgs_sort_variant_count": ([], i32),
                "tdgs_sort_variant_info": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                            ctypes.POINTER(i32), ctypes.POINTER(i32)], st),
                "tdgs_context_set_sort_variant": ([P, i32], st),
                "tdgs_context_set_tuning": ([P, i32, i32], st),
                "tdgs_context_get_tuning": ([P, i32, ctypes.POINTER(i32)], st),
                "tdgs_context_launch_count": ([P], ctypes.c_uint64),
                "tdgs_context_enable_timing": ([P, i32], st),
                "tdgs_context_kernel_times": ([P, ctypes.POINTER(_KernelTime), i32], i32),
                "tdgs_context_depth_passes": ([P, ctypes.POINTER(i32), P], st),
                "tdgs_count_tiles": ([P, P, u32, F, P, P], st),
                "tdgs_scan": ([P, P, u32, P, P, P], st),
                "tdgs_duplicate_keys": ([P, P, P, u32, F, P, P, u32, P], st),
                "tdgs_sort_pairs": ([P, P, P, P, P, u32, u32, u32, ctypes.POINTER(i32), P], st),
                "tdgs_tile_ranges": ([P, P, u32, u32, P, P], st),
                "tdgs_sort_frame": ([P, P, u32, F, ctypes.POINTER(P), ctypes.POINTER(P),
                                     ctypes.POINTER(P), ctypes.POINTER(u32), P], st),
                "tdgs_scan_noalloc": ([P, u32, P, P, P, P], st),
                "tdgs_preprocess": ([P, P, P, u32, P, P, P, P], st),
                "tdgs_sort_pairs_bitonic": ([P, P, P, P, P, u32, P], st),
                "tdgs_diag_barrier_timeout": ([P, P], st),
                "tdgs_render": ([P, P, P, P, u32, P, P, F, P, P, P], st),
                "tdgs_sort_views_3d": ([P, P, P, u32, P, u32, ctypes.POINTER(_ViewResult), P], st),
                "tdgs_context_projected": ([P, ctypes.POINTER(P), ctypes.POINTER(P)], st),
                "tdgs_sort_frame_normalized": ([P, P, u32, F, ctypes.POINTER(P), ctypes.POINTER(P),
                                                ctypes.POINTER(P), ctypes.POINTER(u32), P], st),
                "tdgs_sort_frame_3d": ([P, P, P, u32, P, ctypes.POINTER(P), ctypes.POINTER(P),
                                        ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                        ctypes.POINTER(u32), P], st),
                "tdgs_sort_views": ([P, ctypes.POINTER(_View), u32, ctypes.POINTER(_ViewResult), P], st),
                "tdgs_reserve_views": ([P, ctypes.POINTER(_View), u32, ctypes.c_uint64, P], st),
                "tdgs_sort_views_async": ([P, ctypes.POINTER(_View), u32, P], st),
                "tdgs_views_results": ([P, ctypes.POINTER(_ViewResult), u32, P], st),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(0)


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def records_to_tensor(g: np.ndarray, device="cuda") -> torch.Tensor:
    """16-byte Gaussian records (numpy) -> int32 CUDA tensor of shape (n, 4)."""
    a = np.ascontiguousarray(g).view(np.int32).reshape(-1, 4)
    return torch.from_numpy(a).to(device)


def num_tiles(width: int, height: int) -> int:
    return int(lib().tdgs_num_tiles(_Frame(width, height)))


def tile_bits(width: int, height: int) -> int:
    return int(lib().tdgs_tile_bits(_Frame(width, height)))


def scan_noalloc(counts: torch.Tensor, offsets=None, total=None, error=None):
    """tdgs_scan_noalloc on the current stream (no context, no allocation
    inside the library); returns (offsets, total, error) device tensors."""
    n = counts.shape[0]
    dev = counts.device
    offsets = torch.empty(n, dtype=torch.int32, device=dev) if offsets is None else offsets
    total = torch.zeros(1, dtype=torch.int32, device=dev) if total is None else total
    error = torch.zeros(1, dtype=torch.int32, device=dev) if error is None else error
    st = lib().tdgs_scan_noalloc(_ptr(counts), n, _ptr(offsets), _ptr(total), _ptr(error), _stream(dev))
    if st != OK:
        raise TdgsError(st, "tdgs_scan_noalloc")
    return offsets, total, error


def sort_variants() -> list[tuple[int, int, int, int]]:
    """(digit bits, threads, items per thread, blocks per SM) of each
    compiled pass kernel of tdgs_sort_pairs."""
    L = lib()
    out = []
    for i in range(L.tdgs_sort_variant_count()):
        b, t, it, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.tdgs_sort_variant_info(i, ctypes.byref(b), ctypes.byref(t), ctypes.byref(it), ctypes.byref(o))
        out.append((b.value, t.value, it.value, o.value))
    return out


class _DeviceView:
    """Zero-copy view of a context-owned device buffer (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
            "strides": None, "stream": None}


def _view(ptr: int, n: int, dtype: torch.dtype, device) -> torch.Tensor:
    ts = {torch.int64: "<i8", torch.int32: "<i4", torch.float32: "<f4"}[dtype]
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_DeviceView(ptr, n, ts), device=device)


class Context:
    """One library context (scratch buffers, latched device errors) bound to
    one CUDA device.  Use one context per concurrent stream."""

    def __init__(self, device: int | torch.device = 0):
        if isinstance(device, torch.device):
            device = device.index or 0
        self.device = torch.device("cuda", device)
        self._h = ctypes.c_void_p()
        st = lib().tdgs_context_create(ctypes.byref(self._h), int(device))
        if st != OK:
            raise TdgsError(st, "tdgs_context_create")

    def close(self):
        if self._h:
            torch.cuda.synchronize(self.device)
            lib().tdgs_context_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.tdgs_context_destroy(self._h)
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ helpers
    def _check(self, st: int, where: str):
        if st != OK:
            raise TdgsError(st, where, lib().tdgs_last_error(self._h).decode())

    def sync(self):
        """Wait for the current stream; raise the first device-latched error."""
        self._check(lib().tdgs_context_sync(self._h, _stream(self.device)), "tdgs_context_sync")

    def set_sort_variant(self, variant: int):
        self._check(lib().tdgs_context_set_sort_variant(self._h, int(variant)),
                    "tdgs_context_set_sort_variant")

    def set_tuning(self, key: int, value: int):
        self._check(lib().tdgs_context_set_tuning(self._h, int(key), int(value)), "tdgs_context_set_tuning")

    def get_tuning(self, key: int) -> int:
        v = ctypes.c_int(0)
        self._check(lib().tdgs_context_get_tuning(self._h, int(key), ctypes.byref(v)), "tdgs_context_get_tuning")
        return v.value

    def apply_tuning(self, knobs: dict):
        for k, v in knobs.items():
            self.set_tuning({"sort_variant": TUNE_SORT_VARIANT, "tile_digit_bits": TUNE_TILE_DIGIT_BITS,
                             "ctas_per_sm": TUNE_CTAS_PER_SM, "depth_digit_bits": TUNE_DEPTH_DIGIT_BITS}[k], v)

    @property
    def launches(self) -> int:
        """Kernels launched through this context so far."""
        return int(lib().tdgs_context_launch_count(self._h))

    def enable_timing(self, on: bool = True):
        self._check(lib().tdgs_context_enable_timing(self._h, int(on)), "tdgs_context_enable_timing")

    def kernel_times(self) -> dict:
        """{kernel: {"launches", "items", "ms"}} since the last read (waits
        for the recorded events)."""
        cap = 64  # more than the library's kernel kinds; the call clears the record
        buf = (_KernelTime * cap)()
        n = lib().tdgs_context_kernel_times(self._h, buf, cap)
        if n < 0:
            raise TdgsError(INVALID_ARGUMENT, "tdgs_context_kernel_times")
        return {buf[i].name.decode(): {"launches": int(buf[i].launches), "items": int(buf[i].items),
                                       "ms": float(buf[i].total_ms)} for i in range(min(n, cap))}

    def depth_passes(self) -> int:
        """Digit passes of the last single-launch depth sort (0 if none)."""
        v = ctypes.c_int(0)
        self._check(lib().tdgs_context_depth_passes(self._h, ctypes.byref(v), _stream(self.device)),
                    "tdgs_context_depth_passes")
        return v.value

    # ------------------------------------------------------------ the steps
    def count_tiles(self, g: torch.Tensor, width: int, height: int, out=None) -> torch.Tensor:
        n = g.shape[0]
        out = torch.empty(n, dtype=torch.int32, device=self.device) if out is None else out
        self._check(lib().tdgs_count_tiles(self._h, _ptr(g), n, _Frame(width, height), _ptr(out),
                                           _stream(self.device)), "tdgs_count_tiles")
        return out

    def scan(self, counts: torch.Tensor, out=None, total=None):
        n = counts.shape[0]
        out = torch.empty(n, dtype=torch.int32, device=self.device) if out is None else out
        total = torch.zeros(1, dtype=torch.int32, device=self.device) if total is None else total
        self._check(lib().tdgs_scan(self._h, _ptr(counts), n, _ptr(out), _ptr(total),
                                    _stream(self.device)), "tdgs_scan")
        return out, total

    def duplicate_keys(self, g, offsets, width, height, m, keys=None, values=None):
        n = g.shape[0]
        keys = torch.empty(m, dtype=torch.int64, device=self.device) if keys is None else keys
        values = torch.empty(m, dtype=torch.int32, device=self.device) if values is None else values
        self._check(lib().tdgs_duplicate_keys(self._h, _ptr(g), _ptr(offsets), n,
                                              _Frame(width, height), _ptr(keys), _ptr(values),
                                              min(m, keys.shape[0], values.shape[0]),
                                              _stream(self.device)), "tdgs_duplicate_keys")
        return keys, values

    def sort_pairs(self, keys, values, tile_bits: int, flags: int = 0, keys_alt=None,
                   values_alt=None):
        """Sort in place through the alternate buffers; returns the
        (keys, values) tensors that hold the sorted result."""
        m = keys.shape[0]
        keys_alt = torch.empty_like(keys) if keys_alt is None else keys_alt
        values_alt = torch.empty_like(values) if values_alt is None else values_alt
        alt = ctypes.c_int(0)
        self._check(lib().tdgs_sort_pairs(self._h, _ptr(keys), _ptr(values), _ptr(keys_alt),
                                          _ptr(values_alt), m, tile_bits, flags, ctypes.byref(alt),
                                          _stream(self.device)), "tdgs_sort_pairs")
        return (keys_alt, values_alt) if alt.value else (keys, values)

    def diag_barrier_timeout(self):
        """Failure-detection check: a grid barrier one block never reaches;
        the next sync() raises TdgsError(TIMEOUT) and the context stays
        usable."""
        self._check(lib().tdgs_diag_barrier_timeout(self._h, _stream(self.device)), "tdgs_diag_barrier_timeout")

    def sort_pairs_bitonic(self, keys, values, keys_out=None, values_out=None):
        """The paper's bitonic network: sorts by (key, value); returns
        (keys_out, values_out) (new tensors unless given; may be the inputs)."""
        m = keys.shape[0]
        if keys_out is None:
            keys_out = torch.empty_like(keys)
        if values_out is None:
            values_out = torch.empty_like(values)
        self._check(lib().tdgs_sort_pairs_bitonic(self._h, _ptr(keys), _ptr(values), _ptr(keys_out),
                                                  _ptr(values_out), m, _stream(self.device)),
                    "tdgs_sort_pairs_bitonic")
        return keys_out, values_out

    def tile_ranges(self, sorted_keys, num_tiles: int, m=None, out=None) -> torch.Tensor:
        m = sorted_keys.shape[0] if m is None else m
        out = torch.empty((num_tiles, 2), dtype=torch.int32, device=self.device) if out is None else out
        self._check(lib().tdgs_tile_ranges(self._h, _ptr(sorted_keys), m, num_tiles, _ptr(out),
                                           _stream(self.device)), "tdgs_tile_ranges")
        return out

    def sort_frame(self, g: torch.Tensor, width: int, height: int, copy: bool = False):
        """All five steps.  Returns (keys, values, ranges, m); the tensors are
        views of context buffers valid until the next call on this context
        unless copy=True."""
        n = g.shape[0]
        kp, vp, rp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        m = ctypes.c_uint32(0)
        self._check(lib().tdgs_sort_frame(self._h, _ptr(g), n, _Frame(width, height),
                                          ctypes.byref(kp), ctypes.byref(vp), ctypes.byref(rp),
                                          ctypes.byref(m), _stream(self.device)), "tdgs_sort_frame")
        T = num_tiles(width, height)
        k = _view(kp.value or 0, m.value, torch.int64, self.device)
        v = _view(vp.value or 0, m.value, torch.int32, self.device)
        r = _view(rp.value or 0, 2 * T, torch.int32, self.device).view(T, 2)
        if copy:
            k, v, r = k.clone(), v.clone(), r.clone()
        return k, v, r, int(m.value)

    def sort_views_3d(self, g3: torch.Tensor, cov: torch.Tensor, cams, copy: bool = False):
        """Preprocessing and the sort for every camera of ``cams`` (a CAMERA
        array) over the same 3D Gaussians in one batch.  Returns a list of
        (keys, values, ranges, m) per view (views of context buffers unless
        copy=True)."""
        cams = np.ascontiguousarray(np.asarray(cams).reshape(-1))
        assert cams.dtype.itemsize == 76
        nv = len(cams)
        cb = ctypes.create_string_buffer(cams.tobytes(), 76 * nv)
        res = (_ViewResult * nv)()
        self._check(lib().tdgs_sort_views_3d(self._h, _ptr(g3), _ptr(cov), g3.shape[0],
                                             ctypes.cast(cb, ctypes.c_void_p), nv, res, _stream(self.device)),
                    "tdgs_sort_views_3d")
        return self._results(res, nv, copy)

    def projected(self, n_total: int):
        """(records (n_total, 4) int32, conic (n_total, 4) float32) of the
        last 3D call, view after view."""
        rp, cp = ctypes.c_void_p(), ctypes.c_void_p()
        self._check(lib().tdgs_context_projected(self._h, ctypes.byref(rp), ctypes.byref(cp)),
                    "tdgs_context_projected")
        rec = _view(rp.value or 0, 4 * n_total, torch.int32, self.device).view(n_total, 4)
        con = _view(cp.value or 0, 4 * n_total, torch.float32, self.device).view(n_total, 4)
        return rec, con

    def sort_frame_normalized(self, g: torch.Tensor, width: int, height: int, copy: bool = False):
        """Steps 1-5 with the paper's 32-bit normalised key (tile << 10 |
        10-bit depth).  Returns (keys int32, values int32, ranges, m)."""
        n = g.shape[0]
        kp, vp, rp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        m = ctypes.c_uint32(0)
        self._check(lib().tdgs_sort_frame_normalized(self._h, _ptr(g), n, _Frame(width, height),
                                                     ctypes.byref(kp), ctypes.byref(vp), ctypes.byref(rp),
                                                     ctypes.byref(m), _stream(self.device)),
                    "tdgs_sort_frame_normalized")
        T = num_tiles(width, height)
        k = _view(kp.value or 0, m.value, torch.int32, self.device)
        v = _view(vp.value or 0, m.value, torch.int32, self.device)
        r = _view(rp.value or 0, 2 * T, torch.int32, self.device).view(T, 2)
        if copy:
            k, v, r = k.clone(), v.clone(), r.clone()
        return k, v, r, int(m.value)

    # ------------------------------------------------------ preprocessing
    @staticmethod
    def _camera(cam):
        """One 76-byte camera block (numpy CAMERA record) as a ctypes buffer."""
        a = np.ascontiguousarray(np.asarray(cam).reshape(1))
        assert a.dtype.itemsize == 76
        return ctypes.create_string_buffer(a.tobytes(), 76)

    def preprocess(self, g3: torch.Tensor, cov: torch.Tensor, cam, records=None, conic=None,
                   with_conic: bool = True):
        """Project n 3D Gaussians for one camera.  g3: (n, 4) float32 CUDA
        tensor (mean, opacity); cov: (n, 8) float32 (xx, xy, xz, yy, yz, zz,
        pad, pad); cam: a CAMERA record.  Returns (records (n, 4) int32
        bit-view of the 16-byte records, conic (n, 4) float32 or None)."""
        n = g3.shape[0]
        if records is None:
            records = torch.empty((n, 4), dtype=torch.int32, device=g3.device)
        if conic is None and with_conic:
            conic = torch.empty((n, 4), dtype=torch.float32, device=g3.device)
        cb = self._camera(cam)
        self._check(lib().tdgs_preprocess(self._h, _ptr(g3), _ptr(cov), n, ctypes.cast(cb, ctypes.c_void_p),
                                          _ptr(records), _ptr(conic), _stream(self.device)), "tdgs_preprocess")
        return records, conic

    def sort_frame_3d(self, g3: torch.Tensor, cov: torch.Tensor, cam, copy: bool = False):
        """Preprocessing and steps 1-5.  Returns (keys, values, ranges, m,
        records, conic); the tensors are views of context buffers valid until
        the next call on this context unless copy=True."""
        n = g3.shape[0]
        rp, cp, kp, vp, gp = (ctypes.c_void_p() for _ in range(5))
        m = ctypes.c_uint32(0)
        cb = self._camera(cam)
        self._check(lib().tdgs_sort_frame_3d(self._h, _ptr(g3), _ptr(cov), n, ctypes.cast(cb, ctypes.c_void_p),
                                             ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(kp),
                                             ctypes.byref(vp), ctypes.byref(gp), ctypes.byref(m),
                                             _stream(self.device)), "tdgs_sort_frame_3d")
        c = np.asarray(cam).reshape(())
        T = num_tiles(int(c["width"]), int(c["height"]))
        k = _view(kp.value or 0, m.value, torch.int64, self.device)
        v = _view(vp.value or 0, m.value, torch.int32, self.device)
        r = _view(gp.value or 0, 2 * T, torch.int32, self.device).view(T, 2)
        rec = _view(rp.value or 0, 4 * n, torch.int32, self.device).view(n, 4)
        con = _view(cp.value or 0, 4 * n, torch.float32, self.device).view(n, 4)
        if copy:
            k, v, r, rec, con = k.clone(), v.clone(), r.clone(), rec.clone(), con.clone()
        return k, v, r, int(m.value), rec, con

    def render(self, records, conic, rgb, values, ranges, width: int, height: int,
               background=(0.0, 0.0, 0.0), out=None) -> torch.Tensor:
        """Front-to-back blend of every tile: returns a (height, width, 3)
        float32 image.  records: (n, 4) int32 bit-view of the 16-byte
        records; conic: (n, 4) float32; rgb: (n, 3) float32; values, ranges:
        as sort_frame returns them."""
        n = records.shape[0]
        if out is None:
            out = torch.empty((height, width, 3), dtype=torch.float32, device=self.device)
        bg = (ctypes.c_float * 3)(*background)
        self._check(lib().tdgs_render(self._h, _ptr(records), _ptr(conic), _ptr(rgb), n, _ptr(values),
                                      _ptr(ranges), _Frame(width, height), ctypes.cast(bg, ctypes.c_void_p),
                                      _ptr(out), _stream(self.device)), "tdgs_render")
        return out

    def render_frame_3d(self, g3, cov, rgb, cam, background=(0.0, 0.0, 0.0), out=None):
        """Preprocessing, sort and render of one camera's image: returns
        (image, m)."""
        k, v, r, m, rec, con = self.sort_frame_3d(g3, cov, cam)
        c = np.asarray(cam).reshape(())
        img = self.render(rec, con, rgb, v, r, int(c["width"]), int(c["height"]), background, out)
        return img, m

    # ------------------------------------------------------------ views
    @staticmethod
    def _views(views):
        """views: list of (records tensor (n, 4), width, height)."""
        arr = (_View * len(views))()
        for i, (g, w, h) in enumerate(views):
            arr[i].g = g.data_ptr() if g.numel() else None
            arr[i].n = g.shape[0]
            arr[i].f = _Frame(w, h)
        return arr

    def _results(self, res, n, copy):
        out = []
        for i in range(n):
            r = res[i]
            k = _view(r.keys or 0, r.m, torch.int64, self.device)
            v = _view(r.values or 0, r.m, torch.int32, self.device)
            rg = _view(r.ranges or 0, 2 * r.num_tiles, torch.int32, self.device).view(r.num_tiles, 2)
            if copy:
                k, v, rg = k.clone(), v.clone(), rg.clone()
            out.append((k, v, rg, int(r.m)))
        return out

    def sort_views(self, views, copy: bool = False):
        """All views in one batch; returns [(keys, values, ranges, m)] per
        view (views of context buffers unless copy=True)."""
        arr = self._views(views)
        res = (_ViewResult * len(views))()
        self._check(lib().tdgs_sort_views(self._h, arr, len(views), res, _stream(self.device)),
                    "tdgs_sort_views")
        return self._results(res, len(views), copy)

    def reserve_views(self, views, pair_capacity: int):
        arr = self._views(views)
        self._check(lib().tdgs_reserve_views(self._h, arr, len(views), int(pair_capacity),
                                             _stream(self.device)), "tdgs_reserve_views")

    def sort_views_async(self, views):
        """Graph-capturable batch (after reserve_views); read with views_results()."""
        arr = self._views(views)
        self._check(lib().tdgs_sort_views_async(self._h, arr, len(views), _stream(self.device)),
                    "tdgs_sort_views_async")

    def views_results(self, n: int, copy: bool = False):
        res = (_ViewResult * n)()
        self._check(lib().tdgs_views_results(self._h, res, n, _stream(self.device)), "tdgs_views_results")
        return self._results(res, n, copy)

