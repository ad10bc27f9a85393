"""Frames from host memory to sorted results in host memory, overlapped.

The host link of this GPU moves about 190 GB/s each way, so returning a
frame's sorted pairs (12 bytes per pair) takes longer than sorting it.
``HostPipeline`` keeps ``depth`` slots -- each a library context, a CUDA
stream, a device input buffer and pinned host output buffers -- and runs
frame i in slot i % depth: the upload of its records, ``tdgs_sort_frame``
and the download of its keys, values and ranges are queued on the slot's
stream, so one frame's download overlaps the next frame's upload and sort.
A slot is reused only after its previous download has finished.

Every frame still crosses the host link both ways; results are identical
to ``Context.sort_frame`` followed by copies on one stream.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import tdgs


@dataclasses.dataclass
class HostResult:
    """Sorted output of one frame in pinned host memory (views of the
    slot's buffers, valid until the slot is reused ``depth`` frames later;
    ``copy()`` detaches them)."""

    keys: torch.Tensor    # (m,) int64: (tile << 32 | depth bits)
    values: torch.Tensor  # (m,) int32: Gaussian index
    ranges: torch.Tensor  # (tiles, 2) int32
    m: int

    def copy(self) -> "HostResult":
        return HostResult(self.keys.clone(), self.values.clone(), self.ranges.clone(), self.m)


class _Slot:
    def __init__(self, device: torch.device):
        self.ctx = tdgs.Context(device.index or 0)
        self.stream = torch.cuda.Stream(device)
        self.done = torch.cuda.Event()
        self.busy = False
        self.d_g = torch.empty((0, 4), dtype=torch.int32, device=device)
        self.h_k = torch.empty(0, dtype=torch.int64).pin_memory()
        self.h_v = torch.empty(0, dtype=torch.int32).pin_memory()
        self.h_r = torch.empty((0, 2), dtype=torch.int32).pin_memory()


class HostPipeline:
    """``submit(records, width, height)`` with records a pinned (n, 4)
    int32 host tensor (16-byte Gaussian records) returns a ticket;
    ``result(ticket)`` waits for that frame and returns its HostResult."""

    def __init__(self, device: int | torch.device = 0, depth: int = 2):
        self.device = torch.device("cuda", device) if isinstance(device, int) else device
        self.slots = [_Slot(self.device) for _ in range(max(1, depth))]
        self.count = 0
        self._pending: dict[int, tuple[_Slot, HostResult]] = {}

    def close(self):
        torch.cuda.synchronize(self.device)
        for s in self.slots:
            s.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _grow(t: torch.Tensor, n: int, shape_tail=()) -> torch.Tensor:
        if t.shape[0] >= n:
            return t
        return torch.empty((max(n, int(t.shape[0] * 1.25)),) + tuple(shape_tail), dtype=t.dtype,
                           device=t.device, pin_memory=t.device.type == "cpu")

    def submit(self, records: torch.Tensor, width: int, height: int) -> int:
        ticket = self.count
        self.count += 1
        slot = self.slots[ticket % len(self.slots)]
        if slot.busy:  # the previous download of this slot must be complete
            slot.done.synchronize()
        n = records.shape[0]
        T = tdgs.num_tiles(width, height)
        if slot.d_g.shape[0] < n:
            slot.d_g = torch.empty((int(n * 1.25) + 1, 4), dtype=torch.int32, device=self.device)
        with torch.cuda.stream(slot.stream):
            d_g = slot.d_g[:n]
            d_g.copy_(records, non_blocking=True)
            k, v, r, m = slot.ctx.sort_frame(d_g, width, height)
            slot.h_k = self._grow(slot.h_k, m)
            slot.h_v = self._grow(slot.h_v, m)
            slot.h_r = self._grow(slot.h_r, T, (2,))
            hk, hv, hr = slot.h_k[:m], slot.h_v[:m], slot.h_r[:T]
            hk.copy_(k, non_blocking=True)
            hv.copy_(v, non_blocking=True)
            hr.copy_(r, non_blocking=True)
            slot.done.record(slot.stream)
        slot.busy = True
        self._pending[ticket] = (slot, HostResult(hk, hv, hr, m))
        return ticket

    def result(self, ticket: int) -> HostResult:
        slot, res = self._pending.pop(ticket)
        slot.done.synchronize()
        slot.ctx.sync()
        return res

    def drain(self):
        """Wait for every submitted frame (their results stay retrievable)."""
        for s in self.slots:
            if s.busy:
                s.done.synchronize()
