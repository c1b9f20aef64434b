"""Serving loop: continuous batching of camera requests over resident octrees.

Requests (a tree, a camera pose, a resolution) arrive over time.  The batched server admits
waiting requests into free slots whenever a slot table is free and the output pool has room,
packs them into a slot table (16x8 tiles of every request numbered consecutively), and replays a
CUDA graph captured once per table: host-to-device copy of the table, then dot_render_slots (one
persistent launch that drains the tiles of all admitted requests).  Resident trees that differ in
storage type, SH degree or compression cannot share one slot launch (each is a different build
of the march), so the trees are split into groups that can, a table holds one sub-table per
group, and the graph runs one slot launch per group on forked streams that join again: one
replay renders a mixed batch, and the groups' launches overlap on the device.  Two tables are in
flight at a time on two streams, so requests that arrive while a batch is on the GPU start in the
next one at once and their work overlaps on the device.  The plain server launches dot_render_forward once
per request, in arrival order, on one stream.

Host bookkeeping (pool, packing, trace) is plain Python and runs without a GPU; only
``BatchedServer`` / ``PlainServer`` touch the device.
"""
from __future__ import annotations

import contextlib
import ctypes
import dataclasses
import gc
import time
from collections import deque
from typing import List, Sequence

import numpy as np

SLOT_BYTES = 96
HEADER_BYTES = 16
TILE_W, TILE_H = 16, 8       # the work tile of a slot launch


@dataclasses.dataclass
class Request:
    rid: int
    tree: int
    width: int
    height: int
    camera: np.ndarray          # float32[18] dot_camera record
    arrival: float              # seconds from the start of the trace
    offset: int = -1            # float offset of the output in the pool
    done: float = -1.0          # completion time (seconds from the start)

    @property
    def floats(self) -> int:
        return self.width * self.height * 3

    @property
    def tiles(self) -> int:
        return ((self.width + TILE_W - 1) // TILE_W) * ((self.height + TILE_H - 1) // TILE_H)


class OutputPool:
    """First-fit allocator of output images inside one device buffer (offsets in floats)."""

    def __init__(self, capacity_floats: int, align: int = 64):
        self.capacity = int(capacity_floats)
        self.align = align
        self.free = [(0, self.capacity)]          # sorted (start, length)

    def alloc(self, n: int) -> int:
        n = (n + self.align - 1) // self.align * self.align
        for i, (s, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, l - n)
                return s
        return -1

    def release(self, start: int, n: int):
        n = (n + self.align - 1) // self.align * self.align
        self.free.append((start, n))
        self.free.sort()
        merged = []
        for s, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((s, l))
        self.free = merged

    @property
    def free_floats(self) -> int:
        return sum(l for _, l in self.free)


def slot_groups(trees) -> List[List[int]]:
    """Indices of the trees grouped by what one slot launch can serve together (storage type, SH
    degree, compressed or not), groups in order of first appearance.  Each tree is any object
    with storage, sh_degree and palette_bits attributes."""
    keys: List[tuple] = []
    groups: List[List[int]] = []
    for i, t in enumerate(trees):
        k = (int(t.storage), int(t.sh_degree), int(t.palette_bits) > 0)
        if k not in keys:
            keys.append(k)
            groups.append([])
        groups[keys.index(k)].append(i)
    return groups


def write_slots(buf: np.ndarray, reqs: Sequence[Request], pool_base_ptr: int, max_slots: int,
                tree_index=None) -> None:
    """Writes a slot table in place into the byte buffer `buf` (HEADER_BYTES + SLOT_BYTES *
    max_slots): the header, then one 96-byte dot_slot per request.  Slots past the last request
    keep whatever they held: the kernel reads n_slots of them.  tree_index maps a request's tree
    to its index in the launch's tree list (identity if None)."""
    assert len(reqs) <= max_slots
    begin = 0
    for i, r in enumerate(reqs):
        rec = buf[HEADER_BYTES + SLOT_BYTES * i: HEADER_BYTES + SLOT_BYTES * (i + 1)]
        rec[0:72] = np.ascontiguousarray(r.camera, dtype=np.float32).view(np.uint8)
        t = r.tree if tree_index is None else tree_index[r.tree]
        rec[72:80] = np.array([t, 0], np.int32).view(np.uint8)
        rec[80:96] = np.array([begin, pool_base_ptr + 4 * r.offset], np.uint64).view(np.uint8)
        begin += r.tiles
    buf[0:16] = np.array([len(reqs), 0, begin & 0xFFFFFFFF, begin >> 32], np.uint32).view(np.uint8)


def pack_table(reqs: Sequence[Request], pool_base_ptr: int, max_slots: int,
               tree_index=None) -> np.ndarray:
    """Byte image of a slot table: header then one 96-byte dot_slot per request (zero-filled
    after the last request)."""
    buf = np.zeros(HEADER_BYTES + SLOT_BYTES * max_slots, dtype=np.uint8)
    write_slots(buf, reqs, pool_base_ptr, max_slots, tree_index)
    return buf


def poisson_trace(n: int, rate: float, n_trees: int, resolutions, poses, seed: int) -> List[Request]:
    """n requests with exponential inter-arrival gaps (rate per second), a uniformly drawn tree and
    resolution, and a camera record from poses(rng, tree, w, h) -> float32[18]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        tree = int(rng.integers(0, n_trees))
        w, h = resolutions[int(rng.integers(0, len(resolutions)))]
        out.append(Request(i, tree, w, h, poses(rng, tree, w, h), t))
    return out


def percentiles(reqs: Sequence[Request]):
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}


# ----------------------------------------------------------------------------------------------
# device side
# ----------------------------------------------------------------------------------------------
@contextlib.contextmanager
def _no_gc_pauses():
    """The serving loops run with Python's cyclic garbage collector paused (a full collection of
    a large process can stall the host loop for tens of milliseconds); restored afterwards."""
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


class _Table:
    """One slot table per tree group, back to back in one pinned host buffer and one device
    buffer, a work counter per group, the streams the group launches fork onto, and one CUDA graph
    per set of groups a batch can hold (a batch replays the graph of the groups it uses: no launch
    for an empty group, and only the used sub-tables are copied)."""

    def __init__(self, torch, max_slots, n_groups):
        self.table_bytes = HEADER_BYTES + SLOT_BYTES * max_slots
        nbytes = self.table_bytes * n_groups
        self.host = torch.zeros(nbytes, dtype=torch.uint8, pin_memory=True)
        self.host_np = self.host.numpy()
        self.dev = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
        self.counter = torch.zeros(n_groups, dtype=torch.int64, device="cuda")
        self.stream = torch.cuda.Stream()
        self.forks = [torch.cuda.Stream() for _ in range(n_groups - 1)]
        self.graphs = {}                        # bit mask of the groups used -> CUDA graph
        self.event = torch.cuda.Event()
        self.reqs: List[Request] = []


class BatchedServer:
    # up to this many tree groups, a graph per non-empty set of groups; beyond, one graph of all
    MAX_SUBSET_GROUPS = 4

    def __init__(self, trees, opts, pool_floats: int, max_slots: int = 64, n_tables: int = 2):
        import torch

        from . import dot
        self.torch, self.dot = torch, dot
        self.trees = list(trees)
        self.groups = slot_groups(self.trees)
        self.local = {}                                # tree -> (group, index in the group)
        for g, members in enumerate(self.groups):
            for j, t in enumerate(members):
                self.local[t] = (g, j)
        self.index = [{t: self.local[t][1] for t in m} for m in self.groups]
        self.handles = [(ctypes.c_void_p * len(m))(*[self.trees[t].handle.value for t in m])
                        for m in self.groups]
        self.opts = opts
        self.max_slots = max_slots
        self.pool_t = torch.empty(int(pool_floats), dtype=torch.float32, device="cuda")
        self.pool = OutputPool(pool_floats)
        G = len(self.groups)
        full = (1 << G) - 1
        self.masks = list(range(1, full + 1)) if G <= self.MAX_SUBSET_GROUPS else [full]
        self.tables = [_Table(torch, max_slots, G) for _ in range(n_tables)]
        for tb in self.tables:
            for m in self.masks:
                self._capture(tb, m)

    def _launch(self, tb, g):
        torch = self.torch
        rc = self.dot.lib().dot_render_slots(
            self.handles[g], len(self.groups[g]),
            ctypes.c_void_p(tb.dev.data_ptr() + g * tb.table_bytes), self.max_slots,
            ctypes.byref(self.opts), ctypes.c_void_p(tb.counter.data_ptr() + 8 * g),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise self.dot.DotError(rc, self.dot.dot_last_error())

    def _record(self, tb, mask):
        """The work of one replay for the groups in `mask`: their sub-tables copied, then one slot
        launch per group -- the first on the table's stream, the others on forked streams that
        join it again."""
        torch = self.torch
        used = [g for g in range(len(self.groups)) if mask >> g & 1]
        for g in used:
            a, b = g * tb.table_bytes, (g + 1) * tb.table_bytes
            tb.dev[a:b].copy_(tb.host[a:b], non_blocking=True)
        for g, fork in zip(used[1:], tb.forks):
            fork.wait_stream(tb.stream)
            with torch.cuda.stream(fork):
                self._launch(tb, g)
        self._launch(tb, used[0])
        for _, fork in zip(used[1:], tb.forks):
            tb.stream.wait_stream(fork)

    def _capture(self, tb, mask):
        torch = self.torch
        with torch.cuda.stream(tb.stream):          # one eager run before capture
            self._record(tb, mask)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=tb.stream):
            self._record(tb, mask)
        torch.cuda.synchronize()
        tb.graphs[mask] = graph

    def submit(self, reqs: List[Request], tb: _Table):
        base = self.pool_t.data_ptr()
        by_group = [[] for _ in self.groups]
        for r in reqs:
            by_group[self.local[r.tree][0]].append(r)
        mask = 0
        for g, mine in enumerate(by_group):
            if mine or len(self.masks) == 1:
                mask |= 1 << g
                write_slots(tb.host_np[g * tb.table_bytes:(g + 1) * tb.table_bytes], mine, base,
                            self.max_slots, self.index[g])
        tb.reqs = reqs
        with self.torch.cuda.stream(tb.stream):
            tb.graphs[mask].replay()
            tb.event.record(tb.stream)

    def run(self, trace: Sequence[Request], clock=time.perf_counter):
        """Replays the trace in real time; fills r.done for every request."""
        with _no_gc_pauses():
            return self._run(trace, clock)

    def _run(self, trace: Sequence[Request], clock):
        pending: deque = deque()
        free_tables = list(self.tables)
        busy: List[_Table] = []
        i, n, finished = 0, len(trace), 0
        t0 = clock()
        while finished < n:
            now = clock() - t0
            while i < n and trace[i].arrival <= now:
                pending.append(trace[i])
                i += 1
            for tb in list(busy):
                if tb.event.query():
                    t = clock() - t0
                    for r in tb.reqs:
                        r.done = t
                        self.pool.release(r.offset, r.floats)
                    finished += len(tb.reqs)
                    busy.remove(tb)
                    free_tables.append(tb)
            if pending and free_tables:
                batch = []
                while pending and len(batch) < self.max_slots:
                    r = pending[0]
                    off = self.pool.alloc(r.floats)
                    if off < 0:
                        break                          # admitted later, as memory frees up
                    r.offset = off
                    batch.append(pending.popleft())
                if batch:
                    tb = free_tables.pop()
                    self.submit(batch, tb)
                    busy.append(tb)
        return trace

    def render_alone_and_mixed(self, reqs: List[Request]):
        """Device images of `reqs` rendered all in one table, and each in a table of its own."""
        torch = self.torch
        tb = self.tables[0]
        for r in reqs:
            r.offset = self.pool.alloc(r.floats)
            assert r.offset >= 0
        self.submit(list(reqs), tb)
        torch.cuda.synchronize()
        mixed = [self.pool_t[r.offset: r.offset + r.floats].clone() for r in reqs]
        alone = []
        for r in reqs:
            self.pool_t[r.offset: r.offset + r.floats].fill_(-1.0)
            self.submit([r], tb)
            torch.cuda.synchronize()
            alone.append(self.pool_t[r.offset: r.offset + r.floats].clone())
        for r in reqs:
            self.pool.release(r.offset, r.floats)
        return mixed, alone


class PlainServer:
    """One dot_render_forward launch per request, in arrival order, on one stream."""

    def __init__(self, trees, opts, pool_floats: int):
        import torch

        from . import dot
        self.torch, self.dot = torch, dot
        self.trees = list(trees)
        self.opts = opts
        self.pool_t = torch.empty(int(pool_floats), dtype=torch.float32, device="cuda")
        self.pool = OutputPool(pool_floats)
        self.stream = torch.cuda.Stream()
        self.cams = torch.zeros(18, dtype=torch.float32, pin_memory=True)

    def run(self, trace: Sequence[Request], clock=time.perf_counter):
        """Replays the trace in real time; fills r.done for every request."""
        with _no_gc_pauses():
            return self._run(trace, clock)

    def _run(self, trace: Sequence[Request], clock):
        torch, dot = self.torch, self.dot
        pending: deque = deque()
        inflight: deque = deque()
        i, n, finished = 0, len(trace), 0
        t0 = clock()
        while finished < n:
            now = clock() - t0
            while i < n and trace[i].arrival <= now:
                pending.append(trace[i])
                i += 1
            while inflight and inflight[0][1].query():
                r, ev, cam = inflight.popleft()
                r.done = clock() - t0
                self.pool.release(r.offset, r.floats)
                finished += 1
            while pending:
                r = pending[0]
                off = self.pool.alloc(r.floats)
                if off < 0:
                    break
                pending.popleft()
                r.offset = off
                with torch.cuda.stream(self.stream):
                    cam = torch.from_numpy(np.ascontiguousarray(r.camera)).to("cuda", non_blocking=False).view(1, 18)
                    out = self.pool_t[off: off + r.floats]
                    dot.dot_render_forward(self.trees[r.tree], dot.rays_cameras(cam, r.width, r.height),
                                           self.opts, out, stream=self.stream)
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                inflight.append((r, ev, cam))
        return trace
