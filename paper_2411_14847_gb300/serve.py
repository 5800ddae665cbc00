"""Continuous-batching novel-view render server over resident, streaming scenes.

Each scene's current-timestep Gaussians stay resident on the device; `set_scene` swaps in the
next timestep (requests already launched keep the buffers they started with). Render requests
(scene, camera of any resolution) are queued; a scheduler thread admits them into batches as
launch slots (CUDA streams) and device memory free up: a batch takes queued requests in
arrival order, of any scenes and sizes sharing an SH degree, while its estimated footprint fits
the free HBM (or the configured budget), and renders all of them with one launch of each
kernel (dass_preprocess_scenes_packed -> dass_bin_sort_packed -> dass_render_fwd) on its own
stream, so batches overlap on the GPU. A request's records are packed after the previous
request's (a small scene batched with a large one costs its own records only). Requests that
arrive while batches run are admitted into the next free slot. Per-request results do not
depend on the batch they ran in: every pixel's blend only involves its own camera's records.

Device memory: each launch slot keeps grow-only buffers (records, pairs, sort scratch, image,
transmittance, last index) sized to the largest batch it has run, so steady-state serving
allocates only the per-request result images; the slot streams are shared by every server of the
process, so what a closed server leaves in the allocator's per-stream cache serves the next one.
Stream order: `set_scene` records an event on the
caller's current stream and every batch using that version waits for it; each result is
recorded on the submitting thread's current stream before it is handed out, so the allocator
does not reuse its memory while the caller's work on it is pending.

Only buffer allocation and scheduling happen here; all rendering is libdass.
"""
from __future__ import annotations

import collections
import itertools
import math
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import torch

from . import dass as D

SPLAT_BYTES = 48
PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logit", "sh")


# Launch-slot streams are shared by every server of the process (per device): the caching allocator
# keeps freed blocks per stream, so the slot buffers and result images a closed server leaves behind
# serve the next server instead of staying reserved for streams nobody uses again.
_SLOT_STREAMS = {}
_SLOT_LOCK = threading.Lock()


def _slot_streams(device, n):
    with _SLOT_LOCK:
        pool = _SLOT_STREAMS.setdefault(device, [])
        while len(pool) < n:
            pool.append(torch.cuda.Stream(device))
        return pool[:n]


@dataclass
class Request:
    rid: int
    scene_id: object
    cam: object
    future: Future
    t_submit: float
    stream: object = None      # the submitting thread's current stream (the result is recorded on it)
    t_done: float = 0.0
    batch: int = -1


@dataclass
class _Batch:
    bid: int
    reqs: list
    event: torch.cuda.Event
    scenes: list
    outs: list
    t_launch: float
    capacity: int
    slot: int
    est: int


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    batch_sizes: list = field(default_factory=list)
    rejected: int = 0
    relaunched: int = 0


class _Arena:
    """Grow-only device buffers of one launch slot (reused by every batch the slot runs)."""

    def __init__(self, device):
        self.device = device
        self.bufs = {}

    def get(self, name, numel, dtype):
        t = self.bufs.get(name)
        if t is None or t.numel() < numel or t.dtype != dtype:
            t = torch.empty(max(1, int(numel * 1.25) + 1024), dtype=dtype, device=self.device)
            self.bufs[name] = t
        return t[:max(1, numel)]


class RenderServer:
    def __init__(self, tile=16, batch=128, max_batch=16, n_streams=2, hbm_budget=None, pairs_per_record=8.0,
                 device="cuda"):
        self.tile, self.batch_g, self.max_batch = tile, batch, max_batch
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.hbm_budget = hbm_budget
        self.ppr = float(pairs_per_record)       # running estimate of pairs per projected record
        self._scenes = {}
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._queue = collections.deque()
        self._streams = _slot_streams(self.device, n_streams)
        self._arenas = [_Arena(self.device) for _ in range(n_streams)]
        self._slots = [None] * n_streams
        self._ids = itertools.count()
        self._bids = itertools.count()
        self._inflight_bytes = 0
        self._stop = False
        self.stats = ServeStats()
        self.log = []            # (batch id, [request ids], launch time, estimated bytes)
        self._launched = threading.Event()
        D.load()
        self._thread = threading.Thread(target=self._run, name="dass-render-server", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------- public API

    def set_scene(self, scene_id, params: dict, copy=True):
        """Make `params` (dict of device tensors: means, log_scales, quats, opacity_logit, sh) the
        current timestep of `scene_id`. With copy=True (default) the server renders from its own
        snapshot, taken on the caller's current stream, so the caller may keep updating its
        tensors in place; with copy=False the caller hands the tensors over and must not modify
        them while the scene version is current or in flight. Either way every batch that uses
        this version first waits for the caller's stream to reach this call."""
        cur = torch.cuda.current_stream(self.device)
        if copy:
            snap = {k: params[k].detach().clone(memory_format=torch.contiguous_format) for k in PARAM_KEYS}
        else:
            snap = {k: params[k].contiguous() for k in PARAM_KEYS}
        ready = torch.cuda.Event()
        ready.record(cur)
        snap["_ready"] = ready
        with self._lock:
            self._scenes[scene_id] = snap

    def submit(self, scene_id, cam) -> Future:
        """Queue a novel-view render; the future resolves to a [3, H, W] device tensor, recorded on
        the submitting thread's current stream."""
        fut = Future()
        stream = torch.cuda.current_stream(self.device)
        with self._cv:
            if scene_id not in self._scenes:
                raise KeyError(scene_id)
            self._queue.append(Request(next(self._ids), scene_id, cam, fut, time.perf_counter(), stream))
            self._cv.notify()
        return fut

    def submit_many(self, items):
        """Queue several (scene_id, camera) renders at once: the scheduler sees all of them in the
        same pass, so they can share one batch. Returns their futures in order."""
        stream = torch.cuda.current_stream(self.device)
        futs = []
        with self._cv:
            for scene_id, _ in items:
                if scene_id not in self._scenes:
                    raise KeyError(scene_id)
            for scene_id, cam in items:
                fut = Future()
                self._queue.append(Request(next(self._ids), scene_id, cam, fut, time.perf_counter(), stream))
                futs.append(fut)
            self._cv.notify()
        return futs

    def estimate_bytes(self, scene_id, cam):
        """Estimated device bytes of rendering one request alone (what admission charges)."""
        with self._lock:
            sc = self._scenes[scene_id]
        est = _Estimate(self)
        est.add(cam, sc)
        return est.bytes()[0]

    def wait_launched(self, timeout):
        """Block until the first batch has been launched (True) or the timeout expires (False)."""
        return self._launched.wait(timeout)

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- scheduling

    def _free_bytes(self):
        if self.hbm_budget is not None:
            return self.hbm_budget - self._inflight_bytes
        free, _ = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return free + cached - (256 << 20)

    def _form_batch(self):
        """Take queued requests in order while they fit; returns (reqs, scenes, bytes, cap) or None."""
        if not self._queue:
            return None
        reqs, scenes = [], []
        free = self._free_bytes()
        deg = None
        est = _Estimate(self)
        need, cap = 0, 0
        while self._queue and len(reqs) < self.max_batch:
            r = self._queue[0]
            sc = self._scenes[r.scene_id]
            d = sc["sh"].shape[1]
            if deg is not None and d != deg:
                break
            trial = est.copy()
            trial.add(r.cam, sc)
            n_need, c = trial.bytes()
            if n_need > free:
                if not reqs:
                    if self.hbm_budget is not None and n_need > self.hbm_budget or not any(self._slots):
                        self._queue.popleft()
                        self.stats.rejected += 1
                        r.future.set_exception(MemoryError(
                            f"request {r.rid} needs ~{n_need / 2**20:.0f} MiB, more than the free device memory"))
                        continue
                break
            self._queue.popleft()
            reqs.append(r)
            scenes.append(sc)
            deg = d
            est = trial
            need, cap = n_need, c
        return (reqs, scenes, need, cap) if reqs else None

    def _launch(self, slot, reqs, scenes, est, cap, bid=None):
        stream = self._streams[slot]
        arena = self._arenas[slot]
        cams = D.cameras([r.cam for r in reqs])     # marshalled once for every call below
        offsets = D.record_offsets(scenes)
        n_rec = int(offsets[len(reqs)])
        tiles_total, pixels = D.tile_layout(cams, self.tile)
        with torch.cuda.stream(stream):
            for ev in {id(sc["_ready"]): sc["_ready"] for sc in scenes}.values():
                stream.wait_event(ev)
            splats = arena.get("splats", n_rec * D.SPLAT_FLOATS, torch.float32)
            pair_rec = arena.get("pair_rec", cap, torch.int32)
            ranges = arena.get("ranges", 2 * tiles_total, torch.int32)
            counters = arena.get("counters", 4, torch.int64)       # written by the sort
            image = arena.get("image", 3 * pixels, torch.float32)
            T = arena.get("T", pixels, torch.float32)
            last = arena.get("last", pixels, torch.int32)
            ws = arena.get("ws", D.dass_bin_sort_workspace(n_rec, cap, tiles_total), torch.uint8)
            D.dass_preprocess_scenes_packed(scenes, cams, self.tile, offsets, splats, stream=stream)
            D.dass_bin_sort_packed(splats, offsets, cams, self.tile, pair_rec, ranges, counters, ws, stream=stream)
            D.dass_render_fwd(splats, pair_rec, ranges, cams, self.tile, self.batch_g, image, T, last,
                              stream=stream)
            # each request's result in a tensor of its own (the arena is reused by the next batch)
            outs, off = [], 0
            for r in reqs:
                sz = 3 * r.cam.width * r.cam.height
                out = torch.empty((3, r.cam.height, r.cam.width), dtype=torch.float32, device=self.device)
                out.view(-1).copy_(image[off:off + sz])
                outs.append(out)
                off += sz
            ev = torch.cuda.Event()
            ev.record(stream)
        bid = next(self._bids) if bid is None else bid
        for r in reqs:
            r.batch = bid
        self._slots[slot] = _Batch(bid, reqs, ev, scenes, outs, time.perf_counter(), cap, slot, est)
        self._inflight_bytes += est
        self.log.append((bid, [r.rid for r in reqs], time.perf_counter(), est))
        self.stats.batch_sizes.append(len(reqs))
        self._launched.set()

    def _retire(self, slot):
        b = self._slots[slot]
        if b is None or not b.event.query():
            return False
        self._slots[slot] = None
        self._inflight_bytes -= b.est
        m, over = (int(v) for v in self._arenas[slot].bufs["counters"][:2].tolist())
        n_rec = sum(int(sc["means"].shape[0]) for sc in b.scenes)
        self.ppr = max(self.ppr, m / max(1, n_rec))
        if over:   # pair buffer too small: render the same batch again with the exact size
            self.stats.relaunched += 1
            self._launch(slot, b.reqs, b.scenes, b.est, int(m * 1.1) + 4096, bid=b.bid)
            return True
        now = time.perf_counter()
        for r, out in zip(b.reqs, b.outs):
            if r.stream is not None and r.stream != self._streams[slot]:
                out.record_stream(r.stream)
            r.t_done = now
            self.stats.latencies_ms.append(1e3 * (now - r.t_submit))
            r.future.set_result(out)
        return True

    def _run(self):
        try:
            self._loop()
        except BaseException as exc:        # fail every waiting request instead of hanging it
            with self._lock:
                pending = list(self._queue)
                self._queue.clear()
            for b in self._slots:
                if b is not None:
                    pending += b.reqs
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(exc)
            raise

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                if self._stop and not self._queue and not any(self._slots):
                    return
                if not self._queue and not any(self._slots):
                    self._cv.wait(timeout=0.05)
                    continue
            progressed = False
            for s in range(len(self._slots)):
                progressed |= self._retire(s)
            for s in range(len(self._slots)):
                if self._slots[s] is None:
                    with self._lock:
                        formed = self._form_batch()
                    if formed is None:
                        break
                    self._launch(s, *formed)
                    progressed = True
            if not progressed:
                time.sleep(0.0001)


class _Estimate:
    """Running device-byte estimate of a batch (records, pair buffer from the pairs-per-record
    estimate, sort scratch, image/transmittance/last-index buffers, result images)."""

    def __init__(self, srv):
        self.srv = srv
        self.n_rec = 0
        self.pixels = 0
        self.tiles = 0

    def copy(self):
        e = _Estimate(self.srv)
        e.n_rec, e.pixels, e.tiles = self.n_rec, self.pixels, self.tiles
        return e

    def add(self, cam, scene):
        t = self.srv.tile
        self.n_rec += int(scene["means"].shape[0])
        self.pixels += cam.width * cam.height
        self.tiles += math.ceil(cam.width / t) * math.ceil(cam.height / t)

    def bytes(self):
        cap = int(self.n_rec * self.srv.ppr * 1.25) + 4096
        ws = D.dass_bin_sort_workspace(self.n_rec, cap, self.tiles)
        return self.n_rec * SPLAT_BYTES + cap * 4 + ws + self.pixels * 32 + self.tiles * 8, cap


def percentile(values, q):
    if not values:
        return None
    v = sorted(values)
    return v[min(len(v) - 1, int(q * (len(v) - 1) + 0.5))]
