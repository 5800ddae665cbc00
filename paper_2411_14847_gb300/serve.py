"""Continuous-batching novel-view render server over resident, streaming scenes.

Each scene's current-timestep Gaussians stay resident on the device; `set_scene` swaps in the
next timestep (requests already launched keep the buffers they started with). Render requests
(scene, camera of any resolution) are queued; a scheduler thread admits them into batches as
launch slots (CUDA streams) and device memory free up: a batch takes queued requests in
arrival order, of any scenes and sizes sharing an SH degree, while its estimated footprint fits
the free HBM (or the configured budget), and renders all of them with one launch of each
kernel (dass_preprocess_scenes -> dass_bin_sort -> dass_render_fwd) on its own stream, so
batches overlap on the GPU. Requests that arrive while batches run are admitted into the next
free slot. Per-request results do not depend on the batch they ran in: every pixel's blend
only involves its own camera's records.

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
GRAD_FLOATS = 12


@dataclass
class Request:
    rid: int
    scene_id: object
    cam: object
    future: Future
    t_submit: float
    t_done: float = 0.0
    batch: int = -1


@dataclass
class _Batch:
    bid: int
    reqs: list
    event: torch.cuda.Event
    bufs: dict
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
        self._streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self._slots = [None] * n_streams
        self._ids = itertools.count()
        self._bids = itertools.count()
        self._inflight_bytes = 0
        self._stop = False
        self.stats = ServeStats()
        self.log = []            # (batch id, [request ids], launch time, estimated bytes)
        D.load()
        self._thread = threading.Thread(target=self._run, name="dass-render-server", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------- public API

    def set_scene(self, scene_id, params: dict):
        """Make `params` (dict of device tensors: means, log_scales, quats, opacity_logit, sh) the
        current timestep of `scene_id`."""
        snap = {k: params[k].contiguous() for k in ("means", "log_scales", "quats", "opacity_logit", "sh")}
        with self._lock:
            self._scenes[scene_id] = snap

    def submit(self, scene_id, cam) -> Future:
        """Queue a novel-view render; the future resolves to a [3, H, W] device tensor."""
        fut = Future()
        with self._cv:
            if scene_id not in self._scenes:
                raise KeyError(scene_id)
            self._queue.append(Request(next(self._ids), scene_id, cam, fut, time.perf_counter()))
            self._cv.notify()
        return fut

    def estimate_bytes(self, scene_id, cam):
        """Estimated device bytes of rendering one request alone (what admission charges)."""
        with self._lock:
            sc = self._scenes[scene_id]
        return self._estimate([Request(-1, scene_id, cam, None, 0.0)], [sc])[0]

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

    def _estimate(self, reqs, scenes):
        n_rec = len(reqs) * max(s["means"].shape[0] for s in scenes)
        pixels = sum(r.cam.width * r.cam.height for r in reqs)
        tiles = sum(math.ceil(r.cam.width / self.tile) * math.ceil(r.cam.height / self.tile) for r in reqs)
        cap = int(n_rec * self.ppr * 1.25) + 4096
        ws = D.dass_bin_sort_workspace(n_rec, cap, tiles)
        return n_rec * SPLAT_BYTES + cap * 4 + ws + pixels * 20 + tiles * 8, cap

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
        est, cap = 0, 0
        while self._queue and len(reqs) < self.max_batch:
            r = self._queue[0]
            sc = self._scenes[r.scene_id]
            d = sc["sh"].shape[1]
            if deg is not None and d != deg:
                break
            need, c = self._estimate(reqs + [r], scenes + [sc])
            if need > free:
                if not reqs:
                    if self.hbm_budget is not None and need > self.hbm_budget or not any(self._slots):
                        self._queue.popleft()
                        self.stats.rejected += 1
                        r.future.set_exception(MemoryError(
                            f"request {r.rid} needs ~{need / 2**20:.0f} MiB, more than the free device memory"))
                        continue
                break
            self._queue.popleft()
            reqs.append(r)
            scenes.append(sc)
            deg = d
            est, cap = need, c
        return (reqs, scenes, est, cap) if reqs else None

    def _launch(self, slot, reqs, scenes, est, cap, bid=None):
        stream = self._streams[slot]
        cams = D.cameras([r.cam for r in reqs])     # marshalled once for every call below
        rec_stride = max(s["means"].shape[0] for s in scenes)
        tiles_total, pixels = D.tile_layout(cams, self.tile)
        n_rec = len(reqs) * rec_stride
        with torch.cuda.stream(stream):
            bufs = dict(
                scenes=scenes,
                splats=torch.empty((max(1, n_rec), D.SPLAT_FLOATS), dtype=torch.float32, device=self.device),
                pair_rec=torch.empty(max(1, cap), dtype=torch.int32, device=self.device),
                ranges=torch.empty((max(1, tiles_total), 2), dtype=torch.int32, device=self.device),
                counters=torch.empty(4, dtype=torch.int64, device=self.device),   # written by the sort
                image=torch.empty(3 * pixels, dtype=torch.float32, device=self.device),
                T=torch.empty(pixels, dtype=torch.float32, device=self.device),
                last=torch.empty(pixels, dtype=torch.int32, device=self.device),
                ws=torch.empty(max(1, D.dass_bin_sort_workspace(n_rec, cap, tiles_total)), dtype=torch.uint8,
                               device=self.device),
            )
            D.dass_preprocess_scenes(scenes, cams, self.tile, rec_stride, bufs["splats"], stream=stream)
            D.dass_bin_sort(bufs["splats"], rec_stride, cams, self.tile, bufs["pair_rec"], bufs["ranges"],
                            bufs["counters"], bufs["ws"], stream=stream)
            D.dass_render_fwd(bufs["splats"], bufs["pair_rec"], bufs["ranges"], cams, self.tile, self.batch_g,
                              bufs["image"], bufs["T"], bufs["last"], stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        bid = next(self._bids) if bid is None else bid
        for r in reqs:
            r.batch = bid
        self._slots[slot] = _Batch(bid, reqs, ev, bufs, time.perf_counter(), cap, slot, est)
        self._inflight_bytes += est
        self.log.append((bid, [r.rid for r in reqs], time.perf_counter(), est))
        self.stats.batch_sizes.append(len(reqs))

    def _retire(self, slot):
        b = self._slots[slot]
        if b is None or not b.event.query():
            return False
        self._slots[slot] = None
        self._inflight_bytes -= b.est
        m, over = (int(v) for v in b.bufs["counters"][:2].tolist())
        n_rec = len(b.reqs) * max(s["means"].shape[0] for s in b.bufs["scenes"])
        self.ppr = max(self.ppr, m / max(1, n_rec))
        if over:   # pair buffer too small: render the same batch again with the exact size
            self.stats.relaunched += 1
            est2, _ = self._estimate(b.reqs, b.bufs["scenes"])
            self._launch(slot, b.reqs, b.bufs["scenes"], est2, int(m * 1.1) + 4096, bid=b.bid)
            return True
        off = 0
        now = time.perf_counter()
        for r in b.reqs:
            sz = 3 * r.cam.width * r.cam.height
            img = b.bufs["image"][off:off + sz].view(3, r.cam.height, r.cam.width)
            off += sz
            r.t_done = now
            self.stats.latencies_ms.append(1e3 * (now - r.t_submit))
            r.future.set_result(img)
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


def percentile(values, q):
    if not values:
        return None
    v = sorted(values)
    return v[min(len(v) - 1, int(q * (len(v) - 1) + 0.5))]
