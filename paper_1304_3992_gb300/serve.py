"""Continuous-batching server for the extraction path.

Requests (single-band uint8/uint16 images in host memory) arrive at any time.
The scheduler admits them in arrival order while their device bytes (image +
mask) fit the HBM budget, copies each image to the device on a copy stream,
and launches every request whose copy has finished as one batched
``fx_extract_batch`` call -- the persistent tile-queue kernels -- on one of
several compute streams, each with its own plan.  Requests that arrive while
earlier batches are on the GPU are admitted, copied and launched as soon as
memory and a compute stream free up, so their work overlaps on the device.
A mask stays device-resident until its request is released; completion
(device-side) time minus arrival time is the request's latency.

The device work is behind a small backend interface so that the scheduling
logic (budget, ordering, batching, cancellation, failures) is testable on the
host with a fake backend; ``TorchBackend`` is the GPU one.
"""
from __future__ import annotations

import collections
import dataclasses
import statistics
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    image: np.ndarray            # host image (contiguous rows), uint8 or uint16
    arrival: float               # seconds, on the server's clock
    state: str = "pending"       # pending -> copying -> ready -> running -> done | rejected | cancelled | failed
    dev: object = None           # backend handle (device image and mask)
    copy_event: object = None
    done_at: float | None = None
    error: str | None = None
    held: int = 0                # device bytes this request holds against the budget

    @property
    def pixels(self) -> int:
        return int(self.image.shape[0] * self.image.shape[1])

    @property
    def device_bytes(self) -> int:
        return int(self.image.nbytes + self.pixels)


class BudgetError(RuntimeError):
    pass


class Server:
    """Admission by HBM budget + continuous batching over ``backend``."""

    def __init__(self, backend, budget_bytes: int, max_batch: int = 64, max_running: int = 2,
                 clock=time.perf_counter):
        if max_running < 1 or max_batch < 1:
            raise ValueError("max_running and max_batch must be >= 1")
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.max_running = max_running
        self.clock = clock
        self.t0 = clock()
        self.used = 0
        self.pending = collections.deque()
        self.copying = []
        self.ready = []
        self.running = []            # (slot, event, [requests])
        self.free_slots = list(range(max_running))
        self.finished = []
        self.batches = []            # sizes of launched batches
        self.overlapped_launches = 0  # launches made while another batch's event was still pending

    # -------------------------------------------------------------- client
    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, rid: int, image: np.ndarray, arrival: float | None = None) -> Request:
        if image.ndim != 2 or image.dtype not in (np.uint8, np.uint16) or not image.flags.c_contiguous:
            raise ValueError("image must be a contiguous 2-D uint8/uint16 array")
        r = Request(rid, image, self.now() if arrival is None else arrival)
        if r.device_bytes > self.budget:
            r.state, r.error = "rejected", "FX_ERR_BUDGET: request larger than the HBM budget"
            self.finished.append(r)
            return r
        self.pending.append(r)
        return r

    def cancel(self, r: Request) -> bool:
        """Cancel a request that has not been launched yet."""
        if r.state == "pending":
            self.pending.remove(r)
        elif r.state in ("copying", "ready"):
            (self.copying if r.state == "copying" else self.ready).remove(r)
            self._release(r)
        else:
            return False
        r.state = "cancelled"
        self.finished.append(r)
        return True

    def release(self, r: Request):
        """Drop a finished request's device mask (its bytes return to the budget)."""
        if r.state == "done" and (r.dev is not None or r.held):
            self._release(r)

    # ----------------------------------------------------------- scheduling
    def _release(self, r: Request):
        if r.dev is not None:
            self.backend.free(r.dev)
            r.dev = None
        self.used -= r.held
        r.held = 0

    def step(self) -> bool:
        """One scheduling pass; returns True if anything progressed."""
        progressed = False
        # completions
        for item in list(self.running):
            slot, ev, reqs = item
            if self.backend.done(ev):
                t = self.now()
                for r in reqs:
                    r.state, r.done_at = "done", t
                    self.backend.free_input(r.dev)  # the image is no longer needed
                    self.used -= r.image.nbytes
                    r.held -= r.image.nbytes
                    self.finished.append(r)
                self.running.remove(item)
                self.free_slots.append(slot)
                progressed = True
        # finished copies
        for r in list(self.copying):
            if self.backend.done(r.copy_event):
                self.copying.remove(r)
                r.state = "ready"
                self.ready.append(r)
                progressed = True
        # admission in arrival order, while the budget allows
        while self.pending and self.used + self.pending[0].device_bytes <= self.budget:
            r = self.pending.popleft()
            try:
                r.dev = self.backend.alloc(r.image)
            except Exception as e:  # allocation failure: the request fails, the server goes on
                r.state, r.error = "failed", f"alloc: {e}"
                self.finished.append(r)
                continue
            self.used += r.device_bytes
            r.held = r.device_bytes
            r.copy_event = self.backend.copy_in(r.dev, r.image)
            r.state = "copying"
            self.copying.append(r)
            progressed = True
        # launch every ready request on a free compute stream
        while self.ready and self.free_slots:
            batch, self.ready = self.ready[:self.max_batch], self.ready[self.max_batch:]
            slot = self.free_slots.pop(0)
            if any(not self.backend.done(ev) for _, ev, _ in self.running):
                self.overlapped_launches += 1  # another batch is still executing
            try:
                ev = self.backend.launch(slot, [r.dev for r in batch])
            except Exception as e:
                for r in batch:
                    r.state, r.error = "failed", f"launch: {e}"
                    self._release(r)
                    self.finished.append(r)
                self.free_slots.append(slot)
                continue
            for r in batch:
                r.state = "running"
            self.running.append((slot, ev, batch))
            self.batches.append(len(batch))
            progressed = True
        return progressed

    def idle(self) -> bool:
        return not (self.pending or self.copying or self.ready or self.running)

    def drain(self, timeout: float = 60.0, release: bool = True):
        end = self.clock() + timeout
        while not self.idle():
            if not self.step():
                if self.clock() > end:
                    raise TimeoutError("server did not drain")
                time.sleep(2e-5)
            if release:
                for r in self.finished:
                    if r.state == "done" and r.held:
                        self.release(r)

    # ------------------------------------------------------------- reports
    def stats(self) -> dict:
        done = [r for r in self.finished if r.state == "done"]
        lat = sorted((r.done_at - r.arrival) * 1e3 for r in done)
        if not lat:
            return {"completed": 0}
        span = max(r.done_at for r in done) - min(r.arrival for r in done)
        q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
        return {
            "completed": len(done),
            "rejected": sum(r.state == "rejected" for r in self.finished),
            "failed": sum(r.state == "failed" for r in self.finished),
            "p50_ms": q(0.50), "p99_ms": q(0.99), "mean_ms": statistics.fmean(lat),
            "gpx_s": sum(r.pixels for r in done) / span / 1e9 if span > 0 else None,
            "batches": len(self.batches), "mean_batch": statistics.fmean(self.batches) if self.batches else 0,
            "overlapped_launches": self.overlapped_launches,
        }


def run_stream(server: Server, images, rate_hz: float, duration_s: float, seed: int = 7,
               release: bool = True, on_done=None) -> list:
    """Drive ``server`` with a Poisson stream: request i uses images[i % len(images)].
    ``on_done(request)`` sees each finished request before its mask is released."""
    rng = np.random.default_rng(seed)
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        arrivals.append(t)
    reqs = []
    start = server.now()
    i = 0
    while i < len(arrivals) or not server.idle():
        now = server.now() - start
        while i < len(arrivals) and arrivals[i] <= now:
            reqs.append(server.submit(i, images[i % len(images)], arrival=start + arrivals[i]))
            i += 1
        if not server.step():
            time.sleep(2e-5)
        for r in reqs:
            if r.state == "done" and r.held:
                if on_done is not None and not getattr(r, "seen", False):
                    r.seen = True
                    on_done(r)
                if release:
                    server.release(r)
    return reqs


class TorchBackend:
    """GPU backend: torch device buffers, a copy stream, one plan + stream per slot."""

    def __init__(self, params, slots: int = 2, max_images: int = 64, device: int = 0, specialize: bool = True):
        import torch
        from . import fx
        self.torch, self.fx = torch, fx
        self.device = torch.device("cuda", device)
        self.copy_stream = torch.cuda.Stream(self.device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        # kernels compiled for the served parameters before the plans are made
        # (fx_specialize; a no-op where run-time compilation is unavailable)
        self.specialized = False
        if specialize:
            with torch.cuda.device(self.device):
                for dt in (fx.FX_U16, fx.FX_U8):
                    try:  # parameters that a dtype cannot evaluate exactly stay on the precompiled kernels
                        self.specialized = fx.specialize(params, dt) or self.specialized
                    except fx.FxError:
                        pass
        self.plans = [fx.Plan(params, max_images=max_images, device=device) for _ in range(slots)]

    def alloc(self, image):
        t = self.torch
        dt = t.uint8 if image.dtype == np.uint8 else t.uint16
        img = t.empty(image.shape, dtype=dt, device=self.device)
        out = t.empty(image.shape, dtype=t.uint8, device=self.device)
        return {"img": img, "out": out}

    def copy_in(self, dev, image):
        t = self.torch
        src = t.from_numpy(image)
        with t.cuda.nvtx.range("serve: copy in"), t.cuda.stream(self.copy_stream):
            dev["img"].copy_(src, non_blocking=True)
            ev = t.cuda.Event()
            ev.record(self.copy_stream)
        dev["img"].record_stream(self.copy_stream)
        dev["host"] = src  # keep the host buffer alive until the copy is done
        return ev

    def launch(self, slot, devs):
        t = self.torch
        s = self.streams[slot]
        with t.cuda.nvtx.range(f"serve: launch {len(devs)} requests"):
            self.plans[slot].extract_batch([(d["img"], d["out"]) for d in devs], stream=s)
        ev = t.cuda.Event()
        ev.record(s)
        for d in devs:  # the caching allocator must not recycle these before the kernel ends
            d["img"].record_stream(s)
            d["out"].record_stream(s)
        return ev

    @staticmethod
    def done(ev) -> bool:
        return ev.query()

    @staticmethod
    def free_input(dev):
        dev["img"] = None
        dev.pop("host", None)

    @staticmethod
    def free(dev):
        dev.clear()

    def close(self):
        for p in self.plans:
            p.close()
