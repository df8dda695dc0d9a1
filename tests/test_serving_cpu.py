"""Host-side tests of the continuous-batching scheduler with a fake backend
(no GPU): admission by budget in arrival order, rejection of oversized
requests, overlap of batches, cancellation, and failures injected by the
backend.  Time is simulated: device work completes after fixed delays."""
import numpy as np
import pytest

from paper_1304_3992_gb300.serve import Server, run_stream


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Copies take copy_s, batches take kernel_s of simulated time."""

    def __init__(self, clock, copy_s=0.001, kernel_s=0.005, fail_alloc=(), fail_launch=False):
        self.clock, self.copy_s, self.kernel_s = clock, copy_s, kernel_s
        self.fail_alloc, self.fail_launch = set(fail_alloc), fail_launch
        self.live = 0
        self.launches = []

    def alloc(self, image):
        if image.shape in self.fail_alloc:
            raise MemoryError("out of memory")
        self.live += 1
        return {"shape": image.shape}

    def copy_in(self, dev, image):
        return self.clock() + self.copy_s

    def launch(self, slot, devs):
        if self.fail_launch:
            raise RuntimeError("FX_ERR_CUDA")
        self.launches.append((slot, len(devs), self.clock()))
        return self.clock() + self.kernel_s

    def done(self, ev):
        return self.clock() >= ev

    def free_input(self, dev):
        pass

    def free(self, dev):
        self.live -= 1


def img(h, w, dtype=np.uint16):
    return np.zeros((h, w), dtype=dtype)


def advance(server, clock, dt, steps=20):
    for _ in range(steps):
        clock.t += dt / steps
        server.step()


def test_admission_in_order_under_budget():
    c = Clock()
    be = FakeBackend(c)
    a, b, d = img(100, 100), img(100, 100), img(10, 10)  # 30 000 device bytes each for a, b
    s = Server(be, budget_bytes=45_000, clock=c)
    ra, rb, rd = s.submit(0, a), s.submit(1, b), s.submit(2, d)
    s.step()
    assert ra.state == "copying" and rb.state == "pending" and rd.state == "pending"  # FIFO: d waits behind b
    assert s.used <= s.budget
    advance(s, c, 0.01)
    assert ra.state == "done"
    s.release(ra)
    advance(s, c, 0.02)
    assert rb.state == "done" and rd.state == "done"
    assert s.used == rb.pixels + rd.pixels  # masks stay resident until released
    s.release(rb)
    s.release(rd)
    assert s.used == 0 and be.live == 0


def test_oversized_request_rejected():
    c = Clock()
    s = Server(FakeBackend(c), budget_bytes=1000, clock=c)
    r = s.submit(0, img(100, 100))
    assert r.state == "rejected" and "BUDGET" in r.error
    assert s.idle()


def test_continuous_batching_overlaps():
    c = Clock()
    be = FakeBackend(c, copy_s=0.001, kernel_s=0.01)
    s = Server(be, budget_bytes=10**9, max_running=2, clock=c)
    first = [s.submit(i, img(50, 60)) for i in range(3)]
    advance(s, c, 0.002)  # copies done, first batch launched
    assert be.launches and be.launches[0][1] == 3
    late = [s.submit(10 + i, img(40, 40, np.uint8)) for i in range(4)]
    advance(s, c, 0.002)  # the late requests launch while the first batch still runs
    assert len(be.launches) == 2 and be.launches[1][1] == 4 and s.overlapped_launches == 1
    advance(s, c, 0.05)
    assert all(r.state == "done" for r in first + late)
    st = s.stats()
    assert st["completed"] == 7 and st["batches"] == 2


def test_cancel_and_failures():
    c = Clock()
    be = FakeBackend(c, fail_alloc={(13, 17)})
    s = Server(be, budget_bytes=10**9, clock=c)
    r1 = s.submit(0, img(20, 20))
    r2 = s.submit(1, img(13, 17))
    r3 = s.submit(2, img(30, 30))
    assert s.cancel(r3) and r3.state == "cancelled"
    s.step()
    assert r2.state == "failed" and "alloc" in r2.error
    advance(s, c, 0.02)
    assert r1.state == "done" and not s.cancel(r1)
    be.fail_launch = True
    r4 = s.submit(3, img(20, 20))
    advance(s, c, 0.01)
    assert r4.state == "failed" and "launch" in r4.error
    s.release(r1)
    assert s.used == 0


def test_poisson_stream_with_fake_backend():
    class TickingClock(Clock):
        def __call__(self):  # simulated time moves with every look at the clock
            self.t += 2e-5
            return self.t

    c = TickingClock()
    s = Server(FakeBackend(c, copy_s=0.002, kernel_s=0.004), budget_bytes=10**8, clock=c)
    imgs = [img(64, 64), img(128, 32, np.uint8), img(200, 100)]
    reqs = run_stream(s, imgs, rate_hz=500, duration_s=0.2, seed=3)
    assert reqs and all(r.state == "done" for r in reqs)
    st = s.stats()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    assert s.used == 0
