"""The serving request loop on a fake clock and a fake backend (no GPU):
arrival handling, continuous batching, latency accounting, first-come
first-served order, back-pressure and an injected slow request."""
import numpy as np

from paper_2009_03254_gb300 import serving


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeMesh:
    def __init__(self, n):
        self.num_triangles = n
        self.released = False

    def release(self):
        self.released = True


class FakeBackend:
    """Ticks of up to `batch` requests; a tick costs setup + per_request * k
    of fake time; the isovalue 99 is a slow request (costs `slow` extra)."""

    def __init__(self, clock, batch=4, setup=0.010, per_request=0.002, slow=0.5):
        self.clock, self.batch, self.setup, self.per, self.slow = clock, batch, setup, per_request, slow
        self.queue, self.done, self.next, self.ticks = [], {}, 1, []

    def submit(self, iso):
        t = self.next
        self.next += 1
        self.queue.append((t, iso))
        return t

    def step(self):
        take, self.queue = self.queue[:self.batch], self.queue[self.batch:]
        cost = self.setup + self.per * len(take) + sum(self.slow for _, iso in take if iso == 99)
        self.clock.t += cost
        self.ticks.append([t for t, _ in take])
        for t, iso in take:
            self.done[t] = (serving.ISO_OK, FakeMesh(int(iso)))
        return len(take)

    def take(self, ticket):
        return self.done.pop(ticket) if ticket in self.done else (serving.ISO_PENDING, None)


def test_latency_and_continuous_batching():
    clk = FakeClock()
    be = FakeBackend(clk)
    arrivals = [0.0, 0.001, 0.002, 0.003, 0.004, 0.005, 0.100]
    isos = [1, 2, 3, 4, 5, 6, 7]
    res = serving.RequestLoop(be, clock=clk, sleep=clk.sleep).run(arrivals, isos)
    # tick 0 starts at t=0 with only request 0 (the others have not arrived)
    assert be.ticks[0] == [1]
    # requests 1..5 arrived during tick 0 (ends at 0.012): they share tick 1 (4 of them) and tick 2
    assert be.ticks[1] == [2, 3, 4, 5] and be.ticks[2] == [6]
    assert [r["tick"] for r in res[:6]] == [0, 1, 1, 1, 1, 2]
    assert abs(res[0]["latency"] - 0.012) < 1e-12
    end1 = 0.012 + 0.010 + 0.008
    assert abs(res[1]["latency"] - (end1 - 0.001)) < 1e-12
    assert all(r["status"] == serving.ISO_OK for r in res)
    assert [r["triangles"] for r in res] == isos
    # the last request arrives after the queue drained: the loop slept until it
    assert abs(res[6]["latency"] - 0.012) < 1e-9 and be.ticks[3] == [7]


def test_slow_request_delays_only_later_ticks():
    clk = FakeClock()
    be = FakeBackend(clk, batch=2)
    arrivals = [0.0, 0.0, 0.1, 0.1, 0.1]
    isos = [1, 99, 2, 3, 4]
    res = serving.RequestLoop(be, clock=clk, sleep=clk.sleep).run(arrivals, isos)
    # the slow request holds its tick: its companion waits as long, later requests queue behind it
    assert abs(res[0]["latency"] - res[1]["latency"]) < 1e-12 and res[1]["latency"] > 0.5
    assert min(r["latency"] for r in res[2:]) > 0.4
    assert be.ticks == [[1, 2], [3, 4], [5]]


def test_back_pressure_rejects_when_queue_full():
    clk = FakeClock()
    be = FakeBackend(clk, batch=1, setup=1.0)
    arrivals = [0.0] + [0.5] * 5
    res = serving.RequestLoop(be, clock=clk, sleep=clk.sleep, max_queue=2).run(arrivals, list(range(1, 7)))
    statuses = [r["status"] for r in res]
    # request 0 is alone; at t=1.0 requests 1..5 have arrived but only 2 fit in the queue
    assert statuses[:3] == [serving.ISO_OK] * 3
    assert statuses[3:] == [serving.REJECTED] * 3
    s = serving.latency_summary(res)
    assert s["served"] == 3 and s["rejected"] == 3


def test_meshes_released_unless_kept():
    clk = FakeClock()
    be = FakeBackend(clk)
    res = serving.RequestLoop(be, clock=clk, sleep=clk.sleep, keep_meshes=True).run([0.0, 0.0], [5, 6])
    assert all(r["mesh"] is not None and not r["mesh"].released for r in res)


def test_workload_generators():
    a = serving.poisson_arrivals(20000, 50.0, 1)
    assert np.all(np.diff(a) > 0) and abs(len(a) / a[-1] - 50.0) < 2.0
    w = serving.random_walk_isovalues(5000, -1.0, 2.0, 5)
    assert w.min() >= -1.0 and w.max() <= 2.0
    steps = np.diff(w.astype(np.float64))
    assert 0.03 < np.std(steps) < 0.09          # 0.02 * 3, except where reflected
    assert np.array_equal(w, serving.random_walk_isovalues(5000, -1.0, 2.0, 5))
