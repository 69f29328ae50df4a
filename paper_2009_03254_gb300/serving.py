"""Request loop of the serving path.

Requests arrive over time: a schedule of arrival times (seconds from the
start) with one isovalue each.  The loop submits every request that has
arrived, runs one tick of the backend whenever requests wait (requests that
arrive during a tick join the next one: continuous batching), and records
each request's latency from arrival to the end of the tick that finished
it.  A queue limit gives back-pressure: a request that arrives while
`max_queue` requests wait is rejected.

The backend only needs submit(iso) -> ticket, step() -> finished count and
take(ticket) -> (status, mesh or None); a backend that also has poll()
(advance without blocking) is polled instead of stepped, so arrivals are
submitted while its earlier requests are still on the GPU.  Time comes
from `clock` and `sleep`, so the loop runs against a fake clock.  `Server`
(iso_server_*) is the batched backend; `PlainBackend` answers one request
per step with iso_extract, the plain per-request path.
"""
from __future__ import annotations

import time

ISO_OK = 0
ISO_PENDING = 7
REJECTED = -1


class PlainBackend:
    """One request per tick through Volume.extract, first come first served."""

    def __init__(self, volume):
        self.volume = volume
        self._queue = []
        self._done = {}
        self._next = 1

    def submit(self, iso):
        t = self._next
        self._next += 1
        self._queue.append((t, float(iso)))
        return t

    def queued(self):
        return len(self._queue)

    def step(self):
        if not self._queue:
            return 0
        t, iso = self._queue.pop(0)
        try:
            self._done[t] = (ISO_OK, self.volume.extract(iso))
        except Exception as e:                 # the library's IsoError carries the status
            self._done[t] = (getattr(e, "code", 4), None)
        return 1

    def take(self, ticket):
        if ticket in self._done:
            return self._done.pop(ticket)
        return ISO_PENDING, None


class RequestLoop:
    def __init__(self, backend, clock=time.perf_counter, sleep=time.sleep, max_queue=None, keep_meshes=False):
        self.backend = backend
        self.clock = clock
        self.sleep = sleep
        self.max_queue = max_queue
        self.keep_meshes = keep_meshes

    def run(self, arrivals, isos):
        """Serve the schedule.  Returns one dict per request, in request order:
        status (REJECTED for back-pressure), latency (s, None if rejected),
        triangles, tick (index of the tick that finished it) and mesh (kept
        only with keep_meshes; otherwise released at once)."""
        n = len(arrivals)
        out = [None] * n
        advance = getattr(self.backend, "poll", None) or self.backend.step
        waiting = {}                            # ticket -> request index
        t0 = self.clock()
        i, finished, ticks = 0, 0, 0
        while finished < n:
            now = self.clock() - t0
            while i < n and arrivals[i] <= now:
                if self.max_queue is not None and len(waiting) >= self.max_queue:
                    out[i] = {"status": REJECTED, "latency": None, "triangles": 0, "tick": None, "mesh": None}
                    finished += 1
                else:
                    waiting[self.backend.submit(isos[i])] = i
                i += 1
            if waiting:
                if not advance() and advance is not self.backend.step:
                    continue                    # polled, nothing finished: look for arrivals again
                t_end = self.clock() - t0
                for ticket in list(waiting):
                    status, mesh = self.backend.take(ticket)
                    if status == ISO_PENDING:
                        continue
                    idx = waiting.pop(ticket)
                    tris = mesh.num_triangles if mesh is not None else 0
                    if mesh is not None and not self.keep_meshes:
                        mesh.release()
                        mesh = None
                    out[idx] = {"status": status, "latency": t_end - arrivals[idx], "triangles": tris,
                                "tick": ticks, "mesh": mesh}
                    finished += 1
                ticks += 1
            elif i < n:
                self.sleep(max(0.0, arrivals[i] - (self.clock() - t0)))
        return out


def poisson_arrivals(n, rate, seed):
    """n arrival times of a Poisson process with `rate` requests per second."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def random_walk_isovalues(n, lo, hi, seed, step_frac=0.02):
    """n isovalues: a random walk in [lo, hi] reflected at both ends, steps
    normal with standard deviation step_frac * (hi - lo), starting midway."""
    import numpy as np
    rng = np.random.default_rng(seed)
    x = 0.5 * (lo + hi)
    out = np.empty(n, np.float32)
    w = hi - lo
    for k in range(n):
        x += rng.normal(0.0, step_frac * w)
        while x < lo or x > hi:
            x = 2 * lo - x if x < lo else 2 * hi - x
        out[k] = x
    return out


def latency_summary(results):
    import numpy as np
    lat = np.array([r["latency"] for r in results if r["latency"] is not None and r["status"] == ISO_OK])
    if len(lat) == 0:
        return {"served": 0}
    return {"served": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "rejected": sum(1 for r in results if r["status"] == REJECTED)}
