"""Request loop over the reconstruction server.

Jobs arrive at given times (a seeded Poisson stream in the benchmark); the
loop submits each job once its arrival time has passed, steps the server
(continuous batching: jobs join and leave at iteration boundaries), and
reports per-job latency from the server's own clock.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field


@dataclass
class Request:
    arrival: float          # seconds after the loop starts
    submit: object          # callable(server) -> job handle with .info()
    tag: object = None
    job: object = None
    latency: float = None


@dataclass
class LoopResult:
    latencies: list = field(default_factory=list)
    wall: float = 0.0
    steps: int = 0
    max_running: int = 0

    def percentile(self, q):
        xs = sorted(self.latencies)
        if not xs:
            return None
        i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
        return xs[i]


def run_requests(server, requests, clock=time.perf_counter, sleep=time.sleep, max_idle=1e-3):
    """Drive `server` (submit via each request's callable, then step) until
    every request has completed.  Arrival times are honoured against `clock`;
    latency = completion time - submission time, both on the server clock."""
    pending = sorted(requests, key=lambda r: r.arrival)
    waiting = []
    res = LoopResult()
    t0 = clock()
    i = 0
    while i < len(pending) or waiting:
        now = clock() - t0
        while i < len(pending) and pending[i].arrival <= now:
            r = pending[i]
            r.job = r.submit(server)
            waiting.append(r)
            i += 1
        if not waiting:
            sleep(min(max_idle, max(0.0, pending[i].arrival - now)))
            continue
        running, queued = server.step()
        res.steps += 1
        res.max_running = max(res.max_running, running)
        still = []
        for r in waiting:
            info = r.job.info()
            if info.state >= 2:  # done or cancelled
                r.latency = info.t_done - info.t_submit
                res.latencies.append(r.latency)
            else:
                still.append(r)
        waiting = still
    res.wall = clock() - t0
    return res
