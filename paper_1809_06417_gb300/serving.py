"""Request loop over the reconstruction server.

Jobs arrive at given times (a seeded Poisson stream in the benchmark); the
loop submits each job once its arrival time has passed, steps the server
(continuous batching: jobs join and leave at iteration boundaries), and
reports per-job latency on its own clock, from the job's arrival to the end
of the step that completed it -- the time a job waited for a step in flight
before it could be submitted is part of it.  Requests marked as warm-up run
like the others but stay out of the statistics.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field


@dataclass
class Request:
    arrival: float          # seconds after the loop starts
    submit: object          # callable(server) -> job handle with .info()
    tag: object = None
    warmup: bool = False    # excluded from the latency statistics
    job: object = None
    latency: float = None   # arrival -> completion seen by the loop (loop clock)
    service: float = None   # submission -> completion on the server's clock


@dataclass
class LoopResult:
    latencies: list = field(default_factory=list)   # measured requests only
    services: list = field(default_factory=list)
    wall: float = 0.0
    steps: int = 0
    max_running: int = 0
    measured_start: float = None   # arrival of the first measured request (loop clock)
    measured_end: float = None     # completion of the last measured request

    def percentile(self, q, xs=None):
        xs = sorted(self.latencies if xs is None else xs)
        if not xs:
            return None
        i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
        return xs[i]

    def throughput(self):
        """Measured requests completed per second between the first measured
        arrival and the last measured completion."""
        if not self.latencies or self.measured_end is None:
            return None
        return len(self.latencies) / max(self.measured_end - self.measured_start, 1e-12)


def run_requests(server, requests, clock=time.perf_counter, sleep=time.sleep, max_idle=1e-3):
    """Drive `server` (submit via each request's callable, then step) until
    every request has completed.  Arrival times are honoured against `clock`."""
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
        seen = clock() - t0
        res.steps += 1
        res.max_running = max(res.max_running, running)
        still = []
        for r in waiting:
            info = r.job.info()
            if info.state >= 2:  # done or cancelled
                r.latency = seen - r.arrival
                r.service = info.t_done - info.t_submit
                if not r.warmup:
                    res.latencies.append(r.latency)
                    res.services.append(r.service)
                    if res.measured_start is None or r.arrival < res.measured_start:
                        res.measured_start = r.arrival
                    res.measured_end = seen if res.measured_end is None else max(res.measured_end, seen)
            else:
                still.append(r)
        waiting = still
    res.wall = clock() - t0
    return res
