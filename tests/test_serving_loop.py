"""Host-side logic of the request loop (no GPU): arrivals are honoured on the
loop's clock, every request completes, latency runs from a job's arrival to the
end of the step that completed it (time spent waiting for a step in flight
counts), warm-up requests stay out of the statistics, and a job that the
server refuses surfaces as an error."""
import pytest

from paper_1809_06417_gb300.serving import Request, run_requests


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeJob:
    def __init__(self, server, steps):
        self.server, self.left, self.t_submit, self.t_done, self.state = server, steps, server.clock(), None, 0

    def info(self):
        class I:
            pass
        i = I()
        i.state, i.t_submit, i.t_done = self.state, self.t_submit, self.t_done
        return i


class FakeServer:
    """Each step takes `dt` seconds and advances every resident job by one
    iteration; at most `slots` jobs are resident (admission by capacity)."""

    def __init__(self, clock, dt=0.01, slots=2):
        self.clock, self.dt, self.slots = clock, dt, slots
        self.queue, self.resident = [], []

    def submit(self, steps):
        j = FakeJob(self, steps)
        self.queue.append(j)
        return j

    def step(self):
        while self.queue and len(self.resident) < self.slots:
            j = self.queue.pop(0)
            j.state = 1
            self.resident.append(j)
        self.clock.t += self.dt
        for j in list(self.resident):
            j.left -= 1
            if j.left == 0:
                j.state, j.t_done = 2, self.clock.t
                self.resident.remove(j)
        return len(self.resident), len(self.queue)


def test_loop_completes_every_request_and_measures_latency():
    clk = FakeClock()
    srv = FakeServer(clk, dt=0.01, slots=2)
    reqs = [Request(arrival=0.05 * k, submit=lambda s, n=n: s.submit(n)) for k, n in enumerate([3, 5, 2, 4, 1])]
    res = run_requests(srv, reqs, clock=clk, sleep=clk.sleep)
    assert len(res.latencies) == 5
    assert all(r.latency is not None and r.latency > 0 for r in reqs)
    # a lone job of n steps takes n * dt
    assert reqs[0].latency == pytest.approx(0.03, abs=1e-9)
    assert res.max_running <= 2
    assert res.percentile(50) <= res.percentile(99)


def test_capacity_makes_later_jobs_wait():
    clk = FakeClock()
    srv = FakeServer(clk, dt=0.01, slots=1)
    reqs = [Request(arrival=0.0, submit=lambda s: s.submit(10)) for _ in range(3)]
    res = run_requests(srv, reqs, clock=clk, sleep=clk.sleep)
    lat = sorted(res.latencies)
    assert lat == pytest.approx([0.10, 0.20, 0.30], abs=1e-9)


def test_refused_job_raises():
    clk = FakeClock()
    srv = FakeServer(clk)

    def refuse(s):
        raise MemoryError("job can never fit")

    with pytest.raises(MemoryError):
        run_requests(srv, [Request(arrival=0.0, submit=refuse)], clock=clk, sleep=clk.sleep)


def test_latency_counts_the_wait_for_a_step_in_flight():
    """A job arriving while a long step runs is submitted only after it: its
    latency includes that wait, its service time on the server does not."""
    clk = FakeClock()
    srv = FakeServer(clk, dt=0.05, slots=4)
    reqs = [Request(arrival=0.0, submit=lambda s: s.submit(2)),
            Request(arrival=0.01, submit=lambda s: s.submit(1))]
    res = run_requests(srv, reqs, clock=clk, sleep=clk.sleep)
    # the second job arrives at 0.01 during the first step (0 -> 0.05), is
    # submitted at 0.05 and done after the second step, at 0.10
    assert reqs[1].latency == pytest.approx(0.09, abs=1e-9)
    assert reqs[1].service == pytest.approx(0.05, abs=1e-9)
    assert len(res.latencies) == 2


def test_warmup_requests_are_not_measured():
    clk = FakeClock()
    srv = FakeServer(clk, dt=0.01, slots=8)
    reqs = [Request(arrival=0.01 * k, submit=lambda s: s.submit(3), warmup=k < 5) for k in range(12)]
    res = run_requests(srv, reqs, clock=clk, sleep=clk.sleep)
    assert len(res.latencies) == 7
    assert all(r.latency is not None for r in reqs)
    assert res.measured_start == pytest.approx(0.05)
    assert res.throughput() == pytest.approx(7 / (res.measured_end - 0.05))
