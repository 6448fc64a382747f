"""The end-to-end serving loop of bench.py on CPU with a fake library: every
prepared request is submitted once, finished results are counted, and the
next step's requests are prepared while the current step runs."""
import os
import sys
import threading
import time
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeFeed:
    def __init__(self, delay):
        self.delay, self.next, self.calls = delay, 0, []

    def take(self, k):
        self.calls.append((threading.get_ident(), time.perf_counter()))
        time.sleep(self.delay)                      # relaxation on host threads
        ids = list(range(self.next, self.next + k))
        self.next += k
        return ["P%d" % i for i in ids], ["sdp%d" % i for i in ids]


class FakeBatch:
    def __init__(self, step_s):
        self.step_s, self.submitted, self.steps = step_s, [], []

    def submit(self, sdp, problem):
        assert problem == "P" + sdp[3:]
        self.submitted.append(sdp)
        return len(self.submitted)

    def step(self, iters, stream):
        self.steps.append(time.perf_counter())
        time.sleep(self.step_s)                     # the GPU serving `iters` iterations


def test_e2e_loop_submits_counts_and_overlaps():
    S = SimpleNamespace(STROM_OK=0, transfer_bytes=lambda: (0, 0))
    feed, batch = FakeFeed(0.2), FakeBatch(0.3)
    ok = SimpleNamespace(status=0)
    cert = SimpleNamespace(xi=0.0)

    def harvest(tickets):                           # half of the outstanding tickets finish per step
        n = len(tickets) // 2
        return [(ok, cert, 0.0, 0.0)] * n, tickets[n:]

    steps, per_step = 4, 5
    done, te, b0, b1, rest = bench.run_e2e(S, batch, feed, per_step, steps, 40, None, [], harvest, lambda: None)
    assert batch.submitted == ["sdp%d" % i for i in range(steps * per_step)]
    assert len(feed.calls) == steps + 1                  # one prefetch for a step that is not run
    # outstanding 5, 3+5, 4+5, 5+5 before each harvest: 2 + 4 + 4 + 5 finish, 5 stay
    assert done == 15 and len(rest) == 5
    # preparation overlaps serving: serial would take steps * (0.2 + 0.3) s
    assert te < steps * 0.5 - 0.3
