"""Host logic of the serving client (serving.StreamClient.run) with a fake server and fake
frame preparation, on the CPU: every arrived frame is accounted for at most once (completed,
dropped or failed), a stream has at most one frame in the server, and a frame refused by
admission (EBUSY) is retried and, when a newer frame has arrived meanwhile, replaced by it."""
from types import SimpleNamespace

import numpy as np

from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import serving as SV


class FakeServer:
    """Refuses the first `busy` submissions with EBUSY, then completes every frame after
    `rounds` polls; checks that a stream never has two frames in flight."""

    def __init__(self, busy: int, rounds: int):
        self.busy, self.rounds = busy, rounds
        self.polls, self.stream_of, self.in_flight = {}, {}, set()
        self.next = 1
        self.refused = 0

    def submit(self, fa):
        sid = fa
        if self.busy > 0:
            self.busy -= 1
            self.refused += 1
            raise B.PilotError(B.PILOT_EBUSY, "pending queue full")
        assert sid not in self.in_flight, "two frames of one stream in the server"
        tk = self.next
        self.next += 1
        self.polls[tk], self.stream_of[tk] = 0, sid
        self.in_flight.add(sid)
        return tk

    def poll(self, tk):
        self.polls[tk] += 1
        if self.polls[tk] < self.rounds:
            return False, None, None
        self.in_flight.discard(self.stream_of[tk])
        return True, SimpleNamespace(hyp_iters=7, best=-1), 0.5


def client_with(server, fail_every: int = 0):
    c = SV.StreamClient.__new__(SV.StreamClient)     # no device: preparation is faked
    c.server = server
    calls = []

    def prepare_batch(jobs):
        out = []
        for sid, st, t in jobs:
            calls.append((sid, t))
            failed = fail_every and (t + 1) % fail_every == 0
            out.append(None if failed else (sid, (0.0, 0.0), None))   # (frame args, origin, keep-alive)
        return out

    c.prepare_batch = prepare_batch
    return c, calls


def streams(n_streams, n_frames, period):
    return [SV.StreamState(gt=np.zeros((n_frames, 12)), sensors=[None] * n_frames,
                           arrivals=np.arange(n_frames) * period + 0.0003 * s, estimate=np.zeros(12))
            for s in range(n_streams)]


def check_accounting(st, sts):
    accounted = st["completed_frames"] + st["dropped_frames"] + st["crop_failed"]
    assert accounted <= st["offered_frames"], st
    done = [t for s in sts for t in s.done]
    assert len(done) == st["completed_frames"]
    for s in sts:                                   # each stream's frames complete in arrival order
        assert s.done == sorted(set(s.done))


def test_frames_are_accounted_once_under_overload():
    server = FakeServer(busy=0, rounds=40)          # slower than the arrivals: frames are dropped
    c, _ = client_with(server)
    sts = streams(3, 200, 0.002)
    st = c.run(sts, 0.15)
    check_accounting(st, sts)
    assert st["dropped_frames"] > 0 and st["completed_frames"] > 0
    assert st["hyp_iter_per_s"] > 0 and st["ebusy_retries"] == 0


def test_refused_frames_are_retried_and_replaced_without_double_counting():
    server = FakeServer(busy=60, rounds=3)           # admission refuses for a while
    c, calls = client_with(server)
    sts = streams(2, 300, 0.002)
    st = c.run(sts, 0.2)
    check_accounting(st, sts)
    assert st["ebusy_retries"] == server.refused > 0
    # while refused, newer frames replaced the waiting one: some streams prepared several
    # frames before their first completion
    assert len(calls) > st["completed_frames"] + st["crop_failed"]


def test_failed_crops_are_counted_and_skipped():
    server = FakeServer(busy=0, rounds=2)
    c, _ = client_with(server, fail_every=3)
    sts = streams(2, 100, 0.003)
    st = c.run(sts, 0.12)
    check_accounting(st, sts)
    assert st["crop_failed"] > 0
    assert all((t + 1) % 3 != 0 for s in sts for t in s.done)
