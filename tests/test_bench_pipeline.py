"""Host logic of the double-buffered end-to-end loop (bench.pipelined_run), on the
CPU: CUDA streams and events are replaced by a recorder that builds the
happens-before graph of the enqueued operations (stream order plus event waits),
and the test checks every ordering the reuse of a buffer set needs."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Recorder:
    """Streams as lists of operations; an event remembers the last operation of its
    stream when recorded; a wait makes the waiting stream's next operation depend on it."""

    def __init__(self):
        self.ops = []            # (name, step, buffer set)
        self.preds = []          # predecessor op indices of each op
        self.current = None

    def enqueue(self, stream, label):
        preds = set(stream.pending)
        if stream.last is not None:
            preds.add(stream.last)
        self.ops.append(label)
        self.preds.append(preds)
        stream.last = len(self.ops) - 1
        stream.pending = set()
        return stream.last

    def before(self, a, b):
        """True when op a happens before op b."""
        seen, todo = set(), [b]
        while todo:
            x = todo.pop()
            for p in self.preds[x]:
                if p == a:
                    return True
                if p not in seen:
                    seen.add(p)
                    todo.append(p)
        return False


def fake_cuda(rec):
    class Stream:
        def __init__(self, device=None):
            self.last, self.pending = None, set()

        def wait_event(self, ev):
            if ev.op is not None:
                self.pending.add(ev.op)

    class Event:
        def __init__(self, *a, **k):
            self.op = None

        def record(self, stream):
            self.op = stream.last

    class Ctx:
        def __init__(self, st):
            self.st = st

        def __enter__(self):
            self.prev, rec.current = rec.current, self.st

        def __exit__(self, *exc):
            rec.current = self.prev

    return Stream, Event, Ctx


@pytest.mark.parametrize("steps", [1, 2, 5, 8])
def test_pipelined_run_orders_every_buffer_reuse(monkeypatch, steps):
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench

    rec = Recorder()
    Stream, Event, Ctx = fake_cuda(rec)
    monkeypatch.setattr(torch.cuda, "Stream", Stream)
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "stream", Ctx)
    phase = {"timed": False}
    counter = {"in": 0, "cmp": 0, "out": 0}

    def op(kind):
        def run(b):
            s = counter[kind]
            counter[kind] += 1
            rec.enqueue(rec.current, (kind, s, b, phase["timed"]))
        return run

    parts = [op("in")]

    def sync(*a, **k):
        # the warm-up ends with a synchronize: later ops belong to the timed steps
        phase["timed"] = True
        counter.update({"in": 0, "cmp": 0, "out": 0})
    monkeypatch.setattr(torch.cuda, "synchronize", sync)
    bench.pipelined_run("cpu", steps, parts, op("cmp"), op("out"))
    timed = {(k, s): i for i, (k, s, b, t) in enumerate(rec.ops) if t}
    assert len(timed) == 3 * steps
    for s in range(steps):
        b = s % 2
        assert rec.ops[timed[("in", s)]][2] == b and rec.ops[timed[("cmp", s)]][2] == b
        # a step's call follows its own inputs, and its read-back follows the call
        assert rec.before(timed[("in", s)], timed[("cmp", s)])
        assert rec.before(timed[("cmp", s)], timed[("out", s)])
        if s >= 2:
            # set b's inputs are overwritten only after step s-2 computed on them, and its
            # results only after step s-2's read-back
            assert rec.before(timed[("cmp", s - 2)], timed[("in", s)])
            assert rec.before(timed[("out", s - 2)], timed[("cmp", s)])
    # the three kinds of work are on three different streams, so they can overlap
    if steps >= 2:
        assert not rec.before(timed[("cmp", 0)], timed[("in", 1)])
        assert not rec.before(timed[("out", 0)], timed[("cmp", 1)])
