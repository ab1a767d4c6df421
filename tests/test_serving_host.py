"""Host-side scheduling of the serving loop, with a fake library (CPU only):
first-come first-served admission under a device-memory budget, slot limits,
rejection of requests larger than the budget, memory released on completion."""
import types

import pytest

pytest.importorskip("paper_2412_14973_gb300")
from paper_2412_14973_gb300 import serving  # noqa: E402


class FakeLib:
    """Solves finish after a fixed number of polls; records concurrency."""

    def __init__(self, sizes, polls=3):
        self.sizes = sizes
        self.polls = polls
        self.live = {}
        self.order = []
        self.max_live = 0
        self.next = 1
        self.destroyed, self.moved, self.rebound = [], [], []

    def tlr_mdd_workspace_bytes(self, d):
        return self.sizes[d]

    def tlr_mdd_create(self, d, D, U, stream):
        h = self.next
        self.next += 1
        self.live[h] = self.polls
        self.order.append(d)
        self.max_live = max(self.max_live, len(self.live))
        return h

    def tlr_mdd_solve_async(self, h, theta, opts):
        pass

    def tlr_mdd_solve_query(self, h):
        self.live[h] -= 1
        return self.live[h] <= 0

    def tlr_mdd_solve_wait(self, h):
        return types.SimpleNamespace(gpu_ms=1.0, iters=30)

    def tlr_mdd_destroy(self, h):
        del self.live[h]
        self.destroyed.append(h)

    def tlr_mdd_set_stream(self, h, stream):
        self.moved.append((h, stream))

    def tlr_mdd_set_data(self, h, D, U, mem=0):
        self.live[h] = self.polls
        self.rebound.append(h)


@pytest.fixture
def fake(monkeypatch):
    def install(sizes, polls=3):
        f = FakeLib(sizes, polls)
        for name in ("tlr_mdd_workspace_bytes", "tlr_mdd_create", "tlr_mdd_solve_async",
                     "tlr_mdd_solve_query", "tlr_mdd_solve_wait", "tlr_mdd_destroy",
                     "tlr_mdd_set_stream", "tlr_mdd_set_data"):
            monkeypatch.setattr(serving.T, name, getattr(f, name))
        return f
    return install


def _req(rid, size_key, arrival=0.0):
    return serving.SolveRequest(rid, arrival, size_key, None, None, object(), opts=None)


def test_budget_and_slots_bound_concurrency(fake):
    f = fake({"a": 40, "b": 40, "c": 40, "d": 40})
    srv = serving.Server(100, max_active=3, stream_factory=object, poll_s=0)
    out = srv.run([_req(i, k) for i, k in enumerate("abcd")], realtime=False)
    assert [r.status for r in out] == [0, 0, 0, 0]
    assert f.max_live == 2            # 3 slots, but only two 40-byte requests fit in 100
    assert srv.peak_used <= 100
    srv.close()
    assert srv.used == 0 and not f.live


def test_oversized_request_rejected_and_others_served(fake):
    f = fake({"small": 10, "huge": 1000})
    srv = serving.Server(100, max_active=2, stream_factory=object, poll_s=0)
    out = srv.run([_req(0, "small"), _req(1, "huge"), _req(2, "small")], realtime=False)
    assert out[1].status == -4 and out[1].theta is None
    assert out[0].status == 0 and out[2].status == 0
    assert "huge" not in f.order


def test_first_come_first_served(fake):
    f = fake({"big": 80, "s1": 10, "s2": 10}, polls=2)
    srv = serving.Server(100, max_active=4, stream_factory=object, poll_s=0)
    srv.run([_req(0, "s1"), _req(1, "big"), _req(2, "s2")], realtime=False)
    # s2 does not overtake the big request that arrived before it
    assert f.order == ["s1", "big", "s2"]


def test_records_one_json_line_per_request(fake, monkeypatch, tmp_path):
    import json
    fake({"a": 10, "huge": 1000})
    reqs = [_req(0, "a", 0.0), _req(1, "huge", 0.0)]
    for r in reqs:
        r.desc = types.SimpleNamespace(nr=64, ns=48, tile=16, tiles=None, ntiles=0, rank=3,
                                       precision=serving.T.TLR_PREC_BF16X3, key=r.desc)
    # the fake library keys its sizes by the description
    monkeypatch.setattr(serving.T, "tlr_mdd_workspace_bytes", lambda d: {"a": 10, "huge": 1000}[d.key])
    srv = serving.Server(100, max_active=2, stream_factory=object, poll_s=0)
    out = srv.run(reqs, realtime=False)
    recs = serving.records(reqs, out)
    assert [r["rid"] for r in recs] == [0, 1]
    assert recs[0]["status"] == 0 and recs[0]["iters"] == 30 and recs[0]["precision"] == "bf16x3"
    assert recs[1]["status"] == -4 and recs[1]["tile"] == 16
    p = tmp_path / "log.jsonl"
    serving.write_jsonl(p, recs)
    lines = p.read_text().splitlines()
    assert [json.loads(x)["rid"] for x in lines] == [0, 1]


def test_finished_handles_are_reused_by_requests_of_the_same_shape(fake):
    # a, b, a, a: the later a's take over the first a's handle (no create, no
    # allocation); the b handle stays cached
    f = fake({"a": 30, "b": 30})
    srv = serving.Server(100, max_active=1, stream_factory=object, poll_s=0)
    out = srv.run([_req(i, k) for i, k in enumerate("abaa")], realtime=False)
    assert [r.status for r in out] == [0, 0, 0, 0]
    assert f.order == ["a", "b"] and srv.created == 2 and srv.reused == 2
    assert len(f.rebound) == 2 and len(f.moved) == 2
    assert srv.used == 60 and len(srv.idle) == 2
    srv.close()
    assert srv.used == 0 and not f.live


def test_idle_handles_are_evicted_least_recently_used_first_when_memory_is_needed(fake):
    f = fake({"a": 40, "b": 40, "c": 40})
    srv = serving.Server(100, max_active=1, stream_factory=object, poll_s=0)
    srv.run([_req(0, "a"), _req(1, "b")], realtime=False)
    assert srv.used == 80
    srv.run([_req(2, "c")], realtime=False)     # needs 40: the a handle (oldest) goes
    assert srv.evicted == 1 and f.destroyed == [1] and srv.used == 80
    srv.run([_req(3, "b")], realtime=False)     # cached: reused, nothing evicted
    assert srv.evicted == 1 and srv.reused == 1
    srv.close()


def test_no_reuse_mode_destroys_every_handle(fake):
    f = fake({"a": 30})
    srv = serving.Server(100, max_active=1, stream_factory=object, poll_s=0, reuse=False)
    srv.run([_req(0, "a"), _req(1, "a")], realtime=False)
    assert srv.created == 2 and srv.reused == 0 and srv.used == 0 and not f.live


class FakeBatch:
    made = []

    def __init__(self, handles, stream):
        self.handles = list(handles)
        self.polls = 2
        FakeBatch.made.append(self)

    def solve_async(self, thetas, opts):
        self.n = len(thetas)

    def query(self):
        self.polls -= 1
        return self.polls <= 0

    def wait(self):
        return [types.SimpleNamespace(gpu_ms=2.0, iters=30) for _ in self.handles]

    def destroy(self):
        pass


def _sreq(rid, nr, key, arrival=0.0, prec=1):
    d = types.SimpleNamespace(nr=nr, precision=prec, key=key)
    return serving.SolveRequest(rid, arrival, d, None, None, object(), opts=None)


def test_batching_groups_arrived_requests_of_the_same_size(fake, monkeypatch):
    f = fake({})
    monkeypatch.setattr(serving.T, "tlr_mdd_workspace_bytes", lambda d: 10)
    monkeypatch.setattr(serving.T, "Batch", FakeBatch)
    FakeBatch.made = []
    reqs = [_sreq(0, 1024, "a"), _sreq(1, 2048, "b"), _sreq(2, 1024, "c"), _sreq(3, 1024, "d"),
            _sreq(4, 2048, "e")]
    srv = serving.Server(1000, max_active=2, stream_factory=object, poll_s=0, batch_max=4)
    out = srv.run(reqs, realtime=False)
    assert [r.status for r in out] == [0] * 5 and all(r.iters == 30 for r in out)
    groups = sorted(len(b.handles) for b in FakeBatch.made)
    assert groups == [2, 3] and srv.batches == 2        # the 1024s together, the 2048s together
    srv.close()


def test_fp32_requests_are_never_batched(fake, monkeypatch):
    fake({})
    monkeypatch.setattr(serving.T, "tlr_mdd_workspace_bytes", lambda d: 10)
    monkeypatch.setattr(serving.T, "Batch", FakeBatch)
    FakeBatch.made = []
    reqs = [_sreq(i, 1024, str(i), prec=0) for i in range(3)]
    srv = serving.Server(1000, max_active=1, stream_factory=object, poll_s=0, batch_max=4)
    out = srv.run(reqs, realtime=False)
    assert [r.status for r in out] == [0, 0, 0] and not FakeBatch.made and srv.batches == 0
    srv.close()


def test_batch_members_respect_the_budget(fake, monkeypatch):
    fake({})
    monkeypatch.setattr(serving.T, "tlr_mdd_workspace_bytes", lambda d: 40)
    monkeypatch.setattr(serving.T, "Batch", FakeBatch)
    FakeBatch.made = []
    reqs = [_sreq(i, 1024, str(i)) for i in range(4)]
    srv = serving.Server(100, max_active=1, stream_factory=object, poll_s=0, batch_max=4, reuse=False)
    out = srv.run(reqs, realtime=False)
    assert [r.status for r in out] == [0] * 4
    assert max(len(b.handles) for b in FakeBatch.made) == 2 and srv.peak_used <= 100


def test_mixed_size_batches_take_any_size_of_one_precision(fake, monkeypatch):
    fake({})
    monkeypatch.setattr(serving.T, "tlr_mdd_workspace_bytes", lambda d: 10)
    monkeypatch.setattr(serving.T, "Batch", FakeBatch)
    FakeBatch.made = []
    reqs = [_sreq(0, 1024, "a"), _sreq(1, 2048, "b"), _sreq(2, 4096, "c"), _sreq(3, 1024, "d", prec=0),
            _sreq(4, 8192, "e")]
    srv = serving.Server(1000, max_active=1, stream_factory=object, poll_s=0, batch_max=4, mix_sizes=True)
    out = srv.run(reqs, realtime=False)
    assert [r.status for r in out] == [0] * 5
    # the four tensor-core requests of four sizes in one batch; the FP32 one alone
    assert [len(b.handles) for b in FakeBatch.made] == [4] and srv.batches == 1
    srv.close()


def test_cancelled_requests_end_before_admission(fake):
    f = fake({"a": 60, "b": 60, "c": 60})
    srv = serving.Server(100, max_active=2, stream_factory=object, poll_s=0)
    srv.cancel(1)          # withdrawn before the run serves it; "a" holds the memory meanwhile
    out = srv.run([_req(0, "a"), _req(1, "b"), _req(2, "c")], realtime=False)
    assert [r.status for r in out] == [0, serving.CANCELLED, 0]
    assert out[1].theta is None and out[1].message.startswith("cancelled")
    assert f.order == ["a", "c"]
    # the cancel was consumed: the same id is served on the next run
    out2 = srv.run([_req(1, "b")], realtime=False)
    assert out2[0].status == 0
    srv.close()


def test_cancel_from_another_thread_while_serving(fake):
    import threading
    fake({"a": 60, "b": 60}, polls=200)
    srv = serving.Server(100, max_active=1, stream_factory=object, poll_s=1e-4)
    t = threading.Timer(0.005, srv.cancel, args=(1,))
    t.start()
    out = srv.run([_req(0, "a"), _req(1, "b")], realtime=False)
    t.join()
    assert out[0].status == 0 and out[1].status == serving.CANCELLED
    srv.close()


def test_admission_deadline_expires_queued_requests(fake):
    f = fake({"a": 60, "b": 60, "c": 60}, polls=400)
    reqs = [_req(0, "a"), _req(1, "b"), _req(2, "c")]
    reqs[1].deadline = 0.002    # "a" holds the memory for ~40 ms, so "b" expires in the queue
    reqs[2].deadline = 60.0     # plenty of time
    srv = serving.Server(100, max_active=2, stream_factory=object, poll_s=1e-4)
    out = srv.run(reqs, realtime=True)
    assert [r.status for r in out] == [0, serving.EXPIRED, 0]
    assert f.order == ["a", "c"]
    srv.close()
