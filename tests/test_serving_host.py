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


@pytest.fixture
def fake(monkeypatch):
    def install(sizes, polls=3):
        f = FakeLib(sizes, polls)
        for name in ("tlr_mdd_workspace_bytes", "tlr_mdd_create", "tlr_mdd_solve_async",
                     "tlr_mdd_solve_query", "tlr_mdd_solve_wait", "tlr_mdd_destroy"):
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
    assert srv.peak_used <= 100 and srv.used == 0


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
