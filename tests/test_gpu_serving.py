"""Continuous batching of per-frequency solve requests on one GPU: each
request's result (the default 30-iteration solve) is bit-identical alone and
in the mix, and on a fresh handle or a cached one taken over from an earlier
request of the same shape; admission honours the device-memory budget."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from paper_2412_14973_gb300 import serving  # noqa: E402
from tests._gpu import abi_desc, dev  # noqa: E402

SHAPES = [  # (nx, ny, tile, rank, ns)
    (16, 16, 64, 4, 256), (32, 16, 64, 9, 512), (16, 16, 32, 12, 200),
    (32, 32, 128, 6, 1024), (16, 16, 64, 20, 256), (32, 16, 128, 3, 300),
]


def _requests(prec, arrivals=None):
    reqs = []
    for i, (nx, ny, b, k, ns) in enumerate(SHAPES):
        D, U, perm, lay, _ = problem(nx, ny, b, k, "rule", ns=ns, seed=60 + i, snr_db=10)
        d = abi_desc(lay, ns, nx=nx, ny=ny, precision=prec)
        th0 = (0.2 * synth.planted_theta(lay.nr, b, list(lay.k_diag) + list(lay.k_pair), lay.dense, 70 + i))
        opts = T.solve_opts()
        t = 0.0 if arrivals is None else arrivals[i]
        reqs.append(serving.SolveRequest(i, t, d, dev(D), dev(U), dev(th0), opts))
    return reqs


@pytest.mark.parametrize("prec", [0, 1])
def test_results_identical_alone_and_in_the_mix(prec):
    one = serving.Server(1 << 36, max_active=1, reuse=False)
    alone = one.run(_requests(prec), realtime=False)
    srv = serving.Server(1 << 36, max_active=4)
    mixed = srv.run(_requests(prec), realtime=False)
    assert srv.peak_active > 1
    for a, m in zip(alone, mixed):
        assert a.status == 0 and m.status == 0 and a.iters == 30
        assert torch.equal(a.theta, m.theta)
    # the same requests again: every one runs on a cached handle of its shape
    again = srv.run(_requests(prec), realtime=False)
    assert srv.reused == len(SHAPES) and srv.created == len(SHAPES)
    for a, m in zip(alone, again):
        assert m.status == 0 and torch.equal(a.theta, m.theta)
    srv.close()


def test_budget_admission_and_rejection():
    reqs = _requests(1)
    sizes = [T.tlr_mdd_workspace_bytes(r.desc) for r in reqs]
    budget = max(sizes) + min(sizes)
    srv = serving.Server(budget, max_active=4)
    out = srv.run(reqs, realtime=False)
    assert all(r.status == 0 for r in out)
    assert srv.peak_used <= budget
    srv.close()
    tiny = serving.Server(min(sizes) - 1, max_active=2)
    out = tiny.run(_requests(1)[:2], realtime=False)
    assert [r.status for r in out] == [-4, -4]


def test_poisson_arrivals_latency_accounting():
    g = np.random.default_rng(3)
    arrivals = np.cumsum(g.exponential(0.01, len(SHAPES)))
    out = serving.Server(1 << 36, max_active=3).run(_requests(1, list(arrivals)), realtime=True)
    for r in out:
        assert r.status == 0
        assert r.admitted >= r.arrival - 1e-6
        assert r.latency >= r.gpu_ms / 1e3 * 0.5
    p = serving.percentiles(out)
    assert p[50] <= p[99]


@pytest.mark.parametrize("prec,mix", [(1, False), (2, False), (1, True)])
def test_batched_server_results_identical_to_alone(prec, mix):
    # requests admitted together (of one size, or of any size with mix)
    # run as one lockstep batch (one launch per contraction over all their
    # tiles); results are bitwise those of the requests solved one at a time
    alone = serving.Server(1 << 36, max_active=1, reuse=False).run(_requests(prec), realtime=False)
    srv = serving.Server(1 << 36, max_active=2, batch_max=4, mix_sizes=mix)
    out = srv.run(_requests(prec), realtime=False)
    assert srv.batches >= 2
    for a, m in zip(alone, out):
        assert m.status == 0 and m.iters == 30
        assert torch.equal(a.theta, m.theta)
    srv.close()
