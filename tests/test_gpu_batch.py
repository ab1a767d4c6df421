"""Batched solves (tlr_mdd_batch_*): the solves of several requests of
different sizes in lockstep, each contraction one launch over the tiles of
every member.  Every member's result and solver history are bit for bit its
result alone, in both tensor-core precisions, with the merged launches on
either GEMM form, with checkpoint refreshes, and from host theta buffers."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu, dev, host  # noqa: E402

SHAPES = [  # (nx, ny, b, ranks, mode, ns, tiles)
    (16, 16, 64, 4, "lowrank", 256, None),
    (32, 16, 64, 9, "rule", 300, None),
    (8, 8, 16, [3, 0, 16, 2, 1, 0, 4, 5, 2, 1], [False, True, True, False], 77, None),
    (32, 32, 128, 6, "lowrank", 1024, None),
    (16, 8, None, 4, "lowrank", 90, [48, 16, 64]),
]


def _members(prec):
    out = []
    for i, (nx, ny, b, ranks, mode, ns, tiles) in enumerate(SHAPES):
        D, U, perm, lay, _ = problem(nx, ny, b, ranks, mode, ns=ns, seed=80 + i, snr_db=10, tiles=tiles)
        th0 = (0.2 * synth.cn(synth.rng(90 + i), lay.size)).astype(np.complex64).astype(np.complex128)
        out.append((Gpu(D, U, lay, nx=nx, ny=ny, precision=prec), th0))
    return out


def _alone(members, **kw):
    return [g.solve(th0, **kw) for g, th0 in members]


@pytest.mark.parametrize("prec,persist", [(1, 0), (2, 0), (1, 7)])
def test_batched_results_are_bitwise_the_solves_alone(prec, persist, monkeypatch):
    monkeypatch.setenv("TLR_MDD_PERSIST", str(persist))
    members = _members(prec)
    ref = _alone(members)
    b = T.Batch([g.h for g, _ in members])
    for rep in range(2):   # the batch can be solved again
        thetas = [dev(th0) for _, th0 in members]
        b.solve_async(thetas, T.solve_opts())
        stats = b.wait()
        for (th_ref, st_ref), th, st in zip(ref, thetas, stats):
            assert st.status == 0 and st.iters == 30 and st.restarts == st_ref.restarts
            assert np.array_equal(host(th), th_ref)
            assert list(st.f_hist[:30]) == list(st_ref.f_hist[:30])
    b.destroy()
    for g, _ in members:
        g.close()


def test_batched_refresh_and_host_thetas():
    members = _members(1)
    kw = dict(stages=1, admm_iters=2, lbfgs_iters=3, flags=T.TLR_SOLVE_REFRESH)
    ref = _alone(members, **kw)
    b = T.Batch([g.h for g, _ in members])
    thetas = [np.ascontiguousarray(th0.astype(np.complex64)) for _, th0 in members]
    b.solve_async(thetas, T.solve_opts(theta_memory=T.TLR_MEM_HOST, **kw))
    stats = b.wait()
    for (th_ref, st_ref), th, st in zip(ref, thetas, stats):
        assert st.iters == 6 and np.array_equal(th.astype(np.complex128), th_ref)
    b.destroy()
    for g, _ in members:
        g.close()


def test_batch_rejects_what_it_cannot_run():
    members = _members(1)
    D, U, perm, lay, _ = problem(8, 8, 16, 2, "lowrank", ns=40, seed=5)
    g32 = Gpu(D, U, lay, nx=8, ny=8, precision=T.TLR_PREC_FP32)
    with pytest.raises(T.TLRError) as e:
        T.Batch([members[0][0].h, g32.h])                 # the FP32 path has no packed operands
    assert e.value.code == T.TLR_ERR_UNSUPPORTED
    with pytest.raises(T.TLRError) as e:
        T.Batch([members[0][0].h, members[0][0].h])       # a handle twice
    assert e.value.code == T.TLR_ERR_ARG
    gt = Gpu(D, U, lay, nx=8, ny=8, precision=T.TLR_PREC_TF32)
    with pytest.raises(T.TLRError) as e:
        T.Batch([members[0][0].h, gt.h])                  # mixed tensor-core precisions
    assert e.value.code == T.TLR_ERR_ARG
    for g in [g32, gt] + [g for g, _ in members]:
        g.close()
