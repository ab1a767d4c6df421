"""Device-resident ADMM / L-BFGS solve vs the FP64 oracle (eq. 18-24)."""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import operator, solver
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu, dev, rel  # noqa: E402


def _start(lay, seed=77, scale=0.1):
    th = scale * synth.planted_theta(lay.nr, lay.b, list(lay.k_diag) + list(lay.k_pair), lay.dense, seed)
    return th.astype(np.complex64).astype(np.complex128)


def _oracle_solve(D, U, perm, lay, th0, **kw):
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    th, z, u, st = solver.admm(prob, th0, solver.SolveOpts(**kw))
    return th, st, alpha


def test_nr256_dense_diagonal_final_x_within_1e_3():
    # nr = ns = 256 (16 x 16 grid), tile 64, rank 8, dense diagonal, 20 dB, 30 iterations
    D, U, perm, lay, _ = problem(16, 16, 64, 8, "dense", seed=0, snr_db=20)
    th0 = _start(lay)
    tho, sto, alpha = _oracle_solve(D, U, perm, lay, th0)
    g = Gpu(D, U, lay, nx=16, ny=16, alpha=alpha)
    th, st = g.solve(th0)
    g.close()
    assert st.iters == 30 and st.status == 0
    Xo = operator.unpermute(operator.assemble_xh(tho, lay), perm)
    X = operator.unpermute(operator.assemble_xh(th, lay), perm)
    assert rel(X, Xo) <= 1e-3
    fh = np.array(st.f_hist[:st.n_hist])
    np.testing.assert_allclose(fh, sto.f_hist, rtol=1e-3)
    assert st.restarts == sto.restarts


@pytest.mark.parametrize("mode,ranks", [("lowrank", 3), ("rule", [5, 9, 1, 2, 3, 4])])
def test_small_solves_match_oracle(mode, ranks):
    D, U, perm, lay, _ = problem(8, 6, 16, ranks, mode, ns=60, seed=5, snr_db=10)
    th0 = _start(lay, seed=3, scale=0.3)
    kw = dict(stages=2, admm_iters=2, lbfgs_iters=4, memory=3)
    tho, sto, alpha = _oracle_solve(D, U, perm, lay, th0, **kw)
    g = Gpu(D, U, lay, nx=8, ny=6, alpha=alpha)
    th, st = g.solve(th0, **kw)
    g.close()
    Xo = operator.assemble_xh(tho, lay)
    X = operator.assemble_xh(th, lay)
    assert rel(X, Xo) <= 1e-3
    np.testing.assert_allclose(np.array(st.f_hist[:st.n_hist]), sto.f_hist, rtol=1e-3)


def test_solve_host_theta_matches_device_theta():
    D, U, perm, lay, _ = problem(8, 8, 16, 2, "lowrank", seed=2, snr_db=10)
    th0 = _start(lay, scale=0.3)
    g = Gpu(D, U, lay, nx=8, ny=8)
    th_d, st_d = g.solve(th0, lbfgs_iters=3, stages=1)
    th_h = np.ascontiguousarray(th0.astype(np.complex64))
    st_h = T.tlr_mdd_solve(g.h, th_h, T.solve_opts(lbfgs_iters=3, stages=1, theta_memory=T.TLR_MEM_HOST))
    g.close()
    assert np.array_equal(th_h.astype(np.complex128), th_d)
    assert st_h.iters == st_d.iters


def test_nonfinite_data_reported():
    D, U, perm, lay, _ = problem(4, 4, 8, 2, "lowrank", seed=1)
    D = D.copy()
    D[1, 3] = np.nan
    g = Gpu(D, U, lay, nx=4, ny=4, alpha=1.0)
    with pytest.raises(T.TLRError) as ei:
        g.solve(_start(lay), stages=1, admm_iters=1, lbfgs_iters=2)
    assert ei.value.code == -6
    g.close()


def test_invalid_solver_options():
    D, U, perm, lay, _ = problem(4, 4, 8, 2, "lowrank", seed=1)
    g = Gpu(D, U, lay, nx=4, ny=4)
    for kw in (dict(memory=0), dict(memory=33), dict(rho=0.0), dict(stages=-1)):
        with pytest.raises(T.TLRError) as ei:
            g.solve(_start(lay), **kw)
        assert ei.value.code == -1
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_async_graph_solves_on_two_streams_match_plain_solves(prec, monkeypatch):
    """Concurrent solves (graph replay, two streams) give bit-identical results
    to one-at-a-time solves without graphs: every reduction has a fixed order."""
    import torch
    probs = [problem(8, 8, 16, 3, "lowrank", seed=40 + i, snr_db=10) for i in range(2)]
    th0 = [_start(p[3], seed=50 + i, scale=0.3) for i, p in enumerate(probs)]
    kw = dict(stages=1, admm_iters=2, lbfgs_iters=4)
    # reference: plain launches, one at a time
    monkeypatch.setenv("TLR_MDD_GRAPHS", "0")
    ref = []
    for p, t in zip(probs, th0):
        g = Gpu(p[0], p[1], p[3], nx=8, ny=8, precision=prec)
        th, st = g.solve(t, **kw)
        ref.append(th)
        g.close()
    monkeypatch.setenv("TLR_MDD_GRAPHS", "1")
    streams = [torch.cuda.Stream() for _ in probs]
    gs = [Gpu(p[0], p[1], p[3], nx=8, ny=8, precision=prec, stream=s) for p, s in zip(probs, streams)]
    for rep in range(2):   # the second round replays the recorded graphs
        ths = [dev(t) for t in th0]
        opts = T.solve_opts(**kw)
        for g, th in zip(gs, ths):
            T.tlr_mdd_solve_async(g.h, th, opts)
        for g in gs:
            st = T.tlr_mdd_solve_wait(g.h)
            assert st.iters == 8 and st.status == 0
        for th, r in zip(ths, ref):
            assert np.array_equal(th.cpu().numpy().astype(np.complex128), r)
    for g in gs:
        g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_stationary_start_restarts_like_the_oracle(prec):
    # theta = 0 with low-rank diagonals is a saddle (every product is bilinear
    # in the factors, so g = 0 exactly): each of the 30 iterations restarts
    # and takes no step, on both sides, and X stays 0
    D, U, perm, lay, _ = problem(8, 8, 16, 3, "lowrank", ns=50, seed=6, snr_db=10)
    th0 = np.zeros(lay.size, np.complex128)
    tho, sto, alpha = _oracle_solve(D, U, perm, lay, th0)
    g = Gpu(D, U, lay, nx=8, ny=8, alpha=alpha, precision=prec)
    th, st = g.solve(th0)
    g.close()
    assert sto.restarts == 30 and st.restarts == sto.restarts
    assert st.iters == 30 and st.status == 0
    assert not np.any(th) and not np.any(tho)
    np.testing.assert_allclose(np.array(st.f_hist[:st.n_hist]), sto.f_hist, rtol=1e-5)
