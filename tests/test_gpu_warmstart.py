"""Rank rule, tile-size choice and warm start on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import paper_2412_14973_gb300 as T
import tlr_synth as synth
from oracle import layout, operator, warmstart

from _cases import problem
from _gpu import Gpu, dev, host, rel

pytestmark = pytest.mark.gpu


def _noisy_planted(nr, b, ranks, mode, seed, noise=1e-6):
    lay = layout.make_layout(nr, b, ranks, mode)
    th = synth.planted_theta(nr, b, list(lay.k_diag) + list(lay.k_pair), lay.dense, seed)
    X = operator.assemble_xh(th, lay)
    N = synth.noise(X.shape, seed + 1)
    N = 0.5 * (N + N.T)
    X = X + noise * np.linalg.norm(X) / np.linalg.norm(N) * N
    return X


def _check_ranks(X, b, eps, ranks_gpu, v0_gpu):
    # singular values from FP32 Jacobi (dots of length b, orthogonality to
    # 1e-5): relative accuracy about 1e-5 at b = 256; the bound is 1e-4
    ranks, entries, v0 = warmstart.tile_ranks(X, b, eps)
    assert v0_gpu == pytest.approx(v0, rel=1e-4)
    sv = warmstart.tile_svdvals(X, b)
    for t, (rg, ro) in enumerate(zip(ranks_gpu, ranks)):
        if rg != ro:
            # only a singular value within 1e-4 of the threshold may fall either way
            s = sv[t]
            lo, hi = min(rg, ro), max(rg, ro)
            assert np.all(np.abs(s[lo:hi] - eps * v0) <= 1e-4 * v0), (t, rg, ro, s[lo:hi], eps * v0)
    return ranks, entries


@pytest.mark.parametrize("nr,b,k", [(128, 16, 3), (192, 32, 6), (256, 64, 9)])
def test_tile_ranks_match_oracle(nr, b, k):
    X = _noisy_planted(nr, b, k, "lowrank", 30 + b)
    Xd = dev(X)
    ranks_g, ent_g, v0_g = T.tlr_mdd_tile_ranks(Xd, nr, b, 0.01)
    ranks, ent = _check_ranks(X, b, 0.01, ranks_g, v0_g)
    if ranks_g == ranks:
        assert ent_g == ent
    assert max(ranks_g) <= b


def test_choose_tile_matches_oracle():
    nr = 192
    X = _noisy_planted(nr, 32, 4, "lowrank", 41)
    cands = [8, 16, 24, 32, 48, 64, 7]
    bg, eg = T.tlr_mdd_choose_tile(dev(X), nr, cands, 0.01)
    bo, eo = warmstart.choose_tile(X, cands, 0.01)
    print(f"GPU choice b = {bg} ({eg} entries), oracle b = {bo} ({eo} entries)")
    assert bg == bo


@pytest.mark.parametrize("b", [16, 128])
def test_warm_start_matches_oracle(b):
    # a random complex symmetric X: every kept tile is the truncated SVD
    # (unique: the singular values of a random tile are separated, by about 1%
    # of sigma_max at b = 128).  The GPU's FP32 Jacobi stops at 1e-5 relative
    # orthogonality; a truncation at a 1% gap then moves by ~1e-4, so the bound
    # is the tensor-core path's 1e-3 (the warm start is a starting point)
    nr = 4 * b
    g = synth.rng(50 + b)
    A = synth.cn(g, (nr, nr))
    X = A + A.T
    ks = [b // 4 - 1, 0, b // 2, b // 8] + [(3 * p + 1) % (b // 2) for p in range(6)]
    lay = layout.make_layout(nr, b, ks, [False, False, True, False])
    D = synth.make_d(nr, nr, 1, 3)[0]
    gp = Gpu(D, D, lay, nx=nr // 4, ny=4)
    th = torch.zeros(lay.size, dtype=torch.complex64, device="cuda")
    T.tlr_mdd_warm_start(gp.h, dev(X), th)
    Xg = operator.assemble_xh(host(th), lay)
    Xo = operator.assemble_xh(warmstart.warm_start(X, lay), lay)
    err = rel(Xg, Xo)
    print(f"b = {b}: |X_h(warm, GPU) - X_h(warm, oracle)| = {err:.2e}")
    assert err <= 1e-3


def test_pipeline_benchmark_ranks_warm_start_solve():
    # benchmark solution -> tile ranks -> handle with those ranks -> warm start
    # -> the warm start's misfit is far below the zero start's and the solve
    # continues from it
    D, U, perm, lay0, _ = problem(8, 8, 16, 2, "lowrank", ns=64, seed=60, snr_db=30)
    g0 = Gpu(D, U, lay0, nx=8, ny=8, precision=T.TLR_PREC_BF16X3)
    Xb = torch.empty((64, 64), dtype=torch.complex64, device="cuda")
    T.tlr_mdd_benchmark_solve(g0.h, 1e-3, 300, 1e-6, Xb)
    b, _ = T.tlr_mdd_choose_tile(Xb, 64, [8, 16, 32], 0.01)
    ranks, _, _ = T.tlr_mdd_tile_ranks(Xb, 64, b, 0.01)
    lay = layout.make_layout(64, b, ranks, "rule")
    g = Gpu(D, U, lay, nx=8, ny=8, precision=T.TLR_PREC_BF16X3)
    th = torch.zeros(lay.size, dtype=torch.complex64, device="cuda")
    T.tlr_mdd_warm_start(g.h, Xb, th)
    f_warm, _ = g.grad(host(th))
    f_zero, _ = g.grad(np.zeros(lay.size))
    print(f"tile {b}, ranks {ranks}: f(warm) = {f_warm:.3e}, f(0) = {f_zero:.3e}")
    assert f_warm < 0.1 * f_zero
    th2, st = g.solve(host(th), lam0=0.01, stages=1, admm_iters=1, lbfgs_iters=5)
    assert st.f_hist[st.n_hist - 1] <= f_warm * (1 + 1e-6)


def test_tile_ranks_full_size():
    # nr = 4096, tile 256 (136 tile SVDs of 256 x 256) on a planted rank-20
    # matrix with noise: ranks and v0 as the oracle's
    nr, b = 4096, 256
    X = _noisy_planted(nr, b, 20, "lowrank", 70, noise=1e-4)
    Xd = dev(X)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ranks_g, ent_g, v0_g = T.tlr_mdd_tile_ranks(Xd, nr, b, 0.01)
    e1.record()
    torch.cuda.synchronize()
    print(f"tile ranks at nr {nr}, b {b}: {e0.elapsed_time(e1):.1f} ms; ranks {sorted(set(ranks_g))}")
    _check_ranks(X, b, 0.01, ranks_g, v0_g)


def test_invalid_arguments():
    X = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    for nr, b, eps, code in ((64, 24, 0.01, T.TLR_ERR_SHAPE), (64, 0, 0.01, T.TLR_ERR_SHAPE),
                             (1024, 1024, 0.01, T.TLR_ERR_SHAPE), (64, 16, 0.0, T.TLR_ERR_ARG),
                             (64, 16, 2.0, T.TLR_ERR_ARG)):
        with pytest.raises(T.TLRError) as e:
            T.tlr_mdd_tile_ranks(X, nr, b, eps)
        assert e.value.code == code
    with pytest.raises(T.TLRError) as e:
        T.tlr_mdd_choose_tile(X, 64, [24, 0], 0.01)
    assert e.value.code == T.TLR_ERR_SHAPE
