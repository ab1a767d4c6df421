"""Pins of the oracle's rank rule, tile-size choice and warm start."""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import layout, operator, warmstart


def _planted(nr, b, ranks, mode, seed):
    lay = layout.make_layout(nr, b, ranks, mode)
    th = synth.planted_theta(nr, b, list(lay.k_diag) + list(lay.k_pair), lay.dense, seed)
    return lay, th, operator.assemble_xh(th, lay)


def test_rank_rule_recovers_planted_ranks_and_entry_count():
    # exact low-rank tiles: with a tiny eps the rule counts the nonzero
    # singular values, i.e. the planted ranks; dense diagonal tiles are full
    # rank; the entry count equals the size of the stacked unknown
    nr, b = 48, 8
    n = nr // b
    g = np.random.default_rng(5)
    kd = [int(k) for k in g.integers(0, 4, n)]
    kp = [int(k) for k in g.integers(0, 5, n * (n - 1) // 2)]
    dense = [False, True, False, False, True, False]
    lay, th, X = _planted(nr, b, kd + kp, dense, 6)
    ranks, entries, v0 = warmstart.tile_ranks(X, b, eps=1e-9)
    want = [b if dense[i] else kd[i] for i in range(n)] + kp
    assert ranks == want
    lay_rule = layout.make_layout(nr, b, ranks, "rule")
    assert entries == lay_rule.size
    assert v0 == pytest.approx(max(np.linalg.norm(X[i * b:(i + 1) * b, j * b:(j + 1) * b], 2)
                                   for i, j in warmstart.lower_tiles(nr, b)), rel=1e-12)


def test_rank_rule_threshold_is_relative_to_the_largest_tile_value():
    # one tile with singular values 1, 0.5, 0.02, 0.005, the rest zero: at
    # eps = 0.01 that tile has rank 3 (0.005 < 0.01), every other tile rank 0
    nr, b = 16, 4
    X = np.zeros((nr, nr), np.complex128)
    U = synth.haar_unitary(4, synth.rng(1))
    V = synth.haar_unitary(4, synth.rng(2))
    T = U @ np.diag([1.0, 0.5, 0.02, 0.005]) @ V.conj().T
    X[8:12, 0:4] = T
    X[0:4, 8:12] = T.T
    ranks, entries, v0 = warmstart.tile_ranks(X, b, eps=0.01)
    n = nr // b
    p = layout.pair_index(2, 0, n)
    assert v0 == pytest.approx(1.0)
    assert ranks[n + p] == 3 and sum(ranks) == 3
    assert entries == 2 * b * 3


def test_choose_tile_prefers_the_largest_tile_for_a_rank_one_matrix():
    # X = q q^T: every tile has rank 1, so the entries are nr^2 / b (low-rank
    # diagonals for b > 4) and the largest candidate tile wins
    g = synth.rng(3)
    q = synth.cn(g, 64)
    X = np.outer(q, q)
    b, e = warmstart.choose_tile(X, [8, 16, 32, 5], eps=0.01)
    assert b == 32 and e == 64 * 64 // 32


@pytest.mark.parametrize("k", [10, 4])
def test_takagi_factor(k):
    # Q Q^T equals the symmetric tile (full rank) or its best rank-k
    # truncation (Eckart-Young error sum of the dropped sigma^2)
    g = synth.rng(7)
    A = synth.cn(g, (10, 10))
    S = A + A.T
    Q = warmstart.takagi(S, k)
    s = np.linalg.svd(S, compute_uv=False)
    err = np.linalg.norm(S - Q @ Q.T) ** 2
    assert err == pytest.approx(float(np.sum(s[k:] ** 2)), abs=1e-10 * float(np.sum(s ** 2)))


def test_warm_start_is_the_truncated_svd_of_every_tile():
    # X_h rebuilt from the warm start: pairs and low-rank diagonals are their
    # best rank-k approximations (Eckart-Young), dense diagonals are copied,
    # and the super-diagonal tiles are the plain transposes
    nr, b = 40, 8
    g = synth.rng(9)
    A = synth.cn(g, (nr, nr))
    X = A + A.T
    lay = layout.make_layout(nr, b, [3, 8, 2, 0, 5] + [k % 9 for k in range(10)], [False, True, False, False, False])
    th = warmstart.warm_start(X, lay)
    Xh = operator.assemble_xh(th, lay)
    for i, j in warmstart.lower_tiles(nr, b):
        T = X[lay.rows(i), lay.rows(j)]
        W = Xh[lay.rows(i), lay.rows(j)]
        if i == j and lay.dense[i]:
            np.testing.assert_allclose(W, T, atol=1e-13)
            continue
        k = lay.k_diag[i] if i == j else lay.k_pair[layout.pair_index(i, j, lay.n)]
        s = np.linalg.svd(T, compute_uv=False)
        assert np.linalg.norm(T - W) ** 2 == pytest.approx(float(np.sum(s[k:] ** 2)),
                                                          abs=1e-10 * float(np.sum(s ** 2)))
