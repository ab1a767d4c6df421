"""Pins of the oracle on non-uniform tile partitions (tile sizes d_i, Tile
Low-rank MDD section: equal tiles are not a necessary constraint)."""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import general, layout, operator, solver, tlr, warmstart
from tests._cases import problem

TILES = [3, 5, 2]


def test_offsets_hand_computed():
    # d = (3, 5, 2); diagonals Q_0 (3 x 1), Z_1 (5 x 5), Q_2 (2 x 2); pairs in
    # stacking order (1,0), (2,0), (2,1) with ranks 2, 1, 2:
    # L: 5x2, 2x1, 2x2 = 10, 2, 4; R: 3x2, 3x1, 5x2 = 6, 3, 10
    lay = layout.make_layout(10, None, [1, 2, 2, 2, 1, 2], [False, True, False], tiles=TILES)
    assert lay.off_diag == [0, 3, 28]
    assert lay.off_l == [32, 42, 44]
    assert lay.off_r == [48, 54, 57]
    assert lay.size == 67
    # the entry count sum_{i>j} k_ij (d_i + d_j) + sum_i (d_i k_ii or d_i^2)
    assert lay.size == (2 * (5 + 3) + 1 * (2 + 3) + 2 * (2 + 5)) + (3 * 1 + 25 + 2 * 2)
    assert lay.b is None and lay.roff == [0, 3, 8]


@pytest.mark.parametrize("nr,b,ranks,mode", [(12, 4, [1, 0, 4, 2, 0, 3], [True, False, False]),
                                             (16, 4, 2, "rule"), (8, 8, 3, "lowrank")])
def test_equal_tiles_reproduce_the_uniform_layout(nr, b, ranks, mode):
    u = layout.make_layout(nr, b, ranks, mode)
    t = layout.make_layout(nr, None, ranks, mode, tiles=[b] * (nr // b))
    assert (u.off_diag, u.off_l, u.off_r, u.size, u.dense) == (t.off_diag, t.off_l, t.off_r, t.size, t.dense)
    assert t.b == b
    th = synth.cn(synth.rng(2), u.size)
    assert np.array_equal(operator.assemble_xh(th, u), operator.assemble_xh(th, t))


def _brute_xh(theta, d, kd, dense, kp):
    """Every entry of X_h from the tile formulas, with explicit row offsets."""
    n = len(d)
    roff = [sum(d[:i]) for i in range(n)]
    nr = sum(d)
    X = [[0j] * nr for _ in range(nr)]
    th = [complex(t) for t in theta]
    o = 0
    for i in range(n):
        for r in range(d[i]):
            for c in range(d[i]):
                if dense[i]:
                    v = 0.5 * (th[o + r * d[i] + c] + th[o + c * d[i] + r])
                else:
                    v = sum(th[o + r * kd[i] + q] * th[o + c * kd[i] + q] for q in range(kd[i]))
                X[roff[i] + r][roff[i] + c] = v
        o += d[i] * (d[i] if dense[i] else kd[i])
    pl = [(i, j) for j in range(n) for i in range(j + 1, n)]
    ol = []
    for p, (i, j) in enumerate(pl):
        ol.append(o)
        o += d[i] * kp[p]
    orr = []
    for p, (i, j) in enumerate(pl):
        orr.append(o)
        o += d[j] * kp[p]
    for p, (i, j) in enumerate(pl):
        k = kp[p]
        for r in range(d[i]):
            for c in range(d[j]):
                v = sum(th[ol[p] + r * k + q] * th[orr[p] + c * k + q] for q in range(k))
                X[roff[i] + r][roff[j] + c] = v
                X[roff[j] + c][roff[i] + r] = v
    return np.array(X)


@pytest.mark.parametrize("tiles,ranks,mode", [
    (TILES, [1, 2, 2, 2, 1, 2], [False, True, False]),
    ([1, 4, 2, 5], [1, 0, 2, 3, 1, 1, 0, 2, 1, 2], "lowrank"),
    ([6, 2], [6, 1, 2], "rule"),
])
def test_assembly_matches_brute_force(tiles, ranks, mode):
    nr = sum(tiles)
    lay = layout.make_layout(nr, None, ranks, mode, tiles=tiles)
    th = synth.cn(synth.rng(5), lay.size)
    X = operator.assemble_xh(th, lay)
    n = len(tiles)
    np.testing.assert_allclose(X, _brute_xh(th, tiles, lay.k_diag, lay.dense, lay.k_pair), rtol=0, atol=1e-14)
    assert np.array_equal(X, X.T)
    # every off-diagonal tile is d_i x d_j of rank at most k_ij
    for p, (i, j) in enumerate(lay.pair_list):
        T = X[lay.rows(i), lay.rows(j)]
        assert T.shape == (tiles[i], tiles[j])
        assert np.linalg.matrix_rank(T, tol=1e-10) <= lay.k_pair[p]
    assert n == lay.n


def test_full_rank_tiles_represent_any_symmetric_matrix():
    # ranks min(d_i, d_j) and dense diagonals: every complex symmetric X is a
    # TLR matrix of this partition (the tile SVDs and the diagonal copies
    # reproduce it)
    g = synth.rng(7)
    A = synth.cn(g, (10, 10))
    X = A + A.T
    kp = [min(TILES[i], TILES[j]) for j in range(3) for i in range(j + 1, 3)]
    lay = layout.make_layout(10, None, TILES + kp, "dense", tiles=TILES)
    th = warmstart.warm_start(X, lay)
    np.testing.assert_allclose(operator.assemble_xh(th, lay), X, atol=1e-12)
    # and the general form represents any X (not symmetric)
    B = synth.cn(g, (10, 10))
    gk = [min(TILES[i], TILES[j]) for (i, j) in general.ordered_pairs(3)]
    gl = general.make_general_layout(10, None, TILES + gk, "dense", tiles=TILES)
    tg = np.zeros(gl.size, np.complex128)
    for i in range(3):
        o = gl.off_diag[i]
        tg[o:o + TILES[i] ** 2] = B[gl.rows(i), gl.rows(i)].ravel()
    for p, (i, j) in enumerate(gl.pair_list):
        U, s, Vh = np.linalg.svd(B[gl.rows(i), gl.rows(j)], full_matrices=False)
        k = gl.k_pair[p]
        L, R = U[:, :k] * s[:k], Vh[:k].T
        tg[gl.off_l[p]:gl.off_l[p] + L.size] = L.ravel()
        tg[gl.off_r[p]:gl.off_r[p] + R.size] = R.ravel()
    np.testing.assert_allclose(general.assemble_x(tg, gl), B, atol=1e-12)


def _fd(f, th, idx, h=1e-6):
    out = []
    for e in idx:
        d = np.zeros_like(th)
        d[e] = h
        out.append((f(th + d) - f(th - d)) / (2 * h) + 1j * (f(th + 1j * d) - f(th - 1j * d)) / (2 * h))
    return np.array(out)


def test_gradient_matches_central_differences():
    D, U, perm, lay, _ = problem(4, 3, None, [1, 2, 2, 2, 1, 2], [False, True, False], ns=15, snr_db=10,
                                 planted=False, tiles=[4, 5, 3])
    Dh, Uh, _ = operator.normalise(D, U, perm)
    th = 0.3 * synth.cn(synth.rng(3), lay.size)
    g = operator.gradient(th, lay, Dh, Uh)
    f = lambda t: operator.misfit(t, lay, Dh, Uh)  # noqa: E731
    idx = list(range(0, lay.size, 2))
    fd = _fd(f, th, idx)
    assert np.max(np.abs(fd - g[idx])) <= 1e-6 * np.max(np.abs(g))


def test_general_gradient_matches_central_differences():
    g0 = synth.rng(4)
    tiles = [2, 4, 3]
    ns = 11
    Dh, Uh = synth.cn(g0, (ns, 9)), synth.cn(g0, (ns, 9))
    ranks = [1, 4, 2] + [1, 2, 2, 3, 1, 2]
    lay = general.make_general_layout(9, None, ranks, [False, True, False], tiles=tiles)
    th = 0.5 * synth.cn(synth.rng(5), lay.size)
    gr = general.gradient(th, lay, Dh, Uh)
    f = lambda t: general.misfit(t, lay, Dh, Uh)  # noqa: E731
    idx = list(range(lay.size))
    fd = _fd(f, th, idx)
    assert np.max(np.abs(fd - gr)) <= 1e-6 * np.max(np.abs(gr))


def test_tlr_forms_match_dense_literal():
    D, U, perm, lay, th = problem(6, 4, None, [2, 6, 1, 3, 2, 1], [False, True, False], ns=17, snr_db=20,
                                  tiles=[7, 12, 5])
    Dh, Uh, _ = operator.normalise(D, U, perm)
    f, g, _ = tlr.fgrad(th, lay, Dh.T, Uh.T)
    assert abs(f - operator.misfit(th, lay, Dh, Uh)) <= 1e-12 * f
    go = operator.gradient(th, lay, Dh, Uh)
    assert np.linalg.norm(g - go) <= 1e-12 * np.linalg.norm(go)
    np.testing.assert_allclose(tlr.apply(th, lay, Dh.T), operator.apply_y(th, lay, Dh), atol=1e-12)


def test_planted_recovery_noise_free():
    # tiles 16, 24, 8, 16 (n_r = 64), rank 2: from the truth + 5% the solver
    # recovers X to better than 1e-6 (exact data)
    tiles = [16, 24, 8, 16]
    D, U, perm, lay, th_true = problem(8, 8, None, 2, "lowrank", seed=4, tiles=tiles)
    U = D.astype(np.complex128) @ operator.unpermute(operator.assemble_xh(th_true, lay), perm)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    th0 = th_true + 0.05 * np.abs(th_true).mean() * synth.cn(synth.rng(8), lay.size)
    th, f, gf = solver.lbfgs(prob, th0, np.zeros_like(th0), 0.0, 400, 10)
    X, Xt = operator.assemble_xh(th, lay), operator.assemble_xh(th_true, lay)
    assert np.linalg.norm(X - Xt) <= 1e-6 * np.linalg.norm(Xt)


@pytest.mark.parametrize("tiles,ranks", [([3, 5, 1], 1), ([3, 0, 7], 1), ([2, 8], [3, 1, 1]), ([3, 7], [1, 1, 4])])
def test_invalid_partitions_rejected(tiles, ranks):
    # sizes that do not sum to n_r = 10, an empty tile, a diagonal rank above
    # d_0 = 2, a pair rank above min(d_i, d_j) = 3
    with pytest.raises(ValueError):
        layout.make_layout(10, None, ranks, "lowrank", tiles=tiles)
    with pytest.raises(ValueError):
        general.make_general_layout(10, None, ranks if isinstance(ranks, int) else ranks + [4], "lowrank",
                                    tiles=tiles)


def _eckart_young(X, W, k):
    s = np.linalg.svd(X, compute_uv=False)
    assert np.linalg.norm(X - W) ** 2 == pytest.approx(float(np.sum(s[k:] ** 2)), abs=1e-10 * float(np.sum(s ** 2)))


def test_warm_start_on_unequal_tiles_is_the_truncated_svd_of_every_tile():
    # reciprocal form: each kept tile of X_h (d_i x d_j) is the best rank-k
    # approximation of X's tile, dense diagonals are copied
    g = synth.rng(11)
    tiles = [5, 9, 3, 7]
    A = synth.cn(g, (24, 24))
    X = A + A.T
    lay = layout.make_layout(24, None, [2, 9, 1, 0] + [3, 2, 4, 1, 5, 3], [False, True, False, False],
                             tiles=tiles)
    Xh = operator.assemble_xh(warmstart.warm_start(X, lay), lay)
    for i in range(4):
        for j in range(i + 1):
            T, W = X[lay.rows(i), lay.rows(j)], Xh[lay.rows(i), lay.rows(j)]
            if i == j and lay.dense[i]:
                np.testing.assert_allclose(W, T, atol=1e-13)
                continue
            _eckart_young(T, W, lay.k_diag[i] if i == j else lay.k_pair[layout.pair_index(i, j, 4)])


@pytest.mark.parametrize("tiles", [[4, 4, 4], [3, 6, 2]])
def test_general_warm_start_is_the_truncated_svd_of_every_tile(tiles):
    # general form: every tile, above and below the diagonal and low-rank
    # diagonals, is its own truncated SVD; dense diagonals are copied; full
    # ranks reproduce X
    g = synth.rng(12)
    nr, n = sum(tiles), len(tiles)
    X = synth.cn(g, (nr, nr))
    pl = general.ordered_pairs(n)
    ranks = [2, tiles[1], 1] + [min(tiles[i], tiles[j], 1 + (i + 2 * j) % 3) for (i, j) in pl]
    lay = general.make_general_layout(nr, None, ranks, [False, True, False], tiles=tiles)
    W = general.assemble_x(general.warm_start(X, lay), lay)
    for i in range(n):
        for j in range(n):
            T, Wt = X[lay.rows(i), lay.rows(j)], W[lay.rows(i), lay.rows(j)]
            if i == j and lay.dense[i]:
                np.testing.assert_allclose(Wt, T, atol=1e-13)
                continue
            _eckart_young(T, Wt, lay.k_diag[i] if i == j else lay.k_pair[pl.index((i, j))])
    full = [tiles[i] for i in range(n)] + [min(tiles[i], tiles[j]) for (i, j) in pl]
    lf = general.make_general_layout(nr, None, full, "lowrank", tiles=tiles)
    np.testing.assert_allclose(general.assemble_x(general.warm_start(X, lf), lf), X, atol=1e-12)


@pytest.mark.parametrize("seed", range(8))
def test_random_partitions_gradients_and_structured_forms(seed):
    # random tile sizes, ranks, diagonal modes and data (both forms): the
    # gradients match central differences, and the TLR-structured forms the
    # dense-literal ones
    g = np.random.default_rng(100 + seed)
    n = int(g.integers(1, 5))
    tiles = [int(x) for x in g.integers(1, 6, n)]
    nr, ns = sum(tiles), int(g.integers(3, 9))
    dense = [bool(x) for x in g.integers(0, 2, n)]
    kd = [int(g.integers(0, tiles[i] + 1)) for i in range(n)]
    Dh = synth.cn(synth.rng(200 + seed), (ns, nr))
    Uh = synth.cn(synth.rng(300 + seed), (ns, nr))
    pl = layout.pairs(n)
    kp = [int(g.integers(0, min(tiles[i], tiles[j]) + 1)) for (i, j) in pl]
    lay = layout.make_layout(nr, None, kd + kp, dense, tiles=tiles)
    th = 0.5 * synth.cn(synth.rng(400 + seed), lay.size)
    if lay.size:
        gr = operator.gradient(th, lay, Dh, Uh)
        f = lambda t: operator.misfit(t, lay, Dh, Uh)  # noqa: E731
        idx = sorted(set(int(x) for x in g.integers(0, lay.size, 6)))
        fd = _fd(f, th, idx)
        assert np.max(np.abs(fd - gr[idx])) <= 1e-6 * max(1.0, np.max(np.abs(gr)))
        fs, gs, _ = tlr.fgrad(th, lay, Dh.T, Uh.T)
        assert abs(fs - f(th)) <= 1e-12 * max(1.0, f(th))
        assert np.linalg.norm(gs - gr) <= 1e-12 * max(1.0, np.linalg.norm(gr))
    gp = general.ordered_pairs(n)
    gk = [int(g.integers(0, min(tiles[i], tiles[j]) + 1)) for (i, j) in gp]
    glay = general.make_general_layout(nr, None, kd + gk, dense, tiles=tiles)
    tg = 0.5 * synth.cn(synth.rng(500 + seed), glay.size)
    if glay.size:
        gg = general.gradient(tg, glay, Dh, Uh)
        f2 = lambda t: general.misfit(t, glay, Dh, Uh)  # noqa: E731
        idx = sorted(set(int(x) for x in g.integers(0, glay.size, 6)))
        fd2 = _fd(f2, tg, idx)
        assert np.max(np.abs(fd2 - gg[idx])) <= 1e-6 * max(1.0, np.max(np.abs(gg)))
