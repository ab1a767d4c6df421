"""Pins of the oracle's general (non-reciprocal) TLR form."""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import general, layout, operator, solver


def _theta(lay, seed, scale=0.5):
    return scale * synth.cn(synth.rng(seed), lay.size)


def test_assembly_written_out():
    # N = 2, b = 2, rank 1 everywhere, low-rank diagonals: every entry as an
    # explicit sum over the single factor column
    lay = general.make_general_layout(4, 2, 1, "lowrank")
    th = _theta(lay, 1)
    X = general.assemble_x(th, lay)
    for i in range(2):
        o = lay.off_diag[i]
        L, R = th[o:o + 2], th[o + 2:o + 4]
        for a in range(2):
            for c in range(2):
                assert X[2 * i + a, 2 * i + c] == pytest.approx(L[a] * R[c])
    for p, (i, j) in enumerate(lay.pair_list):
        L, R = th[lay.off_l[p]:lay.off_l[p] + 2], th[lay.off_r[p]:lay.off_r[p] + 2]
        for a in range(2):
            for c in range(2):
                assert X[2 * i + a, 2 * j + c] == pytest.approx(L[a] * R[c])
    assert not np.allclose(X, X.T)


@pytest.mark.parametrize("tiles", [None, [3, 6, 3], [5, 2, 5]])
def test_reduces_to_the_reciprocal_form(tiles):
    # mirrored factors (L_ji = R_ij, R_ji = L_ij, L_ii = R_ii = Q_ii, Z_ii
    # symmetric) give the reciprocal X_h and the same misfit; equal tiles of
    # 4 or the unequal partitions given
    nr, b = 12, 4
    ranks = [2, 2, 0] + [1, 2, 2]
    sym = layout.make_layout(nr, None if tiles else b, ranks, [False, True, False], tiles=tiles)
    ths = _theta(sym, 2)
    n = sym.n
    kp = {}
    for p, (i, j) in enumerate(sym.pair_list):
        kp[(i, j)] = kp[(j, i)] = sym.k_pair[p]
    gen_ranks = list(sym.k_diag) + [kp[(i, j)] for (i, j) in general.ordered_pairs(n)]
    gen = general.make_general_layout(nr, None if tiles else b, gen_ranks, sym.dense, tiles=tiles)
    thg = np.zeros(gen.size, np.complex128)
    for i in range(n):
        B = sym.diag_block(ths, i)
        o = gen.off_diag[i]
        if sym.dense[i]:
            thg[o:o + B.size] = (0.5 * (B + B.T)).ravel()
        else:
            thg[o:o + B.size] = B.ravel()
            thg[o + B.size:o + 2 * B.size] = B.ravel()
    pos = {ij: p for p, ij in enumerate(gen.pair_list)}
    for p, (i, j) in enumerate(sym.pair_list):
        L, R = sym.l_block(ths, p), sym.r_block(ths, p)
        for (a, c), (F, G) in (((i, j), (L, R)), ((j, i), (R, L))):
            q = pos[(a, c)]
            thg[gen.off_l[q]:gen.off_l[q] + F.size] = F.ravel()
            thg[gen.off_r[q]:gen.off_r[q] + G.size] = G.ravel()
    np.testing.assert_allclose(general.assemble_x(thg, gen), operator.assemble_xh(ths, sym), atol=1e-13)


def test_gradient_matches_finite_differences():
    nr, b, ns = 8, 4, 10
    g = synth.rng(3)
    lay = general.make_general_layout(nr, b, [2, 4, 1, 3], [False, True])
    Dh = synth.cn(g, (ns, nr))
    Uh = synth.cn(g, (ns, nr))
    th = _theta(lay, 4)
    gr = general.gradient(th, lay, Dh, Uh)
    h = 1e-6
    for e in list(range(0, lay.size, 3)):
        for unit in (1.0, 1j):
            d = np.zeros(lay.size, np.complex128)
            d[e] = unit * h
            fd = (general.misfit(th + d, lay, Dh, Uh) - general.misfit(th - d, lay, Dh, Uh)) / (2 * h)
            want = gr[e].real if unit == 1.0 else gr[e].imag
            assert fd == pytest.approx(want, rel=1e-6, abs=1e-8)


def test_admm_fixed_point_one_dense_tile():
    # N = 1, dense, general: f + lambda ||Z||^2 is Tikhonov least squares,
    # Z = (D^H D + 2 lambda I)^-1 D^H U; ADMM's fixed point is that minimiser
    nr, ns, lam = 6, 9, 0.2
    g = synth.rng(5)
    Dh = synth.cn(g, (ns, nr))
    Uh = synth.cn(g, (ns, nr))
    lay = general.make_general_layout(nr, nr, 0, "dense")
    prob = general.GeneralProblem(lay, Dh.T, Uh.T)
    opts = solver.SolveOpts(lam0=lam, decay=1.0, stages=1, rho=1.0, admm_iters=300, lbfgs_iters=30, memory=20)
    th, z, u, st = solver.admm(prob, np.zeros(lay.size, np.complex128), opts)
    Zc = np.linalg.solve(Dh.conj().T @ Dh + 2 * lam * np.eye(nr), Dh.conj().T @ Uh)
    assert np.linalg.norm(th.reshape(nr, nr) - Zc) <= 1e-6 * np.linalg.norm(Zc)
