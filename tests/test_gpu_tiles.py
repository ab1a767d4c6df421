"""Non-uniform tile partitions (tile sizes d_i) on the GPU vs the oracle.

Block i of the Hilbert-ordered receivers holds d_i of them; tile (i, j) is
d_i x d_j with L_ij d_i x k and R_ij d_j x k.  Tolerances as for equal tiles:
1e-5 (FP32) and 1e-3 (tensor cores) relative per operator application, 1e-3
on the final X of a solve."""
import numpy as np
import pytest
import torch

import paper_2412_14973_gb300 as T
import tlr_synth as synth
from oracle import general, layout, operator, solver, warmstart

from _cases import problem
from _gpu import Gpu, dev, elem, host, rel

pytestmark = pytest.mark.gpu

CASES = {
    # name: (nx, ny, tiles, ranks (diagonal, then pairs) or int, dense diagonal flags, ns)
    "ragged4": (16, 16, [48, 80, 16, 112], 9, [False, True, False, False], 203),
    "mixed": (12, 8, [40, 8, 31, 17], [5, 8, 0, 17] + [8, 0, 17, 3, 8, 6], [False, False, True, False], 77),
    "big_small": (8, 8, [60, 4], [3, 4, 4], [False, False], 64),
    "many_tc_tiles": (32, 32, [200, 312, 128, 384], 24, [False, False, True, False], 1024),
    # a one-receiver tile (ranks 0 and 1 only), a dense 1 x 1 diagonal, k = 0 pairs
    "unit_tile": (4, 4, [1, 9, 1, 5], [1, 3, 1, 2] + [1, 0, 1, 0, 3, 1], [False, False, True, False], 37),
}
PRECS = [(T.TLR_PREC_FP32, 1e-5), (T.TLR_PREC_BF16X3, 1e-3)]
# per-application bounds of the apply / gradient tests, TF32 included; every
# element within ETOL of the reference's rms
APPLY_PRECS = PRECS + [(T.TLR_PREC_TF32, 1e-3)]
ETOL = {T.TLR_PREC_FP32: 1e-4, T.TLR_PREC_BF16X3: 1e-3, T.TLR_PREC_TF32: 1e-2}


def _setup(name, prec, seed=0):
    nx, ny, tiles, ranks, dense, ns = CASES[name]
    D, U, perm, lay, _ = problem(nx, ny, None, ranks, dense, ns=ns, seed=40 + seed, snr_db=10, planted=False,
                                 tiles=tiles)
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    g = Gpu(D, U, lay, nx=nx, ny=ny, alpha=alpha, precision=prec)
    th = (0.2 * synth.cn(synth.rng(45 + seed), lay.size)).astype(np.complex64).astype(np.complex128)
    return g, lay, th, Dh, Uh, perm


@pytest.mark.parametrize("prec,tol", APPLY_PRECS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_apply_grad_unpermute(name, prec, tol):
    g, lay, th, Dh, Uh, perm = _setup(name, prec)
    Y = g.apply(th)
    Yo = operator.apply_y(th, lay, Dh)
    f, gr = g.grad(th)
    fo = operator.misfit(th, lay, Dh, Uh)
    go = operator.gradient(th, lay, Dh, Uh)
    X = g.unpermute(th)
    Xo = operator.unpermute(operator.assemble_xh(th, lay), perm)
    print(f"tiles {name} prec {prec}: apply {rel(Y, Yo):.2e} grad {rel(gr, go):.2e} f {abs(f - fo) / fo:.2e}")
    assert rel(Y, Yo) <= tol
    assert rel(gr, go) <= tol and abs(f - fo) <= tol * fo
    assert elem(Y, Yo) <= ETOL[prec] and elem(gr, go) <= ETOL[prec]
    assert rel(X, Xo) <= 1e-5
    assert np.array_equal(X, X.T)
    g.close()


@pytest.mark.parametrize("prec", [T.TLR_PREC_FP32, T.TLR_PREC_BF16X3])
@pytest.mark.parametrize("name", ["mixed", "ragged4"])
def test_solve_matches_oracle(name, prec):
    # ragged4's tiles are multiples of 16: the tensor-core solve takes the
    # fused residual step there; mixed's are not
    g, lay, th, Dh, Uh, perm = _setup(name, prec, seed=3)
    th0 = 0.5 * th
    ths, st = g.solve(th0)
    tho, _, _, sto = solver.admm(solver.Problem(lay, Dh.T, Uh.T), th0)
    e = rel(operator.assemble_xh(ths, lay), operator.assemble_xh(tho, lay))
    print(f"tiles solve {name} prec {prec}: rel X {e:.2e}, f {st.f_hist[st.n_hist - 1]:.4e} vs {sto.f_hist[-1]:.4e}")
    assert st.iters == 30 and st.status == 0
    assert e <= 1e-3
    g.close()


@pytest.mark.parametrize("prec", [T.TLR_PREC_FP32, T.TLR_PREC_BF16X3])
def test_explicit_equal_tiles_are_the_uniform_partition(prec):
    # tiles = [b] * N takes exactly the uniform path: bitwise equal results
    D, U, perm, lay, _ = problem(8, 8, 16, 3, "lowrank", ns=70, seed=5, snr_db=10, planted=False)
    th = (0.2 * synth.cn(synth.rng(6), lay.size)).astype(np.complex64)
    out = []
    for tiles in (None, [16] * 4):
        d = T.desc(64, 70, 16, rank=3, nx=8, ny=8, diag_mode=T.TLR_DIAG_LOWRANK, precision=prec, tiles=tiles)
        g = Gpu(D, U, lay, desc=d)
        out.append((g.apply(th), g.grad(th)))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1][0] == out[1][1][0] and np.array_equal(out[0][1][1], out[1][1][1])


@pytest.mark.parametrize("prec,tol", PRECS)
def test_general_form_on_nonuniform_tiles(prec, tol):
    tiles, dense = [20, 36, 8], [False, True, False]
    n = len(tiles)
    rl = [4, 9, 8] + [min(tiles[i], tiles[j], 3 + i + 2 * j) for (i, j) in general.ordered_pairs(n)]
    glay = general.make_general_layout(64, None, rl, dense, tiles=tiles)
    D, U, perm, _, _ = problem(8, 8, 16, 1, "lowrank", ns=90, seed=91, snr_db=10)
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    d = T.desc(64, 90, 0, ranks=rl, nx=8, ny=8, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=dense,
               precision=prec, reciprocity=T.TLR_RECIP_NONE, tiles=tiles, alpha=alpha)
    g = Gpu(D, U, glay, desc=d)
    th = (0.2 * synth.cn(synth.rng(92), glay.size)).astype(np.complex64).astype(np.complex128)
    Y = g.apply(th)
    f, gr = g.grad(th)
    X = g.unpermute(th)
    assert rel(Y, general.apply_y(th, glay, Dh)) <= tol
    go, fo = general.gradient(th, glay, Dh, Uh), general.misfit(th, glay, Dh, Uh)
    assert rel(gr, go) <= tol and abs(f - fo) <= tol * fo
    assert rel(X, operator.unpermute(general.assemble_x(th, glay), perm)) <= 1e-5
    if prec == T.TLR_PREC_FP32:
        ths, st = g.solve(0.5 * th)
        tho, _, _, _ = solver.admm(general.GeneralProblem(glay, Dh.T, Uh.T), 0.5 * th)
        assert st.iters == 30 and st.status == 0
        assert rel(general.assemble_x(ths, glay), general.assemble_x(tho, glay)) <= 1e-3
    g.close()


def test_warm_start_on_unequal_tiles_matches_oracle():
    # a random complex symmetric X on tiles 48, 80, 16, 112: every kept tile is
    # its truncated SVD (wide tiles, e.g. 16 x 80, run the SVD on their
    # transpose), dense diagonals copied.  Bound as for equal tiles: 1e-3
    # (FP32 Jacobi to 1e-5 orthogonality; a starting point)
    tiles = [48, 80, 16, 112]
    nr = sum(tiles)
    g = synth.rng(70)
    A = synth.cn(g, (nr, nr))
    X = A + A.T
    ks = [11, 0, 3, 27] + [13, 4, 30, 9, 41, 2]
    lay = layout.make_layout(nr, None, ks, [False, True, False, False], tiles=tiles)
    D = synth.make_d(nr, nr, 1, 3)[0]
    gp = Gpu(D, D, lay, nx=16, ny=16)
    th = torch.zeros(lay.size, dtype=torch.complex64, device="cuda")
    T.tlr_mdd_warm_start(gp.h, dev(X), th)
    Xg = operator.assemble_xh(host(th), lay)
    Xo = operator.assemble_xh(warmstart.warm_start(X, lay), lay)
    err = rel(Xg, Xo)
    print(f"unequal tiles: |X_h(warm, GPU) - X_h(warm, oracle)| = {err:.2e}")
    assert err <= 1e-3
    gp.close()
