"""General (non-reciprocal) TLR form (reciprocity NONE) on the GPU vs the oracle.

Every tile is free (X_ij = L_ij R_ij^T for all i != j, diagonal tiles L R^T
or dense Z); the library evaluates it with separate expand-side and
compress-side factor panels.  Tolerances as for the reciprocal form: 1e-5
(FP32) and 1e-3 (tensor cores) per operator application, 1e-3 on the final X
of a solve."""
import numpy as np
import pytest
import torch

import paper_2412_14973_gb300 as T
import tlr_synth as synth
from oracle import general, operator, solver

from _cases import problem
from _gpu import Gpu, dev, elem, host, rel

pytestmark = pytest.mark.gpu

CASES = {
    # name: (nx, ny, b, ranks (diagonal, then ordered pairs) or int, dense diagonal flags, ns)
    "lowrank": (8, 8, 16, 3, [False] * 4, 70),
    "mixed": (8, 8, 16, [2, 0, 16, 5] + [(3 * k + 1) % 7 for k in range(12)], [False, False, True, False], 64),
    "ragged": (12, 8, 32, 4, [False, True, False], 203),
}
PRECS = [(T.TLR_PREC_FP32, 1e-5), (T.TLR_PREC_BF16X3, 1e-3)]
# per-application bounds of the apply / gradient tests, TF32 included; every
# element within ETOL of the reference's rms
APPLY_PRECS = PRECS + [(T.TLR_PREC_TF32, 1e-3)]
ETOL = {T.TLR_PREC_FP32: 1e-4, T.TLR_PREC_BF16X3: 1e-3, T.TLR_PREC_TF32: 1e-2}


def _setup(name, prec, seed=0):
    nx, ny, b, ranks, dense, ns = CASES[name]
    nr = nx * ny
    n = nr // b
    rl = ranks if isinstance(ranks, list) else [ranks] * (n + n * (n - 1))
    glay = general.make_general_layout(nr, b, rl, dense)
    D, U, perm, _, _ = problem(nx, ny, b, 1, "lowrank", ns=ns, seed=90 + seed, snr_db=10)
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    d = T.desc(nr, ns, b, ranks=rl, nx=nx, ny=ny, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=dense,
               precision=prec, reciprocity=T.TLR_RECIP_NONE, alpha=alpha)
    g = Gpu(D, U, glay, desc=d)
    th = (0.2 * synth.cn(synth.rng(95 + seed), glay.size)).astype(np.complex64).astype(np.complex128)
    return g, glay, th, Dh, Uh, perm


@pytest.mark.parametrize("prec,tol", APPLY_PRECS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_general_apply_grad_assemble(name, prec, tol):
    g, glay, th, Dh, Uh, perm = _setup(name, prec)
    Y = g.apply(th)
    Yo = general.apply_y(th, glay, Dh)
    f, gr = g.grad(th)
    fo = general.misfit(th, glay, Dh, Uh)
    go = general.gradient(th, glay, Dh, Uh)
    X = g.unpermute(th)
    Xo = operator.unpermute(general.assemble_x(th, glay), perm)
    print(f"general {name} prec {prec}: apply {rel(Y, Yo):.2e} grad {rel(gr, go):.2e} f {abs(f - fo) / fo:.2e}")
    assert rel(Y, Yo) <= tol
    assert rel(gr, go) <= tol and abs(f - fo) <= tol * fo
    assert elem(Y, Yo) <= ETOL[prec] and elem(gr, go) <= ETOL[prec]
    assert rel(X, Xo) <= 1e-5
    assert not np.allclose(X, X.T)
    g.close()


@pytest.mark.parametrize("prec", [T.TLR_PREC_FP32, T.TLR_PREC_BF16X3])
def test_general_solve_matches_oracle(prec):
    g, glay, th, Dh, Uh, perm = _setup("mixed", prec, seed=3)
    th0 = 0.5 * th
    ths, st = g.solve(th0)
    prob = general.GeneralProblem(glay, Dh.T, Uh.T)
    tho, _, _, sto = solver.admm(prob, th0)
    e = rel(general.assemble_x(ths, glay), general.assemble_x(tho, glay))
    print(f"general solve prec {prec}: rel X {e:.2e}, f {st.f_hist[st.n_hist - 1]:.4e} vs {sto.f_hist[-1]:.4e}")
    assert st.iters == 30 and st.status == 0
    assert e <= 1e-3
    g.close()


@pytest.mark.parametrize("tiles", [None, [20, 36, 8]])
def test_general_warm_start_matches_oracle(tiles):
    # a random (non-symmetric) X: every kept tile, diagonal ones included, is
    # its truncated SVD L R^T; dense diagonals copied.  Bound 1e-3 as for the
    # reciprocal warm start
    nr, b = 64, 16
    ts = tiles or [b] * (nr // b)
    n = len(ts)
    X = synth.cn(synth.rng(80), (nr, nr))
    dense = [False, True] + [False] * (n - 2)
    rl = [min(3, ts[i]) for i in range(n)] + [min(ts[i], ts[j], 1 + (2 * i + j) % 5)
                                             for (i, j) in general.ordered_pairs(n)]
    glay = general.make_general_layout(nr, None if tiles else b, rl, dense, tiles=tiles)
    D = synth.make_d(nr, nr, 1, 4)[0]
    d = T.desc(nr, nr, 0 if tiles else b, ranks=rl, nx=8, ny=8, diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=dense,
               reciprocity=T.TLR_RECIP_NONE, tiles=tiles)
    g = Gpu(D, D, glay, desc=d)
    th = torch.zeros(glay.size, dtype=torch.complex64, device="cuda")
    T.tlr_mdd_warm_start(g.h, dev(X), th)
    Xg = general.assemble_x(host(th), glay)
    Xo = general.assemble_x(general.warm_start(X, glay), glay)
    err = rel(Xg, Xo)
    print(f"general warm start, tiles {ts}: rel {err:.2e}")
    assert err <= 1e-3
    g.close()
