"""Benchmark solver of eq. (4) on the GPU against the oracle's CG (FP64).

The oracle normalises D, U itself (its own Hilbert order and alpha = max |D|)
and passes that alpha to the library, so no oracle input comes from the GPU.
"""
import numpy as np
import pytest
import torch

import paper_2412_14973_gb300 as T
import tlr_synth as synth
from oracle import benchmark, layout, operator

from _cases import problem
from _gpu import Gpu, dev, host, rel

pytestmark = pytest.mark.gpu

PRECS = [(T.TLR_PREC_FP32, 1e-4), (T.TLR_PREC_BF16X3, 1e-3)]


def _oracle(D, U, perm, lam, maxit, tol):
    Dh, Uh, _ = operator.normalise(D, U, perm)
    Z = benchmark.solve_eq4(Dh, Uh, lam, tol=tol, maxit=maxit)
    return 0.5 * (Z + Z.T)


def _alpha(D):
    return float(np.max(np.abs(D.astype(np.complex128))))


@pytest.mark.parametrize("prec,tol", PRECS)
def test_converged_solution_matches_oracle(prec, tol):
    # nr = 96 (12 x 8 grid), ns = 120: one ragged 128-row tile on the tensor cores
    D, U, perm, lay, _ = problem(12, 8, 16, 3, "lowrank", ns=120, seed=21, snr_db=10)
    g = Gpu(D, U, lay, nx=12, ny=8, alpha=_alpha(D), precision=prec)
    X, st = g.benchmark(0.3, 400, 1e-6)
    Xo = _oracle(D, U, perm, 0.3, 10000, 1e-13)
    err = rel(X, Xo)
    print(f"precision {prec}: iterations {st.iters}, rel. residual {st.rel_res:.2e}, |X - X_oracle| {err:.2e}")
    assert st.status == 0 and st.rel_res <= 1e-6 * 1.01
    assert err <= tol
    np.testing.assert_array_equal(X, X.T)   # the iterates stay exactly symmetric


def test_fixed_iterations_follow_the_oracle_trajectory():
    # three CG iterations from Z = 0 on both sides: the iterates, not only the
    # fixed point, agree
    D, U, perm, lay, _ = problem(8, 8, 16, 2, "lowrank", ns=64, seed=22, snr_db=20)
    g = Gpu(D, U, lay, nx=8, ny=8, alpha=_alpha(D))
    for it in (1, 3):
        X, st = g.benchmark(0.05, it, 0.0)
        Xo = _oracle(D, U, perm, 0.05, it, 0.0)
        assert st.iters == it
        assert rel(X, Xo) <= 1e-5


def test_unitary_data_converge_in_one_iteration_tensor_cores():
    # nr = ns = 1024 with a unitary D and alpha = 1: the normal operator is
    # (1 + 2 lambda) I on symmetric matrices, so one CG step gives
    # X = P(D^H U) / (1 + 2 lambda) (in Hilbert order)
    nx = ny = 32
    nr = nx * ny
    lay = layout.make_layout(nr, 128, 4, "lowrank")
    gen = synth.rng(23)
    D = synth.phase_dft_unitary(nr, gen).astype(np.complex64)
    U = synth.cn(gen, (nr, nr)).astype(np.complex64)
    g = Gpu(D, U, lay, nx=nx, ny=ny, alpha=1.0, precision=T.TLR_PREC_BF16X3)
    lam = 0.25
    X, st = g.benchmark(lam, 5, 1e-5)
    from oracle import hilbert
    p = hilbert.perm(nx, ny)
    Dh, Uh = D[:, p].astype(np.complex128), U[:, p].astype(np.complex128)    # alpha = 1
    B = Dh.conj().T @ Uh
    Xc = 0.5 * (B + B.T) / (1.0 + 2.0 * lam)
    print(f"iterations {st.iters}, rel. residual {st.rel_res:.2e}, |X - X_closed| {rel(X, Xc):.2e}")
    assert st.iters <= 2
    assert rel(X, Xc) <= 1e-3


def test_zero_iterations_and_invalid_arguments():
    D, U, perm, lay, _ = problem(4, 4, 4, 1, "lowrank", seed=24)
    g = Gpu(D, U, lay, nx=4, ny=4)
    X, st = g.benchmark(0.1, 0, 0.0)
    assert st.iters == 0 and not np.any(X)
    Xd = torch.empty((16, 16), dtype=torch.complex64, device="cuda")
    for lam, it, tol in ((-1.0, 3, 0.0), (float("nan"), 3, 0.0), (0.1, -1, 0.0), (0.1, 3, -1.0)):
        with pytest.raises(T.TLRError) as e:
            T.tlr_mdd_benchmark_solve(g.h, lam, it, tol, Xd)
        assert e.value.code == T.TLR_ERR_ARG
    with pytest.raises(T.TLRError):
        T.tlr_mdd_benchmark_solve(g.h, 0.1, 3, 0.0, None)
