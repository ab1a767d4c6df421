"""Differentiation form (nr = ns = 1024 on a 32 x 32 grid, 16 frequencies in the
workload; one frequency here): the autograd gradient against central complex
finite differences of the FP64 oracle (h = 1e-3) and the oracle's gradient,
then a solve with 30% of the sources dropped and 5 dB noise against the oracle."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from oracle import hilbert, layout, operator, solver, tlr
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from paper_2412_14973_gb300.autograd import misfit  # noqa: E402
from tests._gpu import Gpu, dev, rel  # noqa: E402

NX = NY = 32
B, K = 128, 12


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-3)])
def test_autograd_gradient_vs_finite_differences_and_oracle(prec, tol):
    D, U, perm, lay, _ = problem(NX, NY, B, K, "lowrank", seed=31, snr_db=5, planted=False)
    th = (0.3 * synth.planted_theta(lay.nr, B, K, lay.dense, 32)).astype(np.complex64).astype(np.complex128)
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    g = Gpu(D, U, lay, nx=NX, ny=NY, alpha=alpha, precision=prec)
    t = dev(th).requires_grad_(True)
    f = misfit(t, g.h)
    f.backward()
    grad = t.grad.detach().cpu().numpy().astype(np.complex128)
    Dt, Ut = Dh.T.copy(), Uh.T.copy()
    fo, go, _ = tlr.fgrad(th, lay, Dt, Ut)
    assert abs(f.item() - fo) <= tol * fo
    assert rel(grad, go) <= tol
    # central complex differences of the FP64 misfit on sampled entries
    fx = lambda x: 0.5 * float(np.vdot(tlr.apply(x, lay, Dt) - Ut, tlr.apply(x, lay, Dt) - Ut).real)  # noqa: E731
    h = 1e-3
    idx = synth.rng(5).choice(lay.size, 6, replace=False)
    scale = np.max(np.abs(go))
    for k in idx:
        e = np.zeros(lay.size)
        e[k] = h
        fd = (fx(th + e) - fx(th - e)) / (2 * h) + 1j * (fx(th + 1j * e) - fx(th - 1j * e)) / (2 * h)
        assert abs(fd - grad[k]) <= max(tol, 1e-5) * scale
    g.close()


def test_sparse_sampling_noisy_solve_matches_oracle():
    nr = NX * NY
    D, U, perm, lay, _ = problem(NX, NY, B, K, "lowrank", seed=33, snr_db=5)
    keep = synth.source_keep(nr, 0.7, 34)                    # 717 of 1024 sources
    D, U = np.ascontiguousarray(D[keep]), np.ascontiguousarray(U[keep])
    assert D.shape[0] == 717
    th0 = (0.1 * synth.planted_theta(nr, B, K, lay.dense, 35)).astype(np.complex64).astype(np.complex128)
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    tho, _, _, sto = solver.admm(solver.Problem(lay, Dh.T, Uh.T), th0)
    g = Gpu(D, U, lay, nx=NX, ny=NY, alpha=alpha, precision=T.TLR_PREC_BF16X3)
    th, st = g.solve(th0)
    g.close()
    assert st.iters == 30 and st.status == 0
    e = rel(operator.assemble_xh(th, lay), operator.assemble_xh(tho, lay))
    print(f"nr 1024 sparse-source noisy TC solve: rel X {e:.2e}")
    assert e <= 1e-3
