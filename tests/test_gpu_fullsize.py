"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The batched workload, nr = ns = 4096 (64 x 64 grid), tile 256, ranks 4 and 48, low-rank
diagonals: sampled columns of Y = X_h Dfrak and the full gradient against the
FP64 oracle's TLR-structured forms, on both paths.
The large workload, nr = ns = 9216 (96 x 96 grid), tile 384, rank 64: sampled columns
of Y on the tensor-core path, and the adjoint identity <X Dfrak, V> =
<X, V Dfrak^H> with the GPU's own products at full size.
Inputs: complex Gaussian D (the operator parity does not depend on D's
spectrum) to keep the host-side generation fast; seeded."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from oracle import hilbert, layout, operator, tlr

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu, rel  # noqa: E402


def _big(nx, ny, b, k, seed):
    nr = nx * ny
    lay = layout.make_layout(nr, b, k, "rule")
    D = (synth.cn(synth.rng(seed), (nr, nr)) / np.sqrt(nr)).astype(np.complex64)
    U = (synth.cn(synth.rng(seed + 1), (nr, nr)) / np.sqrt(nr)).astype(np.complex64)
    th = synth.planted_theta(nr, b, k, lay.dense, seed + 2).astype(np.complex64).astype(np.complex128)
    return D, U, lay, th


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-4)])
@pytest.mark.parametrize("k", [4, 48])
def test_nr4096_tile256_columns_and_full_gradient(prec, tol, k):
    D, U, lay, th = _big(64, 64, 256, k, 100 + k)
    g = Gpu(D, U, lay, nx=64, ny=64, precision=prec)
    perm, alpha, Dt, Ut = g.data()
    Y = g.apply(th)
    cols = synth.rng(7).choice(lay.nr, 24, replace=False)
    Dto, Uto = Dt.astype(np.complex128), Ut.astype(np.complex128)
    Yo = tlr.apply(th, lay, Dto[:, cols])
    assert rel(Y[:, cols], Yo) <= tol
    f, gr = g.grad(th)
    fo, go, _ = tlr.fgrad(th, lay, Dto, Uto)
    assert abs(f - fo) <= tol * fo
    assert rel(gr, go) <= tol
    g.close()


def test_nr9216_tile384_columns_tensor_core():
    D, U, lay, th = _big(96, 96, 384, 64, 300)
    g = Gpu(D, U, lay, nx=96, ny=96, precision=T.TLR_PREC_BF16X3)
    perm, alpha, Dt, Ut = g.data()
    assert np.array_equal(perm, hilbert.perm(96, 96))
    Y = g.apply(th)
    cols = synth.rng(9).choice(lay.nr, 8, replace=False)
    Yo = tlr.apply(th, lay, Dt.astype(np.complex128)[:, cols])
    assert rel(Y[:, cols], Yo) <= 1e-4
    # adjoint identity with the GPU's own products: <Y, V> = <X_h, V Dfrak^H>
    V = synth.cn(synth.rng(10), (lay.nr, lay.nr)).astype(np.complex64)
    G = g.adjoint(V)
    Xh = torch.from_numpy(operator.assemble_xh(th, lay).astype(np.complex64)).cuda()
    lhs = np.vdot(Y, V.astype(np.complex128))
    rhs = torch.vdot(Xh.flatten().to(torch.complex128), torch.from_numpy(G).cuda().flatten()).item()
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    g.close()
