"""The allocation-free dense adjoint (tlr_mdd_adjoint_noalloc) against the
handle's adjoint (tlr_mdd_adjoint) and the oracle.

tlr_mdd_adjoint_noalloc serves callers that cannot allocate device memory
(their process gives all device memory to its own pool allocator, or an
allocation on their path may synchronise the device).  It keeps its split-K
scratch in a fixed array inside the library, so this file checks that two
calls in a row, sharing that array, both reproduce the allocating entry point.
Collected last so that a failure here does not hide any other test."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from oracle import operator
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu, dev, host, rel  # noqa: E402

TOL = 1e-5   # the FP32 per-operator tolerance used by the other GPU tests


@pytest.mark.parametrize("nx,ny,b,k,ns", [(16, 16, 64, 8, 300), (16, 8, 32, 4, 4096)])
def test_noalloc_adjoint_matches_allocating_adjoint_on_two_calls(nx, ny, b, k, ns):
    D, U, perm, lay, _ = problem(nx, ny, b, k, "lowrank", ns=ns, snr_db=10, planted=False)
    g = Gpu(D, U, lay, nx=nx, ny=ny)
    _, alpha, Dt, _ = g.data()
    nr = lay.nr
    V = synth.cn(synth.rng(5), (nr, ns)).astype(np.complex64)
    G_ref = g.adjoint(V)
    Vd, Dtd = dev(V), dev(Dt)
    outs = []
    for _ in range(2):
        Gd = torch.full((nr, nr), float("nan"), dtype=torch.complex64, device="cuda")
        T.tlr_mdd_adjoint_noalloc(Vd, Dtd, nr, ns, Gd)
        outs.append(host(Gd))
    g.close()
    for G in outs:
        assert np.all(np.isfinite(G))
        assert rel(G, G_ref) <= TOL
    assert np.array_equal(outs[0], outs[1])
    Dh, _, _ = operator.normalise(D, U, perm, alpha=alpha)
    assert rel(outs[1], operator.adjoint_g(V.astype(np.complex128), Dh)) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    nr_max = int((T.TLR_NOALLOC_SCRATCH_BYTES - 256) // 8) ** 0.5
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_adjoint_noalloc(x, x, int(nr_max) + 1, 16, x)
    assert ei.value.code == -2
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_adjoint_noalloc(None, x, 4, 4, x)
    assert ei.value.code == -1
