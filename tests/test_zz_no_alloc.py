"""The allocation-free dense adjoint (tlr_mdd_adjoint_noalloc) against the
handle's adjoint (tlr_mdd_adjoint) and the oracle.

tlr_mdd_adjoint_noalloc serves callers that cannot allocate device memory
(their process gives all device memory to its own pool allocator, or an
allocation on their path may synchronise the device).  It keeps its split-K
scratch in a fixed array inside the library, so this file checks that two
calls in a row, sharing that array, both reproduce the allocating entry point:
with the split count set by the work (nr = 256), by the array's size (nr =
1024, ns = 2048: two partial slabs fit where five are wanted) and at the
largest accepted size (nr = 1448: one slab fills the array).
Its input panel Dt is built on the host from D by the library's stated
storage rounding (each part of D[s, perm[a]] divided by alpha in IEEE FP32;
bit-exact against the handle's own panel, tests/test_gpu_data.py), not read
back from the GPU.
Collected last so that a failure here does not hide any other test."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from oracle import layout, operator
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu, dev, host, rel  # noqa: E402

TOL = 1e-5   # the FP32 per-operator tolerance used by the other GPU tests


def _panel32(D, perm, alpha):
    """Dfrak = (D[:, perm] / alpha)^T, each part one IEEE FP32 division."""
    a32 = np.float32(alpha)
    Dp = D[:, perm]
    re = np.ascontiguousarray(Dp.real, dtype=np.float32) / a32
    im = np.ascontiguousarray(Dp.imag, dtype=np.float32) / a32
    return np.ascontiguousarray((re + 1j * im).astype(np.complex64).T)


def _check(D, U, perm, lay, nx, ny, ns, seed):
    Dh, _, alpha = operator.normalise(D, U, perm)
    g = Gpu(D, U, lay, nx=nx, ny=ny, alpha=alpha)
    nr = lay.nr
    V = synth.cn(synth.rng(seed), (nr, ns)).astype(np.complex64)
    G_ref = g.adjoint(V)
    Vd, Dtd = dev(V), dev(_panel32(D, perm, alpha))
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
    assert rel(outs[1], operator.adjoint_g(V.astype(np.complex128), Dh)) <= TOL


@pytest.mark.parametrize("nx,ny,b,k,ns", [(16, 16, 64, 8, 300), (16, 8, 32, 4, 4096), (32, 32, 128, 4, 2048)])
def test_noalloc_adjoint_matches_allocating_adjoint_on_two_calls(nx, ny, b, k, ns):
    D, U, perm, lay, _ = problem(nx, ny, b, k, "lowrank", ns=ns, snr_db=10, planted=False)
    _check(D, U, perm, lay, nx, ny, ns, 5)


def test_noalloc_adjoint_at_the_largest_accepted_size():
    # nr = 1448 = 8 x 181: nr^2 complex64 values fill the array (one slab)
    nx, ny, ns = 8, 181, 300
    nr = nx * ny
    assert nr * nr * 8 <= T.TLR_NOALLOC_SCRATCH_BYTES - 256 < (nr + 1) ** 2 * 8
    lay = layout.make_layout(nr, 181, 2, "lowrank")
    from oracle import hilbert
    D = synth.cn(synth.rng(61), (ns, nr)).astype(np.complex64)
    U = synth.cn(synth.rng(62), (ns, nr)).astype(np.complex64)
    _check(D, U, hilbert.perm(nx, ny), lay, nx, ny, ns, 63)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    nr_max = int(((T.TLR_NOALLOC_SCRATCH_BYTES - 256) // 8) ** 0.5)
    # raw device pointers skip the binding's size checks: the library itself
    # refuses nr above its scratch before any work is enqueued
    p = x.data_ptr()
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_adjoint_noalloc(p, p, nr_max + 1, 16, p)
    assert ei.value.code == T.TLR_ERR_SHAPE
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_adjoint_noalloc(None, x, 4, 4, x)
    assert ei.value.code == T.TLR_ERR_ARG
    # a host buffer is refused by the library's device check
    h = torch.zeros(16, dtype=torch.complex64)
    with pytest.raises(T.TLRError) as ei:
        T.tlr_mdd_adjoint_noalloc(p, h.data_ptr(), 2, 2, p)
    assert ei.value.code == T.TLR_ERR_ARG
