"""Hilbert order, alpha and the reordered panels on the GPU vs the oracle (bit-exact)."""
import numpy as np
import pytest
import torch

import tlr_synth as synth
from oracle import hilbert, layout, operator
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu  # noqa: E402


def _div32(z, a32):
    """Part-wise IEEE FP32 division of a complex64 array by a float32."""
    re = np.ascontiguousarray(z.real, dtype=np.float32) / a32
    im = np.ascontiguousarray(z.imag, dtype=np.float32) / a32
    return (re + 1j * im).astype(np.complex64)


@pytest.mark.parametrize("nx,ny", [(1, 1), (16, 16), (64, 32), (5, 3), (177, 90), (96, 96), (128, 64), (7, 33)])
def test_hilbert_perm_bit_exact(nx, ny):
    p = torch.empty(nx * ny, dtype=torch.int32, device="cuda")
    T.tlr_mdd_hilbert_perm(nx, ny, p)
    torch.cuda.synchronize()
    assert np.array_equal(p.cpu().numpy(), hilbert.perm(nx, ny))


@pytest.mark.parametrize("host_inputs", [False, True])
def test_panels_bit_exact(host_inputs):
    D, U, perm, lay, _ = problem(8, 8, 16, 3, "rule", ns=45, snr_db=10)
    a_or = float(np.max(np.abs(D.astype(np.complex128))))
    # explicit alpha: each part of Dfrak = D[:, perm]^T is one IEEE FP32 division by
    # alpha rounded to FP32 (the library's stated storage rounding).  numpy's
    # complex / real divides by multiplying with a rounded reciprocal, so the
    # reference divides the real and imaginary parts as float32 arrays.
    g = Gpu(D, U, lay, nx=8, ny=8, alpha=a_or, host_inputs=host_inputs)
    p, alpha, Dt, Ut = g.data()
    assert np.array_equal(p, perm)
    assert alpha == a_or
    a32 = np.float32(a_or)
    assert np.array_equal(Dt, _div32(D[:, perm], a32).T)
    assert np.array_equal(Ut, _div32(U[:, perm], a32).T)
    # and within one FP32 rounding of the FP64 normalisation of the oracle
    Dh, Uh, _ = operator.normalise(D, U, perm, alpha=a_or)
    assert np.max(np.abs(Dt - Dh.T)) <= 2 * np.finfo(np.float32).eps * np.max(np.abs(Dh))
    g.close()
    # alpha computed on the device: max |D| (FP64 from the complex64 entries)
    g2 = Gpu(D, U, lay, nx=8, ny=8)
    _, alpha2, _, _ = g2.data()
    assert abs(alpha2 - a_or) <= 1e-15 * a_or
    g2.close()


def test_explicit_perm_and_ragged_sizes():
    rng = np.random.default_rng(3)
    nr, ns = 48, 37
    lay = layout.make_layout(nr, 16, 2, "lowrank")
    D = synth.cn(synth.rng(1), (ns, nr)).astype(np.complex64)
    U = synth.cn(synth.rng(2), (ns, nr)).astype(np.complex64)
    perm = rng.permutation(nr).astype(np.int32)
    g = Gpu(D, U, lay, perm=perm, alpha=3.0)
    p, alpha, Dt, Ut = g.data()
    assert np.array_equal(p, perm)
    assert np.array_equal(Dt, _div32(D[:, perm], np.float32(3.0)).T)
    g.close()


def test_invalid_inputs_are_errors_not_faults():
    D = np.zeros((4, 16), np.complex64)
    lay = layout.make_layout(16, 4, 1, "lowrank")
    with pytest.raises(T.TLRError) as ei:
        Gpu(D, D, lay, nx=3, ny=5)            # nx*ny != nr
    assert ei.value.code == -2
    with pytest.raises(T.TLRError) as ei:
        Gpu(D, D, lay, perm=[0] * 16)         # not a permutation
    assert ei.value.code == -1
