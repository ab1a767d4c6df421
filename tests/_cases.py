"""Small seeded problems shared by the oracle and GPU tests (test helper)."""
import numpy as np

import tlr_synth as synth
from oracle import hilbert, layout, operator


def problem(nx, ny, b, ranks, mode, ns=None, seed=0, snr_db=None, planted=True, tiles=None):
    """D, U (paper layout, complex64), perm, layout, planted theta (complex128).

    U = D X + noise is composed by the oracle from the planted factors
    (X = S X_h S^T, eq. 11) in FP64 and cast once to complex64.  ``tiles``:
    block sizes of a non-uniform partition (``b`` is then ignored).
    """
    nr = nx * ny
    ns = nr if ns is None else ns
    lay = layout.make_layout(nr, b, ranks, mode, tiles=tiles)
    D = synth.make_d(ns, nr, 1, seed)[0]
    perm = hilbert.perm(nx, ny)
    th = synth.planted_theta(nr, b, ranks, lay.dense, seed + 1, tiles=tiles)
    X = operator.unpermute(operator.assemble_xh(th, lay), perm)
    U = D.astype(np.complex128) @ X
    if snr_db is not None:
        n = synth.noise(U.shape, seed + 2)
        scale = np.linalg.norm(U) / np.linalg.norm(n) * 10 ** (-snr_db / 20)
        U = U + scale * n
    if not planted:
        th = synth.planted_theta(nr, b, ranks, lay.dense, seed + 3, tiles=tiles)
    return D, U.astype(np.complex64), perm, lay, th
