"""The persistent, double-buffered form of the packed tensor-core GEMM gives
bit for bit the results of the one-tile-per-CTA form: the same K chunks in
the same order into the same accumulators, only the scheduling differs.
Checked for every contraction class (TLR_MDD_PERSIST selects the classes
when a handle is created), both tensor-core formats, equal and unequal tiles,
applies, gradients and 30-iteration solves."""
import numpy as np
import pytest

import tlr_synth as synth
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu  # noqa: E402

CASES = {
    # name: (nx, ny, b, ranks, mode, ns, tiles)
    "equal": (16, 16, 64, 6, "lowrank", 300, None),
    "many_tiles": (32, 16, 32, 3, "lowrank", 130, None),
    "dense_mixed": (8, 8, 16, [3, 0, 16, 2, 1, 0, 4, 5, 2, 1], [False, True, True, False], 77, None),
    "unequal": (16, 8, None, 4, "lowrank", 90, [48, 16, 64]),
}


def _run(name, prec, mask, monkeypatch):
    nx, ny, b, ranks, mode, ns, tiles = CASES[name]
    D, U, perm, lay, _ = problem(nx, ny, b, ranks, mode, ns=ns, seed=7, snr_db=10, planted=False, tiles=tiles)
    th = (0.2 * synth.cn(synth.rng(8), lay.size)).astype(np.complex64).astype(np.complex128)
    monkeypatch.setenv("TLR_MDD_PERSIST", str(mask))
    g = Gpu(D, U, lay, nx=nx, ny=ny, precision=prec)
    Y = g.apply(th)
    f, gr = g.grad(th)
    ths, st = g.solve(th)
    g.close()
    return Y, f, gr, ths, st


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_persistent_kernel_is_bitwise_the_one_tile_kernel(name, prec, monkeypatch):
    ref = _run(name, prec, 0, monkeypatch)
    per = _run(name, prec, 7, monkeypatch)
    assert np.array_equal(ref[0], per[0])
    assert ref[1] == per[1] and np.array_equal(ref[2], per[2])
    assert np.array_equal(ref[3], per[3])
    assert per[4].iters == 30 and per[4].status == 0 and ref[4].f_hist[29] == per[4].f_hist[29]
