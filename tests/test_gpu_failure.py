"""Failure detection without a GPU fault: the tensor-core contraction kernels'
bounded barrier wait gives up on a barrier that nothing completes, records
TLR_ERR_TIMEOUT for the host, and the context stays usable."""
import numpy as np
import pytest

import paper_2412_14973_gb300 as T
import tlr_synth as synth
from oracle import operator

from _cases import problem
from _gpu import Gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_ms", [20, 150])
def test_bounded_wait_runs_out_and_the_context_stays_usable(limit_ms):
    status, waited = T.tlr_mdd_wait_selftest(limit_ms * 1_000_000)
    print(f"limit {limit_ms} ms: status {status}, waited {waited:.1f} ms")
    assert status == T.TLR_ERR_TIMEOUT
    assert limit_ms <= waited < limit_ms + 500
    # a tensor-core product right after it runs and is correct
    D, U, perm, lay, _ = problem(8, 8, 16, 3, "lowrank", ns=70, seed=7, snr_db=10, planted=False)
    Dh, _, alpha = operator.normalise(D, U, perm)
    g = Gpu(D, U, lay, nx=8, ny=8, alpha=alpha, precision=T.TLR_PREC_BF16X3)
    th = (0.2 * synth.cn(synth.rng(8), lay.size)).astype(np.complex64).astype(np.complex128)
    assert rel(g.apply(th), operator.apply_y(th, lay, Dh)) <= 1e-3
    g.close()
