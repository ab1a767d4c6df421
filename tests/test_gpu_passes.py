"""Launch shape of the fused update-and-pack passes: with their grid capped
(each CTA walking several tiles, the last ones ragged) every solve gives the
bits of the uncapped launch, in plain launches and in a recorded graph, in
both tensor-core precisions and on unequal tiles."""
import numpy as np
import pytest

import tlr_synth as synth
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu  # noqa: E402

CASES = [  # (nx, ny, b, rank, mode, ns, tiles)
    (32, 32, 128, 12, "lowrank", 717, None),
    (16, 8, None, 5, "rule", 90, [48, 16, 64]),
]


@pytest.fixture
def restore_cap():
    prev = T.tlr_mdd_set_pass_ctas(0)
    yield
    T.tlr_mdd_set_pass_ctas(prev)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_capped_pass_grid_is_bitwise_the_full_grid(prec, case, restore_cap):
    nx, ny, b, k, mode, ns, tiles = CASES[case]
    D, U, perm, lay, _ = problem(nx, ny, b, k, mode, ns=ns, seed=120 + case, snr_db=10, tiles=tiles)
    th0 = (0.2 * synth.cn(synth.rng(130 + case), lay.size)).astype(np.complex64).astype(np.complex128)
    out = {}
    for cap in (0, 7, 152):
        assert T.tlr_mdd_set_pass_ctas(cap) >= 0
        g = Gpu(D, U, lay, nx=nx, ny=ny, precision=prec)
        # the handle's first solve runs as plain launches, the second records
        # and replays its graph
        out[cap] = [g.solve(th0), g.solve(th0)]
        g.close()
    for cap in (7, 152):
        for (th_ref, st_ref), (th, st) in zip(out[0], out[cap]):
            assert st.status == 0 and st.iters == st_ref.iters == 30
            assert np.array_equal(th, th_ref)
            assert list(st.f_hist[:30]) == list(st_ref.f_hist[:30])


def test_negative_cap_is_rejected(restore_cap):
    with pytest.raises(T.TLRError):
        T.tlr_mdd_set_pass_ctas(-1)
