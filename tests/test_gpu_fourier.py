"""Time <-> frequency stacks on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import paper_2412_14973_gb300 as T
import tlr_synth as synth
from oracle import fourier

pytestmark = pytest.mark.gpu


def _traces(ntr, nt, seed):
    g = synth.rng(seed)
    return g.standard_normal((ntr, nt)).astype(np.float32)


@pytest.mark.parametrize("ntr,nt,f0,nf", [(300, 100, 3, 20), (257, 1125, 0, 563), (70000, 1125, 10, 200)])
def test_forward_stack_matches_oracle(ntr, nt, f0, nf):
    # nt = 1125: 4.5 s at 4 ms as in the examples; 70000 traces take three
    # chunks (the last one short)
    x = _traces(ntr, nt, 92 + nt)
    xd = torch.from_numpy(x).cuda()
    S = torch.empty((nf, ntr), dtype=torch.complex64, device="cuda")
    T.tlr_mdd_time_to_freq(xd, ntr, nt, f0, nf, S)
    So = fourier.time_to_freq(x, f0, nf)
    Sg = S.cpu().numpy().astype(np.complex128)
    err = np.abs(Sg - So).max() / np.abs(So).max()
    print(f"ntr {ntr}, nt {nt}: max error {err:.2e}")
    assert err <= 1e-5


@pytest.mark.parametrize("nt", [64, 1125])
def test_inverse_and_round_trip(nt):
    ntr = 500
    x = _traces(ntr, nt, 93)
    xd = torch.from_numpy(x).cuda()
    nh = nt // 2 + 1
    S = torch.empty((nh, ntr), dtype=torch.complex64, device="cuda")
    T.tlr_mdd_time_to_freq(xd, ntr, nt, 0, nh, S)
    y = torch.empty_like(xd)
    T.tlr_mdd_freq_to_time(S, ntr, nt, 0, nh, y)
    assert np.abs(y.cpu().numpy() - x).max() <= 1e-5 * np.abs(x).max()
    # band-limited inverse vs the oracle's
    f0, nf = 5, nt // 4
    Sb = S[f0:f0 + nf].contiguous()
    T.tlr_mdd_freq_to_time(Sb, ntr, nt, f0, nf, y)
    yo = fourier.freq_to_time(Sb.cpu().numpy(), nt, f0)
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-5 * np.abs(yo).max()


def test_stack_alpha_and_invalid_arguments():
    g = synth.rng(94)
    D = (g.standard_normal((7, 30, 40)) + 1j * g.standard_normal((7, 30, 40))).astype(np.complex64)
    a = T.tlr_mdd_stack_alpha(torch.from_numpy(D).cuda(), D.size)
    assert a == pytest.approx(fourier.stack_alpha(D.astype(np.complex128)), rel=1e-7)
    x = torch.zeros((10, 16), dtype=torch.float32, device="cuda")
    S = torch.zeros((9, 10), dtype=torch.complex64, device="cuda")
    for ntr, nt, f0, nf in ((10, 16, 0, 10), (10, 16, -1, 2), (0, 16, 0, 2), (10, 16, 3, 0)):
        with pytest.raises(T.TLRError) as e:
            T.tlr_mdd_time_to_freq(x, ntr, nt, f0, nf, S)
        assert e.value.code == T.TLR_ERR_ARG
