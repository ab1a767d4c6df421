"""Pins of the oracle's time <-> frequency stacks."""
import numpy as np

import tlr_synth as synth
from oracle import fourier


def test_forward_is_the_dft_sum():
    # the DFT written out as a sum over samples, for an odd and an even nt
    g = synth.rng(90)
    for nt in (9, 12):
        x = g.standard_normal((5, nt))
        S = fourier.time_to_freq(x, 1, nt // 2)
        t = np.arange(nt)
        for f in range(nt // 2):
            k = 1 + f
            want = (x * np.exp(-2j * np.pi * k * t / nt)).sum(axis=1)
            np.testing.assert_allclose(S[f], want, rtol=0, atol=1e-12)


def test_round_trip_and_band_limited_inverse():
    g = synth.rng(91)
    nt = 10
    x = g.standard_normal((4, nt))
    S = fourier.time_to_freq(x, 0, nt // 2 + 1)
    np.testing.assert_allclose(fourier.freq_to_time(S, nt, 0), x, atol=1e-12)
    # a band-limited inverse is the sum of its cosines: bins 2 and 3 only
    Sb = S[2:4]
    y = fourier.freq_to_time(Sb, nt, 2)
    t = np.arange(nt)
    want = sum((2.0 / nt) * np.real(Sb[f][:, None] * np.exp(2j * np.pi * (2 + f) * t / nt)) for f in range(2))
    np.testing.assert_allclose(y, want, atol=1e-12)


def test_stack_alpha_is_the_largest_modulus():
    D = np.zeros((3, 4, 5), np.complex64)
    D[1, 2, 3] = 3 - 4j
    D[2, 0, 0] = -4.5
    assert fourier.stack_alpha(D) == 5.0
