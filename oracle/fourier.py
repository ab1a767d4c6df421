"""Time <-> frequency stacks of the examples (TEST INFRASTRUCTURE ONLY).

The recorded wavefields are transformed to the frequency domain and each
frequency is solved on its own; the Green's function returns to time by the
inverse transform (Numerical Examples).  Conventions: trace-major traces
x[tr, t], nt samples; X(omega_k) = sum_t x(t) exp(-2 pi i k t / nt) for
k = 0 .. nt/2 (numpy's rfft), the stack holds the band k = f0 .. f0+nf-1
frequency-major (stack[f, tr]); the inverse is numpy's irfft of the band with
zeros elsewhere (the 1/nt factor included).  alpha = max |D(omega)| over the
whole stack (hyper-parameter selection section).
"""
from __future__ import annotations

import numpy as np


def time_to_freq(x, f0: int, nf: int) -> np.ndarray:
    X = np.fft.rfft(np.asarray(x, np.float64), axis=-1)
    return np.ascontiguousarray(X[:, f0:f0 + nf].T)


def freq_to_time(S, nt: int, f0: int) -> np.ndarray:
    S = np.asarray(S, np.complex128)
    nf, ntr = S.shape
    spec = np.zeros((ntr, nt // 2 + 1), np.complex128)
    spec[:, f0:f0 + nf] = S.T
    return np.fft.irfft(spec, n=nt, axis=-1)


def stack_alpha(D) -> float:
    return float(np.max(np.abs(np.asarray(D))))
