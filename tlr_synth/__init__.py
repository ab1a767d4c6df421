"""Seeded synthetic inputs for tile low-rank (TLR) multidimensional deconvolution.

This module is shared by the FP64 oracle, the tests and the benchmark.  It only
draws random numbers and builds the synthetic stand-ins for the paper's 3D
Overthrust workload (Numerical Examples section): a receiver grid, a
down-going wavefield D(w) with a decaying singular spectrum, planted factor
values for a symmetric TLR Green's function, complex Gaussian noise, source-drop
masks, rank schedules and a Poisson request stream.  It holds none of the
method's arithmetic: it never forms X from its tiles, never applies the MDD
operator and never computes a residual or a gradient.  Composing the up-going
wavefield U = D X + noise is done by whoever consumes these draws (the oracle
in the tests, the benchmark's own device-side setup at full size).

Every generator takes a seed (or a numpy Generator) so both sides of a parity
test receive the identical complex64 arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng", "cn", "haar_unitary", "phase_dft_unitary", "singular_decay",
    "make_d", "planted_theta", "theta_tiles", "noise", "source_keep",
    "rank_linear", "rank_loguniform", "Request", "request_stream",
]


def rng(seed: int) -> np.random.Generator:
    """A PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(seed))


def cn(g: np.random.Generator, shape) -> np.ndarray:
    """Circular complex Gaussian CN(0, 1) samples, complex128."""
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im) * (1.0 / math.sqrt(2.0))


def haar_unitary(n: int, g: np.random.Generator) -> np.ndarray:
    """Haar-distributed n x n unitary: QR of a complex Gaussian with the
    R-diagonal phase fix (Mezzadri, 2007)."""
    z = cn(g, (n, n))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def phase_dft_unitary(n: int, g: np.random.Generator) -> np.ndarray:
    """Exactly unitary F diag(e^{i phi}) Pi F diag(e^{i psi}) / n built with
    FFTs (O(n^2 log n)); used where a Haar QR is too slow."""
    psi = np.exp(2j * np.pi * g.random(n))
    phi = np.exp(2j * np.pi * g.random(n))
    pi = g.permutation(n)
    m = np.fft.fft(np.diag(psi), axis=0)          # F diag(psi)
    m = m[pi, :] * phi[:, None]                   # diag(phi) Pi (...)
    m = np.fft.fft(m, axis=0)                     # F (...)
    return m / n


def singular_decay(m: int, lo: float = 1e-3) -> np.ndarray:
    """sigma_i = 10^{log10(lo) * i/(m-1)}: geometric decay from 1 to ``lo``."""
    if m == 1:
        return np.ones(1)
    return 10.0 ** (math.log10(lo) * np.arange(m) / (m - 1))


def make_d(ns: int, nr: int, nfreq: int, seed: int, lo: float = 1e-3,
           haar_max: int = 4096) -> np.ndarray:
    """Down-going wavefields D(w_f) = Q diag(sigma * e^{i phi_f}) W^H, f < nfreq.

    Q (ns x ns) and W (nr x nr) are drawn once and shared across frequencies;
    each frequency gets a fresh random phase per singular value.  Returned as
    complex64 [nfreq, ns, nr] (the paper's layout: one row per source).
    """
    g = rng(seed)
    uni = haar_unitary if max(ns, nr) <= haar_max else phase_dft_unitary
    q = uni(ns, g)
    w = uni(nr, g)
    m = min(ns, nr)
    sig = singular_decay(m, lo)
    out = np.empty((nfreq, ns, nr), dtype=np.complex64)
    for f in range(nfreq):
        ph = np.exp(2j * np.pi * g.random(m))
        out[f] = ((q[:, :m] * (sig * ph)[None, :]) @ w[:, :m].conj().T).astype(np.complex64)
    return out


@dataclass(frozen=True)
class TileSpec:
    kind: str      # "Q" (low-rank diagonal), "Z" (dense diagonal), "L", "R"
    i: int         # tile row (block) index
    j: int         # tile column index
    rows: int
    cols: int


def theta_tiles(nr: int, b, ranks, diag_dense, tiles=None) -> list:
    """The tiles of the stacked unknown (Z-bar, L-bar, R-bar) in storage order.

    ``ranks``: an int (uniform) or a sequence of N diagonal ranks followed by
    N(N-1)/2 pair ranks in stacking order (tile column j ascending, then tile
    row i > j ascending).  ``diag_dense``: sequence of N booleans.  ``tiles``:
    the block sizes d_i of a non-uniform partition (None: N = nr / b blocks of
    size b).
    """
    d = [int(b)] * (nr // b) if tiles is None else [int(t) for t in tiles]
    n = len(d)
    pairs = [(i, j) for j in range(n) for i in range(j + 1, n)]
    if isinstance(ranks, (int, np.integer)):
        kd = [int(ranks)] * n
        kp = [int(ranks)] * len(pairs)
    else:
        ranks = [int(r) for r in ranks]
        kd, kp = ranks[:n], ranks[n:]
    tiles = []
    out = []
    for i in range(n):
        if diag_dense[i]:
            out.append(TileSpec("Z", i, i, d[i], d[i]))
        else:
            out.append(TileSpec("Q", i, i, d[i], kd[i]))
    for p, (i, j) in enumerate(pairs):
        out.append(TileSpec("L", i, j, d[i], kp[p]))
    for p, (i, j) in enumerate(pairs):
        out.append(TileSpec("R", i, j, d[j], kp[p]))
    return out


def planted_theta(nr: int, b, ranks, diag_dense, seed: int, tiles=None) -> np.ndarray:
    """Planted factor values, complex128, in the stacked storage order.

    L, R, Q ~ CN(0,1)/sqrt(d k), scaled by 1/(1+|i-j|) so that energy sits near
    the diagonal as it does for Hilbert-ordered Green's functions; a dense
    diagonal tile is a symmetric CN(0, 1/d) block (d: the factor's rows, the
    tile size b of a uniform partition).
    """
    g = rng(seed)
    parts = []
    for t in theta_tiles(nr, b, ranks, diag_dense, tiles):
        if t.kind == "Z":
            a = cn(g, (t.rows, t.rows)) / math.sqrt(t.rows)
            parts.append(((a + a.T) * 0.5).ravel())
        else:
            if t.cols == 0:
                continue
            s = 1.0 / ((1 + abs(t.i - t.j)) * math.sqrt(t.rows * t.cols))
            parts.append((cn(g, (t.rows, t.cols)) * s).ravel())
    if not parts:
        return np.zeros(0, dtype=np.complex128)
    return np.concatenate(parts)


def noise(shape, seed: int) -> np.ndarray:
    """Unit complex Gaussian noise (complex128); the consumer scales it to the SNR."""
    return cn(rng(seed), shape)


def source_keep(ns: int, keep_frac: float, seed: int) -> np.ndarray:
    """Indices of the sources kept after random dropping (ascending)."""
    k = int(round(keep_frac * ns))
    return np.sort(rng(seed).permutation(ns)[:k])


def rank_linear(a: int, b: int, nfreq: int) -> list:
    """Rank rising linearly from a to b over the frequencies:
    k_f = a + floor((b - a) f / (F - 1) + 1/2)."""
    if nfreq == 1:
        return [a]
    return [a + int(math.floor((b - a) * f / (nfreq - 1) + 0.5)) for f in range(nfreq)]


def rank_loguniform(g: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))


@dataclass(frozen=True)
class Request:
    rid: int
    t_arrive: float   # seconds from stream start
    nr: int
    nx: int
    ny: int
    tile: int
    rank: int
    seed: int


_GRIDS = {1024: (32, 32), 2048: (64, 32), 4096: (64, 64), 8192: (128, 64)}


def request_stream(n: int, rate_hz: float, seed: int, sizes=(1024, 2048, 4096, 8192),
                   tiles=(128, 256, 512), rank_lo: int = 2, rank_hi: int = 64) -> list:
    """A Poisson stream of per-frequency solve requests (nr=ns uniform over
    ``sizes``, tile uniform over ``tiles``, rank log-uniform in [lo, hi])."""
    g = rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += g.exponential(1.0 / rate_hz)
        nr = int(g.choice(sizes))
        tile = int(g.choice(tiles))
        k = min(rank_loguniform(g, rank_lo, rank_hi), tile)
        nx, ny = _GRIDS.get(nr, (nr, 1))
        out.append(Request(rid, t, nr, nx, ny, tile, k, int(g.integers(1 << 30))))
    return out
