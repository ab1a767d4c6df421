"""General (non-reciprocal) tile low-rank parametrisation (TEST INFRASTRUCTURE ONLY).

The reciprocity-aware method ties X_ji to X_ij (X = X^T).  Without that
constraint (the general TLR form the paper builds on, Tile Low-rank MDD
section, before the reciprocity reduction) every tile is free:

* diagonal tile i: X_ii = L_ii R_ii^T (low rank, d_i x k each) or X_ii = Z_ii
  (dense, no symmetrisation);
* every off-diagonal tile (i, j), i != j: X_ij = L_ij R_ij^T with L_ij
  d_i x k and R_ij d_j x k (tile sizes d_i as in ``layout``: uniform or not).

Stacking: the diagonal blocks in i order (Z_ii, or L_ii then R_ii), then the
L factors of the ordered pairs (column j outer, row i inner, i != j), then
their R factors in the same order; every block row-major.  The data fit is
the same, f = 0.5 ||D-hat X - U-hat||^2, and with W = D-hat^H (D-hat X - U-hat)
the factor gradients (convention df/dRe + i df/dIm) are
grad L_ij = W_ij conj(R_ij), grad R_ij = W_ij^T conj(L_ij), grad Z_ii = W_ii.
Dense-literal forms only (tests on small sizes).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .layout import partition


def ordered_pairs(n: int) -> list:
    return [(i, j) for j in range(n) for i in range(n) if i != j]


@dataclass
class GeneralLayout:
    nr: int
    b: int | None        # the tile size of a uniform partition, else None
    n: int
    k_diag: list
    dense: list
    k_pair: list
    pair_list: list = field(default_factory=list)
    off_diag: list = field(default_factory=list)   # Z_ii or L_ii (R_ii follows)
    off_l: list = field(default_factory=list)
    off_r: list = field(default_factory=list)
    size: int = 0
    d: list = field(default_factory=list)      # tile sizes d_i
    roff: list = field(default_factory=list)   # first row of block i

    def rows(self, i):
        return slice(self.roff[i], self.roff[i] + self.d[i])


def make_general_layout(nr: int, b, ranks, diag_mode="rule", tiles=None) -> GeneralLayout:
    d, roff = partition(nr, b, tiles)
    n = len(d)
    pl = ordered_pairs(n)
    if isinstance(ranks, (int, np.integer)):
        kd, kp = [int(ranks)] * n, [int(ranks)] * len(pl)
    else:
        ranks = [int(r) for r in ranks]
        if len(ranks) != n + len(pl):
            raise ValueError("need N + N(N-1) ranks")
        kd, kp = ranks[:n], ranks[n:]
    for i in range(n):
        if kd[i] < 0 or kd[i] > d[i]:
            raise ValueError("diagonal ranks must lie in [0, d_i]")
    for p, (i, j) in enumerate(pl):
        if kp[p] < 0 or kp[p] > min(d[i], d[j]):
            raise ValueError("pair ranks must lie in [0, min(d_i, d_j)]")
    if isinstance(diag_mode, str):
        dense = {"rule": [4 * kd[i] >= d[i] for i in range(n)], "lowrank": [False] * n,
                 "dense": [True] * n}[diag_mode]
    else:
        dense = [bool(x) for x in diag_mode]
    uniform = b if tiles is None else (d[0] if len(set(d)) == 1 else None)
    lay = GeneralLayout(nr, uniform, n, kd, dense, kp, pl, d=d, roff=roff)
    o = 0
    for i in range(n):
        lay.off_diag.append(o)
        o += d[i] * d[i] if dense[i] else 2 * d[i] * kd[i]
    for p, (i, j) in enumerate(pl):
        lay.off_l.append(o)
        o += d[i] * kp[p]
    for p, (i, j) in enumerate(pl):
        lay.off_r.append(o)
        o += d[j] * kp[p]
    lay.size = o
    return lay


def _blocks(theta, lay, i=None, p=None):
    if p is None:
        o, di = lay.off_diag[i], lay.d[i]
        if lay.dense[i]:
            return theta[o:o + di * di].reshape(di, di), None
        k = lay.k_diag[i]
        return theta[o:o + di * k].reshape(di, k), theta[o + di * k:o + 2 * di * k].reshape(di, k)
    (i, j), k = lay.pair_list[p], lay.k_pair[p]
    return (theta[lay.off_l[p]:lay.off_l[p] + lay.d[i] * k].reshape(lay.d[i], k),
            theta[lay.off_r[p]:lay.off_r[p] + lay.d[j] * k].reshape(lay.d[j], k))


def assemble_x(theta, lay: GeneralLayout) -> np.ndarray:
    theta = np.asarray(theta, np.complex128)
    X = np.zeros((lay.nr, lay.nr), np.complex128)
    for i in range(lay.n):
        A, B = _blocks(theta, lay, i=i)
        X[lay.rows(i), lay.rows(i)] = A if lay.dense[i] else A @ B.T
    for p, (i, j) in enumerate(lay.pair_list):
        L, R = _blocks(theta, lay, p=p)
        X[lay.rows(i), lay.rows(j)] = L @ R.T
    return X


def misfit(theta, lay, Dh, Uh) -> float:
    E = Dh @ assemble_x(theta, lay) - Uh
    return 0.5 * float(np.vdot(E, E).real)


def gradient(theta, lay, Dh, Uh) -> np.ndarray:
    theta = np.asarray(theta, np.complex128)
    W = Dh.conj().T @ (Dh @ assemble_x(theta, lay) - Uh)
    g = np.zeros(lay.size, np.complex128)
    for i in range(lay.n):
        Wii = W[lay.rows(i), lay.rows(i)]
        o = lay.off_diag[i]
        A, B = _blocks(theta, lay, i=i)
        if lay.dense[i]:
            g[o:o + Wii.size] = Wii.ravel()
        else:
            gl, gr = Wii @ B.conj(), Wii.T @ A.conj()
            g[o:o + gl.size] = gl.ravel()
            g[o + gl.size:o + gl.size + gr.size] = gr.ravel()
    for p, (i, j) in enumerate(lay.pair_list):
        L, R = _blocks(theta, lay, p=p)
        Wij = W[lay.rows(i), lay.rows(j)]
        gl, gr = Wij @ R.conj(), Wij.T @ L.conj()
        g[lay.off_l[p]:lay.off_l[p] + gl.size] = gl.ravel()
        g[lay.off_r[p]:lay.off_r[p] + gr.size] = gr.ravel()
    return g


def warm_start(X, lay: GeneralLayout) -> np.ndarray:
    """theta of ``lay`` initialised from X (Hilbert order), the initialisation
    paragraph's factors without the reciprocal pairing: every low-rank tile,
    diagonal ones included, from its truncated SVD, L = U_k Sigma_k^1/2 and
    R = conj(V_k) Sigma_k^1/2 (so L R^T = U_k Sigma_k V_k^H); a dense diagonal
    tile is copied (X_ii = Z_ii)."""
    X = np.asarray(X, np.complex128)
    th = np.zeros(lay.size, np.complex128)

    def put(o_l, o_r, tile, k):
        U, s, Vh = np.linalg.svd(tile, full_matrices=False)
        rs = np.sqrt(s[:k])
        L, R = U[:, :k] * rs, Vh[:k, :].T * rs
        th[o_l:o_l + L.size] = L.ravel()
        th[o_r:o_r + R.size] = R.ravel()

    for i in range(lay.n):
        T = X[lay.rows(i), lay.rows(i)]
        o = lay.off_diag[i]
        if lay.dense[i]:
            th[o:o + T.size] = T.ravel()
        elif lay.k_diag[i] > 0:
            put(o, o + lay.d[i] * lay.k_diag[i], T, lay.k_diag[i])
    for p, (i, j) in enumerate(lay.pair_list):
        if lay.k_pair[p] > 0:
            put(lay.off_l[p], lay.off_r[p], X[lay.rows(i), lay.rows(j)], lay.k_pair[p])
    return th


def apply_y(theta, lay, Dh) -> np.ndarray:
    """Receiver-major Y = (D-hat X)^T = X^T Dfrak."""
    return (Dh @ assemble_x(theta, lay)).T


class GeneralProblem:
    """f, gradient and line-search quartic for the general form (dense-literal,
    polarisation of the bilinear assembly), for the ADMM / L-BFGS solver."""

    def __init__(self, lay: GeneralLayout, Dt, Ut):
        self.lay = lay
        self.Dh = np.asarray(Dt, np.complex128).T
        self.Uh = np.asarray(Ut, np.complex128).T

    def fgrad(self, theta):
        return misfit(theta, self.lay, self.Dh, self.Uh), gradient(theta, self.lay, self.Dh, self.Uh)

    def coefficients(self, theta, d, rho, v):
        theta = np.asarray(theta, np.complex128)
        d = np.asarray(d, np.complex128)
        X0 = assemble_x(theta, self.lay)
        Xp = assemble_x(theta + d, self.lay)
        Xm = assemble_x(theta - d, self.lay)
        E = self.Dh @ X0 - self.Uh
        A1 = self.Dh @ (0.5 * (Xp - Xm))
        A2 = self.Dh @ (0.5 * (Xp + Xm) - X0)
        re = lambda a, c: float(np.vdot(a, c).real)  # noqa: E731
        c = np.array([0.5 * re(E, E), re(E, A1), 0.5 * re(A1, A1) + re(E, A2), re(A1, A2), 0.5 * re(A2, A2)])
        if rho:
            w = theta - v
            c[0] += 0.5 * rho * re(w, w)
            c[1] += rho * re(w, d)
            c[2] += 0.5 * rho * re(d, d)
        return c
