"""General (non-reciprocal) tile low-rank parametrisation (TEST INFRASTRUCTURE ONLY).

The reciprocity-aware method ties X_ji to X_ij (X = X^T).  Without that
constraint (the general TLR form the paper builds on, Tile Low-rank MDD
section, before the reciprocity reduction) every tile is free:

* diagonal tile i: X_ii = L_ii R_ii^T (low rank, b x k each) or X_ii = Z_ii
  (dense, no symmetrisation);
* every off-diagonal tile (i, j), i != j: X_ij = L_ij R_ij^T.

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


def ordered_pairs(n: int) -> list:
    return [(i, j) for j in range(n) for i in range(n) if i != j]


@dataclass
class GeneralLayout:
    nr: int
    b: int
    n: int
    k_diag: list
    dense: list
    k_pair: list
    pair_list: list = field(default_factory=list)
    off_diag: list = field(default_factory=list)   # Z_ii or L_ii (R_ii follows)
    off_l: list = field(default_factory=list)
    off_r: list = field(default_factory=list)
    size: int = 0

    def rows(self, i):
        return slice(i * self.b, (i + 1) * self.b)


def make_general_layout(nr: int, b: int, ranks, diag_mode="rule") -> GeneralLayout:
    if b <= 0 or nr % b != 0:
        raise ValueError("tile size must divide n_r")
    n = nr // b
    pl = ordered_pairs(n)
    if isinstance(ranks, (int, np.integer)):
        kd, kp = [int(ranks)] * n, [int(ranks)] * len(pl)
    else:
        ranks = [int(r) for r in ranks]
        if len(ranks) != n + len(pl):
            raise ValueError("need N + N(N-1) ranks")
        kd, kp = ranks[:n], ranks[n:]
    if isinstance(diag_mode, str):
        dense = {"rule": [4 * k >= b for k in kd], "lowrank": [False] * n, "dense": [True] * n}[diag_mode]
    else:
        dense = [bool(x) for x in diag_mode]
    lay = GeneralLayout(nr, b, n, kd, dense, kp, pl)
    o = 0
    for i in range(n):
        lay.off_diag.append(o)
        o += b * b if dense[i] else 2 * b * kd[i]
    for p in range(len(pl)):
        lay.off_l.append(o)
        o += b * kp[p]
    for p in range(len(pl)):
        lay.off_r.append(o)
        o += b * kp[p]
    lay.size = o
    return lay


def _blocks(theta, lay, i=None, p=None):
    b = lay.b
    if p is None:
        o = lay.off_diag[i]
        if lay.dense[i]:
            return theta[o:o + b * b].reshape(b, b), None
        k = lay.k_diag[i]
        return theta[o:o + b * k].reshape(b, k), theta[o + b * k:o + 2 * b * k].reshape(b, k)
    k = lay.k_pair[p]
    return (theta[lay.off_l[p]:lay.off_l[p] + b * k].reshape(b, k),
            theta[lay.off_r[p]:lay.off_r[p] + b * k].reshape(b, k))


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
    b = lay.b
    for i in range(lay.n):
        Wii = W[lay.rows(i), lay.rows(i)]
        o = lay.off_diag[i]
        A, B = _blocks(theta, lay, i=i)
        if lay.dense[i]:
            g[o:o + b * b] = Wii.ravel()
        else:
            k = lay.k_diag[i]
            g[o:o + b * k] = (Wii @ B.conj()).ravel()
            g[o + b * k:o + 2 * b * k] = (Wii.T @ A.conj()).ravel()
    for p, (i, j) in enumerate(lay.pair_list):
        L, R = _blocks(theta, lay, p=p)
        Wij = W[lay.rows(i), lay.rows(j)]
        k = lay.k_pair[p]
        g[lay.off_l[p]:lay.off_l[p] + b * k] = (Wij @ R.conj()).ravel()
        g[lay.off_r[p]:lay.off_r[p] + b * k] = (Wij.T @ L.conj()).ravel()
    return g


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
