"""Dense-literal FP64 forms of the TLR MDD operator and its derivatives.

Everything here forms X_h densely, exactly as the paper writes it, and works in
the paper's layout: D-hat, U-hat are n_s x n_r (one row per source) and the
data equation is D-hat X_h = U-hat (eq. 14).  The GPU library stores the
receiver-major transposes; ``apply_y`` and ``adjoint_g`` give the results in
that layout so tests can compare element by element.
"""
from __future__ import annotations

import numpy as np

from .layout import Layout


def normalise(D: np.ndarray, U: np.ndarray, perm: np.ndarray, alpha: float | None = None):
    """Reorder the receivers and scale by alpha (eq. 14; Hyper-parameter
    selection section).

    D-hat = D S / alpha, U-hat = U S / alpha, where (D S)[:, a] = D[:, perm[a]].
    ``alpha`` defaults to the maximum modulus of the given D (the paper takes
    the maximum over all frequencies; a caller holding several frequencies
    passes that value).
    """
    D = np.asarray(D, dtype=np.complex128)
    U = np.asarray(U, dtype=np.complex128)
    if alpha is None:
        alpha = float(np.max(np.abs(D)))
    return D[:, perm] / alpha, U[:, perm] / alpha, alpha


def assemble_xh(theta: np.ndarray, lay: Layout) -> np.ndarray:
    """X_h = C(Z-bar, L-bar, R-bar), eq. (15), tile by tile from eq. (6)-(9).

    Diagonal: X_ii = Q_ii Q_ii^T (eq. 6) or X_ii = P Z_ii = (Z_ii + Z_ii^T)/2
    (eq. 7 with P = (I + Gamma)/2).  Sub-diagonal: X_ij = L_ij R_ij^T (eq. 8).
    Super-diagonal: X_ji = X_ij^T, plain transpose (eq. 9); it is assigned as
    the transpose of the stored tile so X_h equals X_h^T bit for bit.
    """
    theta = np.asarray(theta, dtype=np.complex128)
    X = np.zeros((lay.nr, lay.nr), dtype=np.complex128)
    for i in range(lay.n):
        B = lay.diag_block(theta, i)
        ri = lay.rows(i)
        if lay.dense[i]:
            X[ri, ri] = 0.5 * (B + B.T)
        else:
            X[ri, ri] = B @ B.T
    for p, (i, j) in enumerate(lay.pair_list):
        L = lay.l_block(theta, p)
        R = lay.r_block(theta, p)
        tile = L @ R.T
        X[lay.rows(i), lay.rows(j)] = tile
        X[lay.rows(j), lay.rows(i)] = tile.T
    return X


def residual(theta, lay, Dh, Uh):
    """E = D-hat X_h - U-hat (the quantity inside the norm of eq. 17a)."""
    return Dh @ assemble_xh(theta, lay) - Uh


def misfit(theta, lay, Dh, Uh) -> float:
    """f = 0.5 || D-hat C(theta) - U-hat ||_F^2, eq. (17a)."""
    E = residual(theta, lay, Dh, Uh)
    return 0.5 * float(np.vdot(E, E).real)


def w_matrices(theta, lay, Dh, Uh):
    """W = D-hat^H (D-hat X - U-hat) and W' = W + W^T (Derivatives paragraph)."""
    W = Dh.conj().T @ residual(theta, lay, Dh, Uh)
    return W, W + W.T


def gradient(theta, lay, Dh, Uh) -> np.ndarray:
    """Factor gradients, eq. (25)-(27), stacked like theta.

    grad L_ij = W'_ij conj(R_ij^paper)^T ... in this storage (R_ij^paper = R_ij^T):
      grad L_ij = W'_ij conj(R_ij)                       (eq. 25.1)
      grad R_ij = (L_ij^H W'_ij)^T                       (eq. 25.2, transposed)
      grad Z_ii = 0.5 W'_ii                              (eq. 26)
      grad Q_ii = W'_ii conj(Q_ii)                       (eq. 27)
    The convention is grad = df/dRe(theta) + i df/dIm(theta): the first-order
    change of f along d is Re <grad, d>.
    """
    theta = np.asarray(theta, dtype=np.complex128)
    _, Wp = w_matrices(theta, lay, Dh, Uh)
    g = np.zeros(lay.size, dtype=np.complex128)
    for i in range(lay.n):
        B = lay.diag_block(theta, i)
        Wii = Wp[lay.rows(i), lay.rows(i)]
        o = lay.off_diag[i]
        if lay.dense[i]:
            gi = 0.5 * Wii
        else:
            gi = Wii @ B.conj()
        g[o:o + gi.size] = gi.ravel()
    for p, (i, j) in enumerate(lay.pair_list):
        L = lay.l_block(theta, p)
        R = lay.r_block(theta, p)
        Wij = Wp[lay.rows(i), lay.rows(j)]
        gl = Wij @ R.conj()
        gr = (L.conj().T @ Wij).T
        g[lay.off_l[p]:lay.off_l[p] + gl.size] = gl.ravel()
        g[lay.off_r[p]:lay.off_r[p] + gr.size] = gr.ravel()
    return g


def apply_y(theta, lay, Dh) -> np.ndarray:
    """Receiver-major forward product Y = X_h Dfrak with Dfrak = D-hat^T,
    i.e. Y = (D-hat X_h)^T (X_h is symmetric, eq. 9)."""
    return (Dh @ assemble_xh(theta, lay)).T


def adjoint_g(V, Dh) -> np.ndarray:
    """G = V Dfrak^H = V conj(D-hat) for V n_r x n_s (receiver-major).

    With V = (D-hat X - U-hat)^T this is W^T (W of eq. 25)."""
    return np.asarray(V, dtype=np.complex128) @ Dh.conj()


def unpermute(Xh, perm) -> np.ndarray:
    """X = S X_h S^T, eq. (11): X[perm[a], perm[c]] = X_h[a, c]."""
    n = len(perm)
    X = np.zeros((n, n), dtype=np.complex128)
    X[np.ix_(perm, perm)] = Xh
    return X


def line_coefficients(theta, d, lay, Dh, Uh, rho=0.0, v=None):
    """Dense-literal coefficients of phi(theta + a d) as a quartic in a.

    C(theta + a d) = X0 + a X1 + a^2 X2 because every tile is bilinear (or
    linear) in its factors; with E = D-hat X0 - U-hat, A1 = D-hat X1,
    A2 = D-hat X2 and the ADMM penalty rho/2 ||theta - v + a d||^2 (eq. 19):
      phi(a) = c0 + c1 a + c2 a^2 + c3 a^3 + c4 a^4.
    X1, X2 are formed by polarisation of the assembly (X(t+d) - X(t-d))/2 etc.
    """
    theta = np.asarray(theta, dtype=np.complex128)
    d = np.asarray(d, dtype=np.complex128)
    X0 = assemble_xh(theta, lay)
    Xp = assemble_xh(theta + d, lay)
    Xm = assemble_xh(theta - d, lay)
    X1 = 0.5 * (Xp - Xm)
    X2 = 0.5 * (Xp + Xm) - X0
    E = Dh @ X0 - Uh
    A1 = Dh @ X1
    A2 = Dh @ X2
    return quartic_from_terms(E, A1, A2, theta, d, rho, v)


def quartic_from_terms(E, A1, A2, theta, d, rho=0.0, v=None):
    re = lambda a, b: float(np.vdot(a, b).real)  # noqa: E731
    c0 = 0.5 * re(E, E)
    c1 = re(E, A1)
    c2 = 0.5 * re(A1, A1) + re(E, A2)
    c3 = re(A1, A2)
    c4 = 0.5 * re(A2, A2)
    if rho:
        w = theta - (v if v is not None else 0.0)
        c0 += 0.5 * rho * re(w, w)
        c1 += rho * re(w, d)
        c2 += 0.5 * rho * re(d, d)
    return np.array([c0, c1, c2, c3, c4])
