"""TLR-structured FP64 forms: the operator and its derivatives without forming X.

Same quantities as ``operator`` but evaluated tile by tile through the
factors (X_ij Dfrak_j = L_ij (R_ij^T Dfrak_j), ...), which is associativity of
the products in eq. (6)-(9) and (25)-(27) and nothing else.  These forms keep
the oracle affordable at the workload sizes (n_r up to 9216) and are checked
against the dense-literal forms to 1e-12 in the tests.

Everything is receiver-major: Dfrak = D-hat^T and Ufrak = U-hat^T are n_r x n_s,
Y = X_h Dfrak, and the residual Rf = Y - Ufrak = (D-hat X_h - U-hat)^T.
"""
from __future__ import annotations

import numpy as np

from .layout import Layout


def _bilinear(a, c, lay: Layout, Dt, ns):
    """Sum over low-rank tiles of (a-factor)(c-factor)^T applied to Dfrak.

    Tile (i, j), i > j: a.L c.R^T; its mirror (j, i): (a.L c.R^T)^T = c.R a.L^T;
    low-rank diagonal: a.Q c.Q^T.  With a = c = theta this is the low-rank
    part of X_h Dfrak.
    """
    Y = np.zeros((lay.nr, ns), dtype=np.complex128)
    for i in range(lay.n):
        if lay.dense[i] or lay.k_diag[i] == 0:
            continue
        ri = lay.rows(i)
        Qa = lay.diag_block(a, i)
        Qc = lay.diag_block(c, i)
        Y[ri] += Qa @ (Qc.T @ Dt[ri])
    for p, (i, j) in enumerate(lay.pair_list):
        if lay.k_pair[p] == 0:
            continue
        ri, rj = lay.rows(i), lay.rows(j)
        La = lay.l_block(a, p)
        Rc = lay.r_block(c, p)
        Y[ri] += La @ (Rc.T @ Dt[rj])
        Y[rj] += Rc @ (La.T @ Dt[ri])
    return Y


def _dense_part(a, lay: Layout, Dt, ns):
    """Sum over dense diagonal tiles of P(a.Z) Dfrak_i = 0.5 (Z + Z^T) Dfrak_i."""
    Y = np.zeros((lay.nr, ns), dtype=np.complex128)
    for i in range(lay.n):
        if lay.dense[i]:
            ri = lay.rows(i)
            Z = lay.diag_block(a, i)
            Y[ri] += 0.5 * (Z + Z.T) @ Dt[ri]
    return Y


def apply(theta, lay: Layout, Dt) -> np.ndarray:
    """Y = X_h Dfrak (eq. 15 applied to the receiver-major data)."""
    theta = np.asarray(theta, dtype=np.complex128)
    ns = Dt.shape[1]
    return _bilinear(theta, theta, lay, Dt, ns) + _dense_part(theta, lay, Dt, ns)


def line_terms(theta, d, lay: Layout, Dt):
    """A0 = X0 Dfrak, A1 = X1 Dfrak, A2 = X2 Dfrak where
    C(theta + a d) = X0 + a X1 + a^2 X2 (bilinear tiles, linear dense tiles)."""
    theta = np.asarray(theta, dtype=np.complex128)
    d = np.asarray(d, dtype=np.complex128)
    ns = Dt.shape[1]
    A1 = _bilinear(d, theta, lay, Dt, ns) + _bilinear(theta, d, lay, Dt, ns) \
        + _dense_part(d, lay, Dt, ns)
    A2 = _bilinear(d, d, lay, Dt, ns)
    return A1, A2


def grad_from_residual(theta, lay: Layout, Dt, Rf) -> np.ndarray:
    """Factor gradients eq. (25)-(27) with W' expanded per tile.

    W = D-hat^H (D-hat X - U-hat) = conj(Dfrak) Rf^T, so
    W'_ij = W_ij + (W_ji)^T = conj(Dfrak_i) Rf_j^T + Rf_i Dfrak_j^H, and e.g.
    grad L_ij = W'_ij conj(R_ij) = conj(Dfrak_i) (Rf_j^T conj(R_ij))
                                   + Rf_i (Dfrak_j^H conj(R_ij)).
    """
    theta = np.asarray(theta, dtype=np.complex128)
    g = np.zeros(lay.size, dtype=np.complex128)

    def wprime_times(i, j, M):
        ri, rj = lay.rows(i), lay.rows(j)
        return Dt[ri].conj() @ (Rf[rj].T @ M) + Rf[ri] @ (Dt[rj].conj().T @ M)

    for i in range(lay.n):
        ri = lay.rows(i)
        o = lay.off_diag[i]
        if lay.dense[i]:
            Wii = Dt[ri].conj() @ Rf[ri].T + Rf[ri] @ Dt[ri].conj().T
            gi = 0.5 * Wii
        else:
            if lay.k_diag[i] == 0:
                continue
            Q = lay.diag_block(theta, i)
            gi = wprime_times(i, i, Q.conj())
        g[o:o + gi.size] = gi.ravel()
    for p, (i, j) in enumerate(lay.pair_list):
        if lay.k_pair[p] == 0:
            continue
        L = lay.l_block(theta, p)
        R = lay.r_block(theta, p)
        gl = wprime_times(i, j, R.conj())      # W'_ij conj(R_ij)
        gr = wprime_times(j, i, L.conj())      # W'_ji conj(L_ij) = (L^H W'_ij)^T
        g[lay.off_l[p]:lay.off_l[p] + gl.size] = gl.ravel()
        g[lay.off_r[p]:lay.off_r[p] + gr.size] = gr.ravel()
    return g


def fgrad(theta, lay: Layout, Dt, Ut):
    """f (eq. 17a), its factor gradient (eq. 25-27) and the residual Rf."""
    Rf = apply(theta, lay, Dt) - Ut
    f = 0.5 * float(np.vdot(Rf, Rf).real)
    return f, grad_from_residual(theta, lay, Dt, Rf), Rf
