"""The preconditioned benchmark objective, eq. (4), for one dense tile.

min_Z 0.5 ||D-hat P Z - U-hat||_F^2 + lambda ||Z||_F^2 with P Z = (Z + Z^T)/2.
Its minimiser solves the normal equations (P is self-adjoint for the real
inner product Re tr(A^H B)):

    P(D-hat^H D-hat P(Z)) + 2 lambda Z = P(D-hat^H U-hat),

a symmetric positive definite real-linear system for lambda > 0, solved here by
plain conjugate gradients on the real vector space C^{n x n} ~ R^{2 n^2}.
With one tile (N = 1) and a dense diagonal, the TLR objective f + g of eq. (16)
is exactly eq. (4), so this minimiser pins the ADMM solver's fixed point.
"""
from __future__ import annotations

import numpy as np


def _p(Z):
    return 0.5 * (Z + Z.T)


def solve_eq4(Dh, Uh, lam: float, tol: float = 1e-14, maxit: int = 10000):
    Dh = np.asarray(Dh, np.complex128)
    Uh = np.asarray(Uh, np.complex128)
    G = Dh.conj().T @ Dh

    def op(Z):
        return _p(G @ _p(Z)) + 2.0 * lam * Z

    b = _p(Dh.conj().T @ Uh)
    x = np.zeros_like(b)
    r = b - op(x)
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    bn = float(np.vdot(b, b).real) ** 0.5
    for _ in range(maxit):
        if rr ** 0.5 <= tol * bn:
            break
        Ap = op(p)
        a = rr / float(np.vdot(p, Ap).real)
        x = x + a * p
        r = r - a * Ap
        rr_new = float(np.vdot(r, r).real)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x
