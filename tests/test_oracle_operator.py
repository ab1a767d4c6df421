"""Pins for the dense-literal operator, misfit and gradients (eq. 6-9, 15-17, 25-27)."""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import hilbert, layout, operator
from tests._cases import problem


def _brute_xh(theta, lay):
    """Every entry of X_h written out from the tile formulas with explicit sums."""
    n, b = lay.nr, lay.b
    X = [[0j] * n for _ in range(n)]
    th = [complex(t) for t in theta]
    for i in range(lay.n):
        o = lay.off_diag[i]
        for r in range(b):
            for c in range(b):
                if lay.dense[i]:
                    v = 0.5 * (th[o + r * b + c] + th[o + c * b + r])
                else:
                    k = lay.k_diag[i]
                    v = sum(th[o + r * k + q] * th[o + c * k + q] for q in range(k))
                X[i * b + r][i * b + c] = v
    for p, (i, j) in enumerate(lay.pair_list):
        k = lay.k_pair[p]
        ol, orr = lay.off_l[p], lay.off_r[p]
        for r in range(b):
            for c in range(b):
                v = sum(th[ol + r * k + q] * th[orr + c * k + q] for q in range(k))
                X[i * b + r][j * b + c] = v        # X_ij = L R^T
                X[j * b + c][i * b + r] = v        # X_ji = X_ij^T
    return np.array(X)


@pytest.mark.parametrize("nr,b,ranks,mode", [
    (8, 4, 2, "lowrank"), (8, 4, 3, "dense"), (12, 4, [1, 0, 4, 2, 0, 3], [True, False, False]),
    (16, 4, 1, "rule"), (4, 4, 2, "lowrank"),
])
def test_assembly_matches_brute_force(nr, b, ranks, mode):
    lay = layout.make_layout(nr, b, ranks, mode)
    th = synth.cn(synth.rng(5), lay.size)
    X = operator.assemble_xh(th, lay)
    np.testing.assert_allclose(X, _brute_xh(th, lay), rtol=0, atol=1e-14)
    assert np.array_equal(X, X.T)            # reciprocity: exact plain symmetry
    assert not np.allclose(X, X.conj().T)    # and it is not Hermitian


def test_data_equation_after_reordering():
    # with U = D X (natural order), D-hat X_h = U-hat (eq. 14) holds exactly
    D, U, perm, lay, th = problem(4, 4, 4, 2, "lowrank", ns=20)
    Dh, Uh, _ = operator.normalise(D, U.astype(np.complex128), perm, alpha=1.0)
    E = operator.residual(th, lay, Dh, Uh)
    assert np.linalg.norm(E) < 1e-5 * np.linalg.norm(Uh)   # U was cast to complex64 once
    # the wrong direction (S^T instead of S) does not fit
    inv = np.argsort(perm)
    Dw, Uw, _ = operator.normalise(D, U, inv, alpha=1.0)
    assert np.linalg.norm(operator.residual(th, lay, Dw, Uw)) > 0.1 * np.linalg.norm(Uw)


def test_adjoint_dot_product():
    # <X Dfrak, V> = <X, V Dfrak^H> for the receiver-major forms
    D, U, perm, lay, th = problem(8, 4, 8, 3, "rule", ns=24)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    Y = operator.apply_y(th, lay, Dh)
    V = synth.cn(synth.rng(9), Y.shape)
    G = operator.adjoint_g(V, Dh)
    Xh = operator.assemble_xh(th, lay)
    lhs = np.vdot(Y, V)
    rhs = np.vdot(Xh, G)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    np.testing.assert_allclose(Y, Xh @ Dh.T, rtol=1e-13, atol=1e-13)


def test_adjoint_solution_is_minus_w_at_zero():
    # X_adj = D^H U (cross-correlation) equals -W at X = 0
    D, U, perm, lay, th = problem(4, 4, 4, 2, "lowrank", ns=16)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    W, _ = operator.w_matrices(np.zeros(lay.size), lay, Dh, Uh)
    np.testing.assert_allclose(W, -(Dh.conj().T @ Uh), rtol=1e-14, atol=1e-14)


def _fd_grad(f, theta, idx, h):
    out = []
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        re = (f(theta + e) - f(theta - e)) / (2 * h)
        im = (f(theta + 1j * e) - f(theta - 1j * e)) / (2 * h)
        out.append(re + 1j * im)
    return np.array(out)


@pytest.mark.parametrize("mode", ["lowrank", "dense", [True, False, True, False]])
def test_gradient_matches_central_differences(mode):
    D, U, perm, lay, _ = problem(8, 4, 8, 3, mode, ns=40, snr_db=10, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    th = synth.cn(synth.rng(3), lay.size) * 0.3
    g = operator.gradient(th, lay, Dh, Uh)
    f = lambda t: operator.misfit(t, lay, Dh, Uh)  # noqa: E731
    idx = synth.rng(4).choice(lay.size, 24, replace=False)
    fd = _fd_grad(f, th, idx, 1e-3)
    assert np.max(np.abs(fd - g[idx])) <= 1e-6 * np.max(np.abs(g))


def test_directional_derivative():
    D, U, perm, lay, _ = problem(8, 4, 8, 2, "rule", ns=32, snr_db=20, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    th = synth.cn(synth.rng(6), lay.size) * 0.3
    d = synth.cn(synth.rng(7), lay.size)
    g = operator.gradient(th, lay, Dh, Uh)
    h = 1e-4
    fd = (operator.misfit(th + h * d, lay, Dh, Uh) - operator.misfit(th - h * d, lay, Dh, Uh)) / (2 * h)
    assert abs(fd - np.vdot(g, d).real) <= 1e-7 * abs(fd)


def test_unpermute_matches_matrix_form():
    lay = layout.make_layout(32, 8, 2, "lowrank")
    th = synth.cn(synth.rng(1), lay.size)
    p = hilbert.perm(8, 4)
    S = hilbert.hilbert_matrix(p)
    Xh = operator.assemble_xh(th, lay)
    np.testing.assert_allclose(operator.unpermute(Xh, p), S @ Xh @ S.T, atol=1e-15)


def test_quartic_coefficients_match_direct_evaluation():
    D, U, perm, lay, _ = problem(8, 4, 8, 3, [True, False, False, True], ns=24, snr_db=10, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    th = synth.cn(synth.rng(11), lay.size) * 0.3
    d = synth.cn(synth.rng(12), lay.size) * 0.1
    v = synth.cn(synth.rng(13), lay.size) * 0.1
    rho = 0.7
    c = operator.line_coefficients(th, d, lay, Dh, Uh, rho, v)
    for a in [-1.3, -0.2, 0.0, 0.5, 2.0]:
        t = th + a * d
        direct = operator.misfit(t, lay, Dh, Uh) + 0.5 * rho * np.vdot(t - v, t - v).real
        poly = sum(c[q] * a ** q for q in range(5))
        assert abs(direct - poly) <= 1e-12 * max(1.0, abs(direct))
