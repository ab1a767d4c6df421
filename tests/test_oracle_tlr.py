"""The TLR-structured FP64 forms agree with the dense-literal definitions."""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import operator, tlr
from tests._cases import problem

CASES = [
    (4, 4, 4, 2, "lowrank", 16),
    (8, 4, 8, 3, "dense", 40),
    (8, 8, 16, 5, "rule", 50),
    (8, 4, 8, [2, 0, 8, 1, 0, 3, 2, 0, 1, 4], [False, True, False, False], 33),
]


@pytest.mark.parametrize("nx,ny,b,ranks,mode,ns", CASES)
def test_tlr_forms_match_dense(nx, ny, b, ranks, mode, ns):
    D, U, perm, lay, _ = problem(nx, ny, b, ranks, mode, ns=ns, snr_db=10, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    Dt, Ut = Dh.T.copy(), Uh.T.copy()
    th = synth.cn(synth.rng(21), lay.size) * 0.3
    d = synth.cn(synth.rng(22), lay.size) * 0.2
    Y = tlr.apply(th, lay, Dt)
    Yd = operator.apply_y(th, lay, Dh)
    assert np.linalg.norm(Y - Yd) <= 1e-12 * np.linalg.norm(Yd)
    f, g, Rf = tlr.fgrad(th, lay, Dt, Ut)
    fd = operator.misfit(th, lay, Dh, Uh)
    gd = operator.gradient(th, lay, Dh, Uh)
    assert abs(f - fd) <= 1e-12 * fd
    assert np.linalg.norm(g - gd) <= 1e-12 * np.linalg.norm(gd)
    A1, A2 = tlr.line_terms(th, d, lay, Dt)
    cd = operator.line_coefficients(th, d, lay, Dh, Uh)
    E = Rf
    re = lambda a, b: np.vdot(a, b).real  # noqa: E731
    c = [0.5 * re(E, E), re(E, A1), 0.5 * re(A1, A1) + re(E, A2), re(A1, A2), 0.5 * re(A2, A2)]
    np.testing.assert_allclose(c, cd, rtol=1e-11, atol=1e-12 * abs(cd[0]))
