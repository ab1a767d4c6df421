"""FP32 SIMT operator, adjoint and gradients vs the FP64 oracle (eq. 6-9, 15-17, 25-27).

Tolerances (FP32 path): relative Frobenius error <= 1e-5 per operator
application, and every element within 1e-4 of the reference's rms value.
"""
import numpy as np
import pytest

import tlr_synth as synth
from oracle import layout, operator, tlr
from tests._cases import problem

pytestmark = pytest.mark.gpu
T = pytest.importorskip("paper_2412_14973_gb300")
from tests._gpu import Gpu, elem, rel  # noqa: E402

TOL, ETOL = 1e-5, 1e-4

CASES = {
    # name: (nx, ny, b, ranks, mode, ns)
    "dense256": (16, 16, 64, 8, "dense", 256),
    "ragged": (12, 8, 48, 5, "lowrank", 203),
    "mixed": (8, 8, 16, [3, 0, 16, 2, 1, 0, 4, 5, 2, 1], [False, True, True, False], 77),
    "one_tile_dense": (4, 4, 16, 0, "dense", 33),
    "one_tile_lr": (4, 4, 16, 6, "lowrank", 20),
    "rule_k_big": (16, 8, 32, 9, "rule", 130),
    "many_tiles": (32, 16, 32, 3, "lowrank", 96),
}


def _setup(name):
    nx, ny, b, ranks, mode, ns = CASES[name]
    D, U, perm, lay, _ = problem(nx, ny, b, ranks, mode, ns=ns, snr_db=10, planted=False)
    th = synth.cn(synth.rng(sorted(CASES).index(name)), lay.size) * 0.2
    # the oracle normalises by its own alpha (max |D|) and hands that value to
    # the library explicitly: nothing on the oracle side comes from the GPU
    Dh, Uh, alpha = operator.normalise(D, U, perm)
    g = Gpu(D, U, lay, nx=nx, ny=ny, alpha=alpha)
    return g, lay, th, Dh, Uh, perm


@pytest.mark.parametrize("name", sorted(CASES))
def test_apply(name):
    g, lay, th, Dh, Uh, _ = _setup(name)
    th = th.astype(np.complex64).astype(np.complex128)
    Y = g.apply(th)
    Yo = operator.apply_y(th, lay, Dh)
    assert rel(Y, Yo) <= TOL
    assert elem(Y, Yo) <= ETOL
    g.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_grad_and_misfit(name):
    g, lay, th, Dh, Uh, _ = _setup(name)
    th = th.astype(np.complex64).astype(np.complex128)
    f, gr = g.grad(th)
    fo = operator.misfit(th, lay, Dh, Uh)
    go = operator.gradient(th, lay, Dh, Uh)
    assert abs(f - fo) <= TOL * fo
    assert rel(gr, go) <= TOL
    assert elem(gr, go) <= ETOL
    # bitwise reproducible
    f2, gr2 = g.grad(th)
    assert f2 == f and np.array_equal(gr2, gr)
    g.close()


@pytest.mark.parametrize("name", ["dense256", "ragged", "mixed"])
def test_adjoint_and_dot_product(name):
    g, lay, th, Dh, Uh, _ = _setup(name)
    V = synth.cn(synth.rng(17), (lay.nr, Dh.shape[0])).astype(np.complex64).astype(np.complex128)
    G = g.adjoint(V)
    Go = operator.adjoint_g(V, Dh)
    assert rel(G, Go) <= TOL
    assert elem(G, Go) <= ETOL
    # <X Dfrak, V> = <X, V Dfrak^H> with the GPU's own products
    th32 = th.astype(np.complex64).astype(np.complex128)
    Y = g.apply(th32)
    Xh = operator.assemble_xh(th32, lay)
    lhs, rhs = np.vdot(Y, V), np.vdot(Xh, G)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    g.close()


@pytest.mark.parametrize("name", ["dense256", "mixed", "one_tile_lr"])
def test_unpermute_dense(name):
    g, lay, th, Dh, Uh, perm = _setup(name)
    th = th.astype(np.complex64).astype(np.complex128)
    X = g.unpermute(th)
    Xo = operator.unpermute(operator.assemble_xh(th, lay), perm)
    assert rel(X, Xo) <= TOL
    assert np.array_equal(X, X.T)     # reciprocity survives the back-mapping exactly
    g.close()


def test_gradient_of_zero_theta_is_minus_adjoint_image():
    # at theta = 0 the low-rank gradients vanish and the dense ones are
    # -(D^H U + (D^H U)^T)/2 restricted to the diagonal tiles
    g, lay, th, Dh, Uh, _ = _setup("dense256")
    f, gr = g.grad(np.zeros(lay.size))
    go = operator.gradient(np.zeros(lay.size), lay, Dh, Uh)
    assert rel(gr, go) <= TOL
    assert abs(f - 0.5 * np.vdot(Uh, Uh).real) <= TOL * f
    g.close()
