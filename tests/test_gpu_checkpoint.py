"""Checkpoint / resume of the solver (TLR_SOLVE_RESUME, TLR_SOLVE_REFRESH,
tlr_mdd_get_state / tlr_mdd_set_state): a solve split at ADMM-iteration
boundaries, with the state carried through host-visible z, u, reproduces the
uninterrupted solve bit for bit (the reductions have a fixed order)."""
import numpy as np
import pytest
import torch

import paper_2412_14973_gb300 as T

from _cases import problem
from _gpu import Gpu, dev, host

pytestmark = pytest.mark.gpu

BASE = dict(decay=0.5, rho=1.0, lbfgs_iters=4, memory=6)


def _state(g):
    z = torch.empty(g.lay.size, dtype=torch.complex64, device="cuda")
    u = torch.empty_like(z)
    T.tlr_mdd_get_state(g.h, z, u)
    return z, u


@pytest.mark.parametrize("prec", [T.TLR_PREC_FP32, T.TLR_PREC_BF16X3])
def test_split_solve_is_bit_identical(prec):
    D, U, perm, lay, th0 = problem(8, 8, 16, 2, "lowrank", ns=64, seed=80, snr_db=20, planted=False)
    R = T.TLR_SOLVE_REFRESH
    ga = Gpu(D, U, lay, nx=8, ny=8, precision=prec)
    th_a, st_a = ga.solve(th0, lam0=4.0, stages=3, admm_iters=2, flags=R, **BASE)

    # split at a stage boundary, state moved to a fresh handle through z, u
    gb = Gpu(D, U, lay, nx=8, ny=8, precision=prec)
    th_1, _ = gb.solve(th0, lam0=4.0, stages=1, admm_iters=2, flags=R, **BASE)
    z, u = _state(gb)
    gc = Gpu(D, U, lay, nx=8, ny=8, precision=prec)
    T.tlr_mdd_set_state(gc.h, z, u)
    th_b, _ = gc.solve(th_1, lam0=2.0, stages=2, admm_iters=2, flags=R | T.TLR_SOLVE_RESUME, **BASE)
    np.testing.assert_array_equal(th_b, th_a)

    # split inside the first stage, resumed on the same handle
    gd = Gpu(D, U, lay, nx=8, ny=8, precision=prec)
    t1, _ = gd.solve(th0, lam0=4.0, stages=1, admm_iters=1, flags=R, **BASE)
    t2, _ = gd.solve(t1, lam0=4.0, stages=1, admm_iters=1, flags=R | T.TLR_SOLVE_RESUME, **BASE)
    t3, _ = gd.solve(t2, lam0=2.0, stages=2, admm_iters=2, flags=R | T.TLR_SOLVE_RESUME, **BASE)
    np.testing.assert_array_equal(t3, th_a)
    assert st_a.iters == 3 * 2 * 4


def test_state_round_trip_and_resume_changes_the_start():
    D, U, perm, lay, th0 = problem(4, 4, 8, 2, "lowrank", seed=81, snr_db=20, planted=False)
    g = Gpu(D, U, lay, nx=4, ny=4)
    g.solve(th0, lam0=1.0, stages=1, admm_iters=2, **BASE)
    z, u = _state(g)
    g2 = Gpu(D, U, lay, nx=4, ny=4)
    T.tlr_mdd_set_state(g2.h, z, u)
    z2, u2 = _state(g2)
    assert torch.equal(z, z2) and torch.equal(u, u2)
    assert torch.any(u != 0)
    # resuming from a nonzero dual differs from a cold start at the same theta
    a, _ = g2.solve(th0, lam0=1.0, stages=1, admm_iters=1, flags=T.TLR_SOLVE_RESUME, **BASE)
    g3 = Gpu(D, U, lay, nx=4, ny=4)
    b, _ = g3.solve(th0, lam0=1.0, stages=1, admm_iters=1, **BASE)
    assert not np.array_equal(a, b)


def test_invalid_flags_and_arguments():
    D, U, perm, lay, th0 = problem(4, 4, 8, 2, "lowrank", seed=82)
    g = Gpu(D, U, lay, nx=4, ny=4)
    with pytest.raises(T.TLRError) as e:
        g.solve(th0, flags=4)
    assert e.value.code == T.TLR_ERR_ARG
    z = torch.zeros(lay.size, dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TLRError) as e:
        T.tlr_mdd_set_state(g.h, z, None)
    assert e.value.code == T.TLR_ERR_ARG
