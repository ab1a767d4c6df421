"""Pins for the ADMM / L-BFGS solver pieces (eq. 18-24) of the oracle."""
import numpy as np
import pytest
from scipy.optimize import minimize

import tlr_synth as synth
from oracle import benchmark, layout, operator, solver
from tests._cases import problem


def _as_real(z):
    return np.concatenate([z.real, z.imag])


def _as_cplx(x):
    n = x.size // 2
    return x[:n] + 1j * x[n:]


@pytest.mark.parametrize("lam", [0.0, 0.1, 10.0])
def test_prox_of_squared_frobenius_norm(lam):
    # eq. (21)-(22): prox_{lam ||.||^2}(V) = V / (1 + 2 lam), checked by numeric argmin
    V = synth.cn(synth.rng(1), 6)
    obj = lambda x: lam * np.sum(x ** 2) + 0.5 * np.sum((x - _as_real(V)) ** 2)  # noqa: E731
    num = _as_cplx(minimize(obj, np.zeros(12), tol=1e-14, method="BFGS").x)
    np.testing.assert_allclose(num, V / (1 + 2 * lam), atol=1e-7)


@pytest.mark.parametrize("lam,rho", [(0.1, 1.0), (10.0, 1.0), (1.0, 0.3)])
def test_z_update(lam, rho):
    # eq. (20) and (23): argmin_z lam||z||^2 + rho/2 ||x - z + u||^2 = (x + u)/(1 + 2 lam/rho)
    x = synth.cn(synth.rng(2), 5)
    u = synth.cn(synth.rng(3), 5)
    obj = lambda zr: lam * np.sum(zr ** 2) + 0.5 * rho * np.sum((_as_real(x + u) - zr) ** 2)  # noqa: E731
    num = _as_cplx(minimize(obj, np.zeros(10), tol=1e-14, method="BFGS").x)
    np.testing.assert_allclose(num, (x + u) / (1 + 2 * lam / rho), atol=1e-7)


def test_quartic_argmin_known_polynomial():
    # phi(a) = (a-2)^2 (a+1)^2 = a^4 - 2a^3 - 3a^2 + 4a + 4: minimisers a=2 and a=-1, max at 0.5
    c = [4.0, 4.0, -3.0, -2.0, 1.0]
    assert abs(solver.quartic_argmin(c) - 2.0) < 1e-14


@pytest.mark.parametrize("seed", range(20))
def test_quartic_argmin_vs_grid(seed):
    g = np.random.default_rng(seed)
    c = g.standard_normal(5)
    c[4] = abs(c[4]) + 0.1
    c[1] = -abs(c[1]) - 0.05          # descent at 0
    a = solver.quartic_argmin(c)
    grid = np.linspace(1e-6, 20, 400001)
    vals = c[0] + grid * (c[1] + grid * (c[2] + grid * (c[3] + grid * c[4])))
    assert solver.quartic_eval(c, a) <= vals.min() + 1e-9


def test_quadratic_case_is_a_line_minimum():
    # c3 = c4 = 0 (all tiles dense): a* = -c1 / (2 c2)
    c = [1.0, -3.0, 2.0, 0.0, 0.0]
    assert abs(solver.quartic_argmin(c) - 0.75) < 1e-15


def test_two_loop_secant_equation():
    # the L-BFGS inverse-Hessian maps the newest y to the newest s
    g = np.random.default_rng(0)
    S = [synth.cn(synth.rng(s), 7) for s in range(3)]
    A = g.standard_normal((14, 14))
    A = A @ A.T + 14 * np.eye(14)
    Y = [_as_cplx(A @ _as_real(s)) for s in S]
    d = solver.two_loop(Y[-1], S, Y)
    np.testing.assert_allclose(-d, S[-1], rtol=1e-12, atol=1e-12)


def test_lbfgs_exact_line_search_is_finite_on_quadratic():
    # one dense 4x4 tile and rho = 0: f is a convex quadratic in Z; the iterates
    # stay symmetric (grad Z = W'/2), 20 real unknowns, so L-BFGS with the exact
    # line search (CG-like on a quadratic) reaches the minimiser well within 40 steps
    D, U, perm, lay, _ = problem(2, 2, 4, 0, "dense", ns=12, snr_db=0, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    th0 = np.zeros(lay.size, np.complex128)
    th, f, gf = solver.lbfgs(prob, th0, np.zeros_like(th0), 0.0, 40, 50)
    Zs = benchmark.solve_eq4(Dh, Uh, 0.0 + 1e-300)
    Xs = 0.5 * (Zs + Zs.T)
    Xh = operator.assemble_xh(th, lay)
    assert np.linalg.norm(Xh - Xs) <= 1e-9 * np.linalg.norm(Xs)


def test_admm_reaches_benchmark_minimiser_for_one_dense_tile():
    # N = 1 dense diagonal: f + g of eq. (16) is exactly eq. (4); ADMM's fixed
    # point is its minimiser, the solution of the normal equations (CG, 1e-14)
    D, U, perm, lay, _ = problem(4, 2, 8, 0, "dense", ns=16, snr_db=10, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    lam = 0.1
    Zs = benchmark.solve_eq4(Dh, Uh, lam)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    opts = solver.SolveOpts(lam0=lam, decay=1.0, stages=1, rho=1.0, admm_iters=400,
                            lbfgs_iters=30, memory=20)
    th, z, u, st = solver.admm(prob, np.zeros(lay.size, np.complex128), opts)
    Z = th.reshape(8, 8)
    assert np.linalg.norm(Z - Zs) <= 1e-6 * np.linalg.norm(Zs)
    assert np.linalg.norm(th - z) <= 1e-6 * np.linalg.norm(z)


def test_planted_recovery_noise_free():
    # nr = 64 (8x8 grid), b = 16, k = 2, lambda = rho = 0: from the truth + 5%
    # the solver recovers X to better than 1e-6 (the data are exact)
    D, U, perm, lay, th_true = problem(8, 8, 16, 2, "lowrank", seed=4)
    U = (D.astype(np.complex128) @ operator.unpermute(operator.assemble_xh(th_true, lay), perm))
    Dh, Uh, _ = operator.normalise(D, U, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    th0 = th_true + 0.05 * np.abs(th_true).mean() * synth.cn(synth.rng(8), lay.size)
    th, f, gf = solver.lbfgs(prob, th0, np.zeros_like(th0), 0.0, 400, 10)
    X = operator.assemble_xh(th, lay)
    Xt = operator.assemble_xh(th_true, lay)
    assert np.linalg.norm(X - Xt) <= 1e-6 * np.linalg.norm(Xt)


def test_nr256_dense_diagonal_solve_runs_and_decreases():
    D, U, perm, lay, _ = problem(16, 16, 64, 8, "dense", seed=0, snr_db=20)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    th0 = np.zeros(lay.size, np.complex128)
    th0 += 0.01 * synth.cn(synth.rng(99), lay.size)
    th, z, u, st = solver.admm(prob, th0)
    assert st.iters == 30
    f0 = operator.misfit(th0, lay, Dh, Uh)
    assert st.f_hist[-1] < 0.5 * f0


def test_benchmark_solver_unitary_closed_form():
    # D-hat unitary (ns = nr): on symmetric matrices the normal operator of
    # eq. (4) is (1 + 2 lambda) I, so Z = P(D-hat^H U-hat) / (1 + 2 lambda)
    import tlr_synth as synth
    g = synth.rng(11)
    n, lam = 12, 0.3
    Dh = synth.haar_unitary(n, g)
    Uh = synth.cn(g, (n, n))
    Z = benchmark.solve_eq4(Dh, Uh, lam)
    B = Dh.conj().T @ Uh
    Zc = 0.5 * (B + B.T) / (1.0 + 2.0 * lam)
    assert np.linalg.norm(Z - Zc) <= 1e-12 * np.linalg.norm(Zc)


def test_benchmark_solver_matches_brute_force_real_system():
    # the objective of eq. (4) as a real least-squares problem in the 2 n^2
    # real unknowns of Z, built column by column from its definition and solved
    # densely; the CG minimiser must agree
    import tlr_synth as synth
    g = synth.rng(12)
    n, ns, lam = 3, 5, 0.05
    Dh = synth.cn(g, (ns, n))
    Uh = synth.cn(g, (ns, n))

    def residual_vec(Z):
        R = Dh @ (0.5 * (Z + Z.T))
        return np.concatenate([R.real.ravel(), R.imag.ravel(),
                               np.sqrt(2 * lam) * Z.real.ravel(), np.sqrt(2 * lam) * Z.imag.ravel()])

    cols = []
    for part in (1.0, 1j):
        for idx in range(n * n):
            E = np.zeros(n * n, np.complex128)
            E[idx] = part
            cols.append(residual_vec(E.reshape(n, n)))
    A = np.stack(cols, axis=1)
    rhs = np.concatenate([Uh.real.ravel(), Uh.imag.ravel(), np.zeros(2 * n * n)])
    sol = np.linalg.lstsq(A, rhs, rcond=None)[0]
    Zb = (sol[: n * n] + 1j * sol[n * n:]).reshape(n, n)
    Z = benchmark.solve_eq4(Dh, Uh, lam)
    assert np.linalg.norm(Z - Zb) <= 1e-9 * np.linalg.norm(Zb)


# ---- restart branches of the L-BFGS x-update (reading of the ADMM solver
# section's eq. 19: L-BFGS with the usual steepest-descent restart) ----

def _restart_problem():
    D, U, perm, lay, _ = problem(4, 4, 8, 2, "lowrank", ns=20, seed=21, snr_db=10, planted=False)
    Dh, Uh, _ = operator.normalise(D, U, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    th0 = 0.3 * synth.planted_theta(16, 8, 2, lay.dense, 22)
    v = 0.1 * synth.cn(synth.rng(23), lay.size)
    return prob, lay, Dh, Uh, th0, v


def _phi(th, lay, Dh, Uh, rho, v):
    # the x-update objective of eq. (19), from the dense-literal misfit
    w = th - v
    return operator.misfit(th, lay, Dh, Uh) + 0.5 * rho * float(np.vdot(w, w).real)


def test_ascent_direction_restarts_along_minus_g_in_the_same_iteration(monkeypatch):
    prob, lay, Dh, Uh, th0, v = _restart_problem()
    rho = 0.5
    th2, _, _ = solver.lbfgs(prob, th0, v, rho, 2, 10)
    th3_plain, _, _ = solver.lbfgs(prob, th0, v, rho, 3, 10)
    g2 = operator.gradient(th2, lay, Dh, Uh) + rho * (th2 - v)
    real_two_loop = solver.two_loop
    seen = []

    def forced(g, S, Y):
        seen.append(len(S))
        d = real_two_loop(g, S, Y)
        return g.copy() if len(seen) == 3 else d     # third call: an ascent direction

    monkeypatch.setattr(solver, "two_loop", forced)
    st = solver.SolveStats()
    th3, _, _ = solver.lbfgs(prob, th0, v, rho, 3, 10, st)
    assert seen == [0, 1, 2]              # pairs accumulated before the forced call
    assert st.restarts == 1 and st.iters == 3 and st.alphas[2] > 0.0
    assert not np.allclose(th3_plain, th3)
    # the restart iteration's step is the exact minimiser of phi along -g2,
    # found here by a grid and a bounded scalar search on the dense-literal objective
    from scipy.optimize import minimize_scalar
    phi = lambda a: _phi(th2 - a * g2, lay, Dh, Uh, rho, v)  # noqa: E731
    amax = 10.0 * st.alphas[2]
    grid = np.linspace(0.0, amax, 2001)
    a0 = grid[int(np.argmin([phi(a) for a in grid]))]
    res = minimize_scalar(phi, bounds=(max(0.0, a0 - amax / 1000), a0 + amax / 1000), method="bounded",
                          options={"xatol": 1e-14 * amax})
    step = th3 - th2
    a_taken = float(np.vdot(-g2, step).real / np.vdot(g2, g2).real)
    assert np.linalg.norm(step + a_taken * g2) <= 1e-12 * np.linalg.norm(step)   # along -g2
    assert abs(a_taken - res.x) <= 1e-6 * res.x
    # the memory was cleared: the next direction sees at most the restart's own pair
    seen.clear()
    solver.lbfgs(prob, th0, v, rho, 4, 10)
    assert seen[:3] == [0, 1, 2] and seen[3] <= 1


def test_no_minimiser_on_positive_steps_takes_no_step_and_clears_memory(monkeypatch):
    prob, lay, Dh, Uh, th0, v = _restart_problem()
    rho = 0.5
    th2, _, _ = solver.lbfgs(prob, th0, v, rho, 2, 10)
    real_coef = solver.Problem.coefficients
    calls = []

    def degenerate(self, theta, d, rho_, v_):
        calls.append(1)
        if len(calls) == 3:
            # c1 < 0 (descent) but phi is linear: no stationary point on a > 0
            return np.array([1.0, -1.0, 0.0, 0.0, 0.0])
        return real_coef(self, theta, d, rho_, v_)

    seen = []
    real_two_loop = solver.two_loop

    def spy(g, S, Y):
        seen.append((len(S), g.copy()))
        return real_two_loop(g, S, Y)

    monkeypatch.setattr(solver.Problem, "coefficients", degenerate)
    monkeypatch.setattr(solver, "two_loop", spy)
    st = solver.SolveStats()
    th3, _, _ = solver.lbfgs(prob, th0, v, rho, 3, 10, st)
    assert np.array_equal(th3, th2)                      # no step in the third iteration
    assert st.alphas[2] == 0.0 and st.restarts == 1 and st.iters == 3
    assert st.f_hist[2] == st.f_hist[1]
    seen.clear()
    calls.clear()
    st = solver.SolveStats()
    solver.lbfgs(prob, th0, v, rho, 4, 10, st)
    assert [n for n, _ in seen] == [0, 1, 2, 0]          # memory cleared: the fourth direction is -g
    assert st.restarts == 1


def test_stationary_start_restarts_every_iteration_without_a_step():
    # theta = 0 with low-rank diagonals: every factor product is bilinear, so
    # the gradient vanishes (a saddle): each iteration restarts, d = -g = 0,
    # and no step is taken
    prob, lay, Dh, Uh, _, v = _restart_problem()
    th0 = np.zeros(lay.size, np.complex128)
    st = solver.SolveStats()
    th, f, gf = solver.lbfgs(prob, th0, np.zeros_like(th0), 1.0, 5, 10, st)
    assert np.array_equal(th, th0) and st.restarts == 5 and st.iters == 5
    assert np.all(np.asarray(st.alphas) == 0.0)
    assert abs(f - 0.5 * float(np.vdot(Uh, Uh).real)) <= 1e-12 * f


@pytest.mark.parametrize("c", [[1.0, -1.0, 0.0, 0.0, 0.0],     # linear, decreasing
                               [0.0, -1.0, 0.0, -1.0, 0.0],    # cubic, phi' = -1 - 3a^2 < 0
                               [0.0, 1.0, 1.0, 0.0, 1.0],      # phi' = 1 + 2a + 4a^3 > 0 on a > 0
                               [2.0, 0.0, 0.0, 0.0, 0.0]])     # constant
def test_quartic_without_positive_stationary_point(c):
    assert solver.quartic_argmin(c) is None
