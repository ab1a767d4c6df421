"""ADMM with an L-BFGS x-update for the TLR MDD problem (ADMM solver section).

The paper splits min f(theta) + g(theta) into x- and z-blocks (eq. 18):

* x-update (eq. 19): theta <- argmin f(theta) + rho/2 ||theta - z + u||^2,
  approximately, by limited-memory BFGS (Liu & Nocedal 1989);
* z-update (eq. 20-23): z <- (theta + u) / (1 + 2 lambda / rho), the prox of
  g = lambda(||Z-bar||^2 + ||L-bar||^2 + ||R-bar||^2);
* dual update (eq. 24): u <- u + theta - z.

lambda follows the paper's continuation lambda_{s+1} = 0.1 lambda_s from 10,
three stages (Hyper-parameter selection section).

Readings where the paper is silent (each is listed in the design notes):
* the dual is used in scaled form throughout (eq. 19 and 23 use ||. + Lambda||,
  eq. 24 writes rho(X - Z); with u = Lambda the scaled update is u += theta - z);
* z starts at theta_0 and u at zero; theta, z and u carry across stages;
* rho = 1, 2 ADMM iterations per stage, 5 L-BFGS iterations per x-update,
  memory m = 10, memory cleared at the start of every x-update;
* the line search is exact: C is bilinear in the factors, so
  phi(a) = f(theta + a d) + rho/2 ||theta + a d - v||^2 is a quartic in a; its
  minimiser over a > 0 is taken among the real roots of phi'(a);
* restart (the usual safeguard of L-BFGS, Liu & Nocedal 1989; Nocedal &
  Wright, Numerical Optimization, ch. 7): when the two-loop direction d is not
  a descent direction (Re<g, d> >= 0) the memory is cleared and the same
  iteration continues along d = -g; when the exact line search then finds no
  minimiser on a > 0 (g = 0, a stationary point, or a degenerate quartic) the
  iteration takes no step and clears the memory.  An iteration that does
  either counts as one restart.  A pair (s, y) is kept only if
  <s,y> > 1e-12 |s||y|;
* the returned iterate is theta (the x-block).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import tlr
from .layout import Layout


def _re(a, b) -> float:
    return float(np.vdot(a, b).real)


@dataclass
class SolveOpts:
    lam0: float = 10.0
    decay: float = 0.1
    stages: int = 3
    rho: float = 1.0
    admm_iters: int = 2
    lbfgs_iters: int = 5
    memory: int = 10


@dataclass
class SolveStats:
    f_hist: list = field(default_factory=list)   # data misfit f after every L-BFGS step
    alphas: list = field(default_factory=list)
    restarts: int = 0
    iters: int = 0
    status: str = "ok"


def quartic_eval(c, a: float) -> float:
    return c[0] + a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])))


def quartic_argmin(c):
    """Minimiser over a > 0 of c0 + c1 a + c2 a^2 + c3 a^3 + c4 a^4.

    Candidates are the real roots of the derivative 4c4 a^3 + 3c3 a^2 + 2c2 a + c1
    (numpy's companion-matrix roots, each polished by two Newton steps);
    the positive candidate with the smallest value wins, ties to the smaller a.
    Returns None when there is no positive stationary point.
    """
    coeffs = [4.0 * c[4], 3.0 * c[3], 2.0 * c[2], c[1]]
    while len(coeffs) > 1 and coeffs[0] == 0.0:
        coeffs.pop(0)
    if len(coeffs) == 1:
        return None
    roots = np.roots(coeffs)
    best = None
    for r in roots:
        if abs(r.imag) > 1e-7 * max(1.0, abs(r)):
            continue
        a = float(r.real)
        for _ in range(2):
            d1 = c[1] + a * (2 * c[2] + a * (3 * c[3] + a * 4 * c[4]))
            d2 = 2 * c[2] + a * (6 * c[3] + a * 12 * c[4])
            if d2 != 0.0:
                a -= d1 / d2
        if not (a > 0.0) or not math.isfinite(a):
            continue
        v = quartic_eval(c, a)
        if best is None or v < best[0] or (v == best[0] and a < best[1]):
            best = (v, a)
    return None if best is None else best[1]


def two_loop(g, S, Y):
    """L-BFGS direction -H g by the two-loop recursion with real inner
    products Re<a, b> (theta is treated as a real vector of twice its length);
    H0 = gamma I with gamma = <s,y>/<y,y> of the newest pair (1 if none)."""
    q = g.copy()
    alph = []
    for s, y in zip(reversed(S), reversed(Y)):
        a = _re(s, q) / _re(y, s)
        q = q - a * y
        alph.append(a)
    gamma = _re(S[-1], Y[-1]) / _re(Y[-1], Y[-1]) if S else 1.0
    r = gamma * q
    for (s, y), a in zip(zip(S, Y), reversed(alph)):
        bcoef = _re(y, r) / _re(y, s)
        r = r + (a - bcoef) * s
    return -r


class Problem:
    """f, its gradient and the line-search quartic for one frequency, in the
    TLR-structured FP64 forms (receiver-major Dfrak, Ufrak)."""

    def __init__(self, lay: Layout, Dt, Ut):
        self.lay, self.Dt, self.Ut = lay, np.asarray(Dt, np.complex128), np.asarray(Ut, np.complex128)

    def fgrad(self, theta):
        f, g, Rf = tlr.fgrad(theta, self.lay, self.Dt, self.Ut)
        self._Rf = Rf
        return f, g

    def coefficients(self, theta, d, rho, v):
        Rf = self._Rf
        A1, A2 = tlr.line_terms(theta, d, self.lay, self.Dt)
        c0 = 0.5 * _re(Rf, Rf)
        c1 = _re(Rf, A1)
        c2 = 0.5 * _re(A1, A1) + _re(Rf, A2)
        c3 = _re(A1, A2)
        c4 = 0.5 * _re(A2, A2)
        if rho:
            w = theta - v
            c0 += 0.5 * rho * _re(w, w)
            c1 += rho * _re(w, d)
            c2 += 0.5 * rho * _re(d, d)
        return np.array([c0, c1, c2, c3, c4])


def lbfgs(prob: Problem, theta, v, rho: float, iters: int, memory: int,
          stats: SolveStats | None = None, fg=None):
    """Approximate x-update of eq. (19): ``iters`` L-BFGS steps on
    phi(theta) = f(theta) + rho/2 ||theta - v||^2 with the exact line search.

    Returns (theta, f, grad f) at the final iterate."""
    stats = stats if stats is not None else SolveStats()
    theta = np.asarray(theta, dtype=np.complex128).copy()
    # ``fg`` carries f and grad f at theta from the previous x-update (the
    # z/u updates leave theta, hence the cached residual, unchanged).
    f, gf = fg if fg is not None else prob.fgrad(theta)
    g = gf + rho * (theta - v)
    S, Y = [], []
    for _ in range(iters):
        d = two_loop(g, S, Y)
        restarted = False
        if not (_re(g, d) < 0.0):
            # not a descent direction: clear the memory and continue this
            # iteration along steepest descent
            S, Y = [], []
            d = -g
            restarted = True
            stats.restarts += 1
        c = prob.coefficients(theta, d, rho, v)
        a = quartic_argmin(c) if c[1] < 0.0 else None
        if a is None:
            # no minimiser on a > 0 along d: no step, memory cleared
            S, Y = [], []
            if not restarted:
                stats.restarts += 1
            stats.f_hist.append(f)
            stats.alphas.append(0.0)
            stats.iters += 1
            continue
        s = a * d
        theta = theta + s
        f, gf = prob.fgrad(theta)
        g_new = gf + rho * (theta - v)
        y = g_new - g
        sy, ss, yy = _re(s, y), _re(s, s), _re(y, y)
        if sy > 1e-12 * math.sqrt(ss * yy):
            S.append(s)
            Y.append(y)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        g = g_new
        stats.f_hist.append(f)
        stats.alphas.append(a)
        stats.iters += 1
    return theta, f, gf


def admm(prob: Problem, theta0, opts: SolveOpts = SolveOpts(), stats: SolveStats | None = None):
    """ADMM (eq. 18-24) with lambda continuation; returns (theta, z, u, stats)."""
    stats = stats if stats is not None else SolveStats()
    theta = np.asarray(theta0, dtype=np.complex128).copy()
    z = theta.copy()
    u = np.zeros_like(theta)
    fg = None
    for s in range(opts.stages):
        lam = opts.lam0 * opts.decay ** s
        for _ in range(opts.admm_iters):
            theta, f, gf = lbfgs(prob, theta, z - u, opts.rho, opts.lbfgs_iters,
                                 opts.memory, stats, fg)
            fg = (f, gf)
            z = (theta + u) / (1.0 + 2.0 * lam / opts.rho)
            u = u + theta - z
    return theta, z, u, stats
