"""Limited-memory BFGS for the oracle -- TEST INFRASTRUCTURE ONLY.

The paper minimises its cost with L-BFGS (Sec. II-F): 5 Hessian corrections,
a backtracking line search with a Wolfe condition, and a stop when the metric
has been stable over the last 20 steps or at the iteration limit.  This is a
plain NumPy restatement of the textbook method (two-loop recursion of Nocedal
& Wright, Numerical Optimization, Alg. 7.4) with the line-search constants
this repository adopts:

  * H0 = (s'y / y'y) I from the newest pair; first step of a (re)start has
    length 1 (alpha = 1/||g||), later iterations try alpha = 1;
  * Armijo constant c1 = 1e-4, weak-Wolfe curvature constant c2 = 0.9;
    the step halves when Armijo fails, doubles when only the curvature test
    fails; at most ``max_ls`` trials;
  * stop when |D_k - D_{k-w}| <= rtol * |D_k| for the window w (20; w <= 0
    turns this test off), when the gradient vanishes, or after ``max_iter``
    iterations.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Tuple

import numpy as np


@dataclass
class LbfgsOptions:
    m: int = 5
    max_iter: int = 200
    stable_window: int = 20
    stable_rtol: float = 1e-5
    max_ls: int = 20
    c1: float = 1e-4
    c2: float = 0.9
    shrink: float = 0.5
    grow: float = 2.0


@dataclass
class LbfgsResult:
    x: np.ndarray
    f: float
    n_iter: int
    n_evals: int
    status: str
    history: List[Tuple[int, float, float, float, int]] = field(default_factory=list)


def two_loop(g: np.ndarray, S: List[np.ndarray], Y: List[np.ndarray]) -> np.ndarray:
    """d = -H g by the two-loop recursion over the pairs (S, Y), oldest
    first: the first loop runs newest to oldest with rho_i = 1 / y_i's_i, the
    initial matrix is (s'y / y'y) I of the newest pair, and the second loop
    runs oldest to newest."""
    q = np.array(g, dtype=np.float64, copy=True)
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        alphas.append((a, rho))
        q -= a * y
    if S:
        q *= float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
        b = rho * float(y @ q)
        q += s * (a - b)
    return -q


def minimise(fg: Callable[[np.ndarray], Tuple[float, np.ndarray]], x0: np.ndarray,
             opts: LbfgsOptions = LbfgsOptions()) -> LbfgsResult:
    """Minimise f with gradient from ``fg(x) -> (f, g)`` (all float64)."""
    x = np.array(x0, dtype=np.float64, copy=True).ravel()
    f, g = fg(x)
    g = np.asarray(g, np.float64).ravel()
    n_evals = 1
    S: List[np.ndarray] = []
    Y: List[np.ndarray] = []
    fhist = [f]
    hist = []
    status = "max_iter"
    restart = True
    it = 0
    for it in range(1, opts.max_iter + 1):
        gnorm = float(np.linalg.norm(g))
        if gnorm == 0.0:
            status = "zero_gradient"
            it -= 1
            break
        d = two_loop(g, S, Y)
        gd = float(g @ d)
        if not gd < 0.0:
            S.clear(); Y.clear()
            d = -g
            gd = -gnorm * gnorm
            restart = True
        alpha = 1.0 / float(np.linalg.norm(d)) if restart else 1.0
        # Backtracking line search with the weak Wolfe curvature test.
        accepted = False
        for _ in range(opts.max_ls):
            xn = x + alpha * d
            fn, gn = fg(xn)
            gn = np.asarray(gn, np.float64).ravel()
            n_evals += 1
            if not np.isfinite(fn) or fn > f + opts.c1 * alpha * gd:
                alpha *= opts.shrink
                continue
            if float(gn @ d) < opts.c2 * gd:
                alpha *= opts.grow
                continue
            accepted = True
            break
        if not accepted:
            status = "line_search_failed"
            it -= 1
            break
        s_new, y_new = xn - x, gn - g
        x, f, g = xn, fn, gn
        if float(s_new @ y_new) > 0.0:
            S.append(s_new); Y.append(y_new)
            if len(S) > opts.m:
                S.pop(0); Y.pop(0)
        restart = False
        fhist.append(f)
        hist.append((it, f, float(np.linalg.norm(g)), alpha, n_evals))
        w = opts.stable_window
        if w > 0 and len(fhist) > w and abs(fhist[-1] - fhist[-1 - w]) <= opts.stable_rtol * abs(fhist[-1]):
            status = "stable"
            break
    return LbfgsResult(x, f, it, n_evals, status, hist)
