"""Pins for the oracle's L-BFGS loop (Sec. II-F; Nocedal & Wright Alg. 7.4).

* a strictly convex quadratic is minimised to its closed-form solution;
* the Rosenbrock function converges to (1, 1);
* every accepted step satisfies the Armijo condition (monotone decrease);
* the "stable over the last 20 steps" rule stops a run on a flat function;
* on a small SRWCR problem the registration lowers D monotonically;
* the two-loop recursion alone: with n pairs (s_i, A s_i) whose steps are
  A-conjugate it returns exactly -A^-1 g (the BFGS update keeps H y_j = s_j for
  every earlier conjugate pair), and for any history it meets the secant
  condition of the newest pair, H y = s.
"""
import numpy as np

import oracle
from oracle import lbfgs
import synth


def test_quadratic_reaches_closed_form_minimiser():
    rng = np.random.default_rng(0)
    Q = rng.normal(size=(12, 12))
    H = Q @ Q.T + 12 * np.eye(12)
    b = rng.normal(size=12)
    x_star = np.linalg.solve(H, b)
    res = lbfgs.minimise(lambda x: (0.5 * x @ H @ x - b @ x, H @ x - b), np.zeros(12),
                         lbfgs.LbfgsOptions(max_iter=200, stable_rtol=1e-15))
    assert np.linalg.norm(res.x - x_star) < 1e-6 * np.linalg.norm(x_star)


def test_rosenbrock_converges():
    def fg(x):
        a, b = x
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        g = np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
        return f, g
    res = lbfgs.minimise(fg, np.array([-1.2, 1.0]),
                         lbfgs.LbfgsOptions(max_iter=500, stable_rtol=1e-14))
    assert np.allclose(res.x, [1.0, 1.0], atol=1e-4)
    fs = [h[1] for h in res.history]
    assert all(f1 <= f0 for f0, f1 in zip(fs, fs[1:]))


def test_stable_window_stops_run():
    res = lbfgs.minimise(lambda x: (float(1e-3 * np.tanh(x @ x)), 2e-3 * x / np.cosh(x @ x) ** 2),
                         np.full(4, 0.01), lbfgs.LbfgsOptions(max_iter=500, stable_window=20))
    assert res.status in ("stable", "zero_gradient", "line_search_failed")
    assert res.n_iter < 500


def test_srwcr_registration_decreases_value(oracle_lib):
    pair = synth.make_pair("c1_2d_128")
    prob = pair.prob
    geo = oracle.Geometry.from_problem(prob)
    A, M = oracle.prepare(pair.fixed, pair.moving, prob.n_bins)

    def fg(x):
        D, g, _ = oracle.value_and_grad(geo, A, M, x.reshape(prob.coef_shape))
        return D, g.ravel()

    res = lbfgs.minimise(fg, np.zeros(prob.n_params), lbfgs.LbfgsOptions(max_iter=8))
    fs = [h[1] for h in res.history]
    D0 = fg(np.zeros(prob.n_params))[0]
    assert fs[0] < D0
    assert all(f1 <= f0 for f0, f1 in zip(fs, fs[1:]))
    assert fs[-1] < 0.97 * D0


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, n))
    return Q @ Q.T + n * np.eye(n), rng


def test_two_loop_with_conjugate_pairs_is_the_inverse_hessian():
    n = 7
    A, rng = _spd(n, 3)
    # A-conjugate steps by Gram-Schmidt in the A inner product.
    S = []
    for _ in range(n):
        v = rng.normal(size=n)
        for s in S:
            v -= (s @ A @ v) / (s @ A @ s) * s
        S.append(v)
    Y = [A @ s for s in S]
    for m in range(3):
        g = rng.normal(size=n)
        d = lbfgs.two_loop(g, S, Y)
        ref = -np.linalg.solve(A, g)
        assert np.linalg.norm(d - ref) <= 1e-10 * np.linalg.norm(ref)


def test_two_loop_meets_the_newest_secant_condition():
    n = 9
    A, rng = _spd(n, 4)
    for k in (1, 2, 5):
        S = [rng.normal(size=n) for _ in range(k)]
        Y = [A @ s + 0.1 * rng.normal(size=n) for s in S]
        assert all(s @ y > 0 for s, y in zip(S, Y))
        d = lbfgs.two_loop(Y[-1], S, Y)
        assert np.linalg.norm(d + S[-1]) <= 1e-12 * np.linalg.norm(S[-1])
    # one pair: a g orthogonal to s and y sees only the initial matrix
    # H0 = (s'y / y'y) I
    s1, y1 = S[0], Y[0]
    g = rng.normal(size=n)
    B = np.linalg.qr(np.stack([s1, y1], axis=1))[0]
    g -= B @ (B.T @ g)
    d = lbfgs.two_loop(g, [s1], [y1])
    assert np.linalg.norm(d + (s1 @ y1) / (y1 @ y1) * g) <= 1e-12 * np.linalg.norm(g)
    # no history: the steepest-descent direction
    g = rng.normal(size=n)
    assert np.array_equal(lbfgs.two_loop(g, [], []), -g)
