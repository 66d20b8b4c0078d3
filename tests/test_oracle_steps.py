"""Pins for single steps of the oracle: the canonical reaction sum, Cao 2006 step sizes
on hand-computed states, and the implicit Newton solve against a linear solve."""
import math
from fractions import Fraction

import numpy as np

from paper_1608_07058_gb300 import workloads as W


def test_lane_tree_sum_exact_on_integers(oracle):
    rng = np.random.default_rng(0)
    for n in [1, 2, 5, 31, 32, 33, 64, 100, 257]:
        v = rng.integers(0, 2**20, n).astype(np.float64)
        assert oracle.lane_tree_sum(v) == float(v.sum())


def test_lane_tree_sum_rounding_bound(oracle):
    rng = np.random.default_rng(1)
    for n in [3, 17, 40, 100]:
        v = np.exp(rng.uniform(-30, 30, n))
        exact = sum(Fraction(float(x)) for x in v)
        got = oracle.lane_tree_sum(v)
        # a summation tree of depth d has relative error below d * 2^-53
        depth = 5 + math.ceil(n / 32)
        assert abs(Fraction(got) - exact) <= depth * 2.0**-53 * float(exact)


def test_tau_immigration_death_hand_values(oracle):
    crn = W.immigration_death()
    # x = 100: a = (10, 10); mu = 0, sigma^2 = 20, bound = 0.03*100 = 3 -> tau = 9/20
    assert abs(oracle.tau_select(crn, [10.0, 10.0], [100]) - 0.45) < 1e-15
    # x = 0: a = (10, 0); mu = 10, sigma^2 = 10, bound = max(0, 1) = 1 -> tau = 1/10
    assert abs(oracle.tau_select(crn, [10.0, 0.0], [0]) - 0.1) < 1e-16


def test_tau_pure_decay_hand_value(oracle):
    crn = W.pure_decay(1.0)
    # x = 1000: mu = -1000, sigma^2 = 1000, bound = 30 -> min(30/1000, 900/1000) = 0.03
    assert abs(oracle.tau_select(crn, [1000.0], [1000]) - 0.03) < 1e-16
    # nothing consumes... with the reaction excluded there is no bound at all
    assert math.isinf(oracle.tau_select(crn, [1000.0], [1000], use=[0]))


def test_tau_dimerisation_hand_values(oracle):
    crn = W.dimerisation()
    x = [400, 798, 0]
    a = [400.0, 10.0 * 400 * 399 / 2, 1000.0 * 798, 0.1 * 798]
    # without the pair (2,3): S1: mu = -400, var = 400, h = 2 + 1/399 (2 S1 is a reactant)
    h1 = 2.0 + 1.0 / 399.0
    b1 = 0.03 * 400 / h1
    # S2: mu = -79.8, var = 79.8, h = 1, bound = 23.94 -> 0.3
    want_im = min(b1 / 400.0, b1 * b1 / 400.0, 23.94 / 79.8, 23.94**2 / 79.8)
    got_im = oracle.tau_select(crn, a, x, use=[1, 0, 0, 1])
    assert abs(got_im - want_im) < 1e-15 * want_im
    assert abs(got_im - 4788 / 319600) < 1e-15  # 12 * 399 / (799 * 400)
    # with the pair: S1 var = 400 + 4 (a2 + a3) = 6384400 -> tau = b1^2 / var
    got_ex = oracle.tau_select(crn, a, x)
    assert abs(got_ex - b1 * b1 / 6384400.0) < 1e-12 * got_ex
    # stiffness: the implicit step is more than 100 times longer
    assert got_im > 100 * got_ex


def test_tau_second_order_hor_factor(oracle):
    # 2A -> B at x = 100: h = 2 + 1/99; mu = -2 a, var = 4 a
    crn = W._crn("dim", 2, [({0: 2}, {1: 1}, 1.0)])
    a = 1.0 * 100 * 99 / 2
    h = 2.0 + 1.0 / 99.0
    b = 0.03 * 100 / h
    want = min(b / (2 * a), b * b / (4 * a))
    assert abs(oracle.tau_select(crn, [a], [100, 0]) - want) < 1e-15 * want
    # below two molecules the reaction cannot fire: no change expected, no bound
    assert math.isinf(oracle.tau_select(crn, [0.0], [1, 0]))


def test_tau_third_order_hor_factors(oracle):
    """Cao 2006's highest-order factors of third-order reactions, on hand values:
    3A: 3 + 1/(x-1) + 2/(x-2); 2A + B: 1.5 (2 + 1/(x_A-1)) for A and 3 for B;
    A + B + C: 3 for each."""
    eps = 0.03
    # 3A -> B at x = 1000: a = k C(1000, 3), mu_A = -3a, var_A = 9a, bound eps x / h
    crn = W._crn("tri", 2, [({0: 3}, {1: 1}, 1e-7)])
    a = 1e-7 * 1000 * 999 * 998 / 6
    h = (3.0 + 1.0 / 999.0) + 2.0 / 998.0
    b = eps * 1000 / h
    want = min(b / (3 * a), b * b / (9 * a))
    assert abs(oracle.tau_select(crn, [a], [1000, 0]) - want) < 1e-15 * want
    # at x = 50 the bound eps x / h < 1 is raised to one molecule
    a = 1e-7 * 50 * 49 * 48 / 6
    assert abs(oracle.tau_select(crn, [a], [50, 0]) - min(1 / (3 * a), 1 / (9 * a))) < 1e-15 / a
    # 2A + B -> C at (40, 30): A: h = 1.5 (2 + 1/39), mu = -2a, var = 4a; B: h = 3, mu = -a
    crn = W._crn("dimb", 3, [({0: 2, 1: 1}, {2: 1}, 1e-4)])
    a = 1e-4 * (40 * 39 / 2) * 30
    hA, hB = 1.5 * (2.0 + 1.0 / 39.0), 3.0
    bA, bB = max(eps * 40 / hA, 1.0), max(eps * 30 / hB, 1.0)
    want = min(bA / (2 * a), bA * bA / (4 * a), bB / a, bB * bB / a)
    assert abs(oracle.tau_select(crn, [a], [40, 30, 0]) - want) < 1e-15 * want
    crn = W._crn("dimb", 3, [({0: 2, 1: 1}, {2: 1}, 1e-8)])
    a = 1e-8 * (4000 * 3999 / 2) * 3000
    hA = 1.5 * (2.0 + 1.0 / 3999.0)
    bA, bB = eps * 4000 / hA, eps * 3000 / 3.0
    want = min(bA / (2 * a), bA * bA / (4 * a), bB / a, bB * bB / a)
    assert abs(oracle.tau_select(crn, [a], [4000, 3000, 0]) - want) < 1e-15 * want
    # A + B + C -> D at (2000, 3000, 4000): h = 3 for each, mu = -a, var = a
    crn = W._crn("abc", 4, [({0: 1, 1: 1, 2: 1}, {3: 1}, 1e-9)])
    a = 1e-9 * 2000 * 3000 * 4000
    want = min(min(eps * x / 3 / a, (eps * x / 3) ** 2 / a) for x in (2000, 3000, 4000))
    assert abs(oracle.tau_select(crn, [a], [2000, 3000, 4000, 0]) - want) < 1e-15 * want
    assert abs(want - 20.0 / 24.0) < 1e-12  # species A decides: bound 20 over a = 24


def test_implicit_solve_linear_network_matches_linear_solve(oracle):
    # isomerisation A <-> B: a(y) = (k1 yA, k2 yB) is linear, so the implicit equation
    # y = c + tau nu^T a(y) is the linear system (I - tau nu^T K) y = c.
    k1, k2 = 3.0, 5.0
    crn = W.isomerisation(k1, k2)
    x = np.array([700, 300])
    tau = 0.8
    a_x = np.array([k1 * 700, k2 * 300])
    P = np.array([1650.0, 1540.0])
    rc, y, its = oracle.implicit_solve(crn, [k1, k2], x, [1, 1], P, a_x, tau)
    assert rc == 0 and its <= 3
    nu = crn.stoich.astype(float)              # (M, N)
    Kmat = np.array([[k1, 0.0], [0.0, k2]])    # da/dy
    c = x + nu.T @ (P - a_x * tau)
    y_lin = np.linalg.solve(np.eye(2) - tau * nu.T @ Kmat, c)
    assert np.allclose(y, y_lin, rtol=1e-9, atol=1e-9)


def test_implicit_solve_dimerisation_residual(oracle):
    crn = W.dimerisation()
    th = crn.rates
    x = np.array([400, 798, 0])
    g = np.array([400.0, 400 * 399 / 2, 798.0, 798.0])
    a_x = th * g
    tau = 0.015
    P = np.round(a_x * tau) + np.array([3, -40, 25, 1])
    rc, y, its = oracle.implicit_solve(crn, th, x, [1, 1, 1, 1], P, a_x, tau)
    assert rc == 0 and its < 10
    gy = np.array([y[0], y[0] * (y[0] - 1) / 2, y[1], y[1]])
    resid = y - x - crn.stoich.T @ (P - a_x * tau) - tau * crn.stoich.T @ (th * gy)
    assert np.max(np.abs(resid)) < 1e-6


def _higher_order_network():
    # 3A -> B, 2A + B -> C, A + B + C -> A, C -> 0: derivatives of C(y,3), C(y,2)C(y',1),
    # and a product of three first-order factors
    return W._crn("ho", 3, [({0: 3}, {1: 1}, 2e-4), ({0: 2, 1: 1}, {2: 1}, 3e-5),
                            ({0: 1, 1: 1, 2: 1}, {0: 1}, 1e-6), ({2: 1}, {}, 0.5)])


def _props(crn, th, y):
    from math import comb
    g = np.ones(crn.n_reactions)
    for j in range(crn.n_reactions):
        for s in range(crn.n_species):
            m = crn.orders[j, s]
            if m == 1:
                g[j] *= y[s]
            elif m == 2:
                g[j] *= y[s] * (y[s] - 1) / 2
            elif m == 3:
                g[j] *= y[s] * (y[s] - 1) * (y[s] - 2) / 6
    return th * g


def test_implicit_solve_analytic_jacobian_linear(oracle):
    k1, k2 = 3.0, 5.0
    crn = W.isomerisation(k1, k2)
    x = np.array([700, 300])
    tau, a_x = 0.8, np.array([k1 * 700, k2 * 300])
    P = np.array([1650.0, 1540.0])
    rc, y, its = oracle.implicit_solve(crn, [k1, k2], x, [1, 1], P, a_x, tau,
                                       oracle.Params(jacobian=1))
    c = x + crn.stoich.T.astype(float) @ (P - a_x * tau)
    y_lin = np.linalg.solve(np.eye(2) - tau * crn.stoich.T @ np.diag([k1, k2]), c)
    assert rc == 0 and its <= 2            # exact Jacobian of a linear map: one step
    assert np.allclose(y, y_lin, rtol=1e-12, atol=1e-9)


def test_implicit_solve_analytic_jacobian_converges_quadratically(oracle):
    """With the exact Jacobian Newton converges quadratically: from the state itself it
    reaches 1e-10 in a handful of iterations, as fast as or faster than with forward
    differences, to the same root; a wrong derivative would not."""
    crn = _higher_order_network()
    th = crn.rates
    x = np.array([400, 300, 200])
    a_x = _props(crn, th, x.astype(float))
    for tau in (0.01, 0.1, 1.0):
        P = np.round(a_x * tau) + np.array([3, -2, 1, 4])
        rc_a, y_a, it_a = oracle.implicit_solve(crn, th, x, [1, 1, 1, 1], P, a_x, tau,
                                                oracle.Params(jacobian=1))
        rc_f, y_f, it_f = oracle.implicit_solve(crn, th, x, [1, 1, 1, 1], P, a_x, tau,
                                                oracle.Params(jacobian=0))
        assert rc_a == 0 and rc_f == 0
        assert it_a <= it_f and it_a <= 10
        assert np.allclose(y_a, y_f, rtol=1e-9)
        resid = y_a - x - crn.stoich.T @ (P - a_x * tau) - tau * crn.stoich.T @ _props(crn, th, y_a)
        assert np.max(np.abs(resid)) < 1e-7 * max(1.0, np.max(np.abs(y_a)))


def test_analytic_jacobian_whole_method_same_law(oracle):
    # the dimerisation with either Jacobian: same implicit leaps, statistically equal
    w = W.config(1, n_traj=4000)
    fd = oracle.simulate(w.crn, w.n_traj, w.x0, w.T, params=oracle.Params(jacobian=0), seed=3)
    an = oracle.simulate(w.crn, w.n_traj, w.x0, w.T, params=oracle.Params(jacobian=1), seed=3)
    assert (an["counters"][:, 1] > 0).all()
    # coupled by the same random numbers and converging to the same roots within 1e-10,
    # nearly every trajectory is identical
    same = (fd["X"] == an["X"]).all(1).mean()
    assert same > 0.99
