"""Pins for the decisions of one outer step of the oracle (Section 2): the critical set
and a0c, the inverse-CDF reaction pick (SSA and critical firings), the switch to SSA, and
the rounding and clamp of implicit firing counts.

Each decision is checked twice: on hand-computed single states through the exported
function the trajectory loop itself calls, and through a law of the whole method that a
mistake in the decision would break (binomial and multinomial laws that critical firings
reproduce exactly, and the fraction of first steps that are SSA bursts)."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1608_07058_gb300 import workloads as W


# --------------------------------------------------------------------------------------
# critical set
# --------------------------------------------------------------------------------------
def _critical_net():
    # species A, B, C; n_c = 10 in the tests below
    return W._crn("crit", 3, [
        ({0: 2}, {1: 1}, 1.0),          # R0: 2A -> B        L = floor(x_A / 2)
        ({1: 1}, {}, 1.0),              # R1: B -> 0         L = x_B
        ({2: 1}, {2: 1, 1: 1}, 1.0),    # R2: C -> C + B     C is a catalyst: never critical
        ({0: 1, 1: 1}, {2: 1}, 1.0),    # R3: A + B -> C     L = min(x_A, x_B)
        ({1: 1}, {0: 1}, 1.0),          # R4: B -> A         given a = 0 below
        ({0: 3}, {}, 1.0),              # R5: 3A -> 0        L = floor(x_A / 3)
    ])


def test_critical_set_hand_state_at_threshold(oracle):
    """x = (20, 9, 1), n_c = 10.  R0: L = 20 // 2 = 10 = n_c, not critical (the test is
    L < n_c).  R1: L = 9, critical.  R2 consumes nothing (its only reactant C is a
    catalyst), not critical although C = 1.  R3: L = min(20, 9) = 9, critical.  R4 has
    a = 0, not critical although L = 9.  R5: L = 20 // 3 = 6, critical.
    a0c = a1 + a3 + a5 = 2 + 8 + 32."""
    crn = _critical_net()
    a = [1.0, 2.0, 4.0, 8.0, 0.0, 32.0]
    crit, ac, a0c = oracle.critical_set(crn, a, [20, 9, 1], n_c=10)
    assert crit.tolist() == [False, True, False, True, False, True]
    assert ac.tolist() == [0.0, 2.0, 0.0, 8.0, 0.0, 32.0]
    assert a0c == 42.0


def test_critical_set_hand_state_below_threshold(oracle):
    """x = (19, 10, 0): R0: L = 9 (critical), R1: L = 10 (not), R3: L = min(19, 10) = 10
    (not), R5: L = 6 (critical); R2 with a = 4 at C = 0 still consumes nothing."""
    crn = _critical_net()
    a = [1.0, 2.0, 4.0, 8.0, 16.0, 32.0]
    crit, ac, a0c = oracle.critical_set(crn, a, [19, 10, 0], n_c=10)
    assert crit.tolist() == [True, False, False, False, False, True]
    assert a0c == 33.0
    # R4 (B -> A) at B = 10 with a > 0 is not critical: L = 10
    # n_c = 11 makes every reaction with L <= 10 and a > 0 critical
    crit, _, a0c = oracle.critical_set(crn, a, [19, 10, 0], n_c=11)
    assert crit.tolist() == [True, True, False, True, True, True]
    assert a0c == 1.0 + 2.0 + 8.0 + 16.0 + 32.0
    # n_c = 0 makes nothing critical
    crit, _, a0c = oracle.critical_set(crn, a, [19, 10, 0], n_c=0)
    assert not crit.any() and a0c == 0.0


# --------------------------------------------------------------------------------------
# reaction pick
# --------------------------------------------------------------------------------------
def test_pick_hand_values(oracle):
    w = [0.0, 3.0, 0.0, 1.0, 4.0, 0.0]       # prefix sums 0, 3, 3, 4, 8, 8
    assert oracle.pick(w, 0.0) == 1            # 0 < 0 is false, 0 < 3 is true
    assert oracle.pick(w, 2.999) == 1
    assert oracle.pick(w, 3.0) == 3            # strict: 3 < 3 false, 3 < 4 true
    assert oracle.pick(w, 3.5) == 3
    assert oracle.pick(w, 4.0) == 4
    assert oracle.pick(w, 7.999) == 4
    assert oracle.pick(w, 8.0) == 4            # no prefix exceeds: last positive weight
    assert oracle.pick(w, 100.0) == 4
    assert oracle.pick([0.0, 0.0], 0.0) == -1  # nothing positive


def test_pick_frequencies_follow_weights(oracle):
    """With target = u * sum(w) on a uniform grid of u, reaction j is picked for a
    fraction w_j / sum(w) of the grid (up to one grid cell per boundary)."""
    w = np.array([0.5, 0.0, 2.0, 1.5, 0.0, 4.0])
    tot = w.sum()
    n = 8000
    picks = [oracle.pick(w, (i + 0.5) / n * tot) for i in range(n)]
    counts = np.bincount(picks, minlength=w.size)
    assert np.all(np.abs(counts - n * w / tot) <= 1)


# --------------------------------------------------------------------------------------
# switch to SSA
# --------------------------------------------------------------------------------------
def test_ssa_switch_hand_values(oracle):
    inf = math.inf
    # a0 = 1000, f = 10: threshold f / a0 = 0.01
    assert not oracle.ssa_switch(0.02, inf, 1000.0, 10.0)   # leap: no critical reaction
    assert oracle.ssa_switch(0.005, inf, 1000.0, 10.0)      # the leap itself is too short
    assert oracle.ssa_switch(0.02, 0.009, 1000.0, 10.0)     # the critical wait is too short
    assert not oracle.ssa_switch(0.02, 0.011, 1000.0, 10.0)
    assert not oracle.ssa_switch(0.01, inf, 1000.0, 10.0)   # strict comparison
    assert not oracle.ssa_switch(0.5, 0.3, 1000.0, 0.0)     # f = 0: never
    assert oracle.ssa_switch(inf, 1e-9, 1e9, 10.0)          # tau1 = inf, tau2 decides


def _two_decays(kA, xA_first=False):
    # R0: B -> 0 (k = 1), R1: A -> 0 (k = kA); species 0 = A, 1 = B.  B is listed first so
    # that a pick over all propensities instead of the critical ones would choose B.
    return W._crn("two decays", 2, [({1: 1}, {}, 1.0), ({0: 1}, {}, kA)])


def test_ssa_switch_whole_method_first_step(oracle):
    """One outer step (max_steps = 1) from A = 5 (critical, a_A = 1e6) and B = 1e6
    (non-critical, a_B = 1e6): tau1 = tau_ex(B) = min(3e4 / 1e6, 9e8 / 1e6) = 0.03 and
    f / a0 = 10 / 2e6 = 5e-6, so the step is an SSA burst exactly when the drawn
    tau2 ~ Exp(a0c = 1e6) is below 5e-6: probability 1 - e^-5.  Without a critical
    reaction (A = 0) the step is a leap for f = 10 and a burst for f = 1e5 (f / a0 = 0.1
    exceeds tau1 = 0.03)."""
    crn = _two_decays(2e5)
    n = 10_000
    P = oracle.Params(max_steps=1)
    out = oracle.simulate(crn, n, [5, 1_000_000], [1.0], params=P, seed=4)
    burst = out["counters"][:, 2] > 0
    leap = out["counters"][:, 0] == 1
    assert np.all(burst ^ leap)
    p = 1.0 - math.exp(-5.0)
    sd = math.sqrt(n * p * (1 - p))
    assert abs(burst.sum() - n * p) < 4 * sd
    out = oracle.simulate(crn, 200, [0, 1_000_000], [1.0], params=P, seed=4)
    assert (out["counters"][:, 0] == 1).all() and (out["counters"][:, 2] == 0).all()
    out = oracle.simulate(crn, 200, [0, 1_000_000], [1.0],
                          params=oracle.Params(max_steps=1, ssa_factor=1e5), seed=4)
    assert (out["counters"][:, 2] == 100).all() and (out["counters"][:, 0] == 0).all()


# --------------------------------------------------------------------------------------
# laws that critical firings reproduce exactly
# --------------------------------------------------------------------------------------
def _chisq_p(obs, probs, min_expected=5.0):
    """Chi-square p-value with cells below min_expected pooled into one."""
    obs = np.asarray(obs, float)
    exp = np.asarray(probs, float) * obs.sum()
    small = exp < min_expected
    if small.any():
        obs = np.concatenate([obs[~small], [obs[small].sum()]])
        exp = np.concatenate([exp[~small], [exp[small].sum()]])
    return stats.chisquare(obs, exp).pvalue


def test_pure_decay_all_critical_is_binomial(oracle):
    """A -> 0 (k = 1) from x0 = 5 with n_c = 10: the reaction is critical throughout, so it
    fires once at a time, either in an SSA burst or as the critical firing at tau2 ~
    Exp(a0c) (tau1 is infinite: no non-critical reaction bounds it).  With the default
    ssa_factor = 10 and a0c = a0 a step leaps only when tau2 >= 10 / a0 (probability
    e^-10), so X(T) ~ Bin(5, e^-kT) up to a deviation of order e^-10."""
    crn = W.pure_decay(1.0)
    n = 20_000
    out = oracle.simulate(crn, n, [5], [1.0], seed=12)
    obs = np.bincount(out["X"][:, 0], minlength=6)
    assert obs.size == 6
    assert _chisq_p(obs, stats.binom.pmf(np.arange(6), 5, math.exp(-1.0))) > 1e-3


@pytest.mark.parametrize("f,T", [(0.5, 1.0), (0.25, 2.0), (1.0, 1.5)])
def test_ssa_switch_compares_the_drawn_critical_wait(oracle, f, T):
    """The switch compares the drawn wait tau2 (not its mean 1/a0c) with f / a0, and a leap
    then keeps that tau2.  For one molecule decaying at rate 1 (critical, a0c = a0 = 1,
    tau1 infinite) the first step is an SSA burst with probability 1 - e^-f, after which
    the molecule survives to T with probability e^-T; otherwise tau2 is conditioned on
    tau2 >= f, i.e. tau2 = f + Exp(1), and survives with probability e^-(T - f) for T >= f.
    So P(X(T) = 1) = e^-T (2 - e^-f).  (Comparing the mean wait instead would never switch
    here and give e^-T; leaving tau2 out of the comparison would too.)"""
    n = 40_000
    out = oracle.simulate(W.pure_decay(1.0), n, [1], [T], params=oracle.Params(ssa_factor=f),
                          seed=12)
    p = math.exp(-T) * (2.0 - math.exp(-f))
    got = (out["X"][:, 0] == 1).mean()
    assert abs(got - p) < 4 * math.sqrt(p * (1 - p) / n)


def test_critical_firing_beside_leaps_is_exact_binomial(oracle):
    """A -> 0 (critical, A = 5) beside B -> 0 (B = 1e6, leaped with tau = 0.03): A fires
    only as the critical firing of a leap (tau2 <= tau1) or inside a rare SSA burst, each
    an exponential clock at rate k A, so A(T) ~ Bin(5, e^-1); B's leaps do not touch it.
    (A leap keeps tau2 only when tau2 >= f / a0 = 1e-5, which removes 1e-5 / 0.03 of A's
    hazard, far below what 20,000 trajectories resolve.)  The pick must search the
    critical propensities only: B, listed first, would otherwise always be chosen and A
    would never decay."""
    crn = _two_decays(1.0)
    n = 20_000
    out = oracle.simulate(crn, n, [5, 1_000_000], [1.0], seed=21)
    assert out["counters"][:, 0].mean() > 30          # B is leaped
    A = out["X"][:, 0]
    obs = np.bincount(A, minlength=6)
    assert obs.size == 6
    assert _chisq_p(obs, stats.binom.pmf(np.arange(6), 5, math.exp(-1.0))) > 1e-3


def test_critical_pick_branching_is_multinomial(oracle):
    """A -> 0 (k1 = 1) and A -> B (k2 = 3), both critical from A = 8, beside C -> 0
    (C = 1e6, leaped): each A molecule independently decays by T = 0.25 with probability
    p = 1 - e^-1, through the first channel with probability k1 / (k1 + k2) = 1/4.  So
    (r_1, r_2, survivors) ~ Multinomial(8; p/4, 3p/4, 1 - p) (up to the 1e-5 / 0.03
    hazard deficit of the switch, as above)."""
    crn = W._crn("branch", 3, [({2: 1}, {}, 1.0), ({0: 1}, {}, 1.0), ({0: 1}, {1: 1}, 3.0)])
    n = 20_000
    out = oracle.simulate(crn, n, [8, 0, 1_000_000], [0.25], seed=33)
    r1, r2 = out["r"][:, 1], out["r"][:, 2]
    assert np.array_equal(out["X"][:, 1], r2)
    p = 1.0 - math.exp(-1.0)
    q = [p / 4, 3 * p / 4, 1 - p]
    cells, probs, obs = [], [], []
    for i in range(9):
        for k in range(9 - i):
            probs.append(stats.multinomial.pmf([i, k, 8 - i - k], 8, q))
            obs.append(int(((r1 == i) & (r2 == k)).sum()))
    assert abs(sum(probs) - 1.0) < 1e-12
    assert _chisq_p(obs, probs) > 1e-3


# --------------------------------------------------------------------------------------
# implicit firing counts
# --------------------------------------------------------------------------------------
def test_implicit_count_rounding_and_clamp(oracle):
    # v = (a_y tau + P) - a_x tau, exact in binary floating point
    assert oracle.implicit_count(5.0, 0.5, 2.0, 4.0) == 3     # v = 2.5: half away from zero
    assert oracle.implicit_count(5.0, 0.5, 3.0, 4.0) == 4     # v = 3.5
    assert oracle.implicit_count(7.0, 0.5, 2.0, 4.0) == 4     # v = 3.5
    assert oracle.implicit_count(7.5, 0.5, 2.0, 4.0) == 4     # v = 3.75, not floor
    assert oracle.implicit_count(4.5, 0.5, 2.0, 4.0) == 2     # v = 2.25
    assert oracle.implicit_count(2.0, 0.5, 0.0, 4.0) == 0     # v = -1: clamped
    assert oracle.implicit_count(3.0, 0.5, 0.0, 4.0) == 0     # v = -0.5: rounds to -1, clamped
    assert oracle.implicit_count(0.0, 1.0, 0.0, 0.0) == 0


def test_implicit_leap_competing_decays_closed_form(oracle):
    """B -> 0 (k0 = 1) and B -> C (k1 = 1) at x = (B, C) = (100, 0), tau = 0.5, both in
    the implicit system.  The implicit equation is linear:
    y_B = x_B - (P0 - a0 tau) - (P1 - a1 tau) - tau (k0 + k1) y_B, so
    y_B = x_B - (P0 + P1) / (1 + tau (k0 + k1)) = 100 - (P0 + P1) / 2.
    K_j = max(0, round(k_j y_B tau + P_j - k_j x_B tau)):
      P = (0, 40): y_B = 80, v = (-10, 30)      -> K = (0, 30)   (clamped below zero)
      P = (0, 41): y_B = 79.5, v = (-10.25, 30.75) -> K = (0, 31) (rounded, not floored)
      P = (9, 30): y_B = 80.5, v = (-0.75, 20.25) -> K = (0, 20)."""
    crn = W._crn("competing", 2, [({0: 1}, {}, 1.0), ({0: 1}, {1: 1}, 1.0)])
    x = [100, 0]
    a_x = [100.0, 100.0]
    for P, K_want in [((0, 40), (0, 30)), ((0, 41), (0, 31)), ((9, 30), (0, 20)),
                      ((30, 30), (15, 15))]:
        for jac in (0, 1):
            rc, K, its = oracle.implicit_leap(crn, [1.0, 1.0], x, [1, 1], np.array(P, float),
                                              a_x, 0.5, oracle.Params(jacobian=jac))
            assert rc == 0
            assert tuple(K) == K_want, (P, jac, K)
