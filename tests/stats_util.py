"""Ensemble comparison used by the fast-precision parity tests: per statistic a z-test on
the mean, a z-test on the variance (SE of the variance from the fourth central moment)
and a two-sample Kolmogorov-Smirnov test, with Holm's step-down correction over all
p-values of a family.

Fast precision rounds propensities to FP32, so a G_j whose path is deterministic (an atom:
the reactants never change before T) differs from the FP64 value by up to ~2^-24
relative.  Such differences are below the stated resolution of the fast results, so G is
compared with a slack q = g_res * |mean|: the KS distance is the Levy-type
sup_x max(F_a(x) - F_b(x + q), F_b(x) - F_a(x + q)), and the mean and variance tests
subtract the slack from the observed differences."""
import numpy as np
from scipy import stats

G_RESOLUTION_FAST = 1e-6  # stated relative resolution of G in fast precision


def ks_slack(x, y, q):
    """Two-sample KS with slack q (q = 0: the ordinary statistic); asymptotic p-value."""
    if q <= 0:
        return float(stats.ks_2samp(x, y).pvalue)
    xs, ys = np.sort(x), np.sort(y)
    pts = np.concatenate([xs, ys])
    Fx = lambda t: np.searchsorted(xs, t, side="right") / xs.size
    Fy = lambda t: np.searchsorted(ys, t, side="right") / ys.size
    D = max(float(np.max(Fx(pts) - Fy(pts + q))), float(np.max(Fy(pts) - Fx(pts + q))), 0.0)
    en = np.sqrt(xs.size * ys.size / (xs.size + ys.size))
    return float(stats.kstwobign.sf(D * en))


def _z_p(d, se):
    if se == 0:
        return 1.0 if abs(d) < 1e-9 else 0.0
    return float(2 * stats.norm.sf(abs(d) / se))


def _var_se(x):
    n = x.size
    m = x.mean()
    m4 = np.mean((x - m) ** 4)
    s2 = x.var()
    return np.sqrt(max(m4 - s2 * s2, 0.0) / n)


def compare(a: dict, b: dict, keys=("X", "r", "G"), g_res=0.0):
    """a, b: dicts of (n, k) arrays.  g_res: relative resolution slack for G (0 for an
    exact comparison).  Returns list of (name, test, p, detail)."""
    rows = []
    for key in keys:
        A = np.asarray(a[key], np.float64)
        B = np.asarray(b[key], np.float64)
        for c in range(A.shape[1]):
            x, y = A[:, c], B[:, c]
            name = f"{key}[{c}]"
            q = g_res * abs(float(y.mean())) if key == "G" else 0.0
            scale = max(1.0, abs(y.mean()))
            if max(x.std(), y.std()) <= 1e-6 * scale:
                # a (numerically) constant statistic, e.g. G of a zero-order reaction = T:
                # equal up to single-precision rounding
                same = abs(x.mean() - y.mean()) <= 1e-5 * scale
                rows.append((name, "const", 1.0 if same else 0.0, (x.mean(), y.mean())))
                continue
            dm = x.mean() - y.mean()
            se_m = np.sqrt(x.var() / x.size + y.var() / y.size)
            rows.append((name, "mean", _z_p(max(abs(dm) - q, 0.0), se_m), (dm, se_m)))
            dv = x.var() - y.var()
            se_v = np.sqrt(_var_se(x) ** 2 + _var_se(y) ** 2)
            slack_v = 2 * q * max(x.std(), y.std()) + q * q
            rows.append((name, "var", _z_p(max(abs(dv) - slack_v, 0.0), se_v), (dv, se_v)))
            rows.append((name, "ks", ks_slack(x, y, q), None))
    return rows


def holm_pass(rows, alpha=0.01):
    """Holm's step-down procedure rejects some hypothesis iff the smallest p-value is
    below alpha / m, so the family passes iff min p >= alpha / m."""
    if not rows:
        return True
    return min(r[2] for r in rows) >= alpha / len(rows)


def summary(rows):
    ps = [r[2] for r in rows]
    worst = min(rows, key=lambda r: r[2]) if rows else None
    return {"n_tests": len(rows), "min_p": min(ps) if ps else None,
            "worst": (worst[0], worst[1]) if worst else None,
            "holm_pass_0.01": holm_pass(rows)}
