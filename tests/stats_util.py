"""Ensemble comparison used by the fast-precision parity tests: per statistic a z-test on
the mean, a z-test on the variance (SE of the variance from the fourth central moment)
and a two-sample Kolmogorov-Smirnov test, with Holm's step-down correction over all
p-values of a family."""
import numpy as np
from scipy import stats


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


def compare(a: dict, b: dict, keys=("X", "r", "G")):
    """a, b: dicts of (n, k) arrays.  Returns list of (name, test, p, detail)."""
    rows = []
    for key in keys:
        A = np.asarray(a[key], np.float64)
        B = np.asarray(b[key], np.float64)
        for c in range(A.shape[1]):
            x, y = A[:, c], B[:, c]
            name = f"{key}[{c}]"
            scale = max(1.0, abs(y.mean()))
            if max(x.std(), y.std()) <= 1e-6 * scale:
                # a (numerically) constant statistic, e.g. G of a zero-order reaction = T:
                # equal up to single-precision rounding
                same = abs(x.mean() - y.mean()) <= 1e-5 * scale
                rows.append((name, "const", 1.0 if same else 0.0, (x.mean(), y.mean())))
                continue
            dm = x.mean() - y.mean()
            se_m = np.sqrt(x.var() / x.size + y.var() / y.size)
            rows.append((name, "mean", _z_p(dm, se_m), (dm, se_m)))
            dv = x.var() - y.var()
            se_v = np.sqrt(_var_se(x) ** 2 + _var_se(y) ** 2)
            rows.append((name, "var", _z_p(dv, se_v), (dv, se_v)))
            rows.append((name, "ks", float(stats.ks_2samp(x, y).pvalue), None))
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
