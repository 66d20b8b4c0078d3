"""ctypes binding of the CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this module.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, asdict

import numpy as np

from . import build as _build

MODE_ADAPTIVE, MODE_EXPLICIT_ONLY, MODE_SSA_ONLY = 0, 1, 2
ST_STEP_LIMIT, ST_NEWTON_FAIL, ST_REJECT_LIMIT, ST_PTRS_CAP = 1, 2, 4, 8


class _Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("n_c", C.c_int32), ("ssa_factor", C.c_double),
                ("n_ssa_explicit", C.c_int32), ("n_ssa_implicit", C.c_int32),
                ("pe_delta", C.c_double), ("stiff_ratio", C.c_double),
                ("newton_tol", C.c_double), ("newton_maxit", C.c_int32),
                ("fd_h", C.c_double), ("max_steps", C.c_int64),
                ("max_reject", C.c_int32), ("mode", C.c_int32), ("jacobian", C.c_int32)]


@dataclass
class Params:
    eps: float = 0.03
    n_c: int = 10
    ssa_factor: float = 10.0
    n_ssa_explicit: int = 100
    n_ssa_implicit: int = 10
    pe_delta: float = 0.05
    stiff_ratio: float = 100.0
    newton_tol: float = 1e-10
    newton_maxit: int = 20
    fd_h: float = 1e-7
    max_steps: int = 100_000_000
    max_reject: int = 64
    mode: int = MODE_ADAPTIVE
    jacobian: int = 0  # 0 forward differences, 1 exact (analytic)

    def c(self) -> _Params:
        return _Params(**asdict(self))


_LIBS: dict = {}


def lib(extra_flags=()):
    key = tuple(extra_flags)
    if key not in _LIBS:
        path = _build.build(extra_flags=extra_flags)
        L = C.CDLL(path)
        P = C.POINTER
        L.mlo_simulate.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                   P(C.c_double), C.c_int64, P(C.c_double), P(C.c_int64),
                                   C.c_int32, P(C.c_double), C.c_int32, P(_Params),
                                   C.c_uint64, C.c_uint64, P(C.c_int64), P(C.c_int64),
                                   P(C.c_double), P(C.c_uint32), P(C.c_int64)]
        L.mlo_simulate.restype = C.c_int
        L.mlo_simulate_grid.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                        P(C.c_double), C.c_int64, P(C.c_double), P(C.c_int64),
                                        C.c_int32, P(C.c_double), C.c_int32, P(_Params),
                                        C.c_uint64, C.c_uint64, P(C.c_double), C.c_int32,
                                        P(C.c_int64), P(C.c_int64), P(C.c_int64),
                                        P(C.c_double), P(C.c_uint32), P(C.c_int64)]
        L.mlo_simulate_grid.restype = C.c_int
        L.mlo_kl_sample.argtypes = [C.c_int64, P(C.c_int64), C.c_int64, C.c_int64,
                                    P(C.c_int64), C.c_int64, C.c_int32]
        L.mlo_kl_sample.restype = C.c_double
        L.mlo_kl_grid.argtypes = [C.c_int64, P(C.c_int64), C.c_int64, P(C.c_int64), C.c_int32,
                                  C.c_int32, C.c_int32, P(C.c_double), P(C.c_double)]
        L.mlo_kl_grid.restype = C.c_int
        L.mlo_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.mlo_u01_from_words.argtypes = [C.c_uint32, C.c_uint32]
        L.mlo_u01_from_words.restype = C.c_double
        for f in ("mlo_exp", "mlo_log"):
            getattr(L, f).argtypes = [C.c_double]
            getattr(L, f).restype = C.c_double
        L.mlo_log_factorial.argtypes = [C.c_int64]
        L.mlo_log_factorial.restype = C.c_double
        L.mlo_poisson.argtypes = [C.c_double, C.c_uint64, C.c_uint32, C.c_uint32,
                                  C.c_uint32, P(C.c_uint32)]
        L.mlo_poisson.restype = C.c_int64
        L.mlo_poisson_batch.argtypes = [C.c_double, C.c_uint64, C.c_int64, P(C.c_int64)]
        L.mlo_tau_select.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                     P(C.c_double), P(C.c_int64), P(C.c_uint8), C.c_double]
        L.mlo_tau_select.restype = C.c_double
        L.mlo_critical_set.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                       P(C.c_double), P(C.c_int64), C.c_int32, P(C.c_uint8),
                                       P(C.c_double)]
        L.mlo_critical_set.restype = C.c_double
        L.mlo_pick.argtypes = [C.c_int32, P(C.c_double), C.c_double]
        L.mlo_pick.restype = C.c_int32
        L.mlo_ssa_switch.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.mlo_ssa_switch.restype = C.c_int
        L.mlo_implicit_count.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.mlo_implicit_count.restype = C.c_int64
        L.mlo_implicit_leap.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                        P(C.c_double), P(C.c_int64), P(C.c_uint8),
                                        P(C.c_double), P(C.c_double), C.c_double,
                                        P(_Params), P(C.c_int64), P(C.c_int32)]
        L.mlo_implicit_leap.restype = C.c_int
        L.mlo_lane_tree_sum.argtypes = [P(C.c_double), C.c_int32]
        L.mlo_lane_tree_sum.restype = C.c_double
        L.mlo_implicit_solve.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                         P(C.c_double), P(C.c_int64), P(C.c_uint8),
                                         P(C.c_double), P(C.c_double), C.c_double,
                                         P(_Params), P(C.c_double), P(C.c_int32)]
        L.mlo_implicit_solve.restype = C.c_int
        L.mlo_gamma.argtypes = [C.c_double, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32,
                                P(C.c_uint32)]
        L.mlo_gamma.restype = C.c_double
        L.mlo_posterior_sample.argtypes = [C.c_int64, C.c_int32, P(C.c_double), C.c_int32,
                                           P(C.c_double), C.c_int32, P(C.c_int64),
                                           P(C.c_double), C.c_uint64, C.c_uint64,
                                           P(C.c_double), P(C.c_uint32)]
        L.mlo_resample_systematic.argtypes = [C.c_int64, P(C.c_double), C.c_uint64, C.c_uint64,
                                              P(C.c_int64)]
        _LIBS[key] = L
    return _LIBS[key]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def simulate(crn, n_traj, x0, T, theta=None, params: Params | None = None, seed=0,
             traj_id_base=0, extra_flags=(), t_obs=None):
    """Run the oracle.  x0: (N,) or (n_traj, N); T: scalar, (1,) or (n_traj,);
    theta: None or (n_traj, M); t_obs: None or (K,) observation times.  Returns dict X, r,
    G, status, counters, and X_obs (n_traj, K, N) when t_obs is given."""
    L = lib(extra_flags)
    params = params or Params()
    N, M = crn.n_species, crn.n_reactions
    x0 = np.ascontiguousarray(x0, np.int64)
    T = np.ascontiguousarray(np.atleast_1d(np.asarray(T, np.float64)))
    x0_per = int(x0.ndim == 2)
    T_per = int(T.shape[0] > 1)
    if theta is not None:
        theta = np.ascontiguousarray(theta, np.float64)
        assert theta.shape == (n_traj, M)
    X = np.zeros((n_traj, N), np.int64)
    r = np.zeros((n_traj, M), np.int64)
    G = np.zeros((n_traj, M), np.float64)
    st = np.zeros(n_traj, np.uint32)
    cnt = np.zeros((n_traj, 4), np.int64)
    K = 0 if t_obs is None else int(np.size(t_obs))
    tk = None if t_obs is None else np.ascontiguousarray(np.atleast_1d(t_obs), np.float64)
    Xo = np.zeros((n_traj, K, N), np.int64) if t_obs is not None else None
    pc = params.c()
    rc = L.mlo_simulate_grid(N, M, _p(crn.orders, C.c_int32), _p(crn.stoich, C.c_int32),
                             _p(crn.rates, C.c_double), n_traj,
                             _p(theta, C.c_double) if theta is not None else None,
                             _p(x0, C.c_int64), x0_per, _p(T, C.c_double), T_per,
                             C.byref(pc), seed, traj_id_base,
                             _p(tk, C.c_double) if K else None, K,
                             _p(Xo, C.c_int64) if K else None, _p(X, C.c_int64),
                             _p(r, C.c_int64), _p(G, C.c_double), _p(st, C.c_uint32),
                             _p(cnt, C.c_int64))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    out = {"X": X, "r": r, "G": G, "status": st, "counters": cnt}
    if t_obs is not None:
        out["X_obs"] = Xo
    return out


def kl_sample(a, b, max_bins=1024):
    """KL(p_a || q_b) of two integer samples under the binned, half-count-smoothed reading."""
    a = np.ascontiguousarray(a, np.int64)
    b = np.ascontiguousarray(b, np.int64)
    return lib().mlo_kl_sample(a.size, _p(a, C.c_int64), 1, b.size, _p(b, C.c_int64), 1,
                               max_bins)


def kl_grid(X_ref, X_test, max_bins=1024):
    """Per (time point, species) KL of X_test's marginals from X_ref's, both (n, K, N);
    returns (kl (K, N), mean)."""
    X_ref = np.ascontiguousarray(X_ref, np.int64)
    X_test = np.ascontiguousarray(X_test, np.int64)
    _, K, N = X_ref.shape
    assert X_test.shape[1:] == (K, N)
    kl = np.zeros((K, N))
    mean = C.c_double(0.0)
    if lib().mlo_kl_grid(X_ref.shape[0], _p(X_ref, C.c_int64), X_test.shape[0],
                         _p(X_test, C.c_int64), K, N, max_bins, _p(kl, C.c_double),
                         C.byref(mean)) != 0:
        raise ValueError("oracle rejected the arguments")
    return kl, mean.value


def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    L.mlo_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u01(w0, w1):
    return lib().mlo_u01_from_words(w0, w1)


def exp(x):
    return lib().mlo_exp(float(x))


def log(x):
    return lib().mlo_log(float(x))


def log_factorial(k):
    return lib().mlo_log_factorial(int(k))


def poisson(mu, seed=0, traj_id=0, step=0, stream=0):
    st = C.c_uint32(0)
    k = lib().mlo_poisson(float(mu), seed, traj_id, step, stream, C.byref(st))
    return int(k), int(st.value)


def poisson_batch(mu, n, seed=0):
    out = np.zeros(n, np.int64)
    lib().mlo_poisson_batch(float(mu), seed, n, _p(out, C.c_int64))
    return out


def lane_tree_sum(v):
    v = np.ascontiguousarray(v, np.float64)
    return lib().mlo_lane_tree_sum(_p(v, C.c_double), v.size)


def tau_select(crn, a, x, use=None, eps=0.03):
    a = np.ascontiguousarray(a, np.float64)
    x = np.ascontiguousarray(x, np.int64)
    use = np.ones(crn.n_reactions, np.uint8) if use is None else np.ascontiguousarray(use, np.uint8)
    return lib().mlo_tau_select(crn.n_species, crn.n_reactions, _p(crn.orders, C.c_int32),
                                _p(crn.stoich, C.c_int32), _p(a, C.c_double),
                                _p(x, C.c_int64), _p(use, C.c_uint8), eps)


def critical_set(crn, a, x, n_c=10):
    """Returns (crit mask as a bool array, ac, a0c)."""
    a = np.ascontiguousarray(a, np.float64)
    x = np.ascontiguousarray(x, np.int64)
    crit = np.zeros(crn.n_reactions, np.uint8)
    ac = np.zeros(crn.n_reactions)
    a0c = lib().mlo_critical_set(crn.n_species, crn.n_reactions, _p(crn.orders, C.c_int32),
                                 _p(crn.stoich, C.c_int32), _p(a, C.c_double), _p(x, C.c_int64),
                                 int(n_c), _p(crit, C.c_uint8), _p(ac, C.c_double))
    return crit.astype(bool), ac, a0c


def pick(w, target):
    w = np.ascontiguousarray(w, np.float64)
    return int(lib().mlo_pick(w.size, _p(w, C.c_double), float(target)))


def ssa_switch(tau1, tau2, a0, ssa_factor):
    return bool(lib().mlo_ssa_switch(float(tau1), float(tau2), float(a0), float(ssa_factor)))


def implicit_count(a_y, tau, P, a_x):
    return int(lib().mlo_implicit_count(float(a_y), float(tau), float(P), float(a_x)))


def implicit_leap(crn, theta, x, nc, P, a_x, tau, params: Params | None = None):
    """Returns (rc, K, iterations); K of reactions with nc = 0 is left at 0."""
    params = params or Params()
    theta = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.int64)
    nc = np.ascontiguousarray(nc, np.uint8)
    P = np.ascontiguousarray(P, np.float64)
    a_x = np.ascontiguousarray(a_x, np.float64)
    K = np.zeros(crn.n_reactions, np.int64)
    its = C.c_int32(0)
    pc = params.c()
    rc = lib().mlo_implicit_leap(crn.n_species, crn.n_reactions, _p(crn.orders, C.c_int32),
                                 _p(crn.stoich, C.c_int32), _p(theta, C.c_double),
                                 _p(x, C.c_int64), _p(nc, C.c_uint8), _p(P, C.c_double),
                                 _p(a_x, C.c_double), float(tau), C.byref(pc), _p(K, C.c_int64),
                                 C.byref(its))
    return rc, K, int(its.value)


def implicit_solve(crn, theta, x, nc, P, a_x, tau, params: Params | None = None):
    params = params or Params()
    theta = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.int64)
    nc = np.ascontiguousarray(nc, np.uint8)
    P = np.ascontiguousarray(P, np.float64)
    a_x = np.ascontiguousarray(a_x, np.float64)
    y = np.zeros(crn.n_species)
    its = C.c_int32(0)
    pc = params.c()
    rc = lib().mlo_implicit_solve(crn.n_species, crn.n_reactions, _p(crn.orders, C.c_int32),
                                  _p(crn.stoich, C.c_int32), _p(theta, C.c_double),
                                  _p(x, C.c_int64), _p(nc, C.c_uint8), _p(P, C.c_double),
                                  _p(a_x, C.c_double), float(tau), C.byref(pc),
                                  _p(y, C.c_double), C.byref(its))
    return rc, y, int(its.value)


def gamma(shape, rate, seed=0, traj_id=0, stream=0):
    st = C.c_uint32(0)
    return lib().mlo_gamma(float(shape), float(rate), seed, traj_id, stream, C.byref(st)), st.value


def posterior_sample(alpha, beta, r, G, seed=0, traj_id_base=0):
    """theta[i, j] ~ Gamma(alpha_j + r[i, j], beta_j + G[i, j]); alpha, beta: (M,) or (n, M)."""
    r = np.ascontiguousarray(r, np.int64)
    G = np.ascontiguousarray(G, np.float64)
    n, M = r.shape
    alpha = np.ascontiguousarray(alpha, np.float64)
    beta = np.ascontiguousarray(beta, np.float64)
    th = np.zeros((n, M))
    st = np.zeros(n, np.uint32)
    rc = lib().mlo_posterior_sample(n, M, _p(alpha, C.c_double), int(alpha.ndim == 2),
                                    _p(beta, C.c_double), int(beta.ndim == 2), _p(r, C.c_int64),
                                    _p(G, C.c_double), seed, traj_id_base, _p(th, C.c_double),
                                    _p(st, C.c_uint32))
    if rc != 0:
        raise ValueError("bad arguments")
    return th, st


def resample_systematic(logw, seed=0, id_base=0):
    logw = np.ascontiguousarray(logw, np.float64)
    anc = np.zeros(logw.size, np.int64)
    if lib().mlo_resample_systematic(logw.size, _p(logw, C.c_double), seed, id_base,
                                     _p(anc, C.c_int64)) != 0:
        raise ValueError("no positive weight")
    return anc
