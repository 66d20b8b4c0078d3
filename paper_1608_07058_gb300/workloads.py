"""Seeded synthetic inputs: reaction networks, per-trajectory rate constants, initial
states and horizons.

This module is shared by the CUDA path's callers and by the oracle's tests, so it holds
none of the simulation method's arithmetic: it only builds matrices and draws numbers.
The networks follow the paper's workload shapes (Section 3 "Results": a gene-network
model, a large signalling pathway, the stiff decaying-dimerising set of Rathinam 2003);
the paper's own model files are not available, so these synthetic networks stand in.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class CRN:
    """A mass-action network: orders[j, s] = reactant multiplicity m_js, stoich[j, s] =
    net change nu_js, rates[j] = base rate constant theta_j."""
    name: str
    orders: np.ndarray
    stoich: np.ndarray
    rates: np.ndarray
    species: tuple = ()

    def __post_init__(self):
        self.orders = np.ascontiguousarray(self.orders, dtype=np.int32)
        self.stoich = np.ascontiguousarray(self.stoich, dtype=np.int32)
        self.rates = np.ascontiguousarray(self.rates, dtype=np.float64)
        assert self.orders.shape == self.stoich.shape
        assert self.rates.shape == (self.orders.shape[0],)

    @property
    def n_species(self) -> int:
        return int(self.orders.shape[1])

    @property
    def n_reactions(self) -> int:
        return int(self.orders.shape[0])


def _crn(name, n_species, reactions, species=()):
    """reactions: list of (reactants {s: m}, products {s: m}, rate)."""
    M = len(reactions)
    orders = np.zeros((M, n_species), np.int32)
    stoich = np.zeros((M, n_species), np.int32)
    rates = np.zeros(M)
    for j, (re, pr, k) in enumerate(reactions):
        for s, m in re.items():
            orders[j, s] += m
            stoich[j, s] -= m
        for s, m in pr.items():
            stoich[j, s] += m
        rates[j] = k
    return CRN(name, orders, stoich, rates, tuple(species))


def immigration_death(k1: float = 10.0, k2: float = 0.1) -> CRN:
    """0 -> A (k1), A -> 0 (k2)."""
    return _crn("immigration_death", 1, [({}, {0: 1}, k1), ({0: 1}, {}, k2)], ("A",))


def pure_decay(k: float = 1.0) -> CRN:
    """A -> 0 (k)."""
    return _crn("pure_decay", 1, [({0: 1}, {}, k)], ("A",))


def isomerisation(k1: float = 1.0, k2: float = 2.0) -> CRN:
    """A -> B (k1), B -> A (k2)."""
    return _crn("isomerisation", 2, [({0: 1}, {1: 1}, k1), ({1: 1}, {0: 1}, k2)], ("A", "B"))


def dimerisation(c=(1.0, 10.0, 1000.0, 0.1)) -> CRN:
    """Stiff decaying-dimerising set (Rathinam, Petzold & Cao 2003):
    S1 -> 0, 2 S1 -> S2, S2 -> 2 S1, S2 -> S3."""
    return _crn("dimerisation", 3, [
        ({0: 1}, {}, c[0]),
        ({0: 2}, {1: 1}, c[1]),
        ({1: 1}, {0: 2}, c[2]),
        ({1: 1}, {2: 1}, c[3]),
    ], ("S1", "S2", "S3"))


GENE_THETA_TRUE = (0.05, 0.05, 10.0, 1.0, 5.0, 0.1)


def gene_expression(theta=GENE_THETA_TRUE) -> CRN:
    """Two-state gene expression with species (gene-on count G, mRNA, protein):
    on 0 -> G, off G -> 0, transcription G -> G + mRNA, mRNA decay, translation
    mRNA -> mRNA + protein, protein decay.  With three species under pure mass action the
    gene-on flag is a count (stationary Poisson(on/off))."""
    return _crn("gene_expression", 3, [
        ({}, {0: 1}, theta[0]),
        ({0: 1}, {}, theta[1]),
        ({0: 1}, {0: 1, 1: 1}, theta[2]),
        ({1: 1}, {}, theta[3]),
        ({1: 1}, {1: 1, 2: 1}, theta[4]),
        ({2: 1}, {}, theta[5]),
    ], ("G", "mRNA", "protein"))


def random_crn(seed: int = 3, n_species: int = 50, n_uni: int = 60, n_bi: int = 40,
               n_pairs: int = 10, ratio: float = 1e4):
    """Random large mass-action network and its initial state.

    Each species gets a weight w in {1,2,3}; every reaction keeps the total weight
    sum_s w_s x_s constant or lowers it, so all counts stay below the initial total
    weight (no blow-up by construction).  n_pairs reversible pairs (nu' = -nu) are placed
    near equilibrium at x0; the other reactions are drawn among A->0, A->B, A->2B,
    A->B+C (unimolecular) and A+B->C, 2A->B, A+B->C+D (bimolecular).  Initial counts are
    log-uniform in [10, 1e5].  Effective first-order rates kappa (k for unimolecular,
    k times the partner's initial count for bimolecular) are log-uniform over a span of
    `ratio`, [1e-3, 1e1], so the fast/slow timescale ratio is about `ratio`; weight-losing
    reactions are drawn from the slow decade.  Returns (CRN, x0).
    """
    rng = np.random.default_rng(seed)
    N = n_species
    w = rng.choice([1, 2, 3], size=N, p=[0.5, 0.3, 0.2])
    x0 = np.floor(np.exp(rng.uniform(np.log(10.0), np.log(1e5), size=N))).astype(np.int64)
    by_w = {v: np.flatnonzero(w == v) for v in (1, 2, 3)}
    lo, hi = 1e1 / ratio, 1e1

    def kappa(slow=False):
        if slow:
            return float(np.exp(rng.uniform(np.log(lo), np.log(lo * 10))))
        return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))

    reactions = []
    n_uni_left, n_bi_left = n_uni, n_bi
    # reversible pairs
    made = 0
    while made < n_pairs:
        kind = rng.integers(3)
        if kind == 0:  # A <-> B, equal weights
            cand = [v for v in (1, 2, 3) if len(by_w[v]) >= 2]
            v = cand[rng.integers(len(cand))]
            A, B = rng.choice(by_w[v], 2, replace=False)
            kf = kappa()
            kb = kf * x0[A] / x0[B]
            reactions += [({A: 1}, {B: 1}, kf), ({B: 1}, {A: 1}, kb)]
            n_uni_left -= 2
        elif kind == 1:  # 2A <-> B with w_B = 2 w_A
            v = int(rng.integers(1, 2))
            if len(by_w[v]) == 0 or len(by_w[2 * v]) == 0:
                continue
            A = int(rng.choice(by_w[v])); B = int(rng.choice(by_w[2 * v]))
            kb = kappa()
            kf = kb * x0[B] / (float(x0[A]) * x0[A])
            reactions += [({A: 2}, {B: 1}, kf), ({B: 1}, {A: 2}, kb)]
            n_bi_left -= 1; n_uni_left -= 1
        else:  # A + B <-> C with w_C = w_A + w_B
            wa, wb = (1, 1) if rng.random() < 0.5 else (1, 2)
            if len(by_w[wa]) < 2 or len(by_w[wb]) < 1 or len(by_w[wa + wb]) < 1:
                continue
            A = int(rng.choice(by_w[wa]))
            B = int(rng.choice([b for b in by_w[wb] if b != A]))
            C = int(rng.choice([c for c in by_w[wa + wb] if c not in (A, B)]))
            kb = kappa()
            kf = kb * x0[C] / (float(x0[A]) * x0[B])
            reactions += [({A: 1, B: 1}, {C: 1}, kf), ({C: 1}, {A: 1, B: 1}, kb)]
            n_bi_left -= 1; n_uni_left -= 1
        made += 1
    # remaining unimolecular reactions
    while n_uni_left > 0:
        A = int(rng.integers(N))
        kind = rng.integers(4)
        if kind == 0:
            reactions.append(({A: 1}, {}, kappa(slow=True)))
        elif kind == 1:
            okB = [b for b in range(N) if b != A and w[b] <= w[A]]
            if not okB:
                continue
            B = int(rng.choice(okB))
            reactions.append(({A: 1}, {B: 1}, kappa(slow=w[B] < w[A])))
        elif kind == 2:
            okB = [b for b in range(N) if b != A and 2 * w[b] <= w[A]]
            if not okB:
                continue
            B = int(rng.choice(okB))
            reactions.append(({A: 1}, {B: 2}, kappa(slow=2 * w[B] < w[A])))
        else:
            okB = [b for b in range(N) if b != A and w[b] < w[A]]
            if not okB:
                continue
            B = int(rng.choice(okB))
            okC = [c for c in range(N) if c not in (A, B) and w[B] + w[c] <= w[A]]
            if not okC:
                continue
            C = int(rng.choice(okC))
            reactions.append(({A: 1}, {B: 1, C: 1}, kappa(slow=w[B] + w[C] < w[A])))
        n_uni_left -= 1
    # remaining bimolecular reactions
    while n_bi_left > 0:
        A = int(rng.integers(N)); B = int(rng.integers(N))
        kind = rng.integers(2)
        if A == B:  # 2A -> B'
            okC = [c for c in range(N) if c != A and w[c] <= 2 * w[A]]
            C = int(rng.choice(okC))
            k = kappa(slow=w[C] < 2 * w[A]) / float(x0[A])
            reactions.append(({A: 2}, {C: 1}, k))
        elif kind == 0:  # A + B -> C
            okC = [c for c in range(N) if c not in (A, B) and w[c] <= w[A] + w[B]]
            C = int(rng.choice(okC))
            k = kappa(slow=w[C] < w[A] + w[B]) / float(x0[B])
            reactions.append(({A: 1, B: 1}, {C: 1}, k))
        else:  # A + B -> C + D
            okC = [c for c in range(N) if c not in (A, B) and w[c] < w[A] + w[B]]
            C = int(rng.choice(okC))
            okD = [d for d in range(N) if d not in (A, B, C) and w[C] + w[d] <= w[A] + w[B]]
            if not okD:
                continue
            D = int(rng.choice(okD))
            k = kappa(slow=w[C] + w[D] < w[A] + w[B]) / float(x0[B])
            reactions.append(({A: 1, B: 1}, {C: 1, D: 1}, k))
        n_bi_left -= 1
    order = rng.permutation(len(reactions))
    reactions = [reactions[i] for i in order]
    return _crn(f"random_crn_{N}x{len(reactions)}", N, reactions), x0


@dataclass
class Workload:
    """One simulate call: a network plus per-trajectory inputs and control parameters."""
    name: str
    crn: CRN
    n_traj: int
    x0: np.ndarray               # (N,) broadcast or (n_traj, N)
    T: np.ndarray                # (1,) broadcast or (n_traj,)
    theta: Optional[np.ndarray]  # (n_traj, M) or None (use crn.rates)
    eps: float = 0.03
    n_c: int = 10
    ssa_factor: float = 10.0
    seed: int = 0
    traj_id_base: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def x0_per_traj(self) -> bool:
        return self.x0.ndim == 2

    @property
    def T_per_traj(self) -> bool:
        return self.T.shape[0] > 1


def gene_theta(n_traj: int, seed: int = 0, theta_true=GENE_THETA_TRUE, shape: float = 2.0):
    """Per-trajectory rate constants theta_j ~ Gamma(shape, rate = shape / theta_true_j)."""
    rng = np.random.default_rng(seed)
    tt = np.asarray(theta_true, np.float64)
    return np.ascontiguousarray(rng.gamma(shape, tt / shape, size=(n_traj, tt.size)))


def config(i: int, n_traj: Optional[int] = None, seed: int = 0) -> Workload:
    """The five benchmark configurations (index 0..3; 4 is the serving mix, see
    serving_requests).  n_traj overrides the trajectory count (first n_traj rows of the
    full draw, so a smaller case is a prefix of the full one)."""
    if i == 0:
        B = 10_000 if n_traj is None else n_traj
        return Workload("immigration_death", immigration_death(), B,
                        np.array([0], np.int64), np.array([100.0]), None, seed=seed)
    if i == 1:
        B = 100_000 if n_traj is None else n_traj
        return Workload("dimerisation", dimerisation(), B,
                        np.array([400, 798, 0], np.int64), np.array([0.2]), None, seed=seed)
    if i == 2:
        full = 1_000_000
        B = full if n_traj is None else n_traj
        rng = np.random.default_rng(seed)
        T = rng.uniform(50.0, 200.0, size=full)[:B]
        theta = gene_theta(full, seed=seed + 1)[:B]
        return Workload("gene_expression", gene_expression(), B,
                        np.array([0, 0, 0], np.int64), np.ascontiguousarray(T),
                        np.ascontiguousarray(theta), seed=seed)
    if i == 3:
        B = 65_536 if n_traj is None else n_traj
        crn, x0 = random_crn(seed=3)
        return Workload("random_crn", crn, B, x0, np.array([10.0]), None, seed=seed)
    raise ValueError(f"no workload {i}")


# Horizon of each model's requests as a fraction of its benchmark horizon.  At 200
# requests/s of 1,000-100,000 trajectories (mean 21,500) each model is offered about
# 1.07e6 trajectories/s.  One GB300 simulates immigration-death at T = 100 at about
# 5e6/s, the dimerisation at T = 0.2 at about 3e7/s, gene expression at T ~ 125 at about
# 4.6e5/s (SSA-bound: the offered load would be 2.3 GPUs) and the 50 x 100 network at
# T = 10 at about 2e2/s (5,000 GPUs).  The scales bring every model to a fraction of one
# GPU: immigration-death 0.5 (about 10 %), dimerisation 1 (3 %), gene expression 0.03
# (7 %), random network 5e-5 (about 25 %), so that the mix as a whole is servable.
SERVING_HORIZON_SCALE = {0: 0.5, 1: 1.0, 2: 0.03, 3: 5e-5}
# Shape of the per-request Gamma spread of rate constants around each model's rates: the
# gene-expression workload's shape 2 wherever possible; the dimerisation keeps shape 50
# (about 14 %), because a wider spread pushes its stiff pair out of partial equilibrium
# and turns the model SSA-bound.
SERVING_THETA_SHAPE = {0: 2.0, 1: 50.0, 2: 2.0, 3: 2.0}


def serving_requests(n_requests: int, seed: int = 0, rate_hz: float = 200.0,
                     min_traj: int = 1_000, max_traj: int = 100_000, models=(0, 1, 2, 3),
                     horizon_scale=None, theta_shape=None):
    """Poisson-arrival request stream for the serving mix: each request picks a model
    uniformly from `models`, a log-uniform trajectory count B in [min_traj, max_traj], its
    own per-trajectory rate constants theta ~ Gamma(shape, rate shape / k) around the
    model's rates k (shape from theta_shape, default SERVING_THETA_SHAPE) and its own
    per-trajectory horizons: the model's horizon x horizon_scale[model] x U[0.5, 1]
    (default SERVING_HORIZON_SCALE).

    The rate constants and horizons are drawn once per model into a pool of max_traj
    rows; a request takes B consecutive rows at a random offset (a view, no copy), so a
    stream of thousands of requests holds a few pools in host memory instead of one batch
    per request (the 50 x 100 network's rate constants alone are 800 bytes per
    trajectory).  Requests differ in offset, size, horizon rows and trajectory ids, so
    their random numbers never coincide.  Returns a list of dicts with arrival time (s),
    Workload and a distinct trajectory-id base."""
    scales = dict(SERVING_HORIZON_SCALE if horizon_scale is None else horizon_scale)
    shapes = dict(SERVING_THETA_SHAPE if theta_shape is None else theta_shape)
    rng = np.random.default_rng(seed)
    bases = {m: config(m, n_traj=1) for m in models}
    pools = {}
    for m in models:
        crn = bases[m].crn
        k = shapes.get(m, 2.0)
        Tm = float(bases[m].T[0] if bases[m].T.shape[0] == 1 else 125.0) * scales.get(m, 1.0)
        pools[m] = (np.ascontiguousarray(rng.gamma(k, crn.rates / k,
                                                   size=(max_traj, crn.n_reactions))),
                    np.ascontiguousarray(Tm * rng.uniform(0.5, 1.0, size=max_traj)))
    t = 0.0
    base = 0
    out = []
    for q in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        m = int(models[rng.integers(len(models))])
        B = int(np.floor(np.exp(rng.uniform(np.log(min_traj), np.log(max_traj)))))
        B = min(max(B, 1), max_traj)
        off = int(rng.integers(0, max_traj - B + 1))
        w0 = bases[m]
        th_pool, T_pool = pools[m]
        wl = Workload(f"req{q}_{w0.name}", w0.crn, B, w0.x0.copy(), T_pool[off:off + B],
                      th_pool[off:off + B], seed=seed + 17, traj_id_base=base)
        base += B
        out.append({"arrival_s": t, "workload": wl, "model_index": m})
    return out
