"""Seeded synthetic bi-objective QAP instances and request streams.

This module only draws inputs; it holds none of the annealer's arithmetic,
so both the CUDA path and the CPU oracle may be fed from it.

The paper evaluates on the structured qapStr instances of Knowles and Corne
(Sec. 4.1: n in {25, 50}, objective correlation rho in {-0.75, 0, 0.75}).
Those files are not available here; the generators below stand in for them
with the same sizes, value ranges and correlation structure:

* ``uniform_instance``: D symmetric, off-diagonal uniform integers in
  [1, 99]; F1, F2 independent uniform integers in [0, 99]; zero diagonals.
* ``euclid_instance``: D from n integer points uniform in a 100 x 100 grid,
  d = Euclidean distance rounded half away from zero; flows from a Gaussian
  copula with correlation ``rho`` on each off-diagonal entry, mapped to
  either uniform [0, 99] (floor(100 Phi(z)), clipped to 99) or, with
  ``sparse=True``, to an exponential of mean 100 (floor(-100 ln(1 - Phi(z))
  + 0.5), clipped to 10^4) under one 70 %-zero mask shared by both flows.

Every generator is driven by numpy's PCG64 seeded from a (workload id,
instance index) pair, so an instance is reproducible from its name alone.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

WORKLOAD_IDS = {"P8": 8, "P25": 25, "P50": 50, "P75": 75, "BATCH": 512, "SERVE": 200}


def _rng(workload: str, index: int) -> np.random.Generator:
    ss = np.random.SeedSequence([WORKLOAD_IDS.get(workload, 0), int(index)])
    return np.random.Generator(np.random.PCG64(ss))


def _phi(z: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr
    return ndtr(z)


@dataclass
class QAPInstance:
    name: str
    n: int
    F1: np.ndarray  # int16 [n, n], flows of objective 1
    F2: np.ndarray  # int16 [n, n], flows of objective 2
    D: np.ndarray   # int16 [n, n], symmetric distances, zero diagonal
    rho: float

    def realised_rho(self) -> float:
        """Pearson correlation of the two flow matrices' off-diagonal
        entries."""
        off = ~np.eye(self.n, dtype=bool)
        a = self.F1[off].astype(np.float64)
        b = self.F2[off].astype(np.float64)
        if a.std() == 0 or b.std() == 0:
            return 0.0
        return float(np.corrcoef(a, b)[0, 1])


def uniform_instance(n: int, index: int = 0, workload: str = "P8") -> QAPInstance:
    rng = _rng(workload, index)
    D = rng.integers(1, 100, size=(n, n))
    D = np.triu(D, 1)
    D = D + D.T
    F1 = rng.integers(0, 100, size=(n, n))
    F2 = rng.integers(0, 100, size=(n, n))
    np.fill_diagonal(F1, 0)
    np.fill_diagonal(F2, 0)
    return QAPInstance(f"{workload}.{index}", n, F1.astype(np.int16), F2.astype(np.int16),
                       D.astype(np.int16), 0.0)


def euclid_distances(rng: np.random.Generator, n: int) -> np.ndarray:
    pts = rng.integers(0, 100, size=(n, 2)).astype(np.float64)
    diff = pts[:, None, :] - pts[None, :, :]
    d = np.sqrt((diff ** 2).sum(-1))
    d = np.floor(d + 0.5)  # non-negative, so this rounds half away from zero
    np.fill_diagonal(d, 0)
    return d.astype(np.int16)


def copula_flows(rng: np.random.Generator, n: int, rho: float, sparse: bool):
    z1 = rng.standard_normal((n, n))
    z2 = rho * z1 + np.sqrt(max(0.0, 1.0 - rho * rho)) * rng.standard_normal((n, n))
    u1, u2 = _phi(z1), _phi(z2)
    if sparse:
        f1 = np.floor(-100.0 * np.log1p(-np.minimum(u1, 1 - 1e-16)) + 0.5)
        f2 = np.floor(-100.0 * np.log1p(-np.minimum(u2, 1 - 1e-16)) + 0.5)
        f1 = np.minimum(f1, 10000)
        f2 = np.minimum(f2, 10000)
        mask = rng.random((n, n)) < 0.7
        f1[mask] = 0
        f2[mask] = 0
    else:
        f1 = np.minimum(np.floor(100.0 * u1), 99)
        f2 = np.minimum(np.floor(100.0 * u2), 99)
    np.fill_diagonal(f1, 0)
    np.fill_diagonal(f2, 0)
    return f1.astype(np.int16), f2.astype(np.int16)


def euclid_instance(n: int, rho: float, sparse: bool, index: int = 0,
                    workload: str = "P25") -> QAPInstance:
    rng = _rng(workload, index)
    D = euclid_distances(rng, n)
    F1, F2 = copula_flows(rng, n, rho, sparse)
    return QAPInstance(f"{workload}.{index}", n, F1, F2, D, rho)


def workload_instance(workload: str, index: int = 0) -> QAPInstance:
    """The single-instance workloads: P8 (n=8), P25, P50, P75."""
    if workload == "P8":
        return uniform_instance(8, index, "P8")
    if workload == "P25":
        return euclid_instance(25, 0.5, False, index, "P25")
    if workload == "P50":
        return euclid_instance(50, -0.5, True, index, "P50")
    if workload == "P75":
        return euclid_instance(75, -0.5, True, index, "P75")
    raise KeyError(workload)


# Replicas / iteration budget of each single-instance workload.
WORKLOAD_RUN = {
    "P8": dict(replicas=16, I_max=10_000, seed=0),
    "P25": dict(replicas=128, I_max=100_000, seed=0),
    "P50": dict(replicas=256, I_max=1_000_000, seed=0),
    "P75": dict(replicas=256, I_max=1_000_000, seed=0),
}


def batch_instances(count: int = 512, n_lo: int = 10, n_hi: int = 75):
    """Many instances of uneven size: n uniform in [n_lo, n_hi], uniform
    flows with rho drawn from {-0.7, 0, 0.7}, distances as in P25."""
    out = []
    for k in range(count):
        rng = _rng("BATCH", k)
        n = int(rng.integers(n_lo, n_hi + 1))
        rho = float(rng.choice([-0.7, 0.0, 0.7]))
        D = euclid_distances(rng, n)
        F1, F2 = copula_flows(rng, n, rho, False)
        out.append(QAPInstance(f"BATCH.{k}", n, F1, F2, D, rho))
    return out


@dataclass
class Request:
    arrival_s: float
    instance: QAPInstance
    I_max: int
    seed: int


def serving_requests(count: int, rate_per_s: float = 200.0, sizes=(20, 30, 50, 75),
                     budgets=(10_000, 100_000), index0: int = 0):
    """Poisson arrivals of solves with n drawn from ``sizes`` and I_max from
    ``budgets``; instances are generated as in the batched workload."""
    rng = _rng("SERVE", index0)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(rng.choice(sizes))
        I_max = int(rng.choice(budgets))
        rho = float(rng.choice([-0.7, 0.0, 0.7]))
        irng = _rng("SERVE", 1_000_000 + index0 + k)
        D = euclid_distances(irng, n)
        F1, F2 = copula_flows(irng, n, rho, False)
        out.append(Request(t, QAPInstance(f"SERVE.{index0 + k}", n, F1, F2, D, rho),
                           I_max, index0 + k))
    return out


def random_qubo(K: int, m: int, index: int = 0, lo: int = -100, hi: int = 100) -> np.ndarray:
    """K dense QUBO matrices of m bits, upper triangle uniform integers in
    [lo, hi] (the lower triangle is zero), for the explicit-QUBO path."""
    rng = _rng("QUBO", index)
    Q = rng.integers(lo, hi + 1, (K, m, m)).astype(np.int32)
    return np.triu(Q)
