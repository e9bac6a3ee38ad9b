"""numpy pieces of the CPU oracle (TEST INFRASTRUCTURE ONLY; see the package
docstring): QAP cost, permutation encoding, dominance filter, brute-force
Pareto fronts and the 2-D hypervolume.
"""
from __future__ import annotations

import itertools

import numpy as np


def qap_cost(H, D, perm) -> int:
    """f(sigma) = sum_ij h_ij d_{sigma_i sigma_j} (Sec. 2.1, Eq. nqap).

    ``perm[i]`` is the 0-based location of facility i."""
    H = np.asarray(H, dtype=np.int64)
    D = np.asarray(D, dtype=np.int64)
    p = np.asarray(perm, dtype=np.int64)
    return int((H * D[np.ix_(p, p)]).sum())


def encode_permutation(perm) -> np.ndarray:
    """Two-way one-hot vector of Sec. 2.2: bit i*n + perm[i] is set."""
    n = len(perm)
    x = np.zeros(n * n, dtype=np.uint8)
    for i, a in enumerate(perm):
        x[i * n + int(a)] = 1
    return x


def decode_permutation(x):
    """perm with perm[i] = location of facility i, or None when x is not a
    permutation matrix."""
    x = np.asarray(x, dtype=np.int64).reshape(-1)
    n = int(round(np.sqrt(x.size)))
    X = x.reshape(n, n)
    if not (np.all(X.sum(0) == 1) and np.all(X.sum(1) == 1)):
        return None
    return [int(np.argmax(X[i])) for i in range(n)]


def dominates(a, b) -> bool:
    """a dominates b (Sec. 3.3): no worse in every objective, not equal."""
    return all(x <= y for x, y in zip(a, b)) and tuple(a) != tuple(b)


def nondominated(points):
    """Indices of the points no other point dominates; among equal vectors
    only the first is kept."""
    pts = [tuple(int(v) for v in p) for p in points]
    keep = []
    seen = set()
    for i, p in enumerate(pts):
        if p in seen:
            continue
        if any(dominates(q, p) for q in pts):
            continue
        seen.add(p)
        keep.append(i)
    return keep


def pareto_front_bruteforce(F1, F2, D):
    """Exact Pareto front of a small bi-objective QAP by enumerating every
    permutation: a sorted list of distinct (f1, f2)."""
    F1 = np.asarray(F1, dtype=np.int64)
    F2 = np.asarray(F2, dtype=np.int64)
    D = np.asarray(D, dtype=np.int64)
    n = D.shape[0]
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.int64)
    f1 = np.empty(len(perms), dtype=np.int64)
    f2 = np.empty(len(perms), dtype=np.int64)
    chunk = 8192
    for s in range(0, len(perms), chunk):
        P = perms[s:s + chunk]
        Dp = D[P[:, :, None], P[:, None, :]]  # [B, n, n]
        f1[s:s + chunk] = (Dp * F1[None]).sum((1, 2))
        f2[s:s + chunk] = (Dp * F2[None]).sum((1, 2))
    # 2-D front: sort by f1 then f2, keep strictly decreasing f2.
    order = np.lexsort((f2, f1))
    front = []
    best2 = None
    for i in order:
        a, b = int(f1[i]), int(f2[i])
        if best2 is None or b < best2:
            front.append((a, b))
            best2 = b
    return front


def hypervolume_2d(points, ref) -> float:
    """Area dominated by ``points`` (minimisation) and bounded by ``ref``
    (Sec. 4.3).  Points not strictly better than ``ref`` in both objectives
    contribute nothing."""
    pts = sorted({(float(a), float(b)) for a, b in points
                  if a < ref[0] and b < ref[1]})
    area = 0.0
    prev2 = float(ref[1])
    for a, b in pts:
        if b < prev2:
            area += (ref[0] - a) * (prev2 - b)
            prev2 = b
    return area


def normalised_hypervolume(points, lo, hi) -> float:
    """Sec. 4.3: map each objective from [lo_k, hi_k] to [1, 2] and measure
    against the reference point (2.1, 2.1); the largest value is 1.21."""
    out = []
    for a, b in points:
        na = 1.0 + (a - lo[0]) / (hi[0] - lo[0]) if hi[0] > lo[0] else 1.0
        nb = 1.0 + (b - lo[1]) / (hi[1] - lo[1]) if hi[1] > lo[1] else 1.0
        out.append((na, nb))
    return hypervolume_2d(out, (2.1, 2.1))
