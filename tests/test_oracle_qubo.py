"""Pins of the oracle's QUBO construction against the paper and mathematics.

* Sec. 2.2 worked example (n = 3): C, G, p_g and two evaluated states,
  stored in tests/golden/worked_example_n3.json.
* Sec. 2.2: c(x) equals the QAP cost f(sigma) of Eq. nqap on permutations;
  g(x) >= 0 with equality exactly on permutation matrices.
* Sec. 3.2, Eq. vermap: w is the largest change of the cost one flip can
  make (checked over every state and flip of small instances), which for
  non-negative flows and zero-diagonal distances has a closed form.
* Consequence of that choice with alpha = w/2 (Eq. wvermaa): no single flip
  from a feasible state lowers either penalised energy.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle


def _golden(golden_dir):
    with open(os.path.join(golden_dir, "worked_example_n3.json")) as f:
        return json.load(f)


def test_worked_example_matrices(golden_dir):
    g = _golden(golden_dir)
    C = oracle.cost_qubo(g["H"], g["D"])
    assert np.array_equal(C, np.array(g["C"]))
    G, pg = oracle.constraint_qubo(3)
    assert np.array_equal(G, np.array(g["G"]))
    assert pg == g["p_g"]


def test_worked_example_states(golden_dir):
    g = _golden(golden_dir)
    inst = oracle.Instance(g["H"], g["H"], g["D"])
    for st in g["states"]:
        x = np.array(st["x"], dtype=np.uint8)
        sigma = [s - 1 for s in st["sigma_1based"]]
        assert oracle.qap_cost(g["H"], g["D"], sigma) == st["f"]
        assert inst.cost(0, x) == st["xCx"] + g["p_c"]
        assert inst.constraint(x) == st["g"]
        G = np.array(g["G"])
        assert int(x @ G @ x) == st["xGx"]
        # E = c + alpha g with alpha = w / 2 = 30 for this instance.
        assert inst.w == (60, 60)
        assert inst.energy(0, x) == st["xCx"] + 30 * st["g"]
    # the valid state decodes to sigma = (3, 1, 2)
    assert oracle.decode_permutation(g["states"][0]["x"]) == [2, 0, 1]
    assert oracle.decode_permutation(g["states"][1]["x"]) is None


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 9])
def test_cost_equals_qap_cost_on_permutations(n):
    rng = np.random.default_rng(n)
    # asymmetric flows and distances, negative entries included: the identity
    # c(x) = f(sigma) holds for any matrices
    H = rng.integers(-50, 100, size=(n, n))
    D = rng.integers(-20, 100, size=(n, n))
    C = oracle.cost_qubo(H, D)
    for _ in range(20):
        perm = rng.permutation(n)
        x = oracle.encode_permutation(perm)
        xi = x.astype(np.int64)
        assert int(xi @ C @ xi) == oracle.qap_cost(H, D, perm)


def _all_states(m):
    k = np.arange(2 ** m, dtype=np.int64)
    return ((k[:, None] >> np.arange(m)) & 1).astype(np.int64)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_constraint_exhaustive(n):
    m = n * n
    G, pg = oracle.constraint_qubo(n)
    X = _all_states(m)
    g_qubo = np.einsum("sp,pq,sq->s", X, G, X) + pg
    R = X.reshape(-1, n, n)
    g_def = ((1 - R.sum(2)) ** 2).sum(1) + ((1 - R.sum(1)) ** 2).sum(1)
    assert np.array_equal(g_qubo, g_def)
    assert (g_qubo >= 0).all()
    assert (g_qubo % 2 == 0).all()
    is_perm = (R.sum(2) == 1).all(1) & (R.sum(1) == 1).all(1)
    assert np.array_equal(g_qubo == 0, is_perm)
    assert is_perm.sum() == len(list(itertools.permutations(range(n))))
    # the least g one flip away from a feasible state is 2 (Sec. 3.2)
    feas = X[is_perm]
    for x in feas:
        for p in range(m):
            y = x.copy()
            y[p] ^= 1
            assert int(y @ G @ y) + pg == 2


def _random_nonneg_instance(rng, n, fmax=99, dmax=99):
    F = rng.integers(0, fmax + 1, size=(n, n))
    np.fill_diagonal(F, 0)
    D = rng.integers(1, dmax + 1, size=(n, n))
    D = np.triu(D, 1)
    D = D + D.T
    return F, D


@pytest.mark.parametrize("seed", range(6))
def test_penalty_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 8))
    F, D = _random_nonneg_instance(rng, n)
    C = oracle.cost_qubo(F, D)
    Fs = F + F.T
    closed = int(Fs.sum(1).max() * D.sum(1).max())
    assert oracle.penalty_w(C) == closed


@pytest.mark.parametrize("seed", range(4))
def test_penalty_is_largest_single_flip_change(seed):
    """w of Eq. vermap bounds |c(x with bit i flipped) - c(x)| over all x, i,
    and for non-negative QUBOs the bound is attained (turn bit i on with
    every other bit on)."""
    rng = np.random.default_rng(200 + seed)
    n = 3
    F, D = _random_nonneg_instance(rng, n)
    F[0, 2] = 0  # asymmetric flows
    C = oracle.cost_qubo(F, D)
    m = n * n
    X = _all_states(m)
    base = np.einsum("sp,pq,sq->s", X, C, X)
    worst = 0
    for p in range(m):
        Y = X.copy()
        Y[:, p] ^= 1
        worst = max(worst, int(np.abs(np.einsum("sp,pq,sq->s", Y, C, Y) - base).max()))
    assert oracle.penalty_w(C) == worst


@pytest.mark.parametrize("seed", range(5))
def test_feasible_states_are_flip_stable(seed):
    """With alpha_k = w_k / 2, every single flip from a feasible state has
    Delta E_k >= 0 for both objectives."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(3, 7))
    F1, D = _random_nonneg_instance(rng, n)
    F2, _ = _random_nonneg_instance(rng, n)
    inst = oracle.Instance(F1, F2, D)
    for _ in range(5):
        x = oracle.encode_permutation(rng.permutation(n))
        e = [inst.energy(k, x) for k in range(2)]
        for p in range(n * n):
            y = x.copy()
            y[p] ^= 1
            for k in range(2):
                assert inst.energy(k, y) - e[k] >= 0


@pytest.mark.parametrize("seed", range(4))
def test_energy_is_cost_plus_weighted_constraint(seed):
    """E_k(x) = c_k(x) + (w_k / 2) g(x) (Eq. mqap / wqubom) on random states,
    and w_k comes from the objective's own cost QUBO."""
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(2, 7))
    F1, D = _random_nonneg_instance(rng, n)
    F2, _ = _random_nonneg_instance(rng, n, fmax=9)
    inst = oracle.Instance(F1, F2, D)
    assert inst.w[0] == oracle.penalty_w(oracle.cost_qubo(F1, D))
    assert inst.w[1] == oracle.penalty_w(oracle.cost_qubo(F2, D))
    G, pg = oracle.constraint_qubo(n)
    for _ in range(20):
        x = (rng.random(n * n) < 0.4).astype(np.uint8)
        xi = x.astype(np.int64)
        g = int(xi @ G @ xi) + pg
        R = xi.reshape(n, n)
        assert g == int(((1 - R.sum(1)) ** 2).sum() + ((1 - R.sum(0)) ** 2).sum())
        for k, F in enumerate((F1, F2)):
            c = int(xi @ oracle.cost_qubo(F, D) @ xi)
            assert 2 * inst.energy(k, x) == 2 * c + inst.w[k] * g


def test_explicit_penalty():
    rng = np.random.default_rng(7)
    F1, D = _random_nonneg_instance(rng, 4)
    F2, _ = _random_nonneg_instance(rng, 4)
    inst = oracle.Instance(F1, F2, D, w=(11, 8))
    assert inst.w == (11, 8)
    x = (rng.random(16) < 0.5).astype(np.uint8)
    g = inst.constraint(x)
    assert g % 2 == 0
    assert inst.energy(0, x) == inst.cost(0, x) + 11 * g // 2
    assert inst.energy(1, x) == inst.cost(1, x) + 8 * g // 2
