"""Pins for the factor-graph oracle: brute-force enumeration on factor graphs
that are trees (BP is exact there)."""
import itertools

import numpy as np
import pytest

from oracle import factor


def _brute(g, factors, F, mode):
    nv, M = g.shape
    out = np.zeros((nv, M)) if mode == "sum" else np.full((nv, M), np.iinfo(np.int64).max)
    for x in itertools.product(range(M), repeat=nv):
        if mode == "sum":
            w = np.prod([g[v, x[v]] for v in range(nv)]) * np.prod([F[x[a], x[b], x[c]] for a, b, c in factors])
            for v in range(nv):
                out[v, x[v]] += w
        else:
            e = sum(int(g[v, x[v]]) for v in range(nv)) + sum(int(F[x[a], x[b], x[c]]) for a, b, c in factors)
            for v in range(nv):
                out[v, x[v]] = min(out[v, x[v]], e)
    return out / out.sum(1, keepdims=True) if mode == "sum" else out


TREES = [
    [(0, 1, 2)],                               # one factor
    [(0, 1, 2), (2, 3, 4)],                    # two factors sharing variable 2
    [(1, 0, 2), (3, 2, 4), (4, 5, 6)],         # a chain of three factors, mixed slots
]


@pytest.mark.parametrize("factors", TREES)
def test_sum_product_exact_on_factor_trees(factors):
    rng = np.random.default_rng(len(factors))
    nv = 1 + max(max(f) for f in factors)
    M = 3
    g = rng.uniform(0.05, 1.0, (nv, M))
    trip = [(a, b, c) for a in range(M) for b in range(M) for c in range(M) if rng.random() < 0.3]
    F = factor.dense_table(trip, rng.uniform(0.5, 2.0, len(trip)), 0.2, M)
    _, bel = factor.sum_product(g, factors, F, n_iters=2 * len(factors) + 2)
    np.testing.assert_allclose(bel, _brute(g, factors, F, "sum"), rtol=1e-11)


@pytest.mark.parametrize("factors", TREES)
def test_min_sum_exact_on_factor_trees(factors):
    rng = np.random.default_rng(10 + len(factors))
    nv = 1 + max(max(f) for f in factors)
    M = 3
    E = rng.integers(0, 15, (nv, M))
    trip = [(a, b, c) for a in range(M) for b in range(M) for c in range(M) if rng.random() < 0.3]
    V = factor.dense_table(trip, rng.integers(0, 8, len(trip)), 9, M, dtype=np.int64)
    _, bel = factor.min_sum(E, factors, V, n_iters=2 * len(factors) + 2)
    ref = _brute(E, factors, V, "min")
    np.testing.assert_array_equal(bel - bel.min(1, keepdims=True), ref - ref.min(1, keepdims=True))


def test_dense_table_is_constant_outside_the_triplets():
    F = factor.dense_table([(0, 1, 2), (2, 2, 2)], [5.0, 7.0], 0.5, 3)
    assert F[0, 1, 2] == 5.0 and F[2, 2, 2] == 7.0
    assert np.count_nonzero(F != 0.5) == 2


# Plausible mistakes planted in a private copy of the factor-graph oracle; the
# brute-force tree pins above must fail for each.
FACTOR_MUTANTS = {
    # the variable-to-factor message keeps the factor's own message (Sec. 7's
    # flooding update leaves it out)
    "no_exclusion": ("if (b, t) != (a, s):", "if True:"),
    # slot 1's sum contracts the other two slots' messages against the wrong axes
    "swapped_slots": ('np.einsum("abc,a,c->b", F, n[0], n[2])', 'np.einsum("abc,c,a->b", F, n[0], n[2])'),
    # min-sum slot 2 broadcasts slot 1's message along the wrong axis
    "min_broadcast": ("V + n[0][:, None, None] + n[1][None, :, None], axis=(0, 1)",
                      "V + n[0][:, None, None] + n[1][:, None, None], axis=(0, 1)"),
    # beliefs without the unary
    "no_unary_belief": ("bel = g.copy()", "bel = np.ones_like(g)"),
}


def _mutant_module(name):
    import types
    old, new = FACTOR_MUTANTS[name]
    src = open(factor.__file__).read()
    assert old in src, name
    mod = types.ModuleType(f"factor_{name}")
    exec(compile(src.replace(old, new, 1), f"<factor mutant {name}>", "exec"), mod.__dict__)
    return mod


def _tree_pins_pass(mod):
    ok = True
    for factors in TREES:
        rng = np.random.default_rng(len(factors))
        nv = 1 + max(max(f) for f in factors)
        M = 3
        g = rng.uniform(0.05, 1.0, (nv, M))
        trip = [(a, b, c) for a in range(M) for b in range(M) for c in range(M) if rng.random() < 0.3]
        F = mod.dense_table(trip, rng.uniform(0.5, 2.0, len(trip)), 0.2, M)
        _, bel = mod.sum_product(g, factors, F, n_iters=2 * len(factors) + 2)
        ok &= np.allclose(bel, _brute(g, factors, F, "sum"), rtol=1e-11)
        E = rng.integers(0, 15, (nv, M))
        V = mod.dense_table(trip, rng.integers(0, 8, len(trip)), 9, M, dtype=np.int64)
        _, belm = mod.min_sum(E, factors, V, n_iters=2 * len(factors) + 2)
        ref = _brute(E, factors, V, "min")
        ok &= np.array_equal(belm - belm.min(1, keepdims=True), ref - ref.min(1, keepdims=True))
    return ok


def test_unmutated_factor_oracle_passes_the_tree_pins():
    assert _tree_pins_pass(factor)


@pytest.mark.parametrize("name", sorted(FACTOR_MUTANTS))
def test_factor_mutant_is_caught(name):
    assert not _tree_pins_pass(_mutant_module(name))
