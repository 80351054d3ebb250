"""The pins catch plausible mistakes: each test plants one mistake in a
private copy of the C oracle (on the CPU), rebuilds it, and checks that a
brute-force pin then fails."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import brute_marginals, brute_min_marginals, random_tree, sym_positive

SRC = os.path.join(os.path.dirname(oracle.__file__), "bp_oracle.c")

MUTANTS = {
    # Eq. 5 leaves out the message from j; the mutant keeps it
    "no_exclusion": ("if (src[e2] != j) scratch[n++]", "scratch[n++]"),
    # a dropped unary factor in h
    "no_unary": ("double p = g_i[x];", "double p = 1.0;"),
    # sum over the wrong index of F
    "wrong_index": ("u += F[(size_t)xi * M + xj] * h[xi];", "u += F[(size_t)xi * M + xj] * h[xj];"),
    # max instead of min in min-sum
    "max_not_min": ("if (v < best) best = v;", "if (v > best) best = v;"),
    # colour 1 half-step first
    "colour_order": ("for (int c = 0; c < 2 && rc == 0; ++c) {",
                     "for (int c = 1; c >= 0 && rc == 0; --c) {"),
    # f(x_j, x_i) instead of f(x_i, x_j): invisible with symmetric tables
    "transposed_table": ("u += F[(size_t)xi * M + xj] * h[xi];", "u += F[(size_t)xj * M + xi] * h[xi];"),
}


def _build_mutant(name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert old in text, name
    d = tempfile.mkdtemp()
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    open(c, "w").write(text.replace(old, new, 1))
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", c, "-o", so])
    lib = ctypes.CDLL(so)
    return lib


def _run_with(lib, fn, *args, **kw):
    saved = oracle._lib
    oracle._lib = lib
    I, P = ctypes.c_int, ctypes.c_void_p
    for nm in ("oracle_sum_product", "oracle_min_sum"):
        getattr(lib, nm).argtypes = [I, I, I, P, P, P, P, P, I, I, P]
    for nm in ("oracle_sum_beliefs", "oracle_min_beliefs"):
        getattr(lib, nm).argtypes = [I, I, I, P, P, P, P]
    for nm in ("oracle_sum_edge_update", "oracle_min_edge_update"):
        getattr(lib, nm).argtypes = [I, P, I, P, P, P]
    try:
        return fn(*args, **kw)
    finally:
        oracle._lib = saved


def _sum_pin_passes(lib, schedule="sync", chain=False):
    ok = True
    for seed in range(4):
        rng = np.random.default_rng(seed)
        n, M = 5, 3
        if chain:
            und = [(0, 1), (1, 2)]
            n = 3
            src = np.array([0, 1, 1, 2])
            dst = np.array([1, 0, 2, 1])
            col = np.array([0, 1, 0])
            iters = 1
        else:
            src, dst, und, col = random_tree(n, rng)
            iters = n
        g = rng.uniform(0.05, 1.0, (n, M))
        F = sym_positive(M, rng)

        def go():
            msg = oracle.sum_product(src, dst, g, F, iters, color=col, schedule=schedule)
            return oracle.sum_beliefs(dst, g, msg)
        bel = _run_with(lib, go)
        ok &= np.allclose(bel, brute_marginals(n, M, und, g, F), rtol=1e-10)
    return ok


def _min_pin_passes(lib):
    ok = True
    for seed in range(4):
        rng = np.random.default_rng(50 + seed)
        n, M = 5, 3
        src, dst, und, col = random_tree(n, rng)
        Eu = rng.integers(0, 20, (n, M))
        A = rng.integers(0, 15, (M, M))
        V = np.minimum(A, A.T)

        def go():
            msg = oracle.min_sum(src, dst, Eu, V, n)
            return oracle.min_beliefs(dst, Eu, msg)
        bel = _run_with(lib, go)
        ref = brute_min_marginals(n, M, und, Eu, V)
        ok &= np.array_equal(bel - bel.min(1, keepdims=True), ref - ref.min(1, keepdims=True))
    return ok


def test_unmutated_oracle_passes():
    assert _sum_pin_passes(oracle._load()) and _min_pin_passes(oracle._load())


@pytest.mark.parametrize("name", ["no_exclusion", "no_unary", "wrong_index"])
def test_sum_mutant_is_caught(name):
    assert not _sum_pin_passes(_build_mutant(name))


def test_min_mutant_is_caught():
    assert not _min_pin_passes(_build_mutant("max_not_min"))


def test_schedule_mutant_is_caught():
    lib = _build_mutant("colour_order")
    assert not _sum_pin_passes(lib, schedule="redblack", chain=True)
    assert _sum_pin_passes(oracle._load(), schedule="redblack", chain=True)


def _eq7_pin_passes(lib):
    """The Eq. 7 pin (tests/test_oracle_algebra.py) on asymmetric band tables."""
    from oracle import stereo
    from tests.test_oracle_algebra import eq7
    ok = True
    for M, T in ((5, 1), (16, 2)):
        rng = np.random.default_rng(M + T)
        g = rng.uniform(0.05, 1.0, M)
        incoming = [rng.uniform(0.05, 1.0, M) for _ in range(3)]
        fbar = 0.1
        band = rng.uniform(0.2, 2.0, 2 * T + 1)
        F = stereo.compatibility_matrix(band, T, fbar, M)
        ref = _run_with(lib, oracle.sum_edge_update, g, incoming, F)
        ok &= np.allclose(eq7(g, incoming, band, T, fbar, M), ref, rtol=1e-12, atol=0)
    return ok


def test_transposed_table_mutant_is_caught_by_the_eq7_pin():
    lib = _build_mutant("transposed_table")
    assert _sum_pin_passes(lib)              # the tree pins use symmetric tables: blind to it
    assert not _eq7_pin_passes(lib)
    assert _eq7_pin_passes(oracle._load())
