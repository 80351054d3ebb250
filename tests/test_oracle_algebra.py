"""The paper's rearranged updates against the oracle's plain dense ones.

The oracle computes Eq. 2 (sum-product) and Eq. 9 (max-product in energies)
over all M x M label pairs.  The paper's O(mM) forms are written out here on
their own, term by term as Sec. 4 and Sec. 5 state them:

* Eq. 7: sum over the band of [f - fbar] h, plus fbar times the sum of h,
  valid for any table, including entries below fbar;
* Eq. 8: the band sum alone, which equals Eq. 2 when fbar really is 0;
* Eq. 11: the least of the band minimum and Ebar plus the least h, valid when
  every E(d) <= Ebar (f >= fbar), and wrong otherwise: the negative control.

Agreement on random inputs pins the oracle's dense update (a dropped term, a
wrong index or a transposed table in it would break these identities), and the
identities themselves are the exactness claim the method rests on."""
import numpy as np
import pytest

import oracle
from oracle import stereo


def _messages(rng, M, k, integer=False):
    if integer:
        return [rng.integers(0, 30, M).astype(np.int64) for _ in range(k)]
    out = []
    for _ in range(k):
        m = rng.uniform(0.05, 1.0, M)
        out.append(m / m.sum())
    return out


def eq7(g, incoming, band, T, fbar, M):
    """Eq. 5 then Eq. 7, normalised to sum 1."""
    h = np.array(g, dtype=np.float64)
    for m in incoming:
        h = h * m
    S = h.sum()
    u = np.empty(M)
    for xj in range(M):
        acc = 0.0
        for d in range(-T, T + 1):          # d = x_i - x_j
            xi = xj + d
            if 0 <= xi < M:
                acc += (band[d + T] - fbar) * h[xi]
        u[xj] = acc + fbar * S
    return u / u.sum()


def eq8(g, incoming, band, T, M):
    """Eq. 8: the band sum alone (fbar = 0), normalised."""
    h = np.array(g, dtype=np.float64)
    for m in incoming:
        h = h * m
    u = np.zeros(M)
    for xj in range(M):
        for d in range(-T, T + 1):
            xi = xj + d
            if 0 <= xi < M:
                u[xj] += band[d + T] * h[xi]
    return u / u.sum()


def eq11(E_i, incoming, bandE, T, ebar, M):
    """Eq. 11 in energies (min-sum), minimum subtracted."""
    h = np.array(E_i, dtype=np.int64)
    for m in incoming:
        h = h + m
    outer = ebar + int(h.min())
    u = np.empty(M, dtype=np.int64)
    for xj in range(M):
        best = outer
        for d in range(-T, T + 1):
            xi = xj + d
            if 0 <= xi < M:
                best = min(best, int(bandE[d + T]) + int(h[xi]))
        u[xj] = best
    return u - u.min()


CASES = [(2, 0), (2, 1), (5, 1), (5, 4), (5, 7), (16, 2), (16, 15), (33, 3), (33, 0)]


@pytest.mark.parametrize("M,T", CASES)
@pytest.mark.parametrize("below_fbar", [False, True])
def test_eq7_equals_the_dense_update(M, T, below_fbar):
    rng = np.random.default_rng(1000 * M + T + below_fbar)
    for k in (0, 1, 3):                      # corner, edge and interior sender
        g = rng.uniform(0.05, 1.0, M)
        incoming = _messages(rng, M, k)
        fbar = rng.uniform(0.05, 0.5)
        band = rng.uniform(fbar, 2.0, 2 * T + 1)
        if below_fbar:                       # Sec. 5: sum-product does not need f >= fbar
            band[rng.integers(0, 2 * T + 1)] = 0.5 * fbar
        F = stereo.compatibility_matrix(band, T, fbar, M)
        ref = oracle.sum_edge_update(g, incoming, F)
        np.testing.assert_allclose(eq7(g, incoming, band, T, fbar, M), ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("M,T", CASES)
def test_eq8_equals_the_dense_update_when_fbar_is_zero(M, T):
    rng = np.random.default_rng(77 * M + T)
    g = rng.uniform(0.05, 1.0, M)
    incoming = _messages(rng, M, 3)
    band = rng.uniform(0.1, 2.0, 2 * T + 1)
    F = stereo.compatibility_matrix(band, T, 0.0, M)
    ref = oracle.sum_edge_update(g, incoming, F)
    np.testing.assert_allclose(eq8(g, incoming, band, T, M), ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("M,T", CASES)
def test_eq11_equals_the_dense_update_when_every_energy_is_at_most_ebar(M, T):
    rng = np.random.default_rng(31 * M + T)
    for k in (0, 1, 3):
        E_i = rng.integers(0, 40, M).astype(np.int64)
        incoming = _messages(rng, M, k, integer=True)
        ebar = int(rng.integers(1, 25))
        bandE = rng.integers(0, ebar + 1, 2 * T + 1).astype(np.int64)
        V = stereo.compatibility_matrix(bandE, T, ebar, M, dtype=np.int64)
        ref = oracle.min_edge_update(E_i, incoming, V)
        np.testing.assert_array_equal(eq11(E_i, incoming, bandE, T, ebar, M), ref - ref.min())


def test_eq11_is_wrong_when_some_energy_exceeds_ebar():
    """Negative control of Sec. 5's condition.  Node i strongly prefers label
    0 and E(0) = 10 > Ebar = 3: the true update (Eq. 9) charges 10 for
    keeping x_j = 0, while Eq. 11's outer term offers Ebar + min h = 3 for the
    same pair, so the two disagree."""
    M, T, ebar = 5, 1, 3
    bandE = np.array([0, 10, 0], dtype=np.int64)            # E(-1), E(0), E(1)
    E_i = np.array([0, 100, 100, 100, 100], dtype=np.int64)
    V = stereo.compatibility_matrix(bandE, T, ebar, M, dtype=np.int64)
    ref = oracle.min_edge_update(E_i, [], V)
    assert int(V[0, 0]) == 10
    assert not np.array_equal(eq11(E_i, [], bandE, T, ebar, M), ref - ref.min())
