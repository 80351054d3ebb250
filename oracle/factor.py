"""Factor-graph BP with three-variable factors -- TEST INFRASTRUCTURE.

Sec. 7: for a factor f(x_i, x_j, x_k) the standard factor-BP message update
costs O(M^3); when f equals a constant fbar outside a set of C compatible
triplets the method costs O(C).  This oracle is the standard (dense) update:

  variable -> factor:  n_{v->a}(x) = g_v(x) prod_{b in N(v) \\ a} m_{b->v}(x)    (normalised)
  factor -> variable:  m_{a->v}(x_v) = sum over the other two variables of
                       f(x_0, x_1, x_2) n_{u->a}(x_u) n_{w->a}(x_w)              (normalised)
  beliefs:             b_v(x) = g_v(x) prod_{a in N(v)} m_{a->v}(x) / Z_v

and min-sum with energies (min instead of sum, + instead of *, min shifted to
0).  A flooding iteration updates every variable->factor message, then every
factor->variable message.  Factor a joins variables factors[a] = (v0, v1, v2)
in slot order, and f is indexed f[x_{v0}, x_{v1}, x_{v2}].
"""
from __future__ import annotations

import numpy as np


def dense_table(triplets, vals, fbar, M, dtype=np.float64):
    """F[x0, x1, x2]: vals on the listed triplets, fbar elsewhere."""
    F = np.full((M, M, M), fbar, dtype=dtype)
    for (a, b, c), v in zip(np.asarray(triplets), np.asarray(vals)):
        F[a, b, c] = v
    return F


def _incident(n_vars, factors):
    inc = [[] for _ in range(n_vars)]
    for a, vs in enumerate(factors):
        for s, v in enumerate(vs):
            inc[v].append((a, s))
    return inc


def _f2v_sum(F, n, s):
    """Message from a factor to its slot-s variable from the other two slots' messages."""
    if s == 0:
        return np.einsum("abc,b,c->a", F, n[1], n[2])
    if s == 1:
        return np.einsum("abc,a,c->b", F, n[0], n[2])
    return np.einsum("abc,a,b->c", F, n[0], n[1])


def _f2v_min(V, n, s):
    if s == 0:
        return np.min(V + n[1][None, :, None] + n[2][None, None, :], axis=(1, 2))
    if s == 1:
        return np.min(V + n[0][:, None, None] + n[2][None, None, :], axis=(0, 2))
    return np.min(V + n[0][:, None, None] + n[1][None, :, None], axis=(0, 1))


def sum_product(g, factors, F, n_iters, m0=None):
    """g: [n_vars][M]; factors: [n_f][3]; F: [M][M][M].  Returns
    (factor->variable messages [n_f][3][M], beliefs [n_vars][M])."""
    g = np.asarray(g, dtype=np.float64)
    factors = np.asarray(factors)
    nv, M = g.shape
    nf = len(factors)
    inc = _incident(nv, factors)
    m = np.full((nf, 3, M), 1.0 / M) if m0 is None else np.array(m0, dtype=np.float64)
    for _ in range(n_iters):
        n = np.empty_like(m)
        for v in range(nv):
            for (a, s) in inc[v]:
                p = g[v].copy()
                for (b, t) in inc[v]:
                    if (b, t) != (a, s):
                        p *= m[b, t]
                n[a, s] = p / p.sum()
        for a in range(nf):
            for s in range(3):
                u = _f2v_sum(F, n[a], s)
                m[a, s] = u / u.sum()
    bel = g.copy()
    for v in range(nv):
        for (a, s) in inc[v]:
            bel[v] *= m[a, s]
    return m, bel / bel.sum(axis=1, keepdims=True)


def min_sum(E, factors, V, n_iters, m0=None):
    E = np.asarray(E, dtype=np.int64)
    factors = np.asarray(factors)
    nv, M = E.shape
    nf = len(factors)
    inc = _incident(nv, factors)
    m = np.zeros((nf, 3, M), dtype=np.int64) if m0 is None else np.array(m0, dtype=np.int64)
    for _ in range(n_iters):
        n = np.empty_like(m)
        for v in range(nv):
            for (a, s) in inc[v]:
                p = E[v].copy()
                for (b, t) in inc[v]:
                    if (b, t) != (a, s):
                        p += m[b, t]
                n[a, s] = p - p.min()
        for a in range(nf):
            for s in range(3):
                u = _f2v_min(V, n[a], s)
                m[a, s] = u - u.min()
    bel = E.copy()
    for v in range(nv):
        for (a, s) in inc[v]:
            bel[v] += m[a, s]
    return m, bel
