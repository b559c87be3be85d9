"""Independent exact checkers used to pin the oracle (no shared code with it).

* ``bfs_roots``        -- breadth-first connected components of a periodic
                          bond field (the textbook definition of a cluster).
* ``brute_moments``    -- <E_sat>, <E_sat^2>, <n_max> by enumerating all q^N
                          configurations with Boltzmann weight exp(E_sat/T)
                          (H = -sum delta, J = 1, Eq. 1 up to a constant).
* ``transfer_moments`` -- the same on an L x M torus by a row transfer
                          matrix, for lattices too big to enumerate.
* ``sw_transition``    -- the exact SW transition matrix of a tiny lattice,
                          built from a caller-supplied labeller, for the
                          stationarity / detailed-balance checks.
"""
from collections import deque
import itertools

import numpy as np

RIGHT, DOWN = 1, 2


def neighbours(L):
    """(right, down) neighbour index arrays of the periodic L x L lattice."""
    idx = np.arange(L * L).reshape(L, L)
    return np.roll(idx, -1, axis=1).ravel(), np.roll(idx, -1, axis=0).ravel()


def bfs_roots(b):
    """Connected components of the bond field b (bit0 right, bit1 down) on the
    periodic lattice; each site gets the minimum index of its component."""
    b = np.asarray(b, dtype=np.uint8)
    L = b.shape[0]
    N = L * L
    r_idx, d_idx = neighbours(L)
    flat = b.ravel()
    adj = [[] for _ in range(N)]
    for i in range(N):
        if flat[i] & RIGHT:
            adj[i].append(int(r_idx[i])); adj[int(r_idx[i])].append(i)
        if flat[i] & DOWN:
            adj[i].append(int(d_idx[i])); adj[int(d_idx[i])].append(i)
    root = np.full(N, -1, dtype=np.int64)
    for s in range(N):
        if root[s] >= 0:
            continue
        comp = [s]
        root[s] = s
        dq = deque([s])
        while dq:
            u = dq.popleft()
            for v in adj[u]:
                if root[v] < 0:
                    root[v] = s
                    comp.append(v)
                    dq.append(v)
        m = min(comp)
        root[comp] = m
    return root.reshape(L, L)


def e_sat_all(L, q):
    """E_sat and per-state counts of every configuration of an L x L lattice
    (configurations enumerated in base-q order)."""
    N = L * L
    states = np.array(list(itertools.product(range(q), repeat=N)), dtype=np.int16)
    r_idx, d_idx = neighbours(L)
    E = (states == states[:, r_idx]).sum(1) + (states == states[:, d_idx]).sum(1)
    n = np.stack([(states == k).sum(1) for k in range(q)], axis=1)
    return states, E.astype(np.int64), n


def brute_moments(L, q, T):
    """Exact <E_sat>, <E_sat^2>, <max_s n_s> by enumerating all q^(L*L) states."""
    _, E, n = e_sat_all(L, q)
    w = np.exp((E - E.max()) / T)
    Z = w.sum()
    nmax = n.max(1)
    return (w * E).sum() / Z, (w * E * E).sum() / Z, (w * nmax).sum() / Z


def transfer_moments(L, M, q, T):
    """Exact <E_sat>, <E_sat^2> on an L-wide, M-tall torus by the row transfer
    matrix: Z(beta) = Tr(A^M) with A[a,b] = exp(beta*(h(a)+v(a,b)))."""
    rows = np.array(list(itertools.product(range(q), repeat=L)), dtype=np.int16)
    h = (rows == np.roll(rows, -1, axis=1)).sum(1).astype(np.float64)
    v = (rows[:, None, :] == rows[None, :, :]).sum(2).astype(np.float64)
    X = h[:, None] + v  # bonds owned by row a: its horizontal ones + down to b

    def logZ(beta):
        A = np.exp(beta * (X - X.max()))
        tr = np.trace(np.linalg.matrix_power(A, M))
        return np.log(tr) + M * beta * X.max()

    beta = 1.0 / T
    hstep = 1e-4 * beta
    f0, fp, fm = logZ(beta), logZ(beta + hstep), logZ(beta - hstep)
    fp2, fm2 = logZ(beta + 2 * hstep), logZ(beta - 2 * hstep)
    d1 = (-fp2 + 8 * fp - 8 * fm + fm2) / (12 * hstep)
    d2 = (-fp2 + 16 * fp - 30 * f0 + 16 * fm - fm2) / (12 * hstep * hstep)
    mean = d1
    return mean, d2 + mean * mean


def sw_transition(L, q, p, label_fn):
    """Exact SW transition matrix P[s, s'] of the L x L, q-state lattice.

    For every subset B of the 2N bonds (as a bond field) the labeller gives
    the clusters of B.  Configurations constant on those clusters are exactly
    the ones whose satisfied bonds include B; from such an s, B is the active
    set with probability p^|B| (1-p)^(sat(s)-|B|), and each of the q^nc
    recolourings of the clusters follows with probability q^-nc."""
    N = L * L
    states, E, _ = e_sat_all(L, q)
    S = len(states)
    r_idx, d_idx = neighbours(L)
    P = np.zeros((S, S))
    powers = q ** np.arange(N - 1, -1, -1)
    for mask in range(1 << (2 * N)):
        bits = np.array([(mask >> k) & 1 for k in range(2 * N)], dtype=np.uint8)
        b = (bits[:N] * RIGHT + bits[N:] * DOWN).astype(np.uint8).reshape(L, L)
        roots = np.asarray(label_fn(b)).ravel()
        uniq, cl = np.unique(roots, return_inverse=True)
        nc = len(uniq)
        # every configuration constant on the clusters
        assign = np.array(list(itertools.product(range(q), repeat=nc)), dtype=np.int64)
        cfg = assign[:, cl]
        ids = cfg @ powers
        k = int(bits.sum())
        sat = E[ids]
        w = p ** k * (1 - p) ** (sat - k) / q ** nc
        P[np.ix_(ids, ids)] += w[:, None]
    return P, E
