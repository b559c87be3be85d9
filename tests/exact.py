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
* ``kaufman_mean_esat`` -- exact <E_sat> of q = 2 on an L x L torus of any
                          size from Kaufman's closed-form partition function
                          of the periodic Ising lattice (as written by
                          Ferdinand and Fisher, Phys. Rev. 185, 832 (1969)).
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


def xy_reflect(k, M, j):
    """Angle index of spin k reflected across the line perpendicular to the
    embedding vector r at angle pi j / M - pi / 2, computed with vectors:
    s' = s - 2 (s . r) r (Wolff's embedding step)."""
    th = 2 * np.pi * k / M
    ph = np.pi * j / M - np.pi / 2
    s = np.array([np.cos(th), np.sin(th)])
    r = np.array([np.cos(ph), np.sin(ph)])
    t = s - 2 * (s @ r) * r
    a = np.arctan2(t[1], t[0]) * M / (2 * np.pi)
    kk = int(np.rint(a)) % M
    assert abs(a - np.rint(a)) < 1e-9, "reflection leaves the angle set"
    return kk


def xy_sigma(k, M, j):
    """s . r for spin k and the embedding vector of axis index j."""
    return float(np.cos(2 * np.pi * k / M - (np.pi * j / M - np.pi / 2)))


def xy_energy_all(L, M):
    """All M^(L*L) configurations and their energies H = -sum cos(theta_i -
    theta_j) over the 2N right/down bonds of the periodic L x L lattice."""
    N = L * L
    states = np.array(list(itertools.product(range(M), repeat=N)), dtype=np.int16)
    r_idx, d_idx = neighbours(L)
    ang = 2 * np.pi * states / M
    H = -(np.cos(ang - ang[:, r_idx]).sum(1) + np.cos(ang - ang[:, d_idx]).sum(1))
    return states, H


def xy_transition(L, M, T, label_fn):
    """Exact transition matrix of one embedded-cluster SW sweep (Wolff's
    embedding, every cluster reflected with probability 1/2) of the M-angle
    XY model on the L x L torus, built from vector geometry: axis index j
    uniform in 0..M-1; a bond is eligible iff sigma_i sigma_j > 0 and active
    with probability 1 - exp(-2 sigma_i sigma_j / T)."""
    N = L * L
    states, H = xy_energy_all(L, M)
    S = len(states)
    r_idx, d_idx = neighbours(L)
    powers = M ** np.arange(N - 1, -1, -1)
    refl = np.array([[xy_reflect(k, M, j) for k in range(M)] for j in range(M)])
    P = np.zeros((S, S))
    for si in range(S):
        s = states[si]
        for j in range(M):
            sig = np.array([xy_sigma(int(k), M, j) for k in s])
            sig[np.abs(sig) < 1e-12] = 0.0
            bonds = []  # (site, dir, p)
            for i in range(N):
                for d, nb in ((0, r_idx[i]), (1, d_idx[i])):
                    prod = sig[i] * sig[nb]
                    if prod > 0:
                        bonds.append((i, d, -np.expm1(-2 * prod / T)))
            nbd = len(bonds)
            for mask in range(1 << nbd):
                w = 1.0 / M
                b = np.zeros(N, dtype=np.uint8)
                for t, (i, d, p) in enumerate(bonds):
                    if (mask >> t) & 1:
                        w *= p
                        b[i] |= RIGHT if d == 0 else DOWN
                    else:
                        w *= 1 - p
                if w == 0.0:
                    continue
                roots = np.asarray(label_fn(b.reshape(L, L))).ravel()
                uniq, cl = np.unique(roots, return_inverse=True)
                nc = len(uniq)
                for fm in range(1 << nc):
                    flip = np.array([(fm >> c) & 1 for c in range(nc)])[cl]
                    s2 = np.where(flip == 1, refl[j][s], s)
                    P[si, int(s2 @ powers)] += w / (1 << nc)
    return P, H


def wolff_transition(L, q, p):
    """Exact transition matrix of one Wolff single-cluster step of the
    q-state Potts model on the L x L torus: seed uniform over the N sites,
    new state uniform over the q - 1 others, every bond between two sites in
    the seed's state active with probability p independently; the seed's
    component (breadth-first search) takes the new state."""
    N = L * L
    states, E, _ = e_sat_all(L, q)
    S = len(states)
    r_idx, d_idx = neighbours(L)
    powers = q ** np.arange(N - 1, -1, -1)
    P = np.zeros((S, S))
    for si in range(S):
        s = states[si]
        for i0 in range(N):
            old = s[i0]
            el = [(i, d) for i in range(N) for d, nb in ((0, r_idx[i]), (1, d_idx[i]))
                  if s[i] == old and s[nb] == old]
            for mask in range(1 << len(el)):
                k = bin(mask).count("1")
                w = p ** k * (1 - p) ** (len(el) - k) / N
                b = np.zeros(N, dtype=np.uint8)
                for t, (i, d) in enumerate(el):
                    if (mask >> t) & 1:
                        b[i] |= RIGHT if d == 0 else DOWN
                roots = bfs_roots(b.reshape(L, L)).ravel()
                comp = roots == roots[i0]
                for new in range(q):
                    if new == old:
                        continue
                    s2 = np.where(comp, new, s)
                    P[si, int(s2 @ powers)] += w / (q - 1)
    return P, E


def kaufman_logz(K, m, n):
    """ln Z of the Ising model sum exp(K * sum_<ij> s_i s_j) on an m x n
    periodic lattice (mpmath number):
      Z = 1/2 (2 sinh 2K)^(mn/2) (Z1 + Z2 + Z3 + Z4),
      Z1 = prod_{r<n} 2 cosh(m g_{2r+1}/2),  Z2 = prod 2 sinh(m g_{2r+1}/2),
      Z3 = prod_{r<n} 2 cosh(m g_{2r}/2),    Z4 = prod 2 sinh(m g_{2r}/2),
    with cosh g_l = cosh 2K coth 2K - cos(pi l / n) for l > 0 and
    g_0 = 2K + ln tanh K (negative below T_c, which makes Z4 change sign)."""
    import mpmath as mp
    K = mp.mpf(K)
    c = mp.cosh(2 * K) * mp.coth(2 * K)

    def g(l):
        if l == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(c - mp.cos(mp.pi * l / n))

    z1 = z2 = z3 = z4 = mp.mpf(1)
    for r in range(n):
        a, b = m * g(2 * r + 1) / 2, m * g(2 * r) / 2
        z1 *= 2 * mp.cosh(a)
        z2 *= 2 * mp.sinh(a)
        z3 *= 2 * mp.cosh(b)
        z4 *= 2 * mp.sinh(b)
    return mp.log(mp.mpf(1) / 2) + (m * n / mp.mpf(2)) * mp.log(2 * mp.sinh(2 * K)) + \
        mp.log(z1 + z2 + z3 + z4)


def kaufman_mean_esat(L, T):
    """Exact <E_sat> of the q = 2 Potts model at temperature T on an L x L
    torus (L >= 3): with delta = (1 + s s')/2 the Potts weight exp(E_sat/T)
    is the Ising weight at K = 1/(2T) times exp(N/T), so
    <E_sat> = N + (1/2) d ln Z / dK."""
    import mpmath as mp
    mp.mp.dps = 50
    K = mp.mpf(1) / (2 * mp.mpf(T))
    d = mp.diff(lambda k: kaufman_logz(k, L, L), K)
    return float(L * L + d / 2)
