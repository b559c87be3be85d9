"""Seeded synthetic inputs shared by the tests, the bench and the golden-value
scripts.  Holds none of the method's arithmetic: only parameter draws and
random configurations, from numpy's PCG64 with fixed seeds.

Workloads (the paper measures on synthetic lattices only, Sec. 4):
  * single lattice: q = 2, L up to 65536, T = T_c, all-zero or seeded start;
  * replica batch: R replicas, L = 2^k with k uniform in 6..11 (64..2048),
    q uniform in {2, 3, 4, 5, 8}, T uniform in [0.9, 1.1] T_c(q), one Philox
    key per replica;
  * temperature grids around T_c(q) for q in {2, 3, 4}, L in {512, 1024, 2048}.
"""
import math

import numpy as np

Q_CHOICES = (2, 3, 4, 5, 8)


def critical_temperature(q):
    """T_c = 1/ln(1 + sqrt q) of the 2D q-state Potts model (J = 1); the
    paper quotes 1.1346 for q = 2 (Sec. 4).  Used only to place inputs."""
    return 1.0 / math.log1p(math.sqrt(q))


def replica_batch(R=512, master_seed=6, k_min=6, k_max=11):
    """Parameters of R independent replicas: dict of arrays L, q, T, seed."""
    rng = np.random.Generator(np.random.PCG64(master_seed))
    k = rng.integers(k_min, k_max + 1, size=R)
    L = (1 << k).astype(np.uint64)
    q = rng.choice(np.array(Q_CHOICES, dtype=np.uint32), size=R)
    u = rng.random(R)
    T = np.array([(0.9 + 0.2 * u[i]) * critical_temperature(int(q[i])) for i in range(R)])
    seed = rng.integers(0, 2**63, size=R, dtype=np.uint64)
    return {"L": L, "q": q.astype(np.uint32), "T": T, "seed": seed}


def random_spins(L, q, seed):
    """Uniformly random L x L uint8 configuration with states 0..q-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, q, size=(L, L), dtype=np.uint8)


def random_bonds(L, density, seed):
    """Random bond field (bit0 right, bit1 down), each bond active with the
    given probability."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = (rng.random((L, L)) < density).astype(np.uint8)
    b |= (rng.random((L, L)) < density).astype(np.uint8) << 1
    return b


def temperature_grid(q, n=32, lo=0.9, hi=1.1):
    """Plain uniform grid of n temperatures on [lo, hi] * T_c(q)."""
    return np.linspace(lo, hi, n) * critical_temperature(q)
