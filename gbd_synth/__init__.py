"""Seeded synthetic inputs for the DMRG sweep: active-space integrals and raw
random numbers. This module holds no step of the method itself; it only
draws numbers. Both the CUDA path's tests/bench and the CPU oracle take their
inputs from here.

Integral recipe (the synthetic stand-in for the paper's active-space
integrals h_act and the Cholesky factors B^Q_act, Sec. "The DMRG-QD-NEVPT2
energy" and Sec. "Computational details"):

  * h is symmetric; diagonal h_pp ~ U[-2, 0] Ha; off-diagonal h_pq ~ N(0, 0.05)
    (0.05 is the standard deviation).
  * chol[Q, p, q] ~ N(0, 0.1) * exp(-|p - q| / 3) (0-based |p-q|), symmetric
    in (p, q); the two-electron integrals are (pq|rs) = sum_Q chol[Q,p,q]
    chol[Q,r,s].
  * Draw order: h diagonal (p = 0..n-1), then the h upper triangle row-major
    (p < q), then for Q = 0.. the chol upper triangle row-major (p <= q).
  * Random stream: the splitmix64 generator (Steele, Lea and Flood 2014,
    "Fast splittable pseudorandom number generators"); the i-th 64-bit output
    of the stream seeded with s is mix64(s + (i + 1) * GOLDEN).  Uniform
    doubles take the top 53 bits.  Normals use the Box-Muller cosine branch,
    consuming two uniforms each.

Counter-based values for the initial MPS (mps_init_value) use the same
mix64 on a derived seed and an element key, so any program can recompute
them from the definition without sharing this code.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
MPS_SEED_SALT = 0x4D50535F494E4954  # "MPS_INIT"


def mix64(z: int) -> int:
    """splitmix64 output finalizer (published constants)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential splitmix64 stream: output i = mix64(seed + (i+1)*GOLDEN)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        return mix64(self.state)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self, std: float) -> float:
        """Box-Muller, cosine branch; u1 is mapped to (0, 1]."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return std * math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def make_integrals(n_orb: int, n_chol: int, seed: int):
    """Return (h[n,n], chol[n_chol,n,n]) as float64 arrays (recipe above)."""
    rng = SplitMix64(seed)
    h = np.zeros((n_orb, n_orb))
    for p in range(n_orb):
        h[p, p] = -2.0 * rng.uniform()  # U[-2, 0]
    for p in range(n_orb):
        for q in range(p + 1, n_orb):
            v = rng.normal(0.05)
            h[p, q] = v
            h[q, p] = v
    chol = np.zeros((n_chol, n_orb, n_orb))
    for Q in range(n_chol):
        for p in range(n_orb):
            for q in range(p, n_orb):
                v = rng.normal(0.1) * math.exp(-abs(p - q) / 3.0)
                chol[Q, p, q] = v
                chol[Q, q, p] = v
    return h, chol


def mps_key(site: int, na: int, nb: int, s: int, row: int, col: int) -> int:
    """64-bit element key of an initial-MPS block entry.

    site < 64, na < 64, nb < 64, s < 4, row < 2^20, col < 2^20.
    """
    return (((((site * 64 + na) * 64 + nb) * 4 + s) << 20 | row) << 20) | col


def mps_init_value(seed: int, site: int, na: int, nb: int, s: int, row: int, col: int) -> float:
    """Counter-based uniform value in [-1, 1) for one initial-MPS entry.

    value = 2 * top53(mix64(mix64(seed ^ SALT) + (key + 1) * GOLDEN)) - 1.
    (na, nb) is the left-bond sector of the block, s the local state index.
    """
    base = mix64((seed ^ MPS_SEED_SALT) & MASK64)
    key = mps_key(site, na, nb, s, row, col)
    z = mix64((base + (key + 1) * GOLDEN) & MASK64)
    return 2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0


def mps_init_block(seed: int, site: int, na: int, nb: int, s: int, rows: int, cols: int) -> np.ndarray:
    """Dense (rows x cols) block of initial-MPS values (vectorised form of
    mps_init_value, same definition)."""
    base = np.uint64(mix64((seed ^ MPS_SEED_SALT) & MASK64))
    r = np.arange(rows, dtype=np.uint64)[:, None]
    c = np.arange(cols, dtype=np.uint64)[None, :]
    prefix = np.uint64(((site * 64 + na) * 64 + nb) * 4 + s)
    with np.errstate(over="ignore"):
        key = (((prefix << np.uint64(20)) | r) << np.uint64(20)) | c
        z = base + (key + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)) - 1.0


# Workloads: sizes of the synthetic active spaces (orbitals = electrons,
# S_z = 0) with the Cholesky rank, bond dimension and sweep count.
WORKLOADS = {
    "cas6_m64": dict(n_orb=6, n_elec=6, two_sz=0, n_chol=18, M=64, n_sweeps=4, seed=1),
    "cas12_m256": dict(n_orb=12, n_elec=12, two_sz=0, n_chol=36, M=256, n_sweeps=6, seed=2),
    "cas16_m512": dict(n_orb=16, n_elec=16, two_sz=0, n_chol=48, M=512, n_sweeps=4, seed=3),
    "cas20_m1024": dict(n_orb=20, n_elec=20, two_sz=0, n_chol=60, M=1024, n_sweeps=4, seed=1),
}


def batched_problem_sizes(n_problems: int = 64, seed: int = 1000):
    """Orbital counts U{8..14} and bond dims from {128,256,512} for the
    batch of independent active spaces, drawn from their own stream."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_problems):
        n = 8 + int(rng.uniform() * 7)
        M = (128, 256, 512)[int(rng.uniform() * 3)]
        out.append((n, M))
    return out
