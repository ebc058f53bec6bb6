"""Seeded synthetic COO workloads shaped like the paper's and the benchmark's.

This module only draws random coordinates and values. It holds none of the
contraction's arithmetic (no keys, no grouping, no products), so that both the
CPU oracle and the CUDA path can be fed from it without sharing method code.

Recipe (stated once, used everywhere):

* Random numbers come from NumPy's ``PCG64`` bit generator. The named
  workloads use seed ``20241010 + k`` for workload k (1..5; 6 for wide_keys, 7 for the
  Table 2 shapes, 8 for the Set 1/2 sweeps); 3Z uses the seed
  of workload 3.
* Values are uniform in [-1, 1]; an exact 0.0 is redrawn, because COO lists
  only nonzeros (Section 2.1.2).
* Coordinates are uniform per mode unless a workload says otherwise; repeated
  coordinates are allowed (they are additive COO entries) except where a
  workload asks for distinct ones.
* Mode numbers are 0-based throughout.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 20241010


@dataclass
class COO:
    """A COO tensor: ``coords`` is int32 [nnz, order] (C order), ``vals`` float64 [nnz]."""

    shape: Tuple[int, ...]
    coords: np.ndarray
    vals: np.ndarray

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.coords = np.ascontiguousarray(self.coords, dtype=np.int32).reshape(-1, len(self.shape))
        self.vals = np.ascontiguousarray(self.vals, dtype=np.float64).reshape(-1)
        if self.coords.shape[0] != self.vals.shape[0]:
            raise ValueError("coords and vals disagree on nnz")

    @property
    def order(self) -> int:
        return len(self.shape)

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])

    def take(self, idx) -> "COO":
        return COO(self.shape, self.coords[idx], self.vals[idx])


@dataclass
class Problem:
    """One contraction Z = X (x) Y over paired modes ``cx[i]`` <-> ``cy[i]``."""

    X: COO
    Y: COO
    cx: Tuple[int, ...]
    cy: Tuple[int, ...]
    out_order: Optional[Tuple[int, ...]] = None
    name: str = ""
    meta: dict = field(default_factory=dict)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def nonzero_values(rng: np.random.Generator, n: int) -> np.ndarray:
    """n values uniform in [-1, 1] with exact zeros redrawn."""
    v = rng.uniform(-1.0, 1.0, size=n)
    bad = np.flatnonzero(v == 0.0)
    while bad.size:
        v[bad] = rng.uniform(-1.0, 1.0, size=bad.size)
        bad = bad[v[bad] == 0.0]
    return v


def uniform_coords(rng: np.random.Generator, shape: Sequence[int], nnz: int) -> np.ndarray:
    """nnz coordinates, each mode uniform over its length (repeats allowed)."""
    out = np.empty((nnz, len(shape)), dtype=np.int32)
    for j, s in enumerate(shape):
        out[:, j] = rng.integers(0, s, size=nnz, dtype=np.int64).astype(np.int32)
    return out


def distinct_coords(rng: np.random.Generator, shape: Sequence[int], nnz: int) -> np.ndarray:
    """nnz distinct coordinates drawn without replacement from the whole index space."""
    cells = int(np.prod(shape, dtype=np.int64))
    if nnz > cells:
        raise ValueError("more distinct coordinates than cells")
    flat = rng.choice(cells, size=nnz, replace=False)
    cols = np.unravel_index(flat, tuple(shape))
    return np.stack([c.astype(np.int32) for c in cols], axis=1)


def uniform_coo(rng, shape, nnz, distinct=False) -> COO:
    coords = distinct_coords(rng, shape, nnz) if distinct else uniform_coords(rng, shape, nnz)
    return COO(tuple(shape), coords, nonzero_values(rng, nnz))


def bounded_zipf_ranks(rng: np.random.Generator, n: int, ncats: int, s: float) -> np.ndarray:
    """n draws of a rank in [0, ncats) with P(rank r) proportional to (r+1)^-s (inverse CDF)."""
    w = np.arange(1, ncats + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, ncats - 1)


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------

def plain_small(seed: int = SEED_BASE + 1) -> Problem:
    """Order-3 64^3 tensors, 5,000 distinct coordinates each; X mode 2 with Y mode 0."""
    rng = rng_for(seed)
    X = uniform_coo(rng, (64, 64, 64), 5000, distinct=True)
    Y = uniform_coo(rng, (64, 64, 64), 5000, distinct=True)
    return Problem(X, Y, (2,), (0,), name="plain_small_64^3_5e3")


def plain_large(seed: int = SEED_BASE + 2, nnz: int = 5_000_000, n: int = 256) -> Problem:
    """Order-4 n^4 tensors, ``nnz`` uniform coordinates each; X modes (2,3) with Y modes (0,1)."""
    rng = rng_for(seed)
    X = uniform_coo(rng, (n,) * 4, nnz)
    Y = uniform_coo(rng, (n,) * 4, nnz)
    return Problem(X, Y, (2, 3), (0, 1), name=f"plain_large_{n}^4_{nnz:.0e}")


def imbalanced(seed: int = SEED_BASE + 3, nx: int = 20_000_000, ny: int = 20_000,
               both_zipf: bool = False, s: float = 1.2) -> Problem:
    """X 4096x512x512, Y 512x512x64; X modes (1,2) with Y modes (0,1).

    Y's (mode 0, mode 1) cell is Zipf(s) over the 262,144 cells, through a seeded
    rank -> cell permutation; with ``both_zipf`` X's (mode 1, mode 2) cell follows
    the same law and permutation, otherwise X is uniform.
    """
    rng = rng_for(seed)
    ncells = 512 * 512
    perm = rng.permutation(ncells)
    X = np.empty((nx, 3), dtype=np.int32)
    X[:, 0] = rng.integers(0, 4096, size=nx).astype(np.int32)
    if both_zipf:
        cell = perm[bounded_zipf_ranks(rng, nx, ncells, s)]
        a, b = np.unravel_index(cell, (512, 512))
        X[:, 1], X[:, 2] = a, b
    else:
        X[:, 1] = rng.integers(0, 512, size=nx).astype(np.int32)
        X[:, 2] = rng.integers(0, 512, size=nx).astype(np.int32)
    xv = nonzero_values(rng, nx)
    Y = np.empty((ny, 3), dtype=np.int32)
    cell = perm[bounded_zipf_ranks(rng, ny, ncells, s)]
    a, b = np.unravel_index(cell, (512, 512))
    Y[:, 0], Y[:, 1] = a, b
    Y[:, 2] = rng.integers(0, 64, size=ny).astype(np.int32)
    yv = nonzero_values(rng, ny)
    name = "imbalanced_zipf_both" if both_zipf else "imbalanced_zipf_y"
    return Problem(COO((4096, 512, 512), X, xv), COO((512, 512, 64), Y, yv), (1, 2), (0, 1), name=name)


def wide_keys(seed: int = SEED_BASE + 6, nnz: int = 5_000_000, n: int = 256, length: int = 65536,
              pool: int = 65536, nnz_y: Optional[int] = None) -> Problem:
    """plain_large with its paired modes stretched to ``length`` each: X is n x n x L x L, Y
    is L x L x n x n, X modes (2,3) with Y modes (0,1), a L^2 (2^32) contract key space.

    Both tensors draw their paired (i, j) coordinates uniformly from one shared pool of
    ``pool`` cells, themselves uniform over L x L: a very sparse tensor whose entries sit on
    a few fibres, like the network-traffic tensors of Table 2 (LBNL, 65K^3). Free
    coordinates are uniform; with the defaults the products and output match plain_large's
    in distribution.
    """
    rng = rng_for(seed)
    cells = rng.choice(length * length, size=pool, replace=False)
    ci, cj = np.unravel_index(cells, (length, length))
    ny = nnz if nnz_y is None else nnz_y

    def draw(count, paired_first):
        c = np.empty((count, 4), dtype=np.int32)
        pick = rng.integers(0, pool, size=count)
        a, b = (0, 1) if paired_first else (2, 3)
        f, g = (2, 3) if paired_first else (0, 1)
        c[:, a], c[:, b] = ci[pick], cj[pick]
        c[:, f] = rng.integers(0, n, size=count).astype(np.int32)
        c[:, g] = rng.integers(0, n, size=count).astype(np.int32)
        return c

    X = COO((n, n, length, length), draw(nnz, False), nonzero_values(rng, nnz))
    Y = COO((length, length, n, n), draw(ny, True), nonzero_values(rng, ny))
    return Problem(X, Y, (2, 3), (0, 1), name=f"wide_keys_{length}^2_pool{pool}_{nnz:.0e}")


# Table 2 shapes and entry counts. The paper generated these tensors at random (all but
# NIPS); "65K", "2K" and the like are read as 65,536 and 2,000.
TABLE2 = {
    "enron": ((186, 186, 44), 9_838),
    "lbnl": ((65_536, 65_536, 65_536), 27_269),
    "facebook": ((63_891, 63_890, 1_847), 738_000),
    "hubbard_1d_p": ((4, 4, 93, 36, 432), 300_000),
    "hubbard_1d_t": ((131, 4, 413, 36, 4), 400_000),
    "hubbard_1d_z": ((4, 129, 184, 24, 4), 100_000),
    "hubbard_2d": ((4, 4, 111, 24, 528), 300_000),
    "nips": ((2_000, 3_000, 14_000, 17_000), 3_000_000),
}


def table2(name: str, seed: int = SEED_BASE + 7, nnz: Optional[int] = None) -> Problem:
    """Self-contraction of a random tensor with one of Table 2's shapes over its second and
    third modes (0-based 1 and 2), the paper's stated convention for its experiments.
    ``nnz`` overrides the table's entry count (smaller copies for the oracle)."""
    shape, n0 = TABLE2[name]
    rng = rng_for(seed + sorted(TABLE2).index(name))
    T = uniform_coo(rng, shape, n0 if nnz is None else nnz)
    return Problem(T, T, (1, 2), (1, 2), name=f"table2_{name}")


def set_sweep(set_no: int, pair: str, nnz: int, seed: int = SEED_BASE + 8) -> Problem:
    """A Set 1 (mode length 50) or Set 2 (length 100) case of Table 1: A is order 5, B order 4,
    each with ``nnz`` uniform entries. ``pair`` is "AA" or "BB" (a tensor with itself) or "AB";
    the second and third modes (0-based 1 and 2) of both are paired."""
    length = {1: 50, 2: 100}[set_no]
    rng = rng_for(seed + 10 * set_no + {"AA": 0, "BB": 1, "AB": 2}[pair])
    A = uniform_coo(rng, (length,) * 5, nnz) if pair in ("AA", "AB") else None
    B = uniform_coo(rng, (length,) * 4, nnz) if pair in ("BB", "AB") else None
    X, Y = {"AA": (A, A), "BB": (B, B), "AB": (A, B)}[pair]
    return Problem(X, Y, (1, 2), (1, 2), name=f"set{set_no}_{pair}_{nnz // 1000}K")


def small_pair(rng: np.random.Generator, nnz_lo: float = 1e2, nnz_hi: float = 1e5,
               size_lo: int = 16, size_hi: int = 512) -> Problem:
    """One order-3 pair of the batched mix: sizes uniform in [16, 512], one paired mode
    (its size shared), contracted mode uniform per side, nnz log-uniform per tensor."""
    cx = int(rng.integers(0, 3))
    cy = int(rng.integers(0, 3))
    xs = [int(v) for v in rng.integers(size_lo, size_hi + 1, size=3)]
    ys = [int(v) for v in rng.integers(size_lo, size_hi + 1, size=3)]
    ys[cy] = xs[cx]
    nx = int(round(np.exp(rng.uniform(np.log(nnz_lo), np.log(nnz_hi)))))
    ny = int(round(np.exp(rng.uniform(np.log(nnz_lo), np.log(nnz_hi)))))
    X = uniform_coo(rng, xs, nx)
    Y = uniform_coo(rng, ys, ny)
    return Problem(X, Y, (cx,), (cy,), name="batched_pair")


def batched(seed: int = SEED_BASE + 4, n: int = 2048) -> List[Problem]:
    rng = rng_for(seed)
    return [small_pair(rng) for _ in range(n)]


def served_large(rng: np.random.Generator, nnz: int = 1_000_000, n: int = 128) -> Problem:
    """An order-4 n^4 pair with ``nnz`` entries each, contracting two random paired modes."""
    cx = tuple(int(v) for v in rng.choice(4, size=2, replace=False))
    cy = tuple(int(v) for v in rng.choice(4, size=2, replace=False))
    X = uniform_coo(rng, (n,) * 4, nnz)
    Y = uniform_coo(rng, (n,) * 4, nnz)
    return Problem(X, Y, cx, cy, name="served_large")


def random_case(rng: np.random.Generator, max_order: int = 4, max_size: int = 6,
                max_nnz: int = 40, dup: bool = True) -> Problem:
    """A tiny random problem for property tests: orders 1..max_order, any number of
    paired modes (0..min order), random sizes, optional repeated coordinates."""
    ox = int(rng.integers(1, max_order + 1))
    oy = int(rng.integers(1, max_order + 1))
    m = int(rng.integers(0, min(ox, oy) + 1))
    cx = tuple(int(v) for v in rng.choice(ox, size=m, replace=False))
    cy = tuple(int(v) for v in rng.choice(oy, size=m, replace=False))
    xs = [int(v) for v in rng.integers(1, max_size + 1, size=ox)]
    ys = [int(v) for v in rng.integers(1, max_size + 1, size=oy)]
    for a, b in zip(cx, cy):
        ys[b] = xs[a]
    nx = int(rng.integers(0, max_nnz + 1))
    ny = int(rng.integers(0, max_nnz + 1))
    X = uniform_coo(rng, xs, nx) if dup else uniform_coo(rng, xs, min(nx, int(np.prod(xs))), distinct=True)
    Y = uniform_coo(rng, ys, ny) if dup else uniform_coo(rng, ys, min(ny, int(np.prod(ys))), distinct=True)
    nz_order = (ox - m) + (oy - m)
    out = tuple(int(v) for v in rng.permutation(nz_order)) if rng.random() < 0.5 else None
    return Problem(X, Y, cx, cy, out, name="random_case")


def served_pools(seed: int = SEED_BASE + 5, n_small: int = 96, n_large: int = 12):
    """The distinct problems a served trace draws from: ``n_small`` pairs of the batched mix
    and ``n_large`` order-4 128^4 pairs with 1e6 entries each contracting two random paired
    modes (holding 20,000 distinct 1e6-entry pairs at once would take about 190 GB of HBM)."""
    rng = rng_for(seed)
    small = [small_pair(rng) for _ in range(n_small)]
    large = [served_large(rng) for _ in range(n_large)]
    return small, large, rng


def served_trace(rng: np.random.Generator, n_requests: int, n_small: int, n_large: int,
                 large_fraction: float = 0.2):
    """``n_requests`` draws from the pools: each request is large with probability
    ``large_fraction``, then uniform over its pool. Returns a list of ("small"|"large", index)."""
    is_large = rng.random(n_requests) < large_fraction
    picks = []
    for big in is_large:
        picks.append(("large", int(rng.integers(n_large))) if big else ("small", int(rng.integers(n_small))))
    return picks
