"""Seeded synthetic inputs for exact k-nearest-neighbour search.

This module only draws random numbers; it holds none of the search method's
arithmetic, so both the CUDA path and the CPU oracle may import it.

Every workload is generated on the host with numpy ``Generator(PCG64)`` from
``SeedSequence(BASE_SEED + workload_id)``.  The sequence is split into three
independent child streams: [0] shared model parameters (mixture centres,
linear maps, rotations), [1] reference points, [2] query points.  Arrays are
C-contiguous float32, row-major ``n x d``.

The paper (Curtin et al., "Tree-Independent Dual-Tree Algorithms", ICML 2013)
runs no experiments, so the shapes below are synthetic stand-ins:

1. ``mono_uniform``  -- monochromatic, N=10,000, d=3, U[0,1]^3, k=5, leaf 20.
2. ``gmm16``         -- bichromatic, N_r=4,000,000, N_q=1,000,000, d=16, k=10;
   32 isotropic Gaussian components, centres U[-10,10]^16, sigma=1, each point
   picks its component uniformly.
3. ``batched``       -- 256 monochromatic problems, ln N ~ Normal(ln 14142, 1.32^2)
   clipped to [1000, 200000], d in {3, 8, 32}, k in {1, 10}, U[0,1]^d or N(0, I).
4. ``latent3``       -- N_r=10,000,000, N_q=1,000,000 (+200,000 training queries),
   d=8, x = A z + eps with z ~ U[0,1]^3, A in R^{8x3} with N(0,1) entries,
   eps ~ N(0, 0.01^2 I), k=10.
5. ``powerlaw64``    -- bichromatic, N_r=N_q=2,000,000, d=64, k=50,
   x = Q diag(i^-0.75) z, z ~ N(0, I), Q a random rotation (QR of a Gaussian
   matrix with the sign of R's diagonal folded into Q).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BASE_SEED = 1304_4327_0


@dataclasses.dataclass
class Workload:
    name: str
    ref: np.ndarray                  # (n_ref, d) float32
    query: Optional[np.ndarray]      # (n_query, d) float32, or None = monochromatic
    k: int
    leaf_size: int
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def mono(self) -> bool:
        return self.query is None

    @property
    def d(self) -> int:
        return int(self.ref.shape[1])

    @property
    def n_query(self) -> int:
        return int(self.ref.shape[0] if self.query is None else self.query.shape[0])


def _streams(workload_id: int, n: int = 3):
    ss = np.random.SeedSequence(BASE_SEED + int(workload_id))
    return [np.random.Generator(np.random.PCG64(c)) for c in ss.spawn(n)]


def _query_stream(workload_id: int, shard: int):
    """Query stream of one shard (shard 0 is the workload's own query stream)."""
    return _streams(workload_id, 3 + shard)[2 + shard]


def uniform(n: int, d: int, seed: int) -> np.ndarray:
    """n points U[0,1]^d as float32 from one seed (used by tests)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.random((n, d), dtype=np.float32)


def gaussian(n: int, d: int, seed: int, scale: float = 1.0) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    return (g.standard_normal((n, d), dtype=np.float32) * np.float32(scale)).astype(np.float32)


def duplicate_heavy(n: int, d: int, seed: int, n_distinct: int = 7) -> np.ndarray:
    """n points drawn (with repetition) from n_distinct grid points: many exact ties."""
    g = np.random.Generator(np.random.PCG64(seed))
    base = g.integers(0, 4, size=(n_distinct, d)).astype(np.float32)
    pick = g.integers(0, n_distinct, size=n)
    return np.ascontiguousarray(base[pick])


def collinear(n: int, d: int, seed: int) -> np.ndarray:
    """n points on one random line through R^d (a degenerate, zero-width cloud)."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = g.random(n, dtype=np.float64)
    direction = g.standard_normal(d)
    direction /= np.linalg.norm(direction)
    return (t[:, None] * direction[None, :] * 10.0).astype(np.float32)


def lattice(shape) -> np.ndarray:
    """All integer points of a grid with the given extents, row-major order."""
    axes = [np.arange(s, dtype=np.float32) for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([m.reshape(-1) for m in mesh], axis=1))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def mono_uniform(n: int = 10_000, d: int = 3, k: int = 5, leaf_size: int = 20) -> Workload:
    _, gr, _ = _streams(1)
    ref = gr.random((n, d), dtype=np.float32)
    return Workload("mono_uniform", ref, None, k, leaf_size)


def _gmm(g, centres, n, sigma):
    comp = g.integers(0, centres.shape[0], size=n)
    x = g.standard_normal((n, centres.shape[1]), dtype=np.float32) * np.float32(sigma)
    x += centres[comp]
    return x


def gmm16(n_ref: int = 4_000_000, n_query: int = 1_000_000, d: int = 16, k: int = 10,
          n_comp: int = 32, leaf_size: int = 32, shard: int = 0) -> Workload:
    """``shard`` > 0 draws an independent query set (one per GPU of a weak-scaling run)."""
    gp, gr, _ = _streams(2)
    gq = _query_stream(2, shard)
    centres = gp.uniform(-10.0, 10.0, size=(n_comp, d)).astype(np.float32)
    ref = _gmm(gr, centres, n_ref, 1.0)
    query = _gmm(gq, centres, n_query, 1.0)
    return Workload("gmm16", ref, query, k, leaf_size, {"centres": centres})


def batched_specs(n_problems: int = 256, n_min: int = 1000, n_max: int = 200_000) -> List[dict]:
    """Shape of every problem of the batched workload (no point data)."""
    gp, _, _ = _streams(3)
    specs = []
    for i in range(n_problems):
        n = int(round(math.exp(gp.normal(math.log(14142.0), 1.32))))
        n = max(n_min, min(n_max, n))
        d = int(gp.choice([3, 8, 32]))
        k = int(gp.choice([1, 10]))
        dist = "uniform" if gp.random() < 0.5 else "gaussian"
        specs.append({"n": n, "d": d, "k": k, "dist": dist, "seed": BASE_SEED * 1000 + 3000 + i})
    return specs


def batched_problem(spec: dict, n_cap: Optional[int] = None) -> Workload:
    n = spec["n"] if n_cap is None else min(spec["n"], n_cap)
    if spec["dist"] == "uniform":
        pts = uniform(n, spec["d"], spec["seed"])
    else:
        pts = gaussian(n, spec["d"], spec["seed"])
    return Workload("batched", pts, None, spec["k"], 0, dict(spec))


def latent3(n_ref: int = 10_000_000, n_query: int = 1_000_000, n_train: int = 200_000,
            d: int = 8, k: int = 10, leaf_size: int = 32, shard: int = 0) -> Workload:
    """``shard`` > 0 draws an independent query (and training) set."""
    gp, gr, _ = _streams(4)
    gq = _query_stream(4, shard)
    A = gp.standard_normal((d, 3)).astype(np.float32)

    def draw(g, n):
        z = g.random((n, 3), dtype=np.float32)
        eps = g.standard_normal((n, d), dtype=np.float32) * np.float32(0.01)
        return (z @ A.T + eps).astype(np.float32)

    ref = draw(gr, n_ref)
    query = draw(gq, n_query)
    train = draw(gq, n_train)
    return Workload("latent3", ref, query, k, leaf_size, {"A": A, "train": train})


def powerlaw64(n_ref: int = 2_000_000, n_query: int = 2_000_000, d: int = 64, k: int = 50,
               leaf_size: int = 32, n_train: int = 0, shard: int = 0) -> Workload:
    """``n_train`` > 0 also draws a disjoint training query set (after the
    queries, from their stream); ``shard`` > 0 draws an independent query set."""
    gp, gr, _ = _streams(5)
    gq = _query_stream(5, shard)
    G = gp.standard_normal((d, d))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    scale = np.arange(1, d + 1, dtype=np.float64) ** -0.75
    M = (Q * scale[None, :]).astype(np.float32)       # x = M z

    def draw(g, n):
        z = g.standard_normal((n, d), dtype=np.float32)
        return (z @ M.T).astype(np.float32)

    ref = draw(gr, n_ref)
    query = draw(gq, n_query)
    extra = {"M": M}
    if n_train > 0:
        extra["train"] = draw(gq, n_train)
    return Workload("powerlaw64", ref, query, k, leaf_size, extra)


WORKLOADS = {1: mono_uniform, 2: gmm16, 3: batched_specs, 4: latent3, 5: powerlaw64}
