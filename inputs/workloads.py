"""Named synthetic workloads (edge-list generator + CL-DIAM parameters).

tau is set per workload so that the clustering has about the stated number of
clusters (the paper sets tau for a quotient-size target, Section 5).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable

from . import EdgeList, grid, rmat, road_mesh


@dataclass(frozen=True)
class Workload:
    name: str
    describe: str
    make: Callable[[], EdgeList]
    tau: float
    seed: int
    target_k: int


WORKLOADS = {
    "grid64": Workload("grid64", "64x64 4-neighbour mesh, 8,064 edges, w in [1,100], seed 1",
                       lambda: grid(64, 100, 1), tau=0.3, seed=1, target_k=64),
    "rmat20": Workload("rmat20", "R-MAT scale 20, edge factor 16, (.57,.19,.19,.05), w in [1,2^20], seed 2, LCC",
                       lambda: rmat(20, 16, 1 << 20, 2), tau=4.65, seed=2, target_k=1024),
    "roadmesh4096": Workload("roadmesh4096", "4096x4096 mesh, 10% edges deleted, 0.1% chords, w in [1,1000], seed 3, LCC",
                             lambda: road_mesh(4096, 1000, 3), tau=5.4, seed=3, target_k=4096),
    "rmat22": Workload("rmat22", "R-MAT scale 22, edge factor 16, w in [1,1000], seed 3, LCC (profiling size)",
                       lambda: rmat(22, 16, 1000, 3), tau=10.5, seed=3, target_k=2048),
    "rmat24": Workload("rmat24", "R-MAT scale 24, edge factor 16, w in [1,1000], seed 3, LCC",
                       lambda: rmat(24, 16, 1000, 3), tau=21.0, seed=3, target_k=4096),
}


def mixture_tau(n: int) -> float:
    """tau for about sqrt(n) clusters on a mixture graph of n nodes (each stage draws about
    gamma tau log2 n centers over roughly log2(n)/2 stages)."""
    import math
    L = max(1.0, math.log2(max(n, 2)))
    return max(0.05, math.sqrt(n) / (4 * math.log(2) * L * max(1.0, L / 2)))


MIX_SEED = 4
MIX_COUNT = 2000
MIX_DESCRIBE = ("2,000 graphs, seed 4: each an R-MAT (scale uniform 8..16, edge factor 8) or a mesh "
                "(side round(2^U), U uniform in [5,9)) with probability 1/2; w in [1,1000]; LCC; "
                "tau per graph for about sqrt(n) clusters")


def mixture(count: int = MIX_COUNT, seed: int = MIX_SEED, W: int = 1000):
    """Yield (g, EdgeList) for the many-graph workload."""
    from . import mix_graph
    for g in range(count):
        yield g, mix_graph(seed, g, W)
