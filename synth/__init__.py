"""Seeded synthetic graph generators shared by the tests, the benchmark and
the oracle.

This module produces inputs only: edge lists (src, dst, weight) in the
shapes of the paper's workloads.  It holds none of the method's arithmetic
(no Laplacian, no solve, no resistance, no farness).  The paper evaluates on
real networks (Sec. 6.3, App. A: complex networks and road networks); those
data sets are not available here, so these families stand in for them:

* ``grid2d``     -- 2-D 4-neighbour grid, high diameter (road-network proxy);
* ``barabasi_albert`` -- preferential attachment, skewed degrees
                    (complex-network proxy);
* ``rmat``       -- R-MAT / Kronecker graph with heavy hubs (complex-network
                    proxy, Graph500 parameters), reduced to its LCC as
                    Sec. 6.3 does for every instance.

All random draws use ``numpy.random.Generator(PCG64(seed))``.
"""
from .graphs import (
    grid2d,
    torus2d,
    random_regular,
    barabasi_albert,
    rmat,
    path_graph,
    cycle_graph,
    complete_graph,
    star_graph,
    random_tree,
    erdos_renyi_connected,
    largest_component,
    uniform_weights,
)

__all__ = [
    "grid2d",
    "torus2d",
    "random_regular",
    "barabasi_albert",
    "rmat",
    "path_graph",
    "cycle_graph",
    "complete_graph",
    "star_graph",
    "random_tree",
    "erdos_renyi_connected",
    "largest_component",
    "uniform_weights",
]
