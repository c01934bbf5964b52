"""Seeded synthetic inputs for tree field integration.

This package only *generates* inputs: tree topologies, edge weights, fields and
kernel specifications (a kind name plus parameters). It contains none of the
integration arithmetic, so both the CUDA path and the CPU oracle can use it
without sharing any computation.
"""
from .trees import (  # noqa: F401
    Tree,
    path,
    star,
    spider,
    caterpillar_leaves,
    caterpillar_hanging_paths,
    toothed_spine,
    comb,
    broom,
    double_broom,
    complete_kary,
    complete_binary_n,
    random_recursive,
    caterpillar_rrt,
    random_mst_topology,
    preferential_attachment,
    torus_knn_mst,
    grid_spanning_tree,
    forest,
    prufer_trees,
)
from .fields import normal_field, dirichlet_pairs  # noqa: F401
from .kernels import KernelSpec  # noqa: F401
from . import configs  # noqa: F401
