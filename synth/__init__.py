"""Seeded synthetic inputs for GFD validation: graphs and GFDs.

This package only draws random inputs (graph structure, labels, attributes,
patterns and literals). It contains no matching, no literal evaluation and no
counting: both the CPU oracle and the CUDA path consume what it produces, and
neither depends on the other.
"""
from .graphs import Graph, chung_lu_edges, graph_from_edges, random_small_graph
from .gfds import GFD, Literal, random_pattern_gfd
from . import configs

__all__ = [
    "Graph", "chung_lu_edges", "graph_from_edges", "random_small_graph",
    "GFD", "Literal", "random_pattern_gfd", "configs",
]
