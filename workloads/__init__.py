"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

Holds the model problem (Nedelec discretisations of the shifted curl-curl equation), coefficient
fields and SplitMix64 streams; none of the multigrid method's arithmetic lives here.
"""
from .rng import uniform, uniform01, splitmix64, STREAMS
from .meshes import hex_problem, quad_problem, tri_problem, hex_element_matrices
from . import fields
from .configs import CONFIGS, make_config, describe

__all__ = ["uniform", "uniform01", "splitmix64", "STREAMS", "hex_problem", "quad_problem",
           "tri_problem", "hex_element_matrices", "fields", "CONFIGS", "make_config", "describe"]
