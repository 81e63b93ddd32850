"""Named synthetic workloads on the unit-cube hex mesh (shapes of coefficient-jump experiments)."""
import numpy as np

from . import fields
from .meshes import hex_problem

CONFIGS = {
    # 8^3 hexes, alpha = beta = 1, f ~ U(-1,1) seed 0 (1,176 DoFs)
    "hex8_unit": dict(n=8, alpha="one", beta=1.0, rhs_seed=0),
    # 64^3 hexes, alpha on an 8^3 checkerboard of blocks {1, 1e4}, beta = 1e-2, f seed 1 (762,048 DoFs)
    "hex64_checker": dict(n=64, alpha="checker", beta=1e-2, rhs_seed=1),
    # 32^3 version of the checkerboard workload (92,256 DoFs), for parity tests that span many tiles
    "hex32_checker": dict(n=32, alpha="checker", beta=1e-2, rhs_seed=1),
    # 16^3 version (10,800 DoFs)
    "hex16_checker": dict(n=16, alpha="checker", beta=1e-2, rhs_seed=1),
    # 24^3 version (38,088 DoFs): the bounded CPU sample of the family
    "hex24_checker": dict(n=24, alpha="checker", beta=1e-2, rhs_seed=1),
    # 128^3, log10 alpha ~ U(-3,3) per element with 64 inclusions alpha = 1e6, beta = 1 (6,193,536 DoFs)
    "hex128_spheres": dict(n=128, alpha="spheres", beta=1.0, rhs_seed=2),
    # 96^3 checkerboard (12^3-element blocks), for 64 right-hand sides with seeds 0..63
    "hex96_checker": dict(n=96, alpha="checker", beta=1e-2, rhs_seed=0),
    # 16^3 and 24^3 members of the inclusion family (bounded CPU samples)
    "hex16_spheres": dict(n=16, alpha="spheres", beta=1.0, rhs_seed=2),
    "hex24_spheres": dict(n=24, alpha="spheres", beta=1.0, rhs_seed=2),
}

# one-line descriptions and the 24^3 member of each family (bounded CPU samples)
DESCRIPTIONS = {
    "checker": ("alpha on an 8^3 checkerboard of blocks {1, 1e4}", "hex24_checker"),
    "spheres": ("log10 alpha ~ U(-3,3) per element with 64 spherical inclusions of alpha = 1e6", "hex24_spheres"),
    "one": ("alpha = 1", "hex8_unit"),
}


def describe(name):
    """(description, name of the family's bounded CPU sample) of a named workload."""
    c = CONFIGS[name]
    n = c["n"]
    what, sample = DESCRIPTIONS[c["alpha"]]
    ndof = 3 * n * (n - 1) ** 2
    return ("unit-cube %d^3 hex mesh, lowest-order Nedelec (%s edge DoFs), %s, beta = %g, f ~ U(-1,1) seed %d, "
            "x0 = 0, tol 1e-8" % (n, format(ndof, ","), what, c["beta"], c["rhs_seed"]), sample)


def make_alpha(n, kind, seed=None):
    if kind == "one":
        return np.ones(n ** 3)
    if kind == "checker":
        return fields.checkerboard(n, nb=8, hi=1e4, lo=1.0)
    if kind == "spheres":
        return fields.log_uniform_with_spheres(n)
    raise ValueError(kind)


def make_config(name, with_parts=False):
    """Return dict(A, G, f, n, ndof, ...) for a named workload (scipy CSR, float64)."""
    c = CONFIGS[name]
    n = c["n"]
    prob = hex_problem(n, make_alpha(n, c["alpha"]), c["beta"], with_parts=with_parts)
    prob["f"] = fields.rhs(prob["ndof"], c["rhs_seed"])
    prob["name"] = name
    return prob
