"""Seeded coefficient fields and right-hand sides for the synthetic hex workloads.

Element (i, j, k) of an n^3 mesh has id i + n (j + n k) and centre ((i+.5)/n, (j+.5)/n, (k+.5)/n).
"""
import numpy as np

from .rng import uniform, uniform01


def element_centres(n):
    e = np.arange(n ** 3)
    return np.stack([(e % n + 0.5) / n, ((e // n) % n + 0.5) / n, (e // (n * n) + 0.5) / n], axis=1)


def block_ids(n, nb):
    """Block index of each element when the cube is cut into nb^3 equal blocks (n % nb == 0)."""
    if n % nb:
        raise ValueError("n must be a multiple of the block count")
    s = n // nb
    e = np.arange(n ** 3)
    bx, by, bz = (e % n) // s, ((e // n) % n) // s, (e // (n * n)) // s
    return bx, by, bz


def checkerboard(n, nb=8, hi=1e4, lo=1.0):
    """alpha = hi on blocks with odd bx+by+bz, lo on the others."""
    bx, by, bz = block_ids(n, nb)
    return np.where((bx + by + bz) % 2 == 1, hi, lo)


def log_uniform_with_spheres(n, seed_alpha=3, seed_spheres=4, lo=-3.0, hi=3.0,
                             nspheres=64, rmin=0.02, rmax=0.08, inclusion=1e6):
    """log10 alpha ~ U(lo, hi) per element; elements whose centre lies inside one of ``nspheres``
    balls (centres U(0,1)^3, radii U(rmin, rmax)) get alpha = inclusion."""
    alpha = 10.0 ** uniform("alpha", seed_alpha, n ** 3, lo, hi)
    u = uniform01("sphere", seed_spheres, 4 * nspheres).reshape(nspheres, 4)
    c = element_centres(n)
    inside = np.zeros(n ** 3, dtype=bool)
    for s in range(nspheres):
        r = rmin + (rmax - rmin) * u[s, 3]
        inside |= ((c - u[s, :3]) ** 2).sum(axis=1) <= r * r
    alpha[inside] = inclusion
    return alpha


def log_uniform(n, seed, lo=-4.0, hi=4.0):
    """alpha = 10^U(lo, hi), independently per element."""
    return 10.0 ** uniform("alpha", seed, n ** 3, lo, hi)


def block_log_uniform(n, seed, nb=8, lo=-4.0, hi=4.0):
    """alpha = 10^U(lo, hi), independently per block of an nb^3 partition (n % nb == 0)."""
    bx, by, bz = block_ids(n, nb)
    vals = 10.0 ** uniform("alpha", seed, nb ** 3, lo, hi)
    return vals[bx + nb * (by + nb * bz)]


def random_jump(n, k, seed, nb=8):
    """Each block of an nb^3 partition is 1 or 10^k with probability 1/2 (coin from 'jump')."""
    if n % nb:
        # uneven meshes: block of element = floor(coordinate * nb)
        e = np.arange(n ** 3)
        bx = ((e % n) * nb) // n
        by = (((e // n) % n) * nb) // n
        bz = ((e // (n * n)) * nb) // n
    else:
        bx, by, bz = block_ids(n, nb)
    coin = uniform01("jump", seed, nb ** 3) < 0.5
    return np.where(coin[bx + nb * (by + nb * bz)], 10.0 ** k, 1.0)


def rhs(ndof, seed):
    """f i.i.d. U(-1, 1)."""
    return uniform("rhs", seed, ndof)
