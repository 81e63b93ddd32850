"""Counter-based SplitMix64 streams for every seeded quantity of the synthetic workloads.

A draw is the first output of a SplitMix64 generator (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) whose state is the 64-bit key

    key(stream, seed, i) = stream << 60 | seed << 40 | i      (stream < 16, seed < 2**20, i < 2**40)

so that each named quantity (right-hand side, coefficient field, sphere, ...) draws from its own
stream and any element can be regenerated independently of the others. A uniform double on [0, 1)
takes the top 53 bits of the draw.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)

# one stream per seeded quantity
STREAMS = {
    "rhs": 0,       # right-hand sides f, i.i.d. U(-1, 1) per DoF
    "alpha": 1,     # per-element or per-block coefficient draws
    "sphere": 2,    # inclusion centres and radii
    "sys_n": 3,     # mesh size of each independent system
    "sys_k": 4,     # jump exponent of each independent system
    "jump": 5,      # per-block coin flips of a jump field
    "x0": 6,        # initial guesses
    "mlp": 7,       # network initialisation
    "probe": 8,     # random test vectors (convergence-factor probes)
}


def splitmix64(x):
    """First SplitMix64 output for state ``x`` (uint64 array), with wrap-around arithmetic."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
    return z ^ (z >> np.uint64(31))


def stream_key(stream, seed):
    if isinstance(stream, str):
        stream = STREAMS[stream]
    if not (0 <= stream < 16 and 0 <= seed < 2**20):
        raise ValueError("stream must be < 16 and seed < 2**20")
    return (np.uint64(stream) << np.uint64(60)) | (np.uint64(seed) << np.uint64(40))


def uniform01(stream, seed, count, offset=0):
    """``count`` doubles in [0, 1): element i is draw ``offset + i`` of (stream, seed)."""
    i = np.arange(offset, offset + count, dtype=np.uint64)
    z = splitmix64(stream_key(stream, seed) + i)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(stream, seed, count, lo=-1.0, hi=1.0, offset=0):
    """``count`` doubles, i.i.d. U(lo, hi) from (stream, seed)."""
    return lo + (hi - lo) * uniform01(stream, seed, count, offset)
