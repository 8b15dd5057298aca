"""Counter-based SplitMix64 generator for ACI's random initial guess (oracle side).

Test infrastructure (see the package header). The random initial guess Y^init of
Algorithm 1 ("if nothing is known, initialise randomly", Sec. 2.6) is drawn from
SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output c (0-based) of the stream with seed s is
mix(s + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64) with the finaliser
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
A uniform value in [-1, 1) is (out >> 11) * 2^-52 - 1, exact in binary64.
The CUDA library implements the same definition independently.

Pinned by: the published SplitMix64 reference outputs for seed 1234567 (first five
values, from the authors' reference code as reproduced in many test suites) in
tests/golden/splitmix64.json, and by agreement with a sequential stream.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Raw 64-bit outputs number ``counters`` (0-based) of the stream seeded with ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_uniform(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [-1, 1) from outputs ``counters``."""
    z = splitmix64(seed, counters)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0


def random_tt_counter(seed: int, ranks, dims, complex_values: bool):
    """Random TT whose entries are consecutive counter values, cores in site order, row-major.

    Real entry e of the concatenated cores uses counter e; a complex entry uses 2e (real
    part) and 2e + 1 (imaginary part).
    """
    cores = []
    off = 0
    for s, d in enumerate(dims):
        shape = (ranks[s], d, ranks[s + 1])
        cnt = int(np.prod(shape))
        if complex_values:
            idx = np.arange(2 * off, 2 * (off + cnt), dtype=np.uint64)
            u = splitmix64_uniform(seed, idx)
            core = (u[0::2] + 1j * u[1::2]).reshape(shape)
        else:
            idx = np.arange(off, off + cnt, dtype=np.uint64)
            core = splitmix64_uniform(seed, idx).reshape(shape)
        cores.append(core)
        off += cnt
    return cores
