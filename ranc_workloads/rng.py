"""Counter-based SplitMix64 draws for the seeded synthetic workloads.

This module holds no RANC arithmetic: it only turns (seed, stream, index)
triples into 64-bit pseudo-random words and maps them to Bernoulli and
uniform-integer draws.  Both the CUDA path and the CPU oracle consume the
arrays built from these draws; neither calls this module while simulating.

Definition (SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014):

    splitmix64(x) = mix(x + 0x9E3779B97F4A7C15)
    mix(z)        = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                    z ^= z >> 27; z *= 0x94D049BB133111EB;
                    z ^ (z >> 31)                   (all mod 2**64)

A draw is ``u = splitmix64(seed ^ (stream << 40) ^ index)``; the stream id
separates the fields of one workload, the index is the flat element index.
"""

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """First SplitMix64 output for state ``x`` (uint64 array or scalar)."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def draws(seed, stream, n, offset=0):
    """``n`` consecutive 64-bit draws of ``stream`` starting at ``offset``."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    key = np.uint64(seed) ^ (np.uint64(stream) << np.uint64(40))
    return splitmix64(key ^ idx)


def bernoulli(seed, stream, shape, p, offset=0):
    """0/1 uint8 array: ``(u >> 32) < floor(p * 2**32)``."""
    n = int(np.prod(shape)) if len(shape) else 1
    u = draws(seed, stream, n, offset)
    thr = np.uint64(int(np.floor(p * 2.0**32)))
    return ((u >> np.uint64(32)) < thr).astype(np.uint8).reshape(shape)


def uniform_int(seed, stream, shape, lo, hi, offset=0):
    """int64 array with ``lo + (u mod (hi - lo + 1))`` (inclusive bounds)."""
    n = int(np.prod(shape)) if len(shape) else 1
    u = draws(seed, stream, n, offset)
    span = np.uint64(hi - lo + 1)
    return (u % span).astype(np.int64).reshape(shape) + np.int64(lo)
