"""Counter-based SplitMix64 random numbers (Steele, Lea, Flood 2014).

value(seed, stream, i) = mix(key(seed, stream) + (i + 1) * GAMMA), where mix is
the SplitMix64 output function and key mixes the seed with a stream id.  The
i-th value of a stream does not depend on how many values were drawn before,
so C, numpy and any other implementation produce the same bits.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFF) * STREAM_MUL)
        return _mix(np.array([s], dtype=np.uint64))[0]


def splitmix64(seed, stream, count, start=0):
    """count raw 64-bit values of the given (seed, stream), from index start."""
    k = _key(seed, stream)
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(k + i * GAMMA)


def uniform(seed, stream, count, lo=0.0, hi=1.0, start=0):
    """count doubles uniform in [lo, hi): the top 53 bits of each value."""
    u = (splitmix64(seed, stream, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return lo + (hi - lo) * u


def normal(seed, stream, count, start=0):
    """count standard normal doubles by Box-Muller on consecutive value pairs."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m, start=2 * start)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]
