"""SplitMix64 counter-based values (oracle's own implementation; test infrastructure only).

SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15, then
z = (z ^ z>>30) * 0xBF58476D1CE4E5B9, z = (z ^ z>>27) * 0x94D049BB133111EB, z ^ z>>31.
Value i of stream s under seed k is output i of SplitMix64 seeded with key = output s of
SplitMix64 seeded with k.  Uniform [0,1) values use the top 24 bits.  Used to recompute
device-side initial tables independently, index by index.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def at(seed, i):
    """Output i (0-based; array allowed) of SplitMix64 seeded with `seed`."""
    i = np.asarray(i, np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed) + (i + np.uint64(1)) * GOLDEN)


def uniform_range(seed, stream, idx, lo, hi):
    """float32 value lo + (hi - lo) * U (computed in float64, rounded once) at indices idx."""
    key = at(seed, stream)
    u = (at(key, idx) >> np.uint64(40)).astype(np.float64) * (1.0 / 16777216.0)
    return (lo + (hi - lo) * u).astype(np.float32)


class InitTable:
    """Lazy view of the initial embedding table U(-r, r) (stream 200), rows -> [n][F] values."""

    def __init__(self, seed, F, r=1e-4):
        self.seed, self.F, self.r = seed, F, r

    def __getitem__(self, rows):
        rows = np.asarray(rows, np.int64)
        idx = (rows[..., None] * self.F + np.arange(self.F)).astype(np.uint64)
        return uniform_range(self.seed, 200, idx, -self.r, self.r)


def init_mlp(seed, dims):
    """Initial MLP parameters as the library draws them: layer k's W[out][in] from stream 300 + 2k and
    b[out] from stream 301 + 2k, U(-1/sqrt(fan_in), 1/sqrt(fan_in)); flat layer by layer."""
    parts = []
    for k in range(len(dims) - 1):
        fi, fo = dims[k], dims[k + 1]
        b = 1.0 / np.sqrt(fi)
        parts.append(uniform_range(seed, 300 + 2 * k, np.arange(fo * fi, dtype=np.uint64), -b, b))
        parts.append(uniform_range(seed, 301 + 2 * k, np.arange(fo, dtype=np.uint64), -b, b))
    return np.concatenate(parts)
