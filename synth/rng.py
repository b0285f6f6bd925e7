"""splitmix64 (Steele, Lea & Flood, 2014) as a plain Python/numpy stream.

state <- state + 0x9E3779B97F4A7C15;  z <- mix(state), with the published
xor-shift-multiply finaliser.  Uniform doubles use the top 53 bits.
"""
import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _mix(z):
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


class SplitMix64:
    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        return _mix(self.state)

    def u64_array(self, n: int) -> np.ndarray:
        """n consecutive outputs, vectorised (same values as n next_u64 calls)."""
        n = int(n)
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            s = np.uint64(self.state) + k * np.uint64(_GAMMA)
            z = s
            z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * _GAMMA) & _MASK
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64_array(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def integers(self, n: int, hi: int) -> np.ndarray:
        """n integers uniform in [0, hi) (multiply-shift on 53-bit uniforms)."""
        return np.minimum((self.uniform(n) * hi).astype(np.int64), hi - 1)

    def permutation(self, n: int) -> np.ndarray:
        """Seeded permutation of range(n) (argsort of uniform keys)."""
        return np.argsort(self.uniform(n), kind="stable")
