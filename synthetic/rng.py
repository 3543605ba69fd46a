"""SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the public 64-bit finaliser
variant).  Pure-integer, so the draws are identical on x86_64 and aarch64."""

_MASK = (1 << 64) - 1


class SplitMix64:
    """Counter-based 64-bit generator: state += golden gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform_int(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive); modulo reduction, deterministic."""
        if hi < lo:
            raise ValueError("empty range")
        return lo + self.next_u64() % (hi - lo + 1)

    def uniform01(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def bernoulli(self, p: float) -> bool:
        return self.uniform01() < p

    @staticmethod
    def derive(seed: int, stream: int) -> "SplitMix64":
        """Independent stream for (seed, stream): seeds a fresh generator
        with one mixed draw so nearby seeds do not share prefixes."""
        g = SplitMix64(seed * 0x100000001B3 + stream)
        return SplitMix64(g.next_u64())
