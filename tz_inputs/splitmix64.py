"""SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): a 64-bit Weyl sequence with increment
0x9E3779B97F4A7C15 passed through the published two-multiply finaliser.
Written out here from that definition so the same stream can be produced by
the C++ circuit generator."""

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def next_bit(self) -> int:
        """One fair bit: the top bit of the next draw."""
        return self.next_u64() >> 63
