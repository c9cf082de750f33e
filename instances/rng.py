"""Counter-free seeded generator: SplitMix64 seeding a xoshiro256** stream.

Both are written from their published definitions (Steele/Lea/Flood 2014 for SplitMix64;
Blackman & Vigna 2018 for xoshiro256**). Integer draws are exact on every platform; normal
draws use Box-Muller through the platform libm, so they agree across machines to the last ulp
or so, which is far below every tolerance used with them.
"""
import math

_M64 = (1 << 64) - 1


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & _M64


class Xoshiro256ss:
    def __init__(self, seed: int):
        s = seed & _M64
        st = []
        for _ in range(4):
            s = (s + 0x9E3779B97F4A7C15) & _M64
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
            st.append(z ^ (z >> 31))
        self.s = st
        self._spare = None

    def next_u64(self) -> int:
        s0, s1, s2, s3 = self.s
        result = (_rotl((s1 * 5) & _M64, 7) * 9) & _M64
        t = (s1 << 17) & _M64
        s2 ^= s0
        s3 ^= s1
        s1 ^= s2
        s0 ^= s3
        s2 ^= t
        s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return result

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, k: int) -> int:
        """Integer in [0, k) by multiply-shift of 53 random bits (exact integer arithmetic)."""
        return ((self.next_u64() >> 11) * k) >> 53

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def normal(self) -> float:
        if self._spare is not None:
            v, self._spare = self._spare, None
            return v
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        self._spare = r * math.sin(2.0 * math.pi * u2)
        return r * math.cos(2.0 * math.pi * u2)

    def permutation(self, n: int):
        p = list(range(n))
        for i in range(n - 1, 0, -1):
            j = self.below(i + 1)
            p[i], p[j] = p[j], p[i]
        return p
