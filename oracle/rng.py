"""splitmix64 in counter mode, for the random vectors the Lanczos method draws.

Oracle -- test infrastructure only.  Algorithm 1 (section 3.1) starts from a
vector p_0 the paper leaves unspecified; the oracle draws it, and every
breakdown replacement vector, from splitmix64 (Steele, Lea, Flood 2014):
  mix(z):  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
           z *= 0x94D049BB133111EB; z ^= z >> 31
Counter mode: key_s = mix(seed + (s+1)*GAMMA); value_i = mix(key_s + (i+1)*GAMMA);
uniform in [-1, 1) as 2*(value >> 11)*2^-53 - 1.  Stream 0 is p_0, stream
b+1 the b-th breakdown vector.
"""
MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def uniform_pm1(seed: int, stream: int, n: int):
    """List of n doubles in [-1, 1) (pure Python: counter-mode splitmix64)."""
    key = mix((seed + (stream + 1) * GAMMA) & MASK)
    out = []
    for i in range(n):
        z = mix((key + (i + 1) * GAMMA) & MASK)
        out.append(2.0 * ((z >> 11) * 2.0 ** -53) - 1.0)
    return out
