"""Independent pure-Python splitmix64 (Vigna, public domain), used by tests to
compute the tie-break hash h(seed, a, b) = mix64(seed ^ mix64(a << 32 | b))
without calling the oracle.  Pinned to the published output sequence."""
M64 = (1 << 64) - 1


def mix64(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix64_sequence(seed: int, count: int):
    s = seed & M64
    out = []
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & M64
        out.append(mix64(s))
    return out


def h(seed: int, a: int, b: int) -> int:
    return mix64((seed & M64) ^ mix64(((a & 0xFFFFFFFF) << 32) | (b & 0xFFFFFFFF)))
