"""Pure-Python big-integer rendering of the page hash (test infrastructure only).

Written separately from ``crum_oracle.c`` so the two can be checked against
each other on tiny inputs: integers are unbounded here and every product is
reduced modulo 2**64 explicitly, and words are read with ``int.from_bytes``.

Hash (the dirty test that stands in for the write-fault tracking of
Algorithm 1 / Section 3.2): h = sum over the 8-byte little-endian words w_i
of a byte string of mix(w_i XOR (i * phi)), modulo 2**64, where mix is
splitmix64's output function (Steele, Lea, Flood, OOPSLA 2014) and phi is
the 64-bit golden-ratio constant.  A final partial word is zero-padded.
"""
from __future__ import annotations

M64 = (1 << 64) - 1
PHI = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9
C2 = 0x94D049BB133111EB


def mix(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * C1) & M64
    z = ((z ^ (z >> 27)) * C2) & M64
    return z ^ (z >> 31)


def words(buf: bytes) -> list[int]:
    pad = (-len(buf)) % 8
    b = bytes(buf) + b"\0" * pad
    return [int.from_bytes(b[k:k + 8], "little") for k in range(0, len(b), 8)]


def hash_bytes(buf: bytes, first_index: int = 0) -> int:
    total = 0
    for i, w in enumerate(words(buf)):
        total += mix(w ^ (((first_index + i) * PHI) & M64))
    return total & M64


def splitmix64(seed: int, count: int) -> list[int]:
    """The splitmix64 generator: state += phi, output mix(state)."""
    out, state = [], seed & M64
    for _ in range(count):
        state = (state + PHI) & M64
        out.append(mix(state))
    return out


def unmix(z: int) -> int:
    """Inverse of mix, from the algebra alone: undo each xorshift by
    repeated shifting and each odd multiply by its inverse modulo 2**64."""
    def unxorshift(y: int, s: int) -> int:
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x & M64

    z &= M64
    z = unxorshift(z, 31)
    z = (z * pow(C2, -1, 1 << 64)) & M64
    z = unxorshift(z, 27)
    z = (z * pow(C1, -1, 1 << 64)) & M64
    return unxorshift(z, 30)
