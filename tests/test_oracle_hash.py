"""Pins for the values of the oracle's 64-bit prefix keys (Section 4 and the
duplicate-detection appendix ask only for "a random hash function"; the keys
used here are a Karp-Rabin polynomial over P = 2^61 - 1 in 32-bit limbs of
big-endian 8-character words, zero past the tested length, finished by the
SplitMix64 output function of (h XOR L_eff * gamma)).

None of these checks recomputes the key the way the oracle does:

* The finisher is a bijection of 64-bit words.  Its inverse, built here from
  the inverses of its xor-shifts and of its odd multipliers modulo 2^64, turns
  every key back into the polynomial value h.  A recovered h must lie below P
  (a wrong finisher, multiplier or length term gives a value below P with
  probability 1/8 per key).
* h must equal the polynomial written as a sum of limb_j * B^(2m-1-j) mod P with
  Python's pow() (not a Horner fold), limbs taken from the characters directly.
  A swapped limb order, a little-endian word, padding on the wrong side or a
  dropped limb changes that sum.
* Closed forms: a 1..4-character prefix is one nonzero high limb and a zero low
  limb, so h = hi * B mod P; the empty prefix gives h = 0.
* Linearity: two strings that differ in one limb have h values that differ by
  (limb difference) * B^e mod P.
* The doubling identity the GPU uses: h(2L) = h(L) * B^(L/4) + h(words L/8 ..
  2L/8 - 1) mod P for L >= 8.
"""
import random

import pytest

import datagen
import oracle

P61 = (1 << 61) - 1
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9  # SplitMix64 output multipliers (Steele, Lea, Flood 2014)
C2 = 0x94D049BB133111EB


def _unxorshift(y, s):
    # inverse of x -> x ^ (x >> s) on 64-bit words
    x = y
    for _ in range(64 // s + 1):
        x = y ^ (x >> s)
    return x & M64


def unsmix(z):
    """Inverse of the SplitMix64 output function."""
    z = _unxorshift(z, 31)
    z = (z * pow(C2, -1, 1 << 64)) & M64
    z = _unxorshift(z, 27)
    z = (z * pow(C1, -1, 1 << 64)) & M64
    return _unxorshift(z, 30)


def recovered_h(ss, i, l, seed):
    key = oracle.prefix_key(ss, i, l, seed)
    return unsmix(key) ^ ((l * GAMMA) & M64)


def limbs(s: bytes, l: int):
    padded = s[:l] + b"\x00" * ((-l) % 8)
    out = []
    for j in range(0, len(padded), 8):
        w = int.from_bytes(padded[j:j + 8], "big")
        out += [w >> 32, w & 0xFFFFFFFF]
    return out


def poly_sum(lm, B):
    m = len(lm)
    return sum(x * pow(B, m - 1 - j, P61) for j, x in enumerate(lm)) % P61


def test_unsmix_inverts_published_outputs():
    # the first published SplitMix64 output from state 0 is smix(gamma)
    assert unsmix(0xE220A8397B1DCDAF) == GAMMA


def _cases():
    rnd = random.Random(17)
    strs = [b"A", b"Z", b"AB", b"ABC", b"ABCD", b"ABCDE", b"ABCDEFG", b"ABCDEFGH", b"ABCDEFGHI",
            b"ACGTACGTACGTACGT", b"ACGTACGTACGTACGTA"]
    strs += [bytes(rnd.choice(b"ABCDEFGHIJKLMNOPQRSTUVWXYZ") for _ in range(rnd.randint(1, 70))) for _ in range(12)]
    cases = []
    for i, s in enumerate(strs):
        for l in sorted({0, 1, min(3, len(s)), min(7, len(s)), min(8, len(s)), min(9, len(s)), len(s) // 2, len(s)}):
            cases.append((i, l))
    return strs, cases


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_key_is_the_karp_rabin_polynomial(seed):
    strs, cases = _cases()
    ss = datagen.from_strings(strs)
    B = oracle.hash_base(seed)
    for i, l in cases:
        h = recovered_h(ss, i, l, seed)
        assert h < P61, (strs[i], l)
        assert h == poly_sum(limbs(strs[i], l), B), (strs[i], l)


def test_short_prefix_closed_forms():
    strs = [b"A", b"AB", b"ABC", b"ABCD", b"QRSTUVW"]
    ss = datagen.from_strings(strs)
    B = oracle.hash_base(4)
    assert recovered_h(ss, 0, 0, 4) == 0
    for i, s in enumerate(strs):
        for l in range(1, min(4, len(s)) + 1):
            hi = int.from_bytes(s[:l] + b"\x00" * (4 - l), "big")
            assert recovered_h(ss, i, l, 4) == hi * B % P61


def test_one_limb_difference_is_linear():
    rnd = random.Random(2)
    B = oracle.hash_base(9)
    for _ in range(40):
        n = rnd.randint(8, 48)
        a = bytearray(rnd.choice(b"ACGT") for _ in range(n))
        b = bytearray(a)
        j = rnd.randrange(n)
        b[j] = ord("T") if a[j] != ord("T") else ord("A")
        ss = datagen.from_strings([bytes(a), bytes(b)])
        la, lb = limbs(bytes(a), n), limbs(bytes(b), n)
        e = len(la) - 1 - (j // 4)
        diff = (recovered_h(ss, 0, n, 9) - recovered_h(ss, 1, n, 9)) % P61
        assert diff == (la[j // 4] - lb[j // 4]) * pow(B, e, P61) % P61


def test_doubling_identity():
    rnd = random.Random(8)
    B = oracle.hash_base(21)
    for L in (8, 16, 32, 64):
        s = bytes(rnd.choice(b"ACGTN") for _ in range(2 * L))
        ss = datagen.from_strings([s, s[L:]])
        h_l = recovered_h(ss, 0, L, 21)
        h_2l = recovered_h(ss, 0, 2 * L, 21)
        h_tail = recovered_h(ss, 1, L, 21)  # the words L/8 .. 2L/8-1 hashed on their own
        assert h_2l == (h_l * pow(B, L // 4, P61) + h_tail) % P61
