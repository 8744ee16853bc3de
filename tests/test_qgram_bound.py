"""The 3-gram count bound the string verification uses to skip pairs
(Ukkonen 1992): L1 distance between the two strings' hashed, capped 3-gram
bucket counts <= 6 x edit distance.  Checked against the oracle's exact
edit distance on random and mutated strings, including short strings, long
runs of one letter (capped counts) and the DNA alphabet."""
import numpy as np

import oracle
from synth import mutate, random_strings

MASK32 = 0xFFFFFFFF


def buckets(s: bytes) -> np.ndarray:
    h = np.zeros(64, np.int64)
    for j in range(len(s) - 2):
        x = ((s[j] << 16) | (s[j + 1] << 8) | s[j + 2]) * 0x9E3779B1 & MASK32
        b = (x >> 26) & 63
        h[b] = min(255, h[b] + 1)
    return h


def check(pairs):
    for a, b in pairs:
        d = oracle.edit_full(a, b)
        l1 = int(np.abs(buckets(a) - buckets(b)).sum())
        assert l1 <= 6 * d, (a, b, l1, d)


def test_qgram_bound_random_and_mutated():
    oracle.build()
    rng = np.random.default_rng(7)
    for alphabet, lmax in ((b"ACGT", 120), (b"abcdefghijklmnopqrstuvwxyz", 20), (b"ab", 30)):
        alpha = np.frombuffer(alphabet, np.uint8)
        S = random_strings(300, 0, lmax, alpha, rng)
        pairs = [(S.get(i), S.get((i * 7 + 1) % S.n)) for i in range(S.n)]
        pairs += [(S.get(i), mutate(S.get(i), int(rng.integers(0, 9)), alpha, rng)) for i in range(S.n)]
        check(pairs)


def test_qgram_bound_capped_counts():
    oracle.build()
    check([(b"A" * 400, b"A" * 380 + b"C" * 3), (b"A" * 300, b"AC" * 150), (b"", b"ACG"), (b"AC", b"ACGTA")])
