"""Philox4x32-10, written from its published definition.

Test infrastructure only (see the package header).

Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
a 4x32-bit counter and a 2x32-bit key; each of the ten rounds multiplies counter
words 0 and 2 by two fixed odd constants, splits the 64-bit products into high and
low halves, XORs the high halves with the other counter words and the key, permutes
the words, and then bumps the key by two Weyl constants.

The method draws two kinds of uniforms from it (both sides use the same counters):

* Metropolis test of the sequential sweep (Sec. II A, Eq. (9)):
  counter = (chain, sweep, bond, TAG_METROPOLIS).
* Sign-SGD step (Sec. II B, Eq. (10)): counter = (element & 0xffffffff,
  element >> 32, step, TAG_UPDATE).
* Random-NNASP attempt (Sec. II A, Eq. (prob_r)): counter = (chain, sweep, attempt,
  TAG_RANDOM); word 0 picks the pair, word 1 is the acceptance uniform.

The uniform is r = (word0 >> 8) * 2**-24, exactly representable in float32.
"""
from __future__ import annotations

import numpy as np

MUL0 = 0xD2511F53
MUL1 = 0xCD9E8D57
WEYL0 = 0x9E3779B9
WEYL1 = 0xBB67AE85
MASK = 0xFFFFFFFF

TAG_METROPOLIS = 0x4D455452  # "METR"
TAG_UPDATE = 0x55504454      # "UPDT"
TAG_RANDOM = 0x52414E44      # "RAND"


def philox4x32_10(ctr, key):
    """One block for python-int counter (4 words) and key (2 words)."""
    c0, c1, c2, c3 = (int(x) & MASK for x in ctr)
    k0, k1 = (int(x) & MASK for x in key)
    for _ in range(10):
        p0 = MUL0 * c0
        p1 = MUL1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & MASK, (p0 >> 32) ^ c3 ^ k1, p0 & MASK)
        k0 = (k0 + WEYL0) & MASK
        k1 = (k1 + WEYL1) & MASK
    return c0, c1, c2, c3


def philox4x32_10_np(c0, c1, c2, c3, k0, k1):
    """Vectorised over uint32 arrays (broadcast); returns four uint32 arrays."""
    u64 = np.uint64
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & u64(MASK) for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & u64(MASK)
    k1 = np.asarray(k1, dtype=np.uint64) & u64(MASK)
    for _ in range(10):
        p0 = u64(MUL0) * c0
        p1 = u64(MUL1) * c2
        c0, c1, c2, c3 = ((p1 >> u64(32)) ^ c1 ^ k0, p1 & u64(MASK),
                          (p0 >> u64(32)) ^ c3 ^ k1, p0 & u64(MASK))
        k0 = (k0 + u64(WEYL0)) & u64(MASK)
        k1 = (k1 + u64(WEYL1)) & u64(MASK)
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def uniform24(word0) -> np.ndarray:
    """r in [0, 1) from the top 24 bits of a 32-bit word (float64 holding a float32 value)."""
    return (np.asarray(word0, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def key_of(seed: int):
    return seed & MASK, (seed >> 32) & MASK


def metropolis_uniform(seed: int, chain: int, sweep: int, bond: int) -> float:
    k0, k1 = key_of(seed)
    w = philox4x32_10((chain, sweep, bond, TAG_METROPOLIS), (k0, k1))
    return float(uniform24(w[0]))


def update_uniforms(seed: int, step: int, n: int) -> np.ndarray:
    k0, k1 = key_of(seed)
    e = np.arange(n, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10_np(e & np.uint64(MASK), e >> np.uint64(32), step, TAG_UPDATE, k0, k1)
    return uniform24(w0)


def random_attempt_words(seed: int, chain: int, sweep: int, attempt: int):
    """(pick word, acceptance uniform) of one random-NNASP attempt."""
    k0, k1 = key_of(seed)
    w = philox4x32_10((chain, sweep, attempt, TAG_RANDOM), (k0, k1))
    return int(w[0]), float(uniform24(w[1]))


def pick(word: int, n: int) -> int:
    """Index in [0, n) from the top 24 bits of a word: floor(r n) with r = (word >> 8) 2^-24,
    in integer arithmetic so that both sides agree exactly."""
    return ((word >> 8) * n) >> 24
