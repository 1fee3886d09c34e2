"""Philox4x32-10 counter-based generator, written from its published definition.

Reference: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11, Section 4 (the Philox S-box family).

Definition used here (N = 4 words of 32 bits, R = 10 rounds):
  * a round maps the counter (x0, x1, x2, x3) under round key (k0, k1) to
    (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0));
  * the key is bumped by the Weyl constants (W0, W1) between rounds;
  * M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85.

Test infrastructure only (part of the oracle): nothing in the product imports it.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Apply the 10-round bijection to counters ``ctr`` (..., 4) under keys ``key`` (..., 2).

    Inputs are any integer arrays holding 32-bit values; the result is a uint32
    array of shape (..., 4).  Broadcasting between ``ctr`` and ``key`` is allowed.
    """
    c = np.asarray(ctr, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    x0, x1, x2, x3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * x0  # exact: both factors < 2^32, product < 2^64
        p1 = M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def trial_words(seed: int, problem_id: int, trials, nwords: int):
    """The first ``nwords`` 32-bit words of the stream of each trial in ``trials``.

    Layout (shared convention of the column sampler): word w of trial t is lane
    (w mod 4) of Philox4x32-10 with key (seed mod 2^32, seed >> 32) and counter
    (t mod 2^32, problem_id, w div 4, t >> 32).  Returns a uint32 array
    (len(trials), nwords).
    """
    t = np.asarray(trials, dtype=np.uint64).reshape(-1)
    nblk = (nwords + 3) // 4
    ctr = np.zeros((t.size, nblk, 4), dtype=np.uint64)
    ctr[:, :, 0] = (t & MASK32)[:, None]
    ctr[:, :, 1] = np.uint64(problem_id) & MASK32
    ctr[:, :, 2] = np.arange(nblk, dtype=np.uint64)[None, :]
    ctr[:, :, 3] = (t >> np.uint64(32))[:, None]
    s = np.uint64(seed)
    key = np.array([s & MASK32, s >> np.uint64(32)], dtype=np.uint64)
    out = philox4x32_10(ctr, key)  # (T, nblk, 4)
    return out.reshape(t.size, nblk * 4)[:, :nwords]


def bounded(word, rng: int) -> int:
    """Map a 32-bit word to [0, rng) by multiply-shift: floor(word * rng / 2^32).

    No rejection step, so the number of words a draw consumes is fixed; the bias
    is at most rng / 2^32 per value.
    """
    return int((int(word) * int(rng)) >> 32)
