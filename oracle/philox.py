"""Philox4x32-10 counter-based generator, written from its published definition.

TEST INFRASTRUCTURE ONLY: nothing under ``oracle/`` is part of the product
path; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.

Source: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11, Section 3.3 (Philox).  A Philox4x32
round maps a 4-word counter (c0, c1, c2, c3) under a 2-word key (k0, k1) to

    hi0:lo0 = M0 * c0,   hi1:lo1 = M1 * c2          (32x32 -> 64-bit products)
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)

with M0 = 0xD2511F53 and M1 = 0xCD9E8D57; between rounds the key is bumped by
the Weyl constants (0x9E3779B9, 0xBB67AE85).  Philox4x32-10 applies 10 rounds.

The streaming-GCP sampler draws its random integers from this generator; the
way counters are laid out and how a 32-bit word becomes a bounded integer is
fixed in ``oracle/gcp.py`` (the paper leaves both unstated, Alg. 5 / Alg. 6).
Everything here is vectorised numpy in uint64 arithmetic; it is slow but exact.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
SH32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """Apply Philox4x32-10 to an array of counters.

    ctr: array-like of shape (n, 4) of uint32 counter words (c0, c1, c2, c3).
    key: pair (k0, k1) of uint32 key words.
    Returns an (n, 4) uint32 array of output words.
    """
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy())
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0            # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> SH32, p0 & MASK32
        hi1, lo1 = p1 >> SH32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def bounded(u, n):
    """Map uint32 words u to integers in [0, n) by multiply-shift: (u * n) >> 32.

    n may be a scalar or an array broadcastable against u; n <= 2^32.
    """
    u = np.asarray(u, dtype=np.uint64)
    n = np.asarray(n, dtype=np.uint64)
    return ((u * n) >> SH32).astype(np.int64)
