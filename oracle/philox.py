"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), oracle copy (test infrastructure only).

Round function on counter (c0,c1,c2,c3) and key (k0,k1):
  (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (64-bit products)
  c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key <- key + (W0, W1)
with M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85; ten rounds, the key bumped
between rounds. Vectorised over numpy uint64 arrays holding 32-bit values.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    c = [np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3)]
    k = [np.asarray(x, dtype=np.uint64) & MASK for x in (k0, k1)]
    for r in range(10):
        if r > 0:
            k = [(k[0] + np.uint64(W0)) & MASK, (k[1] + np.uint64(W1)) & MASK]
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
    return [x.astype(np.uint32) for x in c]
