"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), written from its published definition.

Oracle (test infrastructure only).  Used for the random candidate draws of the low-rank
SI (Sec. 3.2): each angle j gets the 32-bit key  philox((j, k, n, TAG), (seed_lo, seed_hi))[0]
at inner iteration k of outer iteration n; a uniformly random q-subset of the unsampled
angles is the q unsampled angles with the smallest (key, j).
"""
MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
SAMPLE_TAG = 0x52544531


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = (p0 >> 32) & MASK32, p0 & MASK32
        hi1, lo1 = (p1 >> 32) & MASK32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0, c1, c2, c3)


def angle_key(seed, n, k, j):
    return philox4x32_10((j, k, n, SAMPLE_TAG), (seed & MASK32, (seed >> 32) & MASK32))[0]


def draw_without_replacement(seed, n, k, candidates, count):
    """The `count` angles of `candidates` with the smallest (key, index)."""
    keyed = sorted((angle_key(seed, n, k, j), j) for j in candidates)
    return [j for _, j in keyed[:count]]
