"""Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11): ten rounds of two 64x64->128-bit multiplies with the
published multipliers and Weyl key increments.

The method draws one uniform number per noise site (Alg. 1, "sample a
trajectory").  Counter layout used by both the oracle and the GPU library:
ctr = (trajectory id, global gate index, slot, 0), key = (seed, DOMAIN).
Slot 0 / 1 are the two gated qubits (q, q+1), slot 2 is the per-gate coin of a
noise channel that acts with probability < 1.  The uniform is the top 53 bits
of the first output word times 2^-53, so u lies in [0, 1).
"""
MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
DOMAIN_TRAJECTORY = 0x4C454D5053545241  # "LEMPSTRA"


def philox4x64_10(ctr, key):
    """Return the four 64-bit output words for a 4x64 counter and 2x64 key."""
    c0, c1, c2, c3 = (int(x) & MASK64 for x in ctr)
    k0, k1 = (int(x) & MASK64 for x in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64,
                          (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)
    return c0, c1, c2, c3


def uniform(seed, traj, gate, slot):
    """u in [0, 1) for one noise-site draw."""
    w = philox4x64_10((traj, gate, slot, 0), (seed, DOMAIN_TRAJECTORY))[0]
    return (w >> 11) * (1.0 / 9007199254740992.0)
