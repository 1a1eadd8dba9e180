"""The split of a node's slot blocks that the staged warp step computes with.

With the counter (t, node, replica, tag | b), the first three Philox rounds of a node's
blocks multiply words that are either the same for a whole launch or the same for all
of the node's blocks; the warp step computes the launch-wide part once per thread
(A, G and H_b, I_b, J_b) and per node only two wide products before round 4.  This
restates that split in plain integers and checks it against the oracle's full ten
rounds (itself pinned to cuRAND in test_oracle_philox.py) for random keys, steps,
replicas, nodes and all four block indices (D2Q9 uses four, D1Q3 and D2Q5 two).
"""
import numpy as np

import oracle as O

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF
TAG_STEP = 1 << 24


def round_keys(k0, k1):
    rk = []
    for r in range(10):
        rk += [(k0 + r * W0) & MASK, (k1 + r * W1) & MASK]
    return rk


def launch_part(t, replica, rk, nb):
    P, R = M0 * t, M1 * replica
    A = ((R >> 32) ^ rk[0]) & MASK
    G = ((P & MASK) ^ rk[3]) & MASK
    H, I, J = [], [], []
    for b in range(nb):
        C = ((P >> 32) ^ (TAG_STEP | b) ^ rk[1]) & MASK
        R1 = M1 * C
        E = ((R1 >> 32) ^ (R & MASK) ^ rk[2]) & MASK
        P2 = M0 * E
        H.append(((R1 & MASK) ^ rk[4]) & MASK)
        I.append(((P2 >> 32) ^ rk[5]) & MASK)
        J.append(P2 & MASK)
    return A, G, H, I, J


def node_blocks(part, rk, node, nb):
    A, G, H, I, J = part
    P1 = M0 * (node ^ A)
    R2 = M1 * (((P1 >> 32) ^ G) & MASK)
    out = []
    for b in range(nb):
        x0, x1, x2, x3 = ((R2 >> 32) ^ H[b]) & MASK, R2 & MASK, ((P1 & MASK) ^ I[b]) & MASK, J[b]
        for r in range(3, 10):
            p0, p1 = M0 * x0, M1 * x2
            x0, x1, x2, x3 = (((p1 >> 32) ^ x1 ^ rk[2 * r]) & MASK, p1 & MASK,
                              ((p0 >> 32) ^ x3 ^ rk[2 * r + 1]) & MASK, p0 & MASK)
        out.append([x0, x1, x2, x3])
    return out


def test_split_blocks_equal_the_full_rounds():
    rng = np.random.Generator(np.random.PCG64(17))
    for trial in range(300):
        k0, k1 = (int(v) for v in rng.integers(0, 2**32, size=2))
        t = int(rng.integers(0, 2**32)) if trial % 2 else int(rng.integers(0, 20000))
        replica = int(rng.integers(0, 2**32)) if trial % 3 == 0 else int(rng.integers(0, 64))
        rk = round_keys(k0, k1)
        part = launch_part(t, replica, rk, 4)
        for node in (0, 1, 2**31 + 5, int(rng.integers(0, 2**32)), int(rng.integers(0, 2**28))):
            got = node_blocks(part, rk, node, 4)
            for b in range(4):
                want = O.philox([t, node, replica, TAG_STEP | b], [k0, k1])
                assert got[b] == [int(w) for w in want], (trial, node, b)


def test_launch_part_is_node_independent():
    # the launch-wide words do not depend on the node; two nodes differ only after
    # round 1 (a planted node term in A or G would break the equality above)
    rk = round_keys(3, 0)
    p = launch_part(41, 7, rk, 2)
    assert launch_part(41, 7, rk, 2) == p
    assert node_blocks(p, rk, 5, 2) != node_blocks(p, rk, 6, 2)
