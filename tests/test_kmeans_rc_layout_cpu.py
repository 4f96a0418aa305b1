"""The rotated-copies K-means pass (kmeans_rc_kernel in
paper_1511_00152_gb300/csrc/kmeans.cu), its shared-memory layout checked on
the host with the kernel's index expressions.

A half-warp holds NP = ceil(K / 2) rows and C = 16 // NP lanes per row; lane
sl < C NP is (c, ph) = (sl // NP, sl % NP).  Coordinate j owns a 32-word
line; word w of it holds, for b = w // 2 < C NP, centre 2 (b % NP) + (w & 1)
of copy b // NP.  At unrolled step q lane (c, ph) reads the pair
(q + ph) mod NP of copy c, words 2 (c NP + (q + ph) mod NP) and the next.
The rows are staged as (idx, val) pairs at a row stride S >= m, the smallest
with (ph S + c) mod 16 distinct over a half-warp's lanes, and an entry's row
within the group is e / m = umulhi(e, floor(2^32 / m) + 1)."""
import numpy as np
import pytest


def rc_layout(K):
    NP = (K + 1) // 2
    C = 16 // NP
    return NP, C


def lanes(NP, C):
    return [(sl // NP, sl % NP) for sl in range(16) if sl < C * NP]


def stage_stride(m, NP, C):
    S = m
    while True:
        pairs = [(ph * S + c) % 16 for ph in range(NP) for c in range(C)]
        if len(set(pairs)) == len(pairs):
            return S
        S += 1


@pytest.mark.parametrize("K", range(1, 33))
def test_centre_loads_hit_distinct_bank_pairs(K):
    NP, C = rc_layout(K)
    assert C * NP <= 16  # the copies fit one 32-word line
    rng = np.random.default_rng(K)
    for _ in range(40):
        j = rng.integers(0, 4096, size=NP)  # any coordinate for each row
        for q in range(NP):
            pairs = []
            for c, ph in lanes(NP, C):
                pi = (q + ph) % NP
                word = int(j[ph]) * 32 + 2 * (c * NP + pi)
                pairs.append((word // 2) % 16)  # the 8-byte bank pair
            assert len(pairs) == len(set(pairs)), (K, q)


@pytest.mark.parametrize("K", range(1, 33))
def test_table_words_and_reads_agree(K):
    """The table build's word -> (copy, centre) map and the read addresses
    describe the same centres; each lane's NP steps cover every pair once,
    and accumulator slot q of lane (c, ph) holds pair (q + ph) mod NP."""
    NP, C = rc_layout(K)
    word_centre = {}
    for w in range(32):
        b = w >> 1
        if b < C * NP:
            cc = b // NP
            word_centre[w] = (cc, 2 * (b - cc * NP) + (w & 1))
    for c, ph in lanes(NP, C):
        seen = []
        for q in range(NP):
            pi = (q + ph) % NP
            base = 2 * (c * NP + pi)
            assert word_centre[base] == (c, 2 * pi)
            assert word_centre[base + 1] == (c, 2 * pi + 1)
            seen.append(pi)
        assert sorted(seen) == list(range(NP))
    # the centres a row's lanes cover: all K (pairs beyond K are padding)
    assert 2 * NP >= K


@pytest.mark.parametrize("K,m", [(10, 51), (5, 8), (8, 102), (20, 51), (32, 205), (1, 7)])
def test_stage_stride_makes_staged_reads_conflict_free(K, m):
    NP, C = rc_layout(K)
    S = stage_stride(m, NP, C)
    assert S >= m
    if (K, m) == (10, 51):
        assert S == m  # the K-means workload stages its rows unpadded
    for h in (0, 1):
        for step in range(0, (m + C - 1) // C):
            pairs = []
            for c, ph in lanes(NP, C):
                rw = h * NP + ph
                t = c + C * step
                pairs.append((rw * S + t) % 16)
            assert len(pairs) == len(set(pairs))


@pytest.mark.parametrize("m", [2, 3, 7, 39, 51, 102, 205, 819, 1024])
def test_row_of_entry_by_multiply_high(m):
    minv = (1 << 32) // m + 1
    NP_max = 16
    e = np.arange(0, 2 * NP_max * m, dtype=np.uint64)  # a group's entries
    r = (e * np.uint64(minv)) >> np.uint64(32)
    assert np.array_equal(r, e // np.uint64(m))
