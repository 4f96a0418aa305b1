"""The K-means pass's shared-memory centre table, checked on the host.

A row is handled by LPR = ceil(K / 2) lanes, each owning two consecutive
centres (Kpad = 2 LPR).  With LPR <= 16 a half-warp holds G = 16 // LPR row
slots; when G >= 2 the table gives coordinate j one 32-word line with a copy
of its Kpad centre values per slot, copy s at words s Kpad .. s Kpad + Kpad - 1,
and the row in slot s reads copy s.  The index expressions below are the
kernel's (slot and lane decomposition, line address j * 32 + s * Kpad +
2 kl); the check is that the lanes of a half-warp read 8-byte pairs at
distinct banks whatever coordinates their rows sampled, so each centre load
is one shared-memory wavefront per half-warp.
"""
import numpy as np
import pytest


def layout(K):
    LPR = (K + 1) // 2
    Kpad = 2 * LPR
    G = 16 // LPR if LPR <= 16 else 0
    return LPR, Kpad, G


@pytest.mark.parametrize("K", [k for k in range(1, 65) if layout(k)[2] >= 2])
def test_half_warp_reads_are_bank_disjoint(K):
    LPR, Kpad, G = layout(K)
    assert G * Kpad <= 32  # the copies fit one 32-word line
    rng = np.random.default_rng(K)
    for _ in range(50):
        for half in (0, 1):
            j = rng.integers(0, 8192, size=G)  # any coordinate per row slot
            banks = []
            for l16 in range(16):
                hs = l16 // LPR
                kl = l16 - hs * LPR
                if hs >= G:
                    continue  # lane without a row
                word = int(j[hs]) * 32 + hs * Kpad + 2 * kl
                assert word % 2 == 0  # 8-byte aligned pair
                banks += [word % 32, (word + 1) % 32]
            assert len(banks) == len(set(banks))
            assert len(banks) == 2 * LPR * G


@pytest.mark.parametrize("K", [k for k in range(1, 65) if layout(k)[2] >= 2])
def test_every_centre_of_a_row_is_read_by_one_lane(K):
    LPR, Kpad, G = layout(K)
    for hs in range(G):
        centres = sorted(2 * kl + q for kl in range(LPR) for q in (0, 1))
        assert centres == list(range(Kpad)) and Kpad >= K
