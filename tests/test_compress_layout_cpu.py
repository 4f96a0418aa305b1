"""The compress kernels' transform layout, checked on the host.

A 1024-element unit (one warp; pt > 1024: G = pt/1024 warps, one unit
each) is transformed in phases: phase A on element bits {0, 1, 7, 8, 9} in
registers (the float4 layout e = 128 ip + 4 lane + q), phase B on bits
{2, ..., 6} after a transpose through shared memory (lane = (ib, q),
register j: e = 128 ib + 4 j + q), phase C on bits 10.. across the group's
warps.  In shared memory element e sits at phys(e) = e + 4 floor(e / 128)
(four floats of padding after every 128), a 1024-element segment taking
1056 floats.  The index expressions below are the kernels'; the checks are
that every phase covers each element once, that the butterflies of all
phases together run over every element bit of a row exactly once (so the
composition is the Walsh-Hadamard transform, whose stages commute), and
that every warp-wide shared-memory access is free of bank conflicts.  Two
more host checks: the split gather (pt > 1024, masks drawn first) covers
each sample once with its early-fetched coordinates, and the masks-alone
kernel's 16-bit virtual Fisher-Yates entries (value and row tag) behave as
a fresh array per row across tag wraps.
"""
import numpy as np
import pytest

SEG = 1024 + 32


def phys(e):
    return e + ((e >> 7) << 2)


def banks_conflict_free(word_addrs_per_lane, width):
    """A warp access of `width` 4-byte words per lane (1, 2 or 4) needs
    32 * width / 32 wavefronts at best; it is conflict free if each group of
    32 / width consecutive lanes touches 32 distinct banks."""
    per = 32 // width
    for g in range(0, 32, per):
        banks = []
        for lane in range(g, g + per):
            for w in range(width):
                banks.append((word_addrs_per_lane[lane] + w) % 32)
        if len(set(banks)) != 32:
            return False
    return True


def test_padded_layout_is_injective_and_fits_a_segment():
    addrs = [phys(e) for e in range(1024)]
    assert len(set(addrs)) == 1024
    assert max(addrs) < SEG


def test_phase_a_covers_the_unit_and_its_stores_are_conflict_free():
    seen = set()
    for lane in range(32):
        for r in range(32):
            seen.add(128 * (r >> 2) + 4 * lane + (r & 3))
    assert seen == set(range(1024))
    # register bit rb of r <-> element bit {0, 1, 7, 8, 9}[rb]
    for rb, eb in enumerate([0, 1, 7, 8, 9]):
        for r in range(32):
            e0 = 128 * (r >> 2) + (r & 3)
            e1 = 128 * ((r ^ (1 << rb)) >> 2) + ((r ^ (1 << rb)) & 3)
            assert e0 ^ e1 == 1 << eb
    # the float4 stores of phase A (16 bytes per lane) and the loads of the
    # staged raw unit (linear)
    for ip in range(8):
        a = [phys(128 * ip + 4 * lane) for lane in range(32)]
        assert all(x % 4 == 0 for x in a)  # 16-byte aligned
        assert banks_conflict_free(a, 4)
        assert banks_conflict_free([128 * ip + 4 * lane for lane in range(32)], 4)


def test_phase_b_covers_the_unit_and_is_conflict_free():
    seen = set()
    for lane in range(32):
        q, ib = lane & 3, lane >> 2
        for j in range(32):
            seen.add(128 * ib + 4 * j + q)
    assert seen == set(range(1024))
    for j in range(32):
        a = [phys(128 * (lane >> 2) + 4 * j + (lane & 3)) for lane in range(32)]
        assert banks_conflict_free(a, 1)
    # register bit rb of j <-> element bit rb + 2
    for rb in range(5):
        for j in range(32):
            assert (4 * j) ^ (4 * (j ^ (1 << rb))) == 1 << (rb + 2)


@pytest.mark.parametrize("L", [11, 12, 13])
def test_phase_c_covers_the_row_and_is_conflict_free(L):
    G = 1 << (L - 10)
    S = 32 // G
    seen = {}
    for wg in range(G):
        for lane in range(32):
            tau = wg * 32 + lane
            for s2 in range(S):
                for w3 in range(0, G, 2):
                    for half in (0, 1):
                        seg, off = w3 + half, tau + 32 * G * s2
                        key = (seg, off)
                        seen[key] = seen.get(key, 0) + 1
    assert set(seen.values()) == {1}
    assert set(seen) == {(s, o) for s in range(G) for o in range(1024)}
    for s2 in range(S):
        for w3 in range(G):
            for wg in range(G):
                a = [SEG * w3 + phys(wg * 32 + lane + 32 * G * s2) for lane in range(32)]
                assert banks_conflict_free(a, 1)
    # a register pair holds segments w3 and w3 + 1 (the in-pair stage: segment
    # bit 0, element bit 10); pair index P = (s2 G + w3) / 2, whose low bits
    # are segment bits 1..: stage rb >= 1 of the packed registers pairs
    # segments differing in bit rb (element bit 10 + rb)
    for s2 in range(S):
        for w3 in range(0, G, 2):
            P = (s2 * G + w3) >> 1
            for rb in range(1, (G).bit_length() - 1):
                Q = P ^ (1 << (rb - 1))
                w3q = 2 * Q - s2 * G
                assert 0 <= w3q < G and (w3 ^ w3q) == 1 << rb


@pytest.mark.parametrize("L", list(range(2, 14)))
def test_every_bit_of_a_row_is_transformed_once(L):
    """Phase A's stages run for element bits below L among {0,1,7,8,9},
    phase B's for bits 2..6 below L, phase C for bits 10..L-1: together each
    bit of a row's index exactly once, and no bit that would mix two rows of
    a unit (pt < 1024 packs 1024 / pt rows in a unit)."""
    bits = [eb for eb in (0, 1, 7, 8, 9) if eb < L]
    bits += [rb + 2 for rb in range(5) if rb + 2 < L]
    bits += list(range(10, L))
    assert sorted(bits) == list(range(L))


def test_unit_addresses_match_the_gather():
    """The gather reads y at yaddr(row offset, index): phys within a unit
    (pt <= 1024, rows at offset b * pt) or segment * 1056 + phys (pt > 1024),
    the same slots the transform wrote."""
    for L in (6, 10):
        pt = 1 << L
        addrs = {phys(b * pt + c) for b in range(1024 // pt) for c in range(pt)}
        assert len(addrs) == 1024 and max(addrs) < SEG  # rows of a unit never overlap
    L = 12
    for c in range(0, 1 << L, 13):
        addr = (c >> 10) * SEG + phys(c & 1023)
        assert addr // SEG == c >> 10 and addr % SEG == phys(c & 1023)


@pytest.mark.parametrize("L", [11, 12, 13])
@pytest.mark.parametrize("m", [1, 41, 64, 205, 819, 1640])
def test_split_gather_covers_each_sample_once(L, m):
    """pt > 1024 with the masks drawn first: the G warps of a row group
    gather its m samples, each lane first the kMI = 2 coordinates it fetched
    before the transform (t = 32 wg + lane + q 32 G), then the rest in steps
    of 32 G; every t in [0, m) exactly once."""
    G, kMI = 1 << (L - 10), 2
    seen = []
    for wg in range(G):
        for lane in range(32):
            for q in range(kMI):
                t = wg * 32 + lane + q * G * 32
                if t < m:
                    seen.append(t)
            t = wg * 32 + lane + kMI * G * 32
            while t < m:
                seen.append(t)
                t += G * 32
    assert sorted(seen) == list(range(m))


@pytest.mark.parametrize("L", [6, 10, 12, 13])
def test_sixteen_bit_fisher_yates_entries(L):
    """The masks-alone kernel's virtual Fisher-Yates array with 16-bit
    entries: an L-bit value under a (16 - L)-bit row tag; a row sees only its
    own writes (other positions read as their own index), and clearing the
    array when the tag wraps keeps an old row's entries from ever matching.
    Checked against a fresh dictionary per row over several wraps."""
    PT, tag_max = 1 << L, (1 << (16 - L)) - 1
    A = np.zeros(PT, dtype=np.uint16)
    rng = np.random.default_rng(L)
    tag = 1
    for row in range(3 * tag_max + 5):
        ref = {}
        for _ in range(40):
            k = int(rng.integers(0, PT))
            if rng.random() < 0.5:
                v = int(rng.integers(0, PT))
                A[k] = (tag << L) | v
                ref[k] = v
            a = int(A[k])
            got = a & (PT - 1) if (a >> L) == tag else k
            assert got == ref.get(k, k)
        tag += 1
        if tag > tag_max:
            A[:] = 0
            tag = 1
