"""The lane-parallel partial Fisher-Yates used by the compress kernels, as a
host model, against the sequential draw of the written spec.

The kernels draw a row's m mask positions 32 at a time, one step per lane:
each lane takes its Lemire draw from the word stream (a rejected word shifts
the stream of the later lanes by one), and the swaps of the 32 steps are
resolved in parallel -- the value a step emits is the value of its target
just before the step: either an earlier step's displaced value in the same
chunk (the latest lane with the same target, found by matching targets) or
the target's state after the earlier chunks (a tagged array).  The value a
step displaces is the one at its own position t, which an earlier lane of
the chunk may have moved there (resolved by following the latest such lane
until nothing changes).

This file restates that scheme lane by lane in Python and checks it against
the plain sequential partial Fisher-Yates (Sec. I-A, sampling m of p
without replacement) on word streams chosen to force rejections and long
chains of collisions, and against the oracle's masks on the real Philox
stream.
"""
import numpy as np
import pytest

import oracle

M32 = (1 << 32) - 1
TAG_MASK = 0x4D41534B


def sequential_mask(pt, m, words):
    """The spec: for t = 0..m-1, k = t + U(pt - t) by Lemire with rejection
    on the next words of the stream, swap a[t] and a[k], emit a[t]."""
    a = list(range(pt))
    w = 0
    out = []
    for t in range(m):
        s = pt - t
        while True:
            prod = words[w] * s
            w += 1
            if (prod & M32) >= (1 << 32) % s:
                break
        k = t + (prod >> 32)
        a[t], a[k] = a[k], a[t]
        out.append(a[t])
    return out


def chunked_mask(pt, m, words):
    """The kernels' scheme, one 32-lane chunk at a time."""
    A = {}  # positions moved by earlier chunks: position -> value
    out = [None] * m
    woff = 0
    for c0 in range(0, m, 32):
        lanes = range(32)
        act = [c0 + l < m for l in lanes]
        s = [pt - (c0 + l) for l in lanes]
        w = [c0 + l + woff for l in lanes]
        prod = [0] * 32
        while True:
            rej = []
            for l in lanes:
                prod[l] = words[w[l]] * s[l] if act[l] else 0
                rej.append(act[l] and (prod[l] & M32) < (1 << 32) % s[l])
            if not any(rej):
                break
            first = rej.index(True)
            for l in lanes:
                if l >= first:
                    w[l] += 1
            woff += 1
        k = [(c0 + l) + (prod[l] >> 32) if act[l] else -1 - l for l in lanes]
        # src: the latest earlier lane whose target is this lane's position
        srcm = [0] * 32
        for l in lanes:
            if act[l]:
                srcm[l] = sum(1 << j for j in range(l) if act[j] and k[j] == c0 + l)
        src = [max(j for j in range(32) if srcm[l] >> j & 1) if srcm[l] else l for l in lanes]
        vbase = [A.get(c0 + l, c0 + l) if act[l] else 0 for l in lanes]
        V = list(vbase)
        while True:
            nv = [V[src[l]] if srcm[l] else vbase[l] for l in lanes]
            changed = nv != V
            V = nv
            if not changed:
                break
        for l in lanes:
            if not act[l]:
                continue
            prevm = [j for j in range(l) if act[j] and k[j] == k[l]]
            omega = V[prevm[-1]] if prevm else A.get(k[l], k[l])
            out[c0 + l] = omega
        # the last lane of each target group leaves its displaced value
        # for later chunks at targets beyond this chunk
        if c0 + 32 < m:
            for l in lanes:
                if act[l] and k[l] >= c0 + 32 and not any(act[j] and k[j] == k[l] for j in range(l + 1, 32)):
                    A[k[l]] = V[l]
    return out


def _stream(rng, n, small_frac, pt):
    """Random 32-bit words with a fraction of tiny ones (tiny words are the
    ones Lemire's test can reject) and a bias towards targets in the chunk
    (words that map to small offsets)."""
    words = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)
    tiny = rng.random(n) < small_frac
    words[tiny] = rng.integers(0, 64, size=int(tiny.sum()), dtype=np.uint64)
    return [int(x) for x in words]


@pytest.mark.parametrize("pt,m", [(8, 8), (16, 5), (64, 40), (64, 64), (128, 70), (1024, 51), (256, 100)])
def test_chunked_draw_equals_sequential_with_forced_rejections(pt, m):
    rng = np.random.default_rng(pt * 1000 + m)
    for _ in range(40):
        words = _stream(rng, 4 * m + 64, 0.15, pt)
        assert chunked_mask(pt, m, words) == sequential_mask(pt, m, words)


@pytest.mark.parametrize("pt,m", [(32, 32), (64, 33), (128, 96)])
def test_chunked_draw_equals_sequential_with_collision_chains(pt, m):
    """Words near the top of the range give k near pt - 1 for every lane,
    and small words give k = t: targets collide often, within and across
    chunks."""
    rng = np.random.default_rng(pt + m)
    for _ in range(40):
        n = 4 * m + 64
        words = [int(x) for x in rng.integers(0, 1 << 32, size=n, dtype=np.uint64)]
        for i in range(n):
            r = rng.random()
            if r < 0.3:
                words[i] = M32 - int(rng.integers(0, 1 << 20))
            elif r < 0.5:
                words[i] = int(rng.integers(1 << 8, 1 << 12))
        assert chunked_mask(pt, m, words) == sequential_mask(pt, m, words)


@pytest.mark.parametrize("pt,m,row", [(1024, 51, 0), (1024, 51, 12345), (64, 40, 7), (4096, 205, 3)])
def test_models_match_the_oracle_on_the_philox_stream(pt, m, row):
    seed = 20240611
    key = [seed & M32, seed >> 32]
    nblocks = (m + 64) // 4 + 1
    words = []
    for b in range(nblocks):
        words += [int(x) for x in oracle.philox4x32_10([b, row & M32, row >> 32, TAG_MASK], key)]
    expected = [int(x) for x in oracle.mask(pt, m, seed, row)]
    assert sequential_mask(pt, m, words) == expected
    assert chunked_mask(pt, m, words) == expected
