"""The DCT plan's choice of FFT stage order (dct_factor in
paper_1511_00152_gb300/csrc/dct.cu), run on the host through a small
harness linked against the library: the order is a permutation of the
length's radices (8, 4, 2 first, then odd primes up to 13), and it is the
cheapest under the plan's model of the warp kernel's shared-memory accesses
(restated here: for each stage, every load in[j + r S], twiddle read
tw(k r st) and store out[(j / Ns) Ns R + k + q Ns] of 8 bytes a lane, a
half-warp at a time, costs as many wavefronts as the most distinct 4-byte
words any one bank holds), over every distinct order of up to six stages."""
import itertools
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def radices(L):
    out = []
    for r in (8, 4, 2):
        while L > 1 and L % r == 0:
            out.append(r)
            L //= r
    for r in (3, 5, 7, 11, 13):
        while L > 1 and L % r == 0:
            out.append(r)
            L //= r
    return out if L == 1 else None


def wavefronts(elems):
    words = {2 * e + h for e in elems for h in (0, 1)}
    per_bank = {}
    for w in words:
        per_bank[w & 31] = per_bank.get(w & 31, 0) + 1
    return max(per_bank.values()) if per_bank else 0


def cost(L, order):
    total, Ns = 0, 1
    for R in order:
        S, st = L // R, L // (Ns * R)
        for t0 in range(0, S, 32):
            for r in range(R):
                for kind in range(3):
                    if kind == 2 and (Ns == 1 or r == 0):
                        continue
                    for half in (0, 1):
                        js = range(t0 + 16 * half, min(t0 + 16 * half + 16, S))
                        if kind == 0:
                            e = [j + r * S for j in js]
                        elif kind == 1:
                            e = [(j // Ns) * Ns * R + (j % Ns) + r * Ns for j in js]
                        else:
                            e = [((j % Ns) * r * st) % L for j in js]
                        total += wavefronts(e)
        Ns *= R
    return total


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    gxx = shutil.which("g++") or shutil.which("c++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    from paper_1511_00152_gb300 import build
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("plan") / "dct_plan")
    subprocess.run([gxx, "-std=c++17", "-O1", os.path.join(HERE, "host_fixture", "dct_plan_main.cpp"),
                    lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", exe], check=True)

    def run(Ls):
        out = subprocess.run([exe] + [str(L) for L in Ls], check=True, capture_output=True,
                             text=True).stdout
        res = {}
        for line in out.strip().splitlines():
            f = [int(x) for x in line.split()]
            res[f[0]] = f[2:] if f[1] else None
        return res
    return run


LENGTHS = [8, 12, 49, 98, 125, 143, 200, 300, 392, 441, 500, 512, 1000, 1001]


def test_order_is_a_permutation_of_the_radices(plan):
    got = plan(LENGTHS + [17, 34])
    for L in LENGTHS:
        assert sorted(got[L]) == sorted(radices(L)), L
    assert got[17] is None and got[34] is None  # 17 is not a supported radix


def test_order_is_the_cheapest_under_the_model(plan):
    got = plan(LENGTHS)
    for L in LENGTHS:
        costs = {o: cost(L, o) for o in set(itertools.permutations(radices(L)))}
        assert cost(L, tuple(got[L])) == min(costs.values()), (L, got[L])
    # p = 784: the radix-8 stage first stores at a stride of 8 elements
    assert got[392][0] == 7
    assert cost(392, (7, 8, 7)) < cost(392, (8, 7, 7))
