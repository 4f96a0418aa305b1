"""Host restatement (numpy) of the arithmetic of the DCT kernels in
paper_1511_00152_gb300/csrc/dct.cu, checked against scipy.fft's orthonormal
DCT-II / DCT-III and numpy's FFT on every radix combination the kernels
take (2, 3, 4, 5, 7, 8, 11, 13) -- the GPU tests cover a few lengths only.

Forward: the even/odd reordering into z of length L = N/2, the self-sorting
mixed-radix FFT with the kernel's stage addressing (input j + r S, twiddle
index k r st, output (j / Ns) Ns R + k + q Ns) and its butterflies (radix
2, 4 and 8 written out, odd radices in the symmetric form), then E, O, V, W and
X_k = Re W_k, X_{N-k} = -Im W_k.  Inverse: the same steps backwards with the
inverse FFT, as the un-mixing kernel runs them.

The library runs the stages in the order its shared-memory cost model rates
cheapest for the length; every distinct order of the radices is checked
here, so whichever it picks is covered."""
import itertools

import numpy as np
import pytest

scipy_fft = pytest.importorskip("scipy.fft")


def factor(L):
    """The kernels' radices, 8, 4, 2 first, then odd primes up to 13 (the
    library may run them in another order)."""
    out = []
    for r in (8, 4, 2):
        while L > 1 and L % r == 0:
            out.append(r)
            L //= r
    for r in (3, 5, 7, 11, 13):
        while L > 1 and L % r == 0:
            out.append(r)
            L //= r
    assert L == 1
    return out


def dft4(x0, x1, x2, x3, d):
    a, b, c, e = x0 + x2, x0 - x2, x1 + x3, x1 - x3
    em = -1j * d * e
    return a + c, b + em, a - c, b - em


def butterfly(x, R, d, rt):
    """The kernels' R-point DFT: radix 2, 4, 8 written out, odd R in the
    symmetric form (a_r = x_r + x_{R-r}, b_r = x_r - x_{R-r})."""
    if R == 2:
        return [x[0] + x[1], x[0] - x[1]]
    if R == 4:
        return list(dft4(*x, d))
    if R == 8:
        e = dft4(x[0], x[2], x[4], x[6], d)
        o = dft4(x[1], x[3], x[5], x[7], d)
        h = np.sqrt(0.5)
        t = [o[0], h * (1 - 1j * d) * o[1], -1j * d * o[2], h * (-1 - 1j * d) * o[3]]
        return [e[q] + t[q] for q in range(4)] + [e[q] - t[q] for q in range(4)]
    H = (R - 1) // 2
    a = [None] + [x[r] + x[R - r] for r in range(1, H + 1)]
    b = [None] + [x[r] - x[R - r] for r in range(1, H + 1)]
    y = [None] * R
    y[0] = x[0] + sum(a[1:])
    for q in range(1, H + 1):
        re = x[0] + sum(a[r] * rt[(r * q) % R].real for r in range(1, H + 1))
        im = sum(b[r] * -rt[(r * q) % R].imag for r in range(1, H + 1))
        y[q], y[R - q] = re - 1j * im, re + 1j * im
    return y


def orders(L, cap=60):
    """Distinct orders of factor(L) (at most cap of them)."""
    return list(itertools.islice(sorted(set(itertools.permutations(factor(L)))), cap))


def fft_stockham(z, direction, order=None):
    L = len(z)
    tw = np.exp(-direction * 2j * np.pi * np.arange(L) / L)
    a, Ns = z.astype(np.complex128).copy(), 1
    for R in (factor(L) if order is None else order):
        S, st = L // R, L // (Ns * R)
        b = np.empty_like(a)
        rt = tw[np.arange(R) * S]
        for j in range(S):
            jq, k = divmod(j, Ns)
            x = a[j + np.arange(R) * S]
            if Ns > 1:
                x = x * tw[k * np.arange(R) * st]
            y = butterfly(list(x), R, direction, rt)
            base = jq * Ns * R + k
            for q in range(R):
                b[base + q * Ns] = y[q]
        a, Ns = b, Ns * R
    return a


def dct2(x, order=None):
    N = len(x)
    L = N // 2
    v = np.empty(N)
    v[:L], v[N - 1 - np.arange(L)] = x[0::2], x[1::2]
    Z = fft_stockham(v[0::2] + 1j * v[1::2], 1, order)
    y = np.empty(N)
    s = np.full(N, np.sqrt(2 / N))
    s[0] = np.sqrt(1 / N)
    for k in range(L + 1):
        Zk, Zc = Z[0 if k == L else k], np.conj(Z[0 if k == 0 else L - k])
        E, O = (Zk + Zc) / 2, (Zk - Zc) / 2j
        W = np.exp(-1j * np.pi * k / (2 * N)) * (E + np.exp(-2j * np.pi * k / N) * O)
        y[k] = s[k] * W.real
        if 0 < k < L:
            y[N - k] = s[N - k] * -W.imag
    return y


def dct3(y, order=None):
    N = len(y)
    L = N // 2
    s = np.full(N, np.sqrt(2 / N))
    s[0] = np.sqrt(1 / N)
    V = np.empty(L + 1, complex)
    for k in range(L + 1):
        Xk = y[k] / s[k]
        Xn = y[N - k] / s[N - k] if k > 0 else 0.0
        V[k] = np.exp(1j * np.pi * k / (2 * N)) * (Xk - 1j * Xn)
    Z = np.empty(L, complex)
    for k in range(L):
        E = (V[k] + np.conj(V[L - k])) / 2
        D = (V[k] - np.conj(V[L - k])) / 2
        Z[k] = E + 1j * D * np.exp(2j * np.pi * k / N)
    z = fft_stockham(Z, -1, order) / L
    v = np.empty(N)
    v[0::2], v[1::2] = z.real, z.imag
    x = np.empty(N)
    x[0::2], x[1::2] = v[:L], v[N - 1 - np.arange(L)]
    return x


@pytest.mark.parametrize("N", [2, 4, 6, 10, 14, 16, 22, 26, 30, 98, 200, 784, 1000, 2 * 8 * 27,
                               2 * 11 * 13, 2 * 4 * 5 * 7, 2 * 2048])
def test_kernel_dct_arithmetic_matches_scipy(N):
    x = np.random.default_rng(N).standard_normal(N)
    assert np.max(np.abs(dct2(x) - scipy_fft.dct(x, type=2, norm="ortho"))) < 1e-11
    assert np.max(np.abs(dct3(x) - scipy_fft.dct(x, type=3, norm="ortho"))) < 1e-11


@pytest.mark.parametrize("L", [8, 12, 49, 98, 125, 143, 200, 392, 500, 1001])
def test_kernel_fft_stage_addressing(L):
    z = np.random.default_rng(L).standard_normal(L) + 1j * np.random.default_rng(L + 1).standard_normal(L)
    for order in orders(L):
        assert np.max(np.abs(fft_stockham(z, 1, order) - np.fft.fft(z))) < 1e-10, order
        assert np.max(np.abs(fft_stockham(z, -1, order) - L * np.fft.ifft(z))) < 1e-10, order


@pytest.mark.parametrize("N", [200, 784, 1000, 2 * 1001])
def test_kernel_dct_every_stage_order(N):
    x = np.random.default_rng(N + 7).standard_normal(N)
    ref2 = scipy_fft.dct(x, type=2, norm="ortho")
    ref3 = scipy_fft.dct(x, type=3, norm="ortho")
    for order in orders(N // 2):
        assert np.max(np.abs(dct2(x, order) - ref2)) < 1e-11, order
        assert np.max(np.abs(dct3(x, order) - ref3)) < 1e-11, order
