"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws data only: it holds none of the method's arithmetic (no
preconditioning, sampling or estimation), so both the CUDA path and the CPU
oracle can consume its output.  Host generators use numpy's PCG64; device
generators use torch's CUDA generator and are meant for full-size runs where
the oracle only sees rows copied back from the device.

Recipes (all float32 output, rows are samples, row-major n x p):

* ``lowrank_spiky`` -- rank-r Gaussian signal plus Gaussian noise, and a
  fraction of rows with one coordinate multiplied by a spike factor.  Mirrors
  the "few large entries" data that motivates preconditioning (Sec. III and
  the spiky-PC experiment of Sec. V).
* ``mixture`` -- K Gaussian clusters with centres N(0,1)*scale and isotropic
  noise, a fraction of rows with Student-t(df) noise instead (heavy tails).
  Stands in for the synthetic and MNIST K-means workloads of Sec. VII.
* ``lowrank_decay`` -- rank-r signal with singular values proportional to
  1/k on orthonormal loadings, plus small Gaussian noise (the rank-k PCA
  model of Sec. V's experiments).
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------------ host (numpy)

def lowrank_spiky(n: int, p: int, seed: int, sv=(10.0, 6.0, 4.0, 2.0, 1.0),
                  noise: float = 0.1, spike_frac: float = 0.05,
                  spike: float = 50.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    r = len(sv)
    loadings = rng.standard_normal((r, p)) / np.sqrt(p)
    scores = rng.standard_normal((n, r)) * np.asarray(sv)[None, :]
    X = scores @ loadings + noise * rng.standard_normal((n, p))
    n_spiky = int(round(spike_frac * n))
    rows = rng.choice(n, size=n_spiky, replace=False)
    cols = rng.integers(0, p, size=n_spiky)
    X[rows, cols] *= spike
    return X.astype(np.float32)


def mixture(n: int, p: int, K: int, seed: int, centre_scale: float = 3.0,
            sigma: float = 0.5, heavy_frac: float = 0.1, df: float = 3.0):
    """Returns (X float32 n x p, true labels int32, true centres float64 K x p)."""
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((K, p)) * centre_scale
    labels = rng.integers(0, K, size=n).astype(np.int32)
    noise = rng.standard_normal((n, p))
    heavy = rng.random(n) < heavy_frac
    if heavy.any():
        noise[heavy] = rng.standard_t(df, size=(int(heavy.sum()), p))
    X = centres[labels] + sigma * noise
    return X.astype(np.float32), labels, centres


def lowrank_decay(n: int, p: int, seed: int, rank: int = 20, noise: float = 0.01,
                  scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((p, rank)))
    sv = scale / np.arange(1, rank + 1)
    scores = rng.standard_normal((n, rank)) * sv[None, :]
    X = scores @ Q.T + noise * rng.standard_normal((n, p))
    return X.astype(np.float32)


def uniform(n: int, p: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, p)).astype(np.float32)


# ------------------------------------------------------------ device (torch CUDA)

def _torch_gen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def mixture_device(n: int, p: int, K: int, seed: int, device="cuda",
                   centre_scale: float = 3.0, sigma: float = 0.5,
                   heavy_frac: float = 0.1, df: float = 3.0, chunk: int = 1 << 18):
    """Device version of ``mixture`` (same recipe, torch's CUDA generator).

    Student-t(df) noise is drawn as N(0,1) / sqrt(chi2(df)/df) with the
    chi-square drawn as a sum of df squared normals (df integer)."""
    import torch
    g = _torch_gen(seed, device)
    centres = torch.randn(K, p, generator=g, device=device, dtype=torch.float32) * centre_scale
    labels = torch.randint(0, K, (n,), generator=g, device=device, dtype=torch.int64)
    X = torch.empty(n, p, device=device, dtype=torch.float32)
    dfi = int(df)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        noise = torch.randn(r1 - r0, p, generator=g, device=device, dtype=torch.float32)
        heavy = torch.rand(r1 - r0, generator=g, device=device) < heavy_frac
        chi = torch.zeros(r1 - r0, 1, device=device, dtype=torch.float32)
        for _ in range(dfi):
            z = torch.randn(r1 - r0, 1, generator=g, device=device, dtype=torch.float32)
            chi += z * z
        tscale = torch.rsqrt(chi / dfi)
        noise = torch.where(heavy[:, None], noise * tscale, noise)
        X[r0:r1] = centres[labels[r0:r1]] + sigma * noise
    return X, labels.to(torch.int32), centres


def lowrank_decay_device(n: int, p: int, seed: int, rank: int = 20, noise: float = 0.01,
                         scale: float = 1.0, device="cuda", chunk: int = 1 << 16):
    import torch
    g = _torch_gen(seed, device)
    G = torch.randn(p, rank, generator=g, device=device, dtype=torch.float64)
    Q, _ = torch.linalg.qr(G.cpu())  # p x rank: small, on the host
    Q = Q.to(device=device, dtype=torch.float32)
    sv = (scale / torch.arange(1, rank + 1, device=device, dtype=torch.float32))
    X = torch.empty(n, p, device=device, dtype=torch.float32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        scores = torch.randn(r1 - r0, rank, generator=g, device=device) * sv[None, :]
        X[r0:r1] = scores @ Q.T + noise * torch.randn(r1 - r0, p, generator=g, device=device)
    return X


def lowrank_spiky_device(n: int, p: int, seed: int, sv=(10.0, 6.0, 4.0, 2.0, 1.0),
                         noise: float = 0.1, spike_frac: float = 0.05,
                         spike: float = 50.0, device="cuda"):
    import torch
    g = _torch_gen(seed, device)
    r = len(sv)
    loadings = torch.randn(r, p, generator=g, device=device) / float(np.sqrt(p))
    scores = torch.randn(n, r, generator=g, device=device) * torch.tensor(sv, device=device)
    X = scores @ loadings + noise * torch.randn(n, p, generator=g, device=device)
    spiky = torch.rand(n, generator=g, device=device) < spike_frac
    cols = torch.randint(0, p, (n,), generator=g, device=device)
    rows = torch.nonzero(spiky).flatten()
    X[rows, cols[rows]] *= spike
    return X.contiguous()


def init_rows(n: int, K: int, seed: int) -> np.ndarray:
    """K distinct row indices of [0, n) for a seeded K-means start (the same
    rows go to the CUDA path and to the oracle)."""
    rng = np.random.default_rng([int(seed), 0x494E4954])
    return np.sort(rng.choice(n, size=K, replace=False)).astype(np.int64)


def lowrank_mixture_chunk_device(n: int, p: int, seed: int, row0: int, rank: int = 50,
                                 offsets: int = 8, noise: float = 0.1, offset_scale: float = 2.0,
                                 device="cuda", stream=None):
    """Rows row0 .. row0+n-1 of a stream drawn from a rank-`rank` Gaussian
    model plus one of `offsets` mixture offsets plus N(0, noise^2) noise (the
    streaming workload).  The loadings and offsets depend on `seed` only and
    the rows on (seed, row0), so a chunk is the same whichever chunks come
    before it."""
    import torch
    gl = _torch_gen(int(seed) * 1000003 + 17, device)
    loadings = torch.randn(rank, p, generator=gl, device=device) / float(np.sqrt(p))
    offs = torch.randn(offsets, p, generator=gl, device=device) * offset_scale
    sv = torch.linspace(3.0, 0.3, rank, device=device)
    g = _torch_gen((int(seed) * 1000003 + int(row0)) & ((1 << 62) - 1), device)
    scores = torch.randn(n, rank, generator=g, device=device) * sv[None, :]
    which = torch.randint(0, offsets, (n,), generator=g, device=device)
    X = scores @ loadings + offs[which] + noise * torch.randn(n, p, generator=g, device=device)
    return X.contiguous()
