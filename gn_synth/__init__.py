"""Seeded synthetic inputs for generalized Nystrom (GN) workloads.

This module only *draws* inputs: dense test matrices shaped like the paper's
experiments (Section 7.1: A = U Sigma V^T with decaying singular values) and the
Gaussian sketch matrices X (n x r), Y (m x (r+l)) of Algorithm 2, step 1.  It
holds none of the method's arithmetic (no sketch products, no QR, no
pseudoinverse), and it is the one module that both the CPU oracle and the CUDA
path's tests / benchmark may share.

Every generator is a pure function of an integer seed.  Draws use
``torch.Generator`` (Mersenne twister on the CPU, Philox on a CUDA device);
a CPU draw is reproducible on the machine that made it, which is all the
parity tests need because they draw once and hand the same arrays to both
sides.  Large workloads may be drawn directly on a CUDA device for speed; the
values then differ from a CPU draw with the same seed, but are still seeded.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

__all__ = [
    "DEFAULT_SEED",
    "gaussian",
    "orthonormal_columns",
    "geometric_usv",
    "lowrank_plus_noise",
    "sketches",
    "batched_shapes",
    "power_decay",
    "GNProblem",
    "config1",
    "config2",
    "config3",
    "config4",
    "config5_problem",
    "dct_sketch_draws",
    "countsketch_draws",
    "sparse_lowrank_plus_noise",
]

DEFAULT_SEED = 20091139

# Stream offsets keep the independent draws of one problem apart.
_STREAM_A1, _STREAM_A2, _STREAM_NOISE, _STREAM_X, _STREAM_Y, _STREAM_G = range(6)


def _seed(seed: int, stream: int) -> int:
    """Mix (seed, stream) into a 63-bit generator seed (splitmix64 finaliser)."""
    z = (seed * 0x9E3779B97F4A7C15 + (stream + 1) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    z ^= z >> 31
    return z & 0x7FFFFFFFFFFFFFFF


def gaussian(shape, seed: int, stream: int = 0, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """i.i.d. N(0, 1) entries, drawn in FP64 (or ``dtype``) from a seeded generator."""
    g = torch.Generator(device=device)
    g.manual_seed(_seed(seed, stream))
    return torch.randn(*shape, generator=g, device=device, dtype=dtype)


def orthonormal_columns(m: int, k: int, seed: int, stream: int, device="cpu") -> torch.Tensor:
    """Q factor of an m x k Gaussian matrix (the paper's 'random orthogonal' U, V)."""
    q, _ = torch.linalg.qr(gaussian((m, k), seed, stream, device=device))
    return q


def geometric_usv(m: int, n: int, seed: int = DEFAULT_SEED, device="cpu") -> torch.Tensor:
    """A = U diag(2^(-i/10)) V^T, i = 1..n (the 1000 x 500 small dense case)."""
    u = orthonormal_columns(m, n, seed, _STREAM_A1, device)
    v = orthonormal_columns(n, n, seed, _STREAM_A2, device)
    sigma = torch.pow(2.0, -torch.arange(1, n + 1, device=device, dtype=torch.float64) / 10.0)
    return (u * sigma) @ v.T


def lowrank_plus_noise(m: int, n: int, k_modes: int, sigma: torch.Tensor, noise: float,
                       seed: int = DEFAULT_SEED, device="cpu",
                       dtype=torch.float64) -> torch.Tensor:
    """A = W1 diag(sigma) W2^T + noise * N(0,1), W1, W2 i.i.d. N(0,1)/sqrt(k_modes).

    ``sigma`` has k_modes entries.  ``dtype`` is the precision the matrix is
    built and returned in (FP64 by default; FP32 for the very large cases drawn
    on a device, where FP64 would only slow the draw)."""
    w1 = gaussian((m, k_modes), seed, _STREAM_A1, device, dtype) / math.sqrt(k_modes)
    w2 = gaussian((n, k_modes), seed, _STREAM_A2, device, dtype) / math.sqrt(k_modes)
    a = (w1 * sigma.to(device=device, dtype=dtype)) @ w2.T
    del w1, w2
    if noise:
        a.add_(gaussian((m, n), seed, _STREAM_NOISE, device, dtype), alpha=noise)
    return a


def sketches(m: int, n: int, r: int, l: int, seed: int = DEFAULT_SEED, device="cpu",
             dtype=torch.float64):
    """Gaussian sketches of Algorithm 2, step 1: X (n x r), Y (m x (r+l))."""
    x = gaussian((n, r), seed, _STREAM_X, device, dtype)
    y = gaussian((m, r + l), seed, _STREAM_Y, device, dtype)
    return x, y


@dataclass
class GNProblem:
    a: torch.Tensor
    x: torch.Tensor
    y: torch.Tensor
    r: int
    l: int
    eps: float
    note: str = ""


def config1(seed: int = DEFAULT_SEED, device="cpu") -> GNProblem:
    """1000 x 500, sigma_i = 2^(-i/10), r = 20, l = 10, eps = 1e-15 * ||A||_2."""
    m, n, r, l = 1000, 500, 20, 10
    a = geometric_usv(m, n, seed, device)
    x, y = sketches(m, n, r, l, seed, device)
    return GNProblem(a, x, y, r, l, 1e-15 * 2.0 ** -0.1, "geometric 2^(-i/10)")


def power_decay(k_modes: int, p: float, device="cpu") -> torch.Tensor:
    return torch.arange(1, k_modes + 1, device=device, dtype=torch.float64) ** (-p)


def config2(seed: int = DEFAULT_SEED, device="cpu", m: int = 20000, n: int = 10000,
            r: int = 500, l: int = 250, dtype=torch.float64) -> GNProblem:
    """W1 diag(i^-2) W2^T + 1e-8 N, 2000 modes; default 20000 x 10000, r = 500."""
    k = 2000
    a = lowrank_plus_noise(m, n, k, power_decay(k, 2.0, device), 1e-8, seed, device, dtype)
    x, y = sketches(m, n, r, l, seed, device, dtype)
    return GNProblem(a, x, y, r, l, 0.0, "i^-2 over 2000 modes + 1e-8 noise")


def config3(r: int = 1000, seed: int = DEFAULT_SEED, device="cpu", m: int = 32768,
            n: int = 16384, dtype=torch.float64) -> GNProblem:
    """Same generator as the 20000 x 10000 case at 32768 x 16384, l = r/2."""
    return config2(seed, device, m, n, r, r // 2, dtype)


def config4(seed: int = DEFAULT_SEED, device="cpu", m: int = 4096, n: int = 4096,
            r: int = 256, l: int = 128, dtype=torch.float64):
    """Differentiation case: sigma_i = i^-1.5 over 1024 modes + 1e-6 noise, G ~ N(0,1)."""
    k = min(1024, m, n)
    a = lowrank_plus_noise(m, n, k, power_decay(k, 1.5, device), 1e-6, seed, device, dtype)
    x, y = sketches(m, n, r, l, seed, device, dtype)
    g = gaussian((m, n), seed, _STREAM_G, device, dtype)
    return GNProblem(a, x, y, r, l, 0.0, "i^-1.5 over 1024 modes + 1e-6 noise"), g


def batched_shapes(count: int = 512, seed: int = DEFAULT_SEED):
    """Uneven problem shapes: m ~ U[256,4096], n ~ U[128,m], r ~ U{16..128}, l = r/2."""
    g = torch.Generator().manual_seed(_seed(seed, 99))
    shapes = []
    for _ in range(count):
        m = int(torch.randint(256, 4097, (1,), generator=g))
        n = int(torch.randint(128, m + 1, (1,), generator=g))
        r = int(torch.randint(16, 129, (1,), generator=g))
        shapes.append((m, n, r, r // 2))
    return shapes


def config5_problem(index: int, shape, seed: int = DEFAULT_SEED, device="cpu",
                    dtype=torch.float64) -> GNProblem:
    """One batched problem: W1 diag(2^(-i/10)) W2^T + 1e-8 N with per-matrix seed."""
    m, n, r, l = shape
    s = seed + index
    k = min(n, 4 * r)
    sigma = torch.pow(2.0, -torch.arange(1, k + 1, device=device, dtype=torch.float64) / 10.0)
    a = lowrank_plus_noise(m, n, k, sigma, 1e-8, s, device, dtype)
    x, y = sketches(m, n, r, l, s, device, dtype)
    return GNProblem(a, x, y, r, l, 0.0, f"batched #{index}")


def dct_sketch_draws(n: int, r: int, seed: int = DEFAULT_SEED, stream: int = _STREAM_X):
    """The random draws of a subsampled DCT sketch (the sketches of Section 7):
    n random signs (+-1) and r distinct frequencies out of n, sorted.  Only the
    draws; the sketch matrix itself is built by whoever applies it."""
    g = torch.Generator()
    g.manual_seed(_seed(seed, stream + 16))
    signs = torch.randint(0, 2, (n,), generator=g).double() * 2.0 - 1.0
    cols = torch.randperm(n, generator=g)[:r].sort().values
    return signs, cols


def countsketch_draws(n: int, r: int, seed: int = DEFAULT_SEED, stream: int = _STREAM_X):
    """The random draws of a CountSketch matrix (Section 2.5: one +-1 per row):
    a bucket in [0, r) and a sign for each of the n rows.  Only the draws."""
    g = torch.Generator()
    g.manual_seed(_seed(seed, stream + 32))
    buckets = torch.randint(0, r, (n,), generator=g)
    signs = torch.randint(0, 2, (n,), generator=g).double() * 2.0 - 1.0
    return buckets, signs


def sparse_lowrank_plus_noise(m: int, n: int, k: int, nnz_per_row: int, seed: int = DEFAULT_SEED):
    """A sparse stand-in for Section 7's sparse experiment (whose matrix is not
    available): the sum of k sparse rank-1 terms u_t v_t^T, each supported on
    `per` random rows and `per` random columns with per^2 ~ nnz_per_row m / k
    (so the k terms hold about nnz_per_row nonzeros per row), term t scaled by
    1 / (t + 1), plus m nnz_per_row / 4 entries of N(0, 1e-8) noise; COO
    triplets (rows, cols, values), duplicates summed by the caller.  Only draws."""
    g = torch.Generator()
    g.manual_seed(_seed(seed, _STREAM_A1 + 48))
    rows, cols, vals = [], [], []
    per = max(1, int(math.sqrt(max(1, nnz_per_row) * m / max(1, k))))
    for t in range(k):
        ri = torch.randperm(m, generator=g)[: max(1, min(m, per))]
        ci = torch.randperm(n, generator=g)[: max(1, min(n, per))]
        ui = torch.randn(len(ri), generator=g, dtype=torch.float64) * (t + 1) ** -1.0
        vi = torch.randn(len(ci), generator=g, dtype=torch.float64)
        rr = ri[:, None].expand(-1, len(ci)).reshape(-1)
        cc = ci[None, :].expand(len(ri), -1).reshape(-1)
        rows.append(rr)
        cols.append(cc)
        vals.append((ui[:, None] * vi[None, :]).reshape(-1))
    nz = m * max(1, nnz_per_row) // 4
    rows.append(torch.randint(0, m, (nz,), generator=g))
    cols.append(torch.randint(0, n, (nz,), generator=g))
    vals.append(1e-8 * torch.randn(nz, generator=g, dtype=torch.float64))
    return torch.cat(rows), torch.cat(cols), torch.cat(vals)
