"""Seeded synthetic inputs for the hierarchical merge-and-truncate SVD.

This module only *makes matrices*; it holds none of the method's arithmetic.
It is shared by the tests, the bench and the scripts that write stored
expected values, so both sides of every comparison consume identical bytes.

Every matrix is dense and low rank with a decaying spectrum, the character of
the paper's CFD velocity/density snapshots and face images (Section 4), which
are not available here; the synthetic recipes below stand in for them.

Recipes (all seeds are ``SeedSequence(17100281 + tag)``):

* ``planted(m, n, s, noise)``: ``A = U diag(s) V^T + noise * N(0, 1)`` where
  ``U`` (m x r) and ``V`` (n x r) are the Q factors of seeded Gaussian
  matrices, so the singular values of the noise-free part are exactly ``s``.
* ``fixed_rank_512``: 512 x 512, r = 10, s_i = 10^(-i/3), noise 1e-6,
  4 x 4 grid of 128 x 128 blocks, k = 10, FP64.
* ``exp_decay_8192``: 8192 x 8192, r = 512, s_i = exp(-i/20), noise 1e-5,
  16 x 16 grid of 512 x 512 blocks, k = 64, FP32.
* ``pod_fourier``: POD-like snapshot matrix. Column t is
  sum_{j=1..40} c_j(t) phi_j(x) + noise; phi are unit-norm sine/cosine modes
  on a uniform grid, c_j(t) ~ N(0, 1) / j^2. Stored in BF16 (round to nearest
  even) when asked.
* ``ragged_batch``: many independent FP32 matrices whose sizes are not
  multiples of the block size, rank r ~ U{8..64}, s_i = exp(-i/r) / r,
  noise 1e-4.
* ``power_law``: s_i = (i + 1)^-1.5 over 512 modes plus 1e-6 noise.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 17100281


def rng(tag: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(SEED_BASE + int(tag)))


def orthonormal(g: np.random.Generator, m: int, r: int) -> np.ndarray:
    """Q factor of a seeded Gaussian m x r matrix (columns orthonormal)."""
    q, rr = np.linalg.qr(g.standard_normal((m, r)))
    # Fix the sign convention of the QR so the result does not depend on the
    # LAPACK build: make diag(R) positive.
    q *= np.sign(np.where(np.diag(rr) == 0, 1.0, np.diag(rr)))[None, :]
    return q


def planted(m: int, n: int, s, noise: float = 0.0, tag: int = 0,
            dtype=np.float64, return_factors: bool = False):
    """A = U diag(s) V^T + noise * N(0,1), built in float64 then cast."""
    s = np.asarray(s, dtype=np.float64)
    r = s.shape[0]
    g = rng(tag)
    u = orthonormal(g, m, r)
    v = orthonormal(g, n, r)
    a = (u * s[None, :]) @ v.T
    if noise:
        a += noise * g.standard_normal((m, n))
    a = np.ascontiguousarray(a.astype(dtype))
    if return_factors:
        return a, u, s, v
    return a


def planted_band(m: int, n: int, s, noise: float = 0.0, tag: int = 0, rows: int = 1, cols: int = 1,
                 dtype=np.float32):
    """Rows 0..rows and columns 0..cols of ``planted(m, n, s, noise, tag)``
    without building the m x n matrix: the same U, V and noise stream (the
    generator fills row by row, so the first rows x n draws are the noise of
    the first rows).  Equal to the slice of the full matrix up to the rounding
    order of the product."""
    s = np.asarray(s, dtype=np.float64)
    r = s.shape[0]
    g = rng(tag)
    u = orthonormal(g, m, r)
    v = orthonormal(g, n, r)
    a = (u[:rows] * s[None, :]) @ v[:cols].T
    if noise:
        a += noise * g.standard_normal((rows, n))[:, :cols]
    return np.ascontiguousarray(a.astype(dtype))


def fixed_rank_512(dtype=np.float64):
    """512^2, r = 10, s_i = 10^(-i/3), noise 1e-6 (the FP64 parity case)."""
    s = 10.0 ** (-np.arange(10) / 3.0)
    a = planted(512, 512, s, noise=1e-6, tag=1, dtype=dtype)
    return a, dict(block_rows=128, block_cols=128, k=10)


def exp_decay(m: int = 8192, n: int = 8192, r: int = 512, noise: float = 1e-5,
              tag: int = 2, dtype=np.float32):
    s = np.exp(-np.arange(r) / 20.0)
    return planted(m, n, s, noise=noise, tag=tag, dtype=dtype)


def exp_decay_8192(dtype=np.float32):
    """8192^2 FP32, s_i = exp(-i/20) over 512 modes, noise 1e-5."""
    return exp_decay(dtype=dtype), dict(block_rows=512, block_cols=512, k=64)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even); returns
    float32 holding exactly representable bfloat16 values."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (x >> 16) & 1
    rounded = (x + 0x7FFF + lsb) >> 16
    out = (rounded << 16).astype(np.uint32).view(np.float32)
    return out


def bf16_bits(a32: np.ndarray) -> np.ndarray:
    """The uint16 bit patterns of float32 values that are exact bfloat16."""
    return (np.ascontiguousarray(a32, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def pod_fourier(m: int = 32768, n: int = 16384, modes: int = 40,
                noise: float = 1e-3, tag: int = 3, bf16: bool = True):
    """POD-like snapshots: unit-norm Fourier modes with 1/j^2 coefficients."""
    g = rng(tag)
    x = np.arange(m, dtype=np.float64) / m
    phi = np.empty((m, modes))
    for j in range(modes):
        q = j // 2 + 1
        phi[:, j] = np.cos(2 * np.pi * q * x) if j % 2 == 0 else np.sin(2 * np.pi * q * x)
    phi /= np.linalg.norm(phi, axis=0, keepdims=True)
    c = g.standard_normal((modes, n)) / (np.arange(1, modes + 1, dtype=np.float64) ** 2)[:, None]
    a = (phi @ c).astype(np.float32)
    a += (noise * g.standard_normal((m, n))).astype(np.float32)
    if bf16:
        a = bf16_round(a)
    return a


def ragged_sizes(count: int = 256, lo: int = 1024, hi: int = 8192, tag: int = 4,
                 block: int = 1024):
    """Matrix sizes for the many-matrix batch: uniform in [lo, hi], redrawn
    when a multiple of the block size; ranks r ~ U{8..64}."""
    g = rng(tag)
    sizes = []
    for _ in range(count):
        dims = []
        for _d in range(2):
            while True:
                v = int(g.integers(lo, hi + 1))
                if v % block:
                    break
            dims.append(v)
        r = int(g.integers(8, 65))
        sizes.append((dims[0], dims[1], r))
    return sizes


def ragged_matrix(m: int, n: int, r: int, noise: float = 1e-4, tag: int = 0,
                  dtype=np.float32):
    s = np.exp(-np.arange(r) / r) / r
    return planted(m, n, s, noise=noise, tag=tag, dtype=dtype)


def power_law(m: int, n: int, modes: int = 512, noise: float = 1e-6, tag: int = 5,
              dtype=np.float32):
    s = (np.arange(modes) + 1.0) ** -1.5
    return planted(m, n, s, noise=noise, tag=tag, dtype=dtype)


# ---------------------------------------------------------------- on-device recipes
# The largest configurations (a 65536 x 65536 FP32 matrix is 17 GB; the
# 256-matrix batch is ~22 GB) are generated directly in device memory with
# torch's seeded generator: the same recipes as above, a different random
# stream.  They serve the full-size GPU tests, which check properties that
# hold at any size and, where the oracle can afford it, individual matrices
# copied back to the host.

def _torch_gen(tag: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(SEED_BASE + int(tag))
    return g


def orthonormal_device(m: int, r: int, g, device):
    """Q factor (diag(R) > 0) of a seeded m x r Gaussian, FP64 on the device
    (the Gaussian drawn on the device, the QR by LAPACK on the host, so the
    recipe needs no device linear-algebra library)."""
    import torch
    a = torch.randn((m, r), generator=g, device=device, dtype=torch.float64).cpu().numpy()
    q, rr = np.linalg.qr(a)
    d = np.sign(np.diag(rr))
    d[d == 0] = 1
    return torch.from_numpy(q * d[None, :]).to(device)


def planted_device(m: int, n: int, s, noise: float = 0.0, tag: int = 0, device="cuda",
                   chunk_rows: int = 4096, rows=None):
    """A = U diag(s) V^T + noise * N(0, 1) as FP32 on the device (U, V with
    orthonormal columns; the noise-free part has singular values exactly s
    up to FP32 storage).  rows = (r0, r1): only those rows of the same
    matrix (the noise of the other chunks is still drawn, to keep the
    generator's stream)."""
    import torch
    s = torch.as_tensor(np.asarray(s, dtype=np.float64), device=device)
    g = _torch_gen(tag, device)
    u = orthonormal_device(m, s.numel(), g, device)
    v = orthonormal_device(n, s.numel(), g, device)
    us = (u * s[None, :]).to(torch.float32)
    vt = v.t().contiguous().to(torch.float32)
    b0, b1 = (0, m) if rows is None else (int(rows[0]), int(rows[1]))
    a = torch.empty((b1 - b0, n), dtype=torch.float32, device=device)
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        lo, hi = max(r0, b0), min(r1, b1)
        nz = noise * torch.randn((r1 - r0, n), generator=g, device=device, dtype=torch.float32) if noise else None
        if lo >= hi:
            continue
        blk = us[lo:hi] @ vt
        if nz is not None:
            blk += nz[lo - r0:hi - r0]
        a[lo - b0:hi - b0] = blk
    return a


def power_law_65536(device="cuda"):
    """65536^2 FP32, s_i = (i+1)^-1.5 over 512 modes, noise 1e-6; 64 x 64
    grid of 1024^2 blocks, k = 128."""
    s = (np.arange(512) + 1.0) ** -1.5
    return planted_device(65536, 65536, s, noise=1e-6, tag=5, device=device), \
        dict(block_rows=1024, block_cols=1024, k=128, s=s)


def pod_fourier_device(m: int = 32768, n: int = 16384, modes: int = 40, noise: float = 1e-3,
                       tag: int = 3, device="cuda", chunk_rows: int = 4096, stats=None,
                       keep_rounding: bool = False):
    """pod_fourier on the device, BF16 storage; also returns the coefficient
    matrix C (modes x n, FP64 on the host), whose singular values are those of
    the noise-free part (the modes are orthonormal).  stats (a dict), if
    given, receives the Frobenius norm of the BF16 storage rounding and, with
    keep_rounding, the rounding itself (stored BF16 value minus the FP32
    snapshot, m x n FP32 on the device) under "rounding"."""
    import torch
    g = _torch_gen(tag, device)
    xg = torch.arange(m, dtype=torch.float64, device=device) / m
    phi = torch.empty((m, modes), dtype=torch.float64, device=device)
    for j in range(modes):
        q = j // 2 + 1
        phi[:, j] = torch.cos(2 * np.pi * q * xg) if j % 2 == 0 else torch.sin(2 * np.pi * q * xg)
    phi /= torch.linalg.norm(phi, dim=0, keepdim=True)
    c = torch.randn((modes, n), generator=g, device=device, dtype=torch.float64)
    c /= (torch.arange(1, modes + 1, dtype=torch.float64, device=device) ** 2)[:, None]
    phif, cf = phi.to(torch.float32), c.to(torch.float32)
    a = torch.empty((m, n), dtype=torch.bfloat16, device=device)
    rounding2 = 0.0
    rnd = torch.empty((m, n), dtype=torch.float32, device=device) if keep_rounding else None
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        blk = phif[r0:r1] @ cf
        blk += noise * torch.randn((r1 - r0, n), generator=g, device=device, dtype=torch.float32)
        a[r0:r1] = blk.to(torch.bfloat16)
        d = a[r0:r1].float() - blk
        rounding2 += float((d.double() ** 2).sum())
        if rnd is not None:
            rnd[r0:r1] = d
    if stats is not None:
        stats["rounding_fro"] = rounding2 ** 0.5
        if rnd is not None:
            stats["rounding"] = rnd
    return a, c.cpu().numpy()


def ragged_batch_device(count: int = 256, tag: int = 4, device="cuda", noise: float = 1e-4):
    """The many-matrix batch on the device: sizes from ragged_sizes, each
    matrix planted with s_i = exp(-i/r) / r; returns (matrices, sizes)."""
    sizes = ragged_sizes(count, tag=tag)
    mats = []
    for i, (m, n, r) in enumerate(sizes):
        s = np.exp(-np.arange(r) / r) / r
        mats.append(planted_device(m, n, s, noise=noise, tag=10000 + 7 * tag + i, device=device))
    return mats, sizes
