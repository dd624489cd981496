"""Seeded synthetic inputs for block orthogonalization.

This module only draws random matrices with a prescribed singular spectrum;
it holds none of the orthogonalization arithmetic (no Gram product, no
Cholesky, no eigensolver of the method).  Both the CUDA path's tests and the
CPU oracle take their inputs from here.

Recipe (the paper tests on synthetic matrices over a range of condition
numbers, Sec. 4.2, one-iteration accuracy figure; it does not give the
generator):

* Haar-random orthonormal factors: a standard-normal matrix from
  ``numpy.random.Generator(PCG64(seed))``, its Householder QR
  (``numpy.linalg.qr``), and each column multiplied by the sign of the
  corresponding diagonal entry of R.
* X = U diag(sigma) W^T with U (n-by-k) and W (k-by-k) Haar-random and sigma
  log-spaced from 1 down to 1/kappa; for k = 1, sigma = [1].
* All matrices are FP64, column-major (numpy Fortran order), leading
  dimension n.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20180604


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar(g: np.random.Generator, n: int, k: int) -> np.ndarray:
    """n-by-k matrix with orthonormal columns, Haar-distributed (n >= k)."""
    a = g.standard_normal((n, k))
    q, r = np.linalg.qr(a)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.asfortranarray(q * s)


def logspace_sigma(k: int, kappa: float) -> np.ndarray:
    if k == 1:
        return np.ones(1)
    return np.logspace(0.0, -np.log10(kappa), k)


def conditioned(n: int, k: int, kappa: float, seed: int, sigma: np.ndarray | None = None) -> np.ndarray:
    """X = U diag(sigma) W^T with sigma log-spaced 1 .. 1/kappa (column-major FP64)."""
    g = rng(seed)
    u = haar(g, n, k)
    w = haar(g, k, k)
    s = logspace_sigma(k, kappa) if sigma is None else np.asarray(sigma, dtype=np.float64)
    return np.asfortranarray((u * s) @ w.T)


def gaussian(n: int, k: int, seed: int) -> np.ndarray:
    return np.asfortranarray(rng(seed).standard_normal((n, k)))


def hadamard_basis(n: int, k: int, seed: int) -> np.ndarray:
    """n-by-k basis that is orthonormal exactly in FP64.

    Columns of the Sylvester-Hadamard matrix (entries (-1)^popcount(i & j)),
    scaled by 1/sqrt(n), which is a power of two when n is a power of 4; the
    rows are permuted and sign-flipped at random (seeded), which keeps every
    entry exact and the columns exactly orthonormal."""
    if n & (n - 1) or (n.bit_length() - 1) % 2:
        raise ValueError("n must be a power of 4")
    if k > n:
        raise ValueError("k must not exceed n")
    g = rng(seed)
    cols = g.choice(n, size=k, replace=False)
    i = np.arange(n)[:, None]
    pc = np.vectorize(lambda v: bin(int(v)).count("1") & 1)(i & cols[None, :])
    h = np.where(pc == 1, -1.0, 1.0) / np.sqrt(float(n))
    perm = g.permutation(n)
    signs = np.where(g.random(n) < 0.5, -1.0, 1.0)
    return np.asfortranarray(h[perm] * signs[:, None])


def orthonormal_basis(n: int, k: int, seed: int) -> np.ndarray:
    """Orthonormal n-by-k basis V (Householder QR of a seeded Gaussian)."""
    return haar(rng(seed), n, k)


def with_ld(a: np.ndarray, ld: int, fill: float = np.nan) -> np.ndarray:
    """Copy of the column-major matrix a stored with leading dimension ld >= rows.

    Returns the full (ld, cols) buffer; the padding rows hold `fill`."""
    n, k = a.shape
    assert ld >= n
    buf = np.full((ld, k), fill, dtype=a.dtype, order="F")
    buf[:n, :] = a
    return buf


# ---------------------------------------------------------------- workloads

def single_cholqr(seed: int = SEED_BASE + 0, n: int = 100_000, k: int = 8, kappa: float = 1e6) -> np.ndarray:
    """Single CholQR block: n-by-k FP64, sigma log-spaced 1 .. 1e-6."""
    return conditioned(n, k, kappa, seed)


def project_block(seed: int = SEED_BASE + 1, n: int = 4_000_000, kv: int = 64, k: int = 16,
                  kappa: float = 1e10) -> tuple[np.ndarray, np.ndarray]:
    """Projection workload: orthonormal V (n-by-kv) and Y (n-by-k), sigma 1 .. 1e-10."""
    v = orthonormal_basis(n, kv, seed)
    y = conditioned(n, k, kappa, seed + 1000)
    return v, y


def near_span(v: np.ndarray, k: int, kappa_xw: float, seed: int, kappa: float = 1.0) -> np.ndarray:
    """Block X whose component outside span(V) is 1/kappa_xw of its size.

    X = V A + B / kappa_xw with A a seeded Gaussian kv-by-k and B a
    conditioned n-by-k block (condition kappa); kappa(X, W) in the sense of
    the paper's accuracy figure grows with kappa_xw."""
    n, kv = v.shape
    g = rng(seed)
    a = g.standard_normal((kv, k))
    b = conditioned(n, k, kappa, seed + 1)
    return np.asfortranarray(v @ a + b / kappa_xw)
