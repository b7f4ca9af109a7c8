"""Seeded synthetic inputs for Gauss-Jordan inversion.

This module holds only random-number generation and matrix assembly; it contains
none of the inversion's arithmetic, so both the CPU oracle (tests) and the CUDA
path (tests, benchmark) can draw their inputs from it.

All generators use ``numpy.random.Generator(PCG64(seed))`` and return
column-major (Fortran-ordered) float64 arrays unless stated otherwise.

Workload shapes:
  * the paper's worked example (Section 3, the program's default array ``c``);
  * one n x n matrix with i.i.d. N(0,1) entries (128 x 128 for the full-pivoting case);
  * one large n x n matrix N(0,1) + 0.1 n I (8192 x 8192, partial pivoting, blocked);
  * a batch of matrices with orders drawn uniformly from 4..64, entries U[-1,1],
    each diagonal entry set to 1 + sum of the absolute off-diagonal entries of its row;
  * U diag(sigma) V^T with Haar U, V and log-spaced sigma (mixed precision);
  * a batch of such matrices, orders uniform in 128..1024, condition numbers
    log-uniform in [1e2, 1e8] (batched mixed precision).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1401


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def paper_example() -> np.ndarray:
    """The default 3x3 matrix of the paper's program (Section 3, array c)."""
    return np.asfortranarray(np.array([[1.0, 1.0, 1.0], [1.0, 2.0, 3.0], [1.0, 3.0, 6.0]]))


def gaussian(n: int, seed: int, shift: float = 0.0) -> np.ndarray:
    """n x n i.i.d. N(0,1) entries plus ``shift`` on the diagonal, column-major float64."""
    g = rng(seed)
    # draw column by column in storage order so a prefix of columns is seed-stable
    A = g.standard_normal((n, n)).T.copy(order="F") if n > 0 else np.zeros((0, 0), order="F")
    A = np.asfortranarray(A)
    if shift != 0.0 and n > 0:
        A[np.arange(n), np.arange(n)] += shift
    return A


def diag_dominant_batch(count: int, seed: int, n_min: int = 4, n_max: int = 64):
    """Batch of diagonally dominant matrices with uneven orders.

    Orders are drawn uniformly from ``n_min..n_max`` (inclusive); entries are
    U[-1,1]; each diagonal entry is then 1 + sum_{j != i} |a_ij| over its row.
    Returns ``(sizes[int32], packed[float64], offsets[int64])``: matrix m occupies
    ``packed[offsets[m] : offsets[m] + sizes[m]**2]`` in column-major order.
    """
    g = rng(seed)
    sizes = g.integers(n_min, n_max + 1, size=count, dtype=np.int64).astype(np.int32)
    sq = sizes.astype(np.int64) ** 2
    offsets = np.zeros(count, dtype=np.int64)
    if count > 1:
        offsets[1:] = np.cumsum(sq)[:-1]
    packed = np.empty(int(sq.sum()), dtype=np.float64)
    for n in range(n_min, n_max + 1):
        idx = np.nonzero(sizes == n)[0]
        if idx.size == 0:
            continue
        M = g.uniform(-1.0, 1.0, size=(idx.size, n, n))  # M[m, i, j]
        off = M.copy()
        off[:, np.arange(n), np.arange(n)] = 0.0
        M[:, np.arange(n), np.arange(n)] = 1.0 + np.abs(off).sum(axis=2)
        # column-major per matrix: element (i, j) at i + j n  ->  transpose to [m, j, i]
        flat = np.ascontiguousarray(M.transpose(0, 2, 1)).reshape(idx.size, n * n)
        dst = offsets[idx][:, None] + np.arange(n * n)[None, :]
        packed[dst] = flat
    return sizes, packed, offsets


def unpack(sizes: np.ndarray, packed: np.ndarray, offsets: np.ndarray, m: int) -> np.ndarray:
    """Matrix m of a packed batch as an (n, n) column-major array (a view)."""
    n = int(sizes[m])
    return packed[offsets[m]: offsets[m] + n * n].reshape(n, n, order="F")


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of an N(0,1) matrix, columns sign-fixed by diag(R)."""
    Z = g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def svd_conditioned(n: int, kappa: float, seed: int, dtype=np.float32) -> np.ndarray:
    """A = U diag(sigma) V^T, U and V Haar, sigma log-spaced from 1 to kappa, stored as ``dtype``."""
    g = rng(seed)
    U = haar_orthogonal(n, g)
    V = haar_orthogonal(n, g)
    sigma = np.logspace(0.0, np.log10(kappa), n) if n > 1 else np.ones(n)
    A = (U * sigma[None, :]) @ V.T
    return np.asfortranarray(A.astype(dtype))


def svd_conditioned_device(n: int, kappa: float, seed: int, device="cuda"):
    """U diag(sigma) V^T on the GPU in FP32 (torch): U, V Haar (QR of a seeded N(0,1) matrix,
    columns sign-fixed by diag(R)), sigma log-spaced from 1 to kappa.  Column-major
    (Fortran-ordered) FP32 tensor.  For sizes where a host QR would take minutes."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def haar():
        Z = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
        Q, R = torch.linalg.qr(Z)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1.0
        return Q * d[None, :]

    U = haar()
    V = haar()
    sigma = torch.logspace(0.0, float(np.log10(kappa)), n, device=device, dtype=torch.float32)
    A = (U * sigma[None, :]) @ V.T
    return A.t().contiguous().t()


def mixed_batch_params(count: int, seed: int, n_min: int = 128, n_max: int = 1024, kappa_min: float = 1e2,
                       kappa_max: float = 1e8):
    """Orders uniform in ``n_min..n_max`` (inclusive) and condition numbers log-uniform in
    ``[kappa_min, kappa_max]`` for a batch of U diag(sigma) V^T matrices.  Returns
    ``(sizes[int32], kappas[float64], offsets[int64])``; matrix m occupies
    ``offsets[m] : offsets[m] + sizes[m]**2`` of a packed column-major buffer."""
    g = rng(seed)
    sizes = g.integers(n_min, n_max + 1, size=count, dtype=np.int64).astype(np.int32)
    kappas = 10.0 ** g.uniform(np.log10(kappa_min), np.log10(kappa_max), size=count)
    sq = sizes.astype(np.int64) ** 2
    offsets = np.zeros(count, dtype=np.int64)
    if count > 1:
        offsets[1:] = np.cumsum(sq)[:-1]
    return sizes, kappas, offsets


def mixed_batch_seed(seed: int, m: int) -> int:
    """Seed of matrix m of a mixed batch drawn with ``seed``."""
    return seed * 100003 + m


def mixed_batch_host(sizes: np.ndarray, kappas: np.ndarray, offsets: np.ndarray, seed: int) -> np.ndarray:
    """Packed FP32 buffer of the batch: matrix m is ``svd_conditioned`` of its order and kappa
    with seed ``mixed_batch_seed(seed, m)``."""
    total = int(offsets[-1] + int(sizes[-1]) ** 2) if len(sizes) else 0
    packed = np.empty(total, dtype=np.float32)
    for m, (n, k) in enumerate(zip(sizes, kappas)):
        n = int(n)
        A = svd_conditioned(n, float(k), mixed_batch_seed(seed, m), dtype=np.float32)
        packed[offsets[m]: offsets[m] + n * n] = A.reshape(-1, order="F")
    return packed


def mixed_batch_device(sizes: np.ndarray, kappas: np.ndarray, offsets: np.ndarray, seed: int, device="cuda"):
    """Packed FP32 device buffer of the batch: matrix m is ``svd_conditioned_device`` of its
    order and kappa with seed ``mixed_batch_seed(seed, m)`` (the GPU's generator, so not the
    same numbers as ``mixed_batch_host``)."""
    import torch
    total = int(offsets[-1] + int(sizes[-1]) ** 2) if len(sizes) else 0
    flat = torch.empty(total, dtype=torch.float32, device=device)
    for m, (n, k) in enumerate(zip(sizes, kappas)):
        n = int(n)
        A = svd_conditioned_device(n, float(k), mixed_batch_seed(seed, m), device=device)
        matrix_view(flat, n, int(offsets[m])).copy_(A)
    return flat


def matrix_view(flat, n: int, offset: int):
    """Column-major (n, n) view of ``flat[offset : offset + n * n]`` (torch tensor)."""
    return flat[offset: offset + n * n].view(n, n).t()
