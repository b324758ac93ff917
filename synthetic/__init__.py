"""Seeded synthetic inputs for rand_cholQR tests, smoke and bench.

This module is shared by the CPU oracle's tests and the CUDA path's tests and holds none
of the method's arithmetic: it only draws random numbers and calls library routines
(numpy / torch QR) to build test matrices.

Workload recipe (the paper's Sec. 6.3 construction, with the sigma range of the
benchmarked configurations): V = U diag(sigma) W^T, with U (m x n) and W (n x n) the
orthonormal factors of seeded N(0, 1) matrices and sigma_j = kappa^{-j/(n-1)}, log-spaced
from 1 down to 1/kappa, so kappa(V) = kappa and ||V||_2 = 1.  The paper's own scaling
([kappa^-1/2, kappa^1/2]) differs only by the factor kappa^1/2, which every relative
error measure ignores.
"""
import math

import numpy as np

__all__ = ["sigmas", "make_v", "make_v_torch", "make_v_block_torch", "integer_matrix", "default_sketch_sizes",
           "paper_multisketch_sizes", "paper_single_sketch_sizes", "rng"]


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Counter-based numpy generator (Philox4x64) for (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=np.array([seed & (2**64 - 1), stream],
                                                              dtype=np.uint64)))


def sigmas(n: int, kappa: float) -> np.ndarray:
    if n == 1:
        return np.ones(1)
    j = np.arange(n, dtype=np.float64)
    return kappa ** (-j / (n - 1))


def make_v(m: int, n: int, kappa: float, seed: int = 0) -> np.ndarray:
    """V = U diag(sigma) W^T (row-major float64, m x n) with kappa(V) = kappa."""
    G = rng(seed, 0).standard_normal((m, n))
    U, _ = np.linalg.qr(G)
    H = rng(seed, 2).standard_normal((n, n))
    W, _ = np.linalg.qr(H)
    return np.ascontiguousarray((U * sigmas(n, kappa)) @ W.T)


def make_v_torch(m: int, n: int, kappa: float, seed: int = 0, device="cuda"):
    """Same recipe drawn with torch on `device` (for sizes where a host QR is slow).

    Uses torch's generator and QR (library routines); the result is an input only."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 17)
    G = torch.randn((m, n), generator=g, device=device, dtype=torch.float64)
    U, _ = torch.linalg.qr(G)
    del G
    H = torch.randn((n, n), generator=g, device=device, dtype=torch.float64)
    W, _ = torch.linalg.qr(H)
    s = torch.as_tensor(sigmas(n, kappa), device=device, dtype=torch.float64)
    U.mul_(s)
    return (U @ W.T).contiguous()


def make_v_block_torch(m: int, n: int, kappa: float, shard: int, shards: int, seed: int = 0,
                       device="cuda"):
    """Rows [shard m, (shard + 1) m) of an (shards m) x n matrix V = U diag(sigma) W^T with
    kappa(V) = kappa, drawn without the other blocks: U = [U_0; ...; U_{P-1}] / sqrt(P) with
    each U_k the orthonormal factor of its own seeded N(0, 1) block (so U^T U = I), and W
    common to all blocks.  With shards = 1 this is another draw of the same recipe."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 7919 * (shard + 1))
    G = torch.randn((m, n), generator=g, device=device, dtype=torch.float64)
    U, _ = torch.linalg.qr(G)
    del G
    gw = torch.Generator(device=device)
    gw.manual_seed(int(seed) * 1000003 + 5)
    H = torch.randn((n, n), generator=gw, device=device, dtype=torch.float64)
    W, _ = torch.linalg.qr(H)
    s = torch.as_tensor(sigmas(n, kappa) / math.sqrt(shards), device=device, dtype=torch.float64)
    U.mul_(s)
    return (U @ W.T).contiguous()


def integer_matrix(m: int, n: int, bound: int = 2**20, seed: int = 0) -> np.ndarray:
    """Integer-valued float64 matrix with entries in [-bound, bound]: every sum of a few
    million such entries is exact in FP64, whatever the order."""
    return rng(seed, 5).integers(-bound, bound + 1, size=(m, n)).astype(np.float64)


def default_sketch_sizes(n: int):
    """(s1, s2) = (2 (n^2 + n), 4 n): the sketch sizes of the benchmarked configurations."""
    return 2 * (n * n + n), 4 * n


def paper_multisketch_sizes(n: int):
    """The paper's multisketch sizes (Sec. 6.2): p1 = ceil(8.24 (n^2 + n)) for a CountSketch
    with eps1 = 0.9, p2 = ceil(74.3 ln p1) for a Gaussian with eps2 = 0.49 (natural log)."""
    p1 = math.ceil(8.24 * (n * n + n))
    p2 = math.ceil(74.3 * math.log(p1))
    return p1, p2


def paper_single_sketch_sizes(n: int):
    """The paper's single-sketch sizes (Sec. 6.2): a CountSketch alone with ceil(6.8 (n^2 + n))
    rows, a Gaussian alone with ceil(36.01 ln n) rows (natural log; at least n)."""
    return math.ceil(6.8 * (n * n + n)), max(n, math.ceil(36.01 * math.log(n)))
