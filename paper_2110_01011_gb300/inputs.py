"""Seeded synthetic inputs for Rand-QLP: test matrices A and Gaussian test matrices Omega.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle's
tests. It holds none of the factorisation's arithmetic: it only draws random
numbers (numpy's Philox-4x32 counter-based generator, Salmon et al. 2011) and
assembles A = U diag(sigma) V^T + noise from them.

Workload families (the paper's own test data, section 5.2, and the configured
workloads of this library):

* ``omega``: standard Gaussian Omega, m x d (the paper draws it m x n, section
  3.1; the truncated chain draws d = k + p columns).
* ``step_spectrum``: sigma_i = 1 for i <= k, then 0.1^(i-k) (1000 x 1000, k=20).
* ``exp_spectrum``: sigma_i = exp(-i / rate) (20000^2 workload, rate 50).
* ``poly_spectrum``: sigma_i = i^(-alpha) (accuracy stress, alpha 1.5).
* ``low_rank_plus_noise`` etc.: the four families of section 5.2.

Haar-distributed orthonormal factors are the Q factor of a Gaussian matrix
with the column signs fixed by sign(diag(R)) (Mezzadri 2007); that QR is a
LAPACK call (numpy), never this library's code.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng", "omega", "round_to_bf16", "haar_columns", "step_spectrum",
    "exp_spectrum", "poly_spectrum", "low_rank_matrix", "low_rank_matrix_torch",
    "omega_torch", "Problem", "random_batch", "e3_spectrum", "SPARSE_SIZES", "sparse_matrix",
    "csr_to_dense",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox-4x32 stream for ``seed`` (platform independent)."""
    return np.random.Generator(np.random.Philox(int(seed)))


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16-representable FP32 value.

    IEEE round-to-nearest-even on the upper 16 bits of the binary32 pattern.
    Used to make Omega exactly representable in BF16 so that its low part in a
    hi + lo split is zero.
    """
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def omega(m: int, d: int, seed: int, bf16_exact: bool = False) -> np.ndarray:
    """Standard Gaussian test matrix Omega (m x d, FP32, row-major)."""
    w = rng(seed).standard_normal((m, d), dtype=np.float64).astype(np.float32)
    if bf16_exact:
        w = round_to_bf16(w)
    return np.ascontiguousarray(w)


def haar_columns(n: int, r: int, g: np.random.Generator) -> np.ndarray:
    """n x r matrix with Haar-distributed orthonormal columns (FP64).

    The Q factor (positive-diagonal R) of an n x r Gaussian. Large tall draws
    (n >= 4 r, n r >= 4e6) are well conditioned (kappa <= ~3), so Q comes from
    the Cholesky factor of G^T G (LAPACK potrf + trsm) instead of a slower
    Householder QR; both give the same Q up to rounding.
    """
    G = g.standard_normal((n, r))
    if n >= 4 * r and n * r >= 4_000_000:
        import scipy.linalg as sla
        Rc = np.linalg.cholesky(G.T @ G).T
        return sla.solve_triangular(Rc, G.T, trans="T", lower=False).T
    Qh, Rh = np.linalg.qr(G)
    s = np.sign(np.diag(Rh))
    s[s == 0] = 1.0
    return Qh * s


def step_spectrum(n: int, k: int = 20, tail: float = 0.1) -> np.ndarray:
    """sigma_i = 1 for i <= k and tail^(i-k) after (1-based i)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.where(i <= k, 1.0, tail ** np.maximum(i - k, 0))


def exp_spectrum(n: int, rate: float = 50.0) -> np.ndarray:
    """sigma_i = exp(-i / rate) (1-based i)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.exp(-i / rate)


def poly_spectrum(n: int, alpha: float = 1.5) -> np.ndarray:
    """sigma_i = i^(-alpha) (1-based i)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return i ** (-alpha)


def e3_spectrum(name: str, n: int = 1000, k: int = 200) -> np.ndarray:
    """The singular-value families of section 5.2 (n = 1000 in the paper).

    'plus_noise': linear-in-log decay from 1 to 1e-20 over i <= k, zero after
    (the Gaussian noise term is added by ``low_rank_matrix``); 'fast': i^-2;
    's_shaped': about 1, a fast drop, then a floor at 0.01; 'slow': ones for
    i <= 100 then 2^-1, 3^-1, ...
    """
    i = np.arange(1, n + 1, dtype=np.float64)
    if name == "plus_noise":
        s = np.zeros(n)
        s[:k] = np.logspace(0, -20, k)
        return s
    if name == "fast":
        return i ** -2.0
    if name == "s_shaped":
        return 0.01 + 0.99 / (1.0 + np.exp((i - n / 10.0) / (n / 100.0)))
    if name == "slow":
        kk = 100
        s = np.ones(n)
        s[kk:] = 1.0 / np.arange(2, n - kk + 2)
        return s
    raise ValueError(name)


def low_rank_matrix(m: int, n: int, sigma: np.ndarray, noise: float, seed: int,
                    rank: int | None = None, dtype=np.float32) -> np.ndarray:
    """A = U_r diag(sigma_1..r) V_r^T + noise * G / sqrt(n)  (host, numpy).

    U_r, V_r Haar (m x r, n x r); G standard Gaussian m x n. ``rank`` defaults
    to min(m, n, len(sigma)).
    """
    g = rng(seed)
    r = min(m, n, len(sigma)) if rank is None else int(rank)
    U = haar_columns(m, r, g)
    V = haar_columns(n, r, g)
    A = (U * sigma[:r]) @ V.T
    if noise:
        A += (noise / math.sqrt(n)) * g.standard_normal((m, n))
    return np.ascontiguousarray(A.astype(dtype))


def low_rank_matrix_torch(m: int, n: int, sigma: np.ndarray, noise: float, seed: int,
                          rank: int, device="cuda"):
    """Same family as ``low_rank_matrix`` assembled on a device (FP32 out).

    For the 20000 x 20000 class the host product is too slow: U_r and V_r are
    drawn on the host (Philox, LAPACK QR) and the product U_r diag(sigma) V_r^T
    is one FP32 matmul on the device (TF32 disabled); the Gaussian noise is
    drawn by torch's seeded device generator.
    """
    import torch
    g = rng(seed)
    U = haar_columns(m, rank, g) * np.asarray(sigma[:rank], dtype=np.float64)
    V = haar_columns(n, rank, g)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        Ud = torch.from_numpy(U.astype(np.float32)).to(device)
        Vd = torch.from_numpy(V.astype(np.float32)).to(device)
        A = Ud @ Vd.T
        del Ud, Vd
        if noise:
            gen = torch.Generator(device=device)
            gen.manual_seed(int(seed))
            A.add_(torch.randn(m, n, generator=gen, device=device, dtype=torch.float32),
                   alpha=noise / math.sqrt(n))
        return A.contiguous()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def low_rank_matrix_reflect(m: int, n: int, sigma: np.ndarray, seed: int, device="cuda", reflectors: int = 4):
    """A = U diag(sigma) V^T (FP32, on ``device``) with U, V the first
    r = min(m, n) columns of products of ``reflectors`` random Householder
    reflectors: exactly orthonormal, dense, and built from elementwise ops and
    one matmul only (no device QR). A Gaussian Omega is rotation invariant,
    so the sketch's error law depends on sigma alone; these matrices stand in
    for Haar ones where many large matrices are needed quickly."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    r = min(m, n)

    def basis(rows):
        X = torch.zeros(rows, r, device=device, dtype=torch.float32)
        X.diagonal().fill_(1.0)
        for _ in range(reflectors):
            v = torch.randn(rows, generator=gen, device=device, dtype=torch.float32)
            v /= torch.sqrt((v * v).sum())
            X -= 2.0 * torch.outer(v, v @ X)
        return X

    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        U = basis(m) * torch.as_tensor(np.asarray(sigma[:r], dtype=np.float32), device=device)
        return (U @ basis(n).T).contiguous()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def omega_torch(m: int, d: int, seed: int, device="cuda", bf16_exact: bool = False):
    """Gaussian Omega drawn on the host (``omega``) and copied to ``device``."""
    import torch
    return torch.from_numpy(omega(m, d, seed, bf16_exact)).to(device)


@dataclass
class Problem:
    """One matrix of a batched workload (sizes and spectrum recipe)."""
    m: int
    n: int
    k: int
    p: int
    q: int
    kind: str        # "exp" or "poly"
    param: float     # rate for "exp", alpha for "poly"
    seed: int

    @property
    def d(self) -> int:
        return self.k + self.p

    def sigma(self) -> np.ndarray:
        r = min(self.m, self.n)
        if self.kind == "exp":
            return exp_spectrum(r, self.param)
        return poly_spectrum(r, self.param)


def random_batch(count: int, seed: int, m_range=(256, 4096), n_range=(256, 2048),
                 k_range=(8, 64), p: int = 5, q: int = 1) -> list[Problem]:
    """Uneven batch: m, n, k uniform in the given ranges; half exponential
    spectra (rate uniform in [5, 100]) and half polynomial (alpha in [0.5, 3])."""
    g = rng(seed)
    out = []
    for t in range(count):
        m = int(g.integers(m_range[0], m_range[1] + 1))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        k = int(g.integers(k_range[0], k_range[1] + 1))
        k = min(k, min(m, n) - p)
        if t % 2 == 0:
            kind, par = "exp", float(g.uniform(5.0, 100.0))
        else:
            kind, par = "poly", float(g.uniform(0.5, 3.0))
        out.append(Problem(m, n, k, p, q, kind, par, seed * 100003 + t))
    return out


# Square sizes of the sparse test matrices of section 5.1 (Table 1); the
# matrices themselves are not available here, so seeded stand-ins of those
# sizes take their place (``sparse_matrix``).
SPARSE_SIZES = (1856, 2904, 4929, 6747, 7320)


def sparse_matrix(m: int, n: int, seed: int, band: int = 2, extra: int = 8):
    """Seeded sparse stand-in in CSR form: a band |i - j| <= band (clipped to
    the matrix) plus ``extra`` uniformly random columns per row, standard
    normal values, rows sorted by column, no duplicates. Returns (row_ptr
    int64 (m + 1), col_idx int32, vals float32)."""
    g = rng(seed)
    rows, cols = [], []
    for i in range(m):
        c = set(range(max(0, i - band), min(n, i + band + 1)))
        c.update(int(x) for x in g.integers(0, n, size=extra))
        c = sorted(c)
        rows.append(len(c))
        cols.extend(c)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(rows)
    col_idx = np.asarray(cols, dtype=np.int32)
    vals = g.standard_normal(col_idx.size).astype(np.float32)
    return row_ptr, col_idx, vals


def csr_to_dense(m: int, n: int, row_ptr, col_idx, vals) -> np.ndarray:
    """The dense m x n FP64 matrix of a CSR triple (for the oracle)."""
    A = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        s, e = int(row_ptr[i]), int(row_ptr[i + 1])
        A[i, col_idx[s:e]] = vals[s:e]
    return A
