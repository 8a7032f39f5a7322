"""Seeded synthetic inputs shaped like the paper's workloads.

This module generates inputs only; it holds none of the factorisation's
arithmetic.  Both the CUDA path's tests/benchmark and the CPU oracle draw
their inputs from here.

Test matrices (Sec. 4.1 of the paper): A = U diag(s) V^T with U (m x n) and
V (n x n) random orthonormal factors of seeded Gaussian matrices and
singular values s_i log-spaced between 1 and kappa.  The paper prints them
from 1 up to kappa (||A||_2 = kappa); by default they run from 1 down to
1/kappa (||A||_2 = 1), the same matrix divided by kappa up to rounding.
The methods are invariant under that scaling (their shifts scale with the
Gramian they factor) except isCholQR, which reuses the shift of the first
Gramian, of norm ||A||^2, on later Gramians of norm about 1: the Fig. 1
reproduction takes the paper's scale (paper_scale=True).  The paper varies
the seed with the dimensions and the condition number; here the seed is a
splitmix64 hash of (m, n, round(log10 kappa), rep, salt).

Update blocks (basis growth): block_k = Q_prev G 0.1 + N eta with G (q x p)
and N (m x p) Gaussian and eta log-uniform in [1e-12, 1]; the first block
(q = 0) is plain Gaussian N.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One step of the splitmix64 mixer (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _MASK
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def seed_for(*parts: int) -> int:
    h = 0x243F6A8885A308D3
    for p in parts:
        h = splitmix64(h ^ (int(p) & _MASK))
    return h


def _orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    # fix signs so the factor does not depend on LAPACK's sign convention
    q = q * np.sign(np.where(np.diag(r) == 0, 1.0, np.diag(r)))
    return q


def singular_values(n: int, kappa: float) -> np.ndarray:
    """log-spaced 1 -> 1/kappa (Sec. 4.1 up to the factor kappa)."""
    if n == 1:
        return np.ones(1)
    return np.logspace(0.0, -math.log10(kappa), n)


def test_matrix(m: int, n: int, kappa: float, rep: int = 0, salt: int = 0,
                paper_scale: bool = False) -> np.ndarray:
    """A = U diag(s) V^T, column-major float64 (m x n); with paper_scale the
    singular values run from 1 up to kappa (Sec. 4.1), else from 1 down to
    1/kappa."""
    rng = np.random.default_rng(seed_for(m, n, round(math.log10(max(kappa, 1.0))), rep, salt))
    U = _orthonormal(rng, m, n)
    V = _orthonormal(rng, n, n)
    s = singular_values(n, kappa)
    if paper_scale:
        s = s * kappa
    return np.asfortranarray((U * s) @ V.T)


def orthonormal(m: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed_for(m, n, seed, 0x0F))
    return np.asfortranarray(_orthonormal(rng, m, n))


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed_for(m, n, seed, 0x6A))
    return np.asfortranarray(rng.standard_normal((m, n)))


def update_block(Q_prev: np.ndarray | None, m: int, p: int, k: int, seed: int = 0):
    """Block k of a basis-growth run: Q_prev G 0.1 + N eta (Q_prev may be None).

    Returns (block, eta)."""
    rng = np.random.default_rng(seed_for(m, p, k, seed, 0xB1))
    N = rng.standard_normal((m, p))
    if Q_prev is None or Q_prev.shape[1] == 0:
        return np.asfortranarray(N), 1.0
    q = Q_prev.shape[1]
    G = rng.standard_normal((q, p))
    eta = 10.0 ** rng.uniform(-12.0, 0.0)
    return np.asfortranarray(Q_prev @ G * 0.1 + N * eta), float(eta)


def basis_growth_blocks(m: int, p: int, count: int, seed: int = 0):
    """Blocks 0..count-1 of a basis-growth run for tests: block k is
    update_block(Q_prev, ...) with Q_prev an orthonormal basis (LAPACK QR,
    used here only as a data generator) of blocks 0..k-1.
    Returns (blocks, etas)."""
    blocks, etas = [], []
    Qp = None
    for k in range(count):
        b, eta = update_block(Qp, m, p, k, seed)
        blocks.append(b)
        etas.append(eta)
        Qp, _ = np.linalg.qr(np.hstack(blocks))
    return blocks, etas
