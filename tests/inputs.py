"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: only random-number draws and parameter grids.
Ising inputs need no randomness (they are fixed by d, beta, h, Dcut); random tensors are used
where a test needs generic (non-degenerate) spectra.
"""
import numpy as np


def random_site_tensor(dims, seed: int) -> np.ndarray:
    """Gaussian rank-2d tensor with legs [u_0..u_{d-1}, p_0..p_{d-1}] of the given dims."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(tuple(dims) * 2)


def random_matrix(m: int, n: int, seed: int, scale_spread: float = 0.0) -> np.ndarray:
    """Gaussian m x n matrix; with scale_spread > 0 each entry is multiplied by
    10**uniform(-spread, spread) to exercise a wide exponent range."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    if scale_spread > 0:
        A *= 10.0 ** rng.uniform(-scale_spread, scale_spread, size=(m, n))
    return A


def random_symmetric_psd(n: int, seed: int, rank: int | None = None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, rank or n))
    return X @ X.T


def beta_scan(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n)


def random_z2_site_tensor(dims, evens, seed: int) -> np.ndarray:
    """Gaussian rank-2d tensor with the zero-field (spin-flip) block structure: the values of leg
    b are ordered even-parity first, evens[b] of them even, and every entry whose legs' parities
    add up to odd is set to zero."""
    T = random_site_tensor(dims, seed)
    d = len(dims)
    par = np.zeros(T.shape, dtype=int)
    for axis in range(2 * d):
        b = axis % d
        p = (np.arange(dims[b]) >= evens[b]).astype(int)
        shape = [1] * (2 * d)
        shape[axis] = dims[b]
        par = par ^ p.reshape(shape)
    T[par == 1] = 0.0
    return T
