"""Independent exact references that pin the HOTRG oracle (arXiv:1906.06060, Sec. 2).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg and reference arm may use it.

None of these functions uses the tensor network: they evaluate the partition function of
Eq. (pf) by other means (enumeration, textbook closed forms), or restate the closed form of
T^(0). They are what a mistake in `hotrg_ref` would disagree with.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import integrate


def lnz_bruteforce(beta: float, h: float, L: tuple[int, ...]) -> float:
    """ln Z of Eq. (pf) on a periodic L_0 x ... x L_{d-1} lattice by enumerating all 2^N
    spin configurations (N <= 20).

    Bonds: one per (site i, axis a), joining i to i + e_a mod L_a. For L_a = 1 this is a
    self-bond (factor e^beta); for L_a = 2 the pair is joined twice. That is exactly what the
    periodic trace of Eq. (tTr) closes after the coarse-graining steps have merged 2^k sites.
    """
    L = tuple(int(x) for x in L)
    N = int(np.prod(L))
    if N > 20:
        raise ValueError("enumeration limited to 20 spins")
    sites = list(itertools.product(*[range(n) for n in L]))
    index = {s: i for i, s in enumerate(sites)}
    bonds = []
    for s in sites:
        for a, La in enumerate(L):
            t = list(s)
            t[a] = (t[a] + 1) % La
            bonds.append((index[s], index[tuple(t)]))
    cfg = ((np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1).astype(np.int8)
    spins = 1 - 2 * cfg.astype(np.float64)          # bit 0 -> +1, bit 1 -> -1
    i, j = np.array(bonds).T
    e_bond = np.sum(spins[:, i] * spins[:, j], axis=1)
    e_field = np.sum(spins, axis=1)
    expo = beta * e_bond + beta * h * e_field
    m = expo.max()
    return float(m + math.log(np.sum(np.exp(expo - m))))


def moments_bruteforce(beta: float, h: float, L: tuple[int, ...]) -> tuple[float, float]:
    """(<sum over bonds s_i s_j> / N, <sum over sites s_i> / N) on the same periodic lattice as
    lnz_bruteforce, by enumeration. With H = -sum_bonds s s' - h sum s these give
    d(ln Z/N)/d beta = e_bond + h m and d(ln Z/N)/d h = beta m."""
    L = tuple(int(x) for x in L)
    N = int(np.prod(L))
    if N > 20:
        raise ValueError("enumeration limited to 20 spins")
    sites = list(itertools.product(*[range(n) for n in L]))
    index = {s: i for i, s in enumerate(sites)}
    bonds = []
    for s in sites:
        for a, La in enumerate(L):
            t = list(s)
            t[a] = (t[a] + 1) % La
            bonds.append((index[s], index[tuple(t)]))
    cfg = ((np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1).astype(np.int8)
    spins = 1 - 2 * cfg.astype(np.float64)
    i, j = np.array(bonds).T
    e_bond = np.sum(spins[:, i] * spins[:, j], axis=1)
    e_field = np.sum(spins, axis=1)
    expo = beta * e_bond + beta * h * e_field
    w = np.exp(expo - expo.max())
    z = w.sum()
    return float(np.dot(w, e_bond) / z / N), float(np.dot(w, e_field) / z / N)


def pair_and_spin_bruteforce(beta: float, h: float, L: tuple[int, ...], axis: int) -> tuple[float, float]:
    """(<s_0 s_{0 + e_axis}>, <s_0>) on the same periodic lattice as lnz_bruteforce, by
    enumeration (site 0 is the origin; with L_axis = 1 the neighbour is the site itself)."""
    L = tuple(int(x) for x in L)
    N = int(np.prod(L))
    if N > 20:
        raise ValueError("enumeration limited to 20 spins")
    sites = list(itertools.product(*[range(n) for n in L]))
    index = {s: i for i, s in enumerate(sites)}
    bonds = []
    for s in sites:
        for a, La in enumerate(L):
            t = list(s)
            t[a] = (t[a] + 1) % La
            bonds.append((index[s], index[tuple(t)]))
    cfg = ((np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1).astype(np.int8)
    spins = 1 - 2 * cfg.astype(np.float64)
    i, j = np.array(bonds).T
    expo = beta * np.sum(spins[:, i] * spins[:, j], axis=1) + beta * h * np.sum(spins, axis=1)
    w = np.exp(expo - expo.max())
    o = [0] * len(L)
    nb = list(o)
    nb[axis] = 1 % L[axis]
    s0, s1 = spins[:, index[tuple(o)]], spins[:, index[tuple(nb)]]
    return float(np.dot(w, s0 * s1) / w.sum()), float(np.dot(w, s0) / w.sum())


def dlnz_1d(beta: float, h: float, N: int) -> tuple[float, float]:
    """(d/d beta, d/d h) of lnz_1d(beta, h, N) / N, differentiating the transfer-matrix
    eigenvalues: with q = (lam-/lam+)^N, d(ln Z)/N = (dlam+/lam+ + q dlam-/lam-) / (1 + q)."""
    eb = math.exp(beta)
    sh, ch = math.sinh(beta * h), math.cosh(beta * h)
    r = math.sqrt(eb * eb * sh * sh + 1.0 / (eb * eb))
    lp, lm = eb * ch + r, eb * ch - r
    # r^2 = e^{2b} sinh^2(bh) + e^{-2b}
    dr_db = (eb * eb * sh * sh + eb * eb * sh * ch * h - 1.0 / (eb * eb)) / r
    dr_dh = eb * eb * sh * ch * beta / r
    dlp_db, dlm_db = eb * ch + eb * sh * h + dr_db, eb * ch + eb * sh * h - dr_db
    dlp_dh, dlm_dh = eb * sh * beta + dr_dh, eb * sh * beta - dr_dh
    q = (lm / lp) ** N
    return ((dlp_db / lp + q * dlm_db / lm) / (1.0 + q), (dlp_dh / lp + q * dlm_dh / lm) / (1.0 + q))


def lnz_1d(beta: float, h: float, N: int) -> float:
    """ln Z of the periodic Ising chain: ln(lam+^N + lam-^N), transfer-matrix eigenvalues
    lam_pm = e^b cosh(bh) +- sqrt(e^{2b} sinh^2(bh) + e^{-2b})."""
    eb = math.exp(beta)
    r = math.sqrt(eb * eb * math.sinh(beta * h) ** 2 + 1.0 / (eb * eb))
    lp = eb * math.cosh(beta * h) + r
    lm = eb * math.cosh(beta * h) - r          # >= 0 for beta >= 0
    return N * math.log(lp) + math.log1p((lm / lp) ** N)


def x_1d(beta: float, h: float, N: int) -> float:
    """X of Eq. (x) for the periodic Ising chain of N sites. In one dimension the coarse-grained
    tensor after n steps is (up to normalisation) the site matrix to the power N = 2^n, whose
    eigenvalues are those of the transfer matrix, lam+^N and lam-^N, so with q = (lam-/lam+)^N:
        X = (Tr A)^2 / Tr A^2 = (lam+^N + lam-^N)^2 / (lam+^{2N} + lam-^{2N}) = (1 + q)^2 / (1 + q^2).
    """
    eb = math.exp(beta)
    r = math.sqrt(eb * eb * math.sinh(beta * h) ** 2 + 1.0 / (eb * eb))
    q = ((eb * math.cosh(beta * h) - r) / (eb * math.cosh(beta * h) + r)) ** N
    return (1.0 + q) ** 2 / (1.0 + q * q)


def lnz_onsager(beta: float) -> float:
    """Onsager's free energy of the 2D square-lattice Ising model at h = 0, per site:
    ln(2 cosh 2b) + (1/pi) int_0^{pi/2} ln[(1 + sqrt(1 - k^2 sin^2 t)) / 2] dt,
    k = 2 sinh 2b / cosh^2 2b."""
    k = 2.0 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    f = lambda t: math.log(0.5 * (1.0 + math.sqrt(max(0.0, 1.0 - (k * math.sin(t)) ** 2))))
    val, _ = integrate.quad(f, 0.0, 0.5 * math.pi, epsabs=1e-15, epsrel=1e-14, limit=400)
    return math.log(2.0 * math.cosh(2 * beta)) + val / math.pi


def lnz_onsager_double(beta: float) -> float:
    """The double-integral form of the same result:
    ln 2 + 1/(8 pi^2) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)] dt1 dt2 over [0, 2pi]^2."""
    c2, s2 = math.cosh(2 * beta), math.sinh(2 * beta)
    f = lambda t1, t2: math.log(c2 * c2 - s2 * (math.cos(t1) + math.cos(t2)))
    val, _ = integrate.dblquad(f, 0.0, 2 * math.pi, 0.0, 2 * math.pi, epsabs=1e-13, epsrel=1e-12)
    return math.log(2.0) + val / (8 * math.pi ** 2)


def initial_tensor_closed_form(d: int, beta: float, h: float) -> np.ndarray:
    """Closed form of T^(0): with n1 = number of legs carrying index 1,
    T = cosh^{(2d-n1)/2}(b) sinh^{n1/2}(b) * (2 cosh(bh) if n1 is even else 2 sinh(bh))."""
    T = np.empty((2,) * (2 * d))
    cb, sb = math.cosh(beta), math.sinh(beta)
    for idx in itertools.product((0, 1), repeat=2 * d):
        n1 = sum(idx)
        v = 2.0 * (math.cosh(beta * h) if n1 % 2 == 0 else math.sinh(beta * h))
        T[idx] = cb ** ((2 * d - n1) / 2) * sb ** (n1 / 2) * v
    return T


def lnz_high_temperature_4d(beta: float) -> float:
    """Leading terms of the 4D high-temperature series at h = 0:
    ln 2 + 4 ln cosh b + 6 tanh^4 b (the next term is O(tanh^6 b))."""
    return math.log(2.0) + 4 * math.log(math.cosh(beta)) + 6 * math.tanh(beta) ** 4


def lnz_periodic_2x2_xy(T2: np.ndarray) -> float:
    """ln of the exact contraction of a periodic 2 x 2 network (axes x, y) of copies of
    A[x, y; x', y'] = sum_{z,t} T2[x, y, z, t; x', y', z, t] (rank-8 tensor in natural layout).

    On a 2-site periodic ring the two sites are joined by two distinct bonds, so the network
    has 8 bonds. Site (i, j) carries legs x = X[i-1, j], x' = X[i, j], y = Y[i, j-1], y' = Y[i, j].
    """
    A = np.einsum("abcdefcd->abef", T2)
    # bond letters: X[i,j] -> 'p','q','r','s' for (0,0),(1,0),(0,1),(1,1); Y similarly
    X = {(0, 0): "p", (1, 0): "q", (0, 1): "r", (1, 1): "s"}
    Y = {(0, 0): "w", (1, 0): "x", (0, 1): "y", (1, 1): "z"}
    subs = []
    for i in range(2):
        for j in range(2):
            subs.append(X[((i - 1) % 2, j)] + Y[(i, (j - 1) % 2)] + X[(i, j)] + Y[(i, j)])
    val = np.einsum(",".join(subs) + "->", A, A, A, A, optimize=True)
    return float(math.log(val))
