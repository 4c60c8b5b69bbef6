"""HOTRG for the d-dimensional Ising model, plain FP64 NumPy (arXiv:1906.06060, Sec. 2).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg and reference arm may use it. It shares no code with the CUDA library.

Everything here follows the paper's order of operations; NumPy/LAPACK primitives (tensordot,
einsum, eigh) serve as single steps. Where the paper is silent, the reading used is stated at
the function that applies it.

Tensor layout (used by every function in this module)
-----------------------------------------------------
A site tensor of a d-dimensional lattice has 2d legs. They are stored in the "natural" order

    T[u_0, ..., u_{d-1}, p_0, ..., p_{d-1}]

where u_b is the leg pointing to the lower neighbour along axis b (the paper's unprimed index,
x, y, z, t) and p_b the leg pointing to the upper neighbour (the primed index x', y', z', t').
Axis 0 is x, 1 is y, 2 is z, 3 is t. With this order the periodic trace of Eq. (tTr) is the
matrix trace of T reshaped to (P, P), P = prod of the bond dimensions.

Readings of silent points (Sec. 2 and Xie et al.'s HOTRG, which the paper defers to)
-----------------------------------------------------------------------------------------
R1  Step along axis a: site 1 is the lower site. Its p_a contracts with u_a of site 2. The new
    u_a is site 1's u_a, the new p_a is site 2's p_a. A transverse leg b fuses as
    (site-1 leg, site-2 leg) with the site-1 index as the slow index.
R2  The isometry of transverse axis b comes from the Gram matrix of the unprimed pair
    (u_b of site 1, u_b of site 2). The same U is applied to the primed pair ("the same U on x
    and x'", Eq. (SS)). For this model the primed-side Gram has the same spectrum; the tests
    check that.
R3  chi_b = min(D_b^2, Dcut). Eigenvalues are sorted descending (stable). Each kept
    eigenvector is sign-fixed so that its largest-magnitude component is positive (lowest
    index on a tie).
R4  Normalisation (not written in the paper; implied by lattices of 2^40 sites, Sec. 2 end):
    c_n = ||T^(n)||_F for n >= 0, T <- T / c_n, and
    ln Z_N / N = sum_{k=0}^{n} 2^{-k} ln c_k + 2^{-n} ln Tr T^(n)   (N = 2^n).
R5  Axis cycle: t, z, y, x (axes d-1, ..., 0), repeated.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

AXIS_NAMES = "xyzt"


# ---------------------------------------------------------------------------------------------
# Initial tensor (Sec. 2, Eq. (pf) and the definition of T^(0) below it)
# ---------------------------------------------------------------------------------------------
def bond_weight(beta: float) -> np.ndarray:
    """W = U sqrt(Lambda) for the bond matrix e^{beta s s'} (Sec. 2, after Eq. (pf)).

    Rows are the spin s = +1, -1; columns the bond index 0, 1. The eigenvectors of
    [[e^b, e^-b], [e^-b, e^b]] are (1, 1)/sqrt2 (eigenvalue 2 cosh b) and (1, -1)/sqrt2
    (eigenvalue 2 sinh b), so sum_k W[s,k] W[s',k] = e^{beta s s'}.
    """
    lam = np.array([2.0 * math.cosh(beta), 2.0 * math.sinh(beta)])
    U = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    return U * np.sqrt(lam)[None, :]


def site_weight(beta: float, h: float) -> np.ndarray:
    """V_s = e^{beta h s} for s = +1, -1 (Sec. 2, after Eq. (pf))."""
    return np.array([math.exp(beta * h), math.exp(-beta * h)])


def initial_tensor(d: int, beta: float, h: float, spin_insertion: bool = False) -> np.ndarray:
    """T^(0) = sum_s V_s prod_{2d legs} W[s, leg] by explicit summation over the spin (Sec. 2).

    With spin_insertion=True the summand carries an extra factor s: this is the impure tensor
    S^(0) of Sec. 2.
    """
    W = bond_weight(beta)
    V = site_weight(beta, h)
    T = np.zeros((2,) * (2 * d))
    for si, s in enumerate((1.0, -1.0)):
        t = np.array(V[si] * (s if spin_insertion else 1.0))
        for _ in range(2 * d):
            t = np.multiply.outer(t, W[si])
        T += t
    return T


# ---------------------------------------------------------------------------------------------
# Measurements on a coarse-grained tensor (Eqs. (tTr), (matA), (x))
# ---------------------------------------------------------------------------------------------
def dims_of(T: np.ndarray) -> tuple[int, ...]:
    d = T.ndim // 2
    assert T.shape[:d] == T.shape[d:], "unprimed and primed legs must have equal dimensions"
    return T.shape[:d]


def trace(T: np.ndarray) -> float:
    """Eq. (tTr): sum over x,y,z,t of T[x,y,z,t; x,y,z,t] (periodic closure)."""
    P = int(np.prod(dims_of(T)))
    return float(np.trace(T.reshape(P, P)))


def frobenius(T: np.ndarray) -> float:
    return float(np.sqrt(np.sum(T * T)))


def x_indicator(T: np.ndarray, axis: int) -> float:
    """X^(n) = (Tr A)^2 / Tr A^2 with A_{aa'} = sum over the other axes of the traced tensor
    (Eqs. (matA), (x)); `axis` is the last coarse-grained direction."""
    d = T.ndim // 2
    letters = "abcdefgh"
    u = [letters[b] for b in range(d)]
    p = list(u)
    p[axis] = "z"
    A = np.einsum("".join(u + p) + "->" + u[axis] + "z", T)
    return float(np.trace(A) ** 2 / np.trace(A @ A))


# ---------------------------------------------------------------------------------------------
# Isometries: Gram matrices of the two-site unfolding and their truncated eigenbasis
# (Sec. 2, Eq. (SS) "U determined within the original algorithm"; HOSVD of Xie et al.)
# ---------------------------------------------------------------------------------------------
def half_gram(T: np.ndarray, leg_b: int, leg_alpha: int) -> np.ndarray:
    """Q[i, i~, al, al~] = sum over all other legs of T[..i..al..] T[..i~..al~..].

    leg_b / leg_alpha are positions in the natural layout. Site 1 of a step along a uses
    (u_b, p_a); site 2 uses (u_b, u_a).
    """
    X = np.moveaxis(T, (leg_b, leg_alpha), (0, 1))
    Db, Da = X.shape[0], X.shape[1]
    X = X.reshape(Db * Da, -1)
    Q = (X @ X.T).reshape(Db, Da, Db, Da)
    return Q.transpose(0, 2, 1, 3)


def gram(T: np.ndarray, a: int, b: int, side: str = "unprimed") -> np.ndarray:
    """Gram matrix G_b of the two-site tensor M (two copies of T merged along a), for the pair
    of b-legs (site 1, site 2) on the given side:

        G_b[(b1 b2), (b1~ b2~)] = sum over every other leg of M of M[..b1 b2..] M[..b1~ b2~..]
                                = sum_{al, al~} Q1[b1, b1~, al, al~] Q2[b2, b2~, al, al~]

    where al is the contracted bond (site 1's p_a = site 2's u_a). Reading R2."""
    d = T.ndim // 2
    leg = b if side == "unprimed" else d + b
    Q1 = half_gram(T, leg, d + a)
    Q2 = half_gram(T, leg, a)
    Db = T.shape[b]
    G = np.einsum("ikab,jlab->ijkl", Q1, Q2)
    return G.reshape(Db * Db, Db * Db)


@dataclass
class Isometry:
    U: np.ndarray            # [b1, b2, k], shape (D_b, D_b, chi)
    eigenvalues: np.ndarray  # all D_b^2 eigenvalues of G_b, descending
    chi: int
    gap: float               # (lam_chi - lam_{chi+1}) / lam_chi at the cut; inf if lossless


def isometry_from_gram(G: np.ndarray, Db: int, Dcut: int) -> Isometry:
    """Symmetric eigendecomposition of G_b, truncated to chi = min(D_b^2, Dcut). Reading R3."""
    lam, V = np.linalg.eigh(G)
    order = np.argsort(-lam, kind="stable")
    lam, V = lam[order], V[:, order]
    chi = min(Db * Db, Dcut)
    Vk = V[:, :chi].copy()
    for k in range(chi):
        i = int(np.argmax(np.abs(Vk[:, k])))
        if Vk[i, k] < 0:
            Vk[:, k] = -Vk[:, k]
    gap = math.inf
    if chi < lam.size:
        gap = float((lam[chi - 1] - lam[chi]) / lam[chi - 1]) if lam[chi - 1] != 0 else 0.0
    return Isometry(U=Vk.reshape(Db, Db, chi), eigenvalues=lam, chi=chi, gap=gap)


# ---------------------------------------------------------------------------------------------
# Squeeze: T' = U U (T T) U U ... (Eqs. (SS), (ST) with S -> T; 4D extension of Sec. 2)
# ---------------------------------------------------------------------------------------------
def _new_dims(dims, a, U):
    nd = list(dims)
    for b, u in U.items():
        nd[b] = u.shape[2]
    return nd


def squeeze(T1: np.ndarray, T2: np.ndarray, a: int, U: dict[int, np.ndarray],
            max_slices: int | None = None, slices=None) -> np.ndarray:
    """Coarse-grained tensor of the pair (T1 lower, T2 upper along a), slice by slice.

    For each slice s = (k_b for the transverse axes b):
      producer : A_s = T1 with every unprimed transverse leg b1 mapped to b2 by U_b[:, :, k_b]
      GEMM     : O_s = sum over (b2 for all b, al) of A_s * T2     (the O(D^15) contraction)
      epilogue : T'[s, a1; k'.., a2'] = sum over (b1', b2') of U_b[b1', b2', k'_b] O_s
    No intermediate larger than one slice (D^8 entries) is formed. max_slices stops after that
    many slices (leaving the rest zero): only for timing a bounded sample of the work. slices (a
    set of (k_b for the transverse axes b, in axis order) tuples) computes only those slices,
    leaving the rest zero: for checking sampled slices of a large squeeze.
    """
    d = T1.ndim // 2
    dims = dims_of(T1)
    trans = [b for b in range(d) if b != a]
    nd = _new_dims(dims, a, U)
    out = np.zeros(nd + nd)
    chis = [U[b].shape[2] for b in trans]
    for count, ks in enumerate(itertools.product(*[range(c) for c in chis])):
        if max_slices is not None and count >= max_slices:
            break
        if slices is not None and tuple(ks) not in slices:
            continue
        A = T1
        for b, k in zip(trans, ks):
            A = np.moveaxis(np.tensordot(U[b][:, :, k], A, axes=([0], [b])), 0, b)
        # A legs: u_b = b2 (b != a), u_a = a1, p_b = b1', p_a = al
        O = np.tensordot(A, T2, axes=(trans + [d + a], trans + [a]))
        # O legs: [a1, b1' for b in trans (in order), then T2 primed p_0..p_{d-1}]
        # epilogue: contract (b1', b2') -> k'_b for each transverse b
        letters = iter("abcdefghijklmnopqrstuvwxyz")
        a1 = next(letters)
        b1p = {b: next(letters) for b in trans}
        p2 = [next(letters) for _ in range(d)]
        kp = {b: next(letters) for b in trans}
        operands, subs = [O], [a1 + "".join(b1p[b] for b in trans) + "".join(p2)]
        for b in trans:
            operands.append(U[b])
            subs.append(b1p[b] + p2[b] + kp[b])
        outsub = a1 + "".join(kp[b] if b != a else p2[a] for b in range(d))
        R = np.einsum(",".join(subs) + "->" + outsub, *operands, optimize=True)
        idx = [slice(None)] * d
        for b, k in zip(trans, ks):
            idx[b] = k
        # R legs: [a1, primed natural order]; out[u with u_b = k_b, u_a = a1 ; primed]
        out[tuple(idx)] = R
    return out


def two_site_tensor(T1: np.ndarray, T2: np.ndarray, a: int) -> np.ndarray:
    """M = sum_al T1[.., p_a = al] T2[u_a = al, ..] with legs ordered
    [for each axis b: (b1, b2) if b != a else (a1)] then the same for the primed side.
    Only for tiny bond dimensions (it has prod D_b^4 * D_a^2 entries)."""
    d = T1.ndim // 2
    L = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJ")
    u1 = [next(L) for _ in range(d)]
    p1 = [next(L) for _ in range(d)]
    u2 = [next(L) for _ in range(d)]
    p2 = [next(L) for _ in range(d)]
    p1[a] = u2[a]
    outu, outp = [], []
    for b in range(d):
        outu += [u1[b]] if b == a else [u1[b], u2[b]]
        outp += [p2[b]] if b == a else [p1[b], p2[b]]
    spec = "".join(u1 + p1) + "," + "".join(u2 + p2) + "->" + "".join(outu + outp)
    return np.einsum(spec, T1, T2)


def squeeze_direct(T1: np.ndarray, T2: np.ndarray, a: int, U: dict[int, np.ndarray]) -> np.ndarray:
    """The whole network (2 T's and 2(d-1) U's) as one einsum: the definition of the
    coarse-grained tensor, used to pin `squeeze` at tiny bond dimension."""
    d = T1.ndim // 2
    L = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    u1 = [next(L) for _ in range(d)]
    p1 = [next(L) for _ in range(d)]
    u2 = [next(L) for _ in range(d)]
    p2 = [next(L) for _ in range(d)]
    p1[a] = u2[a]
    k = {b: next(L) for b in range(d) if b != a}
    kp = {b: next(L) for b in range(d) if b != a}
    subs = ["".join(u1 + p1), "".join(u2 + p2)]
    ops = [T1, T2]
    for b in k:
        subs += [u1[b] + u2[b] + k[b], p1[b] + p2[b] + kp[b]]
        ops += [U[b], U[b]]
    out = "".join(k[b] if b != a else u1[a] for b in range(d)) + "".join(
        kp[b] if b != a else p2[a] for b in range(d))
    return np.einsum(",".join(subs) + "->" + out, *ops, optimize=True)


# ---------------------------------------------------------------------------------------------
# One coarse-graining step and the full flow
# ---------------------------------------------------------------------------------------------
@dataclass
class StepInfo:
    axis: int
    isometries: dict[int, Isometry]
    ln_c: float = 0.0


def coarse_grain(T: np.ndarray, a: int, Dcut: int,
                 isometries: dict[int, np.ndarray] | None = None) -> tuple[np.ndarray, StepInfo]:
    """One HOTRG step along axis a (Sec. 2): isometries from the Gram matrices, then squeeze.
    Passing `isometries` freezes U (used for fixed-isometry derivatives)."""
    d = T.ndim // 2
    info = StepInfo(axis=a, isometries={})
    U = {}
    for b in range(d):
        if b == a:
            continue
        if isometries is not None:
            U[b] = isometries[b]
            continue
        iso = isometry_from_gram(gram(T, a, b), T.shape[b], Dcut)
        info.isometries[b] = iso
        U[b] = iso.U
    return squeeze(T, T, a, U), info


def default_order(d: int) -> list[int]:
    """Reading R5: t, z, y, x (axes d-1 .. 0)."""
    return list(range(d - 1, -1, -1))


@dataclass
class Flow:
    d: int
    beta: float
    h: float
    Dcut: int
    ln_c: list[float] = field(default_factory=list)        # ln c_0 .. ln c_n
    lnz: list[float] = field(default_factory=list)         # estimate of ln Z_N / N after step n
    axes: list[int] = field(default_factory=list)
    dims: list[tuple[int, ...]] = field(default_factory=list)
    spectra: list[dict[int, np.ndarray]] = field(default_factory=list)
    gaps: list[dict[int, float]] = field(default_factory=list)
    x: list[float] = field(default_factory=list)
    isometries: list[dict[int, np.ndarray]] = field(default_factory=list)   # U of every step
    tensor: np.ndarray | None = None

    @property
    def lnz_per_site(self) -> float:
        return self.lnz[-1]

    @property
    def free_energy(self) -> float:
        """f = -(ln Z / N) / beta."""
        return -self.lnz[-1] / self.beta


def run(d: int, beta: float, h: float, Dcut: int, nsteps: int, order: list[int] | None = None,
        norm=frobenius, T0: np.ndarray | None = None, keep_tensor: bool = False,
        isometries: list[dict[int, np.ndarray]] | None = None) -> Flow:
    """Full flow (reading R4): normalise T^(0), then n steps with ln-norm accumulation.
    `isometries` (one dict per step, as recorded in Flow.isometries) freezes U at every step."""
    order = default_order(d) if order is None else list(order)
    T = initial_tensor(d, beta, h) if T0 is None else np.array(T0, dtype=np.float64)
    flow = Flow(d=d, beta=beta, h=h, Dcut=Dcut)
    c = norm(T)
    T = T / c
    L = math.log(c)
    flow.ln_c.append(math.log(c))
    flow.lnz.append(L + math.log(trace(T)))
    for n in range(1, nsteps + 1):
        a = order[(n - 1) % len(order)]
        T, info = coarse_grain(T, a, Dcut, None if isometries is None else isometries[n - 1])
        c = norm(T)
        if not np.isfinite(c) or c <= 0:
            raise FloatingPointError(f"step {n}: norm {c}")
        T = T / c
        L += math.ldexp(math.log(c), -n)
        tr = trace(T)
        if tr <= 0:
            raise FloatingPointError(f"step {n}: trace {tr}")
        flow.ln_c.append(math.log(c))
        flow.lnz.append(L + math.ldexp(math.log(tr), -n))
        flow.axes.append(a)
        flow.dims.append(dims_of(T))
        flow.spectra.append({b: iso.eigenvalues for b, iso in info.isometries.items()})
        flow.gaps.append({b: iso.gap for b, iso in info.isometries.items()})
        flow.x.append(x_indicator(T, a))
        flow.isometries.append({b: iso.U for b, iso in info.isometries.items()}
                               if isometries is None else isometries[n - 1])
    if keep_tensor:
        flow.tensor = T
    return flow


@dataclass
class ImpurityFlow:
    nn: list[float] = field(default_factory=list)     # <s_i s_j> estimate after step n (n >= 1)
    spin: list[float] = field(default_factory=list)   # <s_i> estimate after step n (n >= 0)


def impurity_flow(d: int, beta: float, h: float, Dcut: int, nsteps: int,
                  order: list[int] | None = None) -> ImpurityFlow:
    """The impure-tensor estimates of Sec. 2, Eqs. (impTN), (SS), (ST), (energy), (spin).

    Energy: impure tensors S^(0) (spin inserted) on two neighbouring sites, site 1 and its
    neighbour along the first coarse-graining axis; step 1 merges the two (Eq. (SS)), every later
    step merges the impure site 1 with a pure site 2 (Eq. (ST)). Magnetisation: one impure tensor,
    merged with a pure site from step 1 on. The isometries are always the pure flow's; the impure
    tensors are divided by the pure flow's norm c_n at every step, so the ratio
    Tr S^(n) / Tr T^(n) (Eq. (tTr) on both) is the estimate of <s_i s_j> resp. <s_i>.
    """
    order = default_order(d) if order is None else list(order)
    T = initial_tensor(d, beta, h)
    S0 = initial_tensor(d, beta, h, spin_insertion=True)
    c = frobenius(T)
    T, SE, SM = T / c, S0 / c, S0 / c
    out = ImpurityFlow()
    out.spin.append(trace(SM) / trace(T))
    for n in range(1, nsteps + 1):
        a = order[(n - 1) % len(order)]
        Tn, info = coarse_grain(T, a, Dcut)
        U = {b: iso.U for b, iso in info.isometries.items()}
        SEn = squeeze(SE, SE if n == 1 else T, a, U)
        SMn = squeeze(SM, T, a, U)
        c = frobenius(Tn)
        T, SE, SM = Tn / c, SEn / c, SMn / c
        tr = trace(T)
        out.nn.append(trace(SE) / tr)
        out.spin.append(trace(SM) / tr)
    return out


def fixed_isometry_derivatives(d: int, beta: float, h: float, Dcut: int, nsteps: int,
                               eps: float = 1e-3) -> tuple[np.ndarray, np.ndarray]:
    """d/d beta and d/d h of the ln Z_N / N estimate after every step 0..nsteps, with the
    isometries of every step frozen at their values at (beta, h) (reading R9).

    Central differences of the frozen flow, Richardson-extrapolated from steps eps and eps/2
    (truncation error O(eps^4)). Where every step is lossless (chi = D^2), the frozen U is an
    orthogonal change of basis and these are the exact derivatives of ln Z / N of the lattice;
    with H = -sum s s' - h sum s they give <H>/N = -d/d beta and <s> = (d/d h) / beta."""
    base = run(d, beta, h, Dcut, nsteps)
    U = base.isometries

    def lnz(b, hh):
        return np.array(run(d, b, hh, Dcut, nsteps, isometries=U).lnz)

    def central(f, e):
        return (f(e) - f(-e)) / (2.0 * e)

    out = []
    for f in (lambda e: lnz(beta + e, h), lambda e: lnz(beta, h + e)):
        d1, d2 = central(f, eps), central(f, eps / 2)
        out.append((4.0 * d2 - d1) / 3.0)
    return out[0], out[1]


def flow_derivatives(d: int, beta: float, h: float, Dcut: int, nsteps: int,
                     eps: float = 1e-4) -> tuple[np.ndarray, np.ndarray]:
    """d/d beta and d/d h of the ln Z_N / N estimate after every step 0..nsteps of the truncated
    flow itself (isometries recomputed at every point), by central differences Richardson-
    extrapolated from steps eps and eps/2. This is what differentiating the isometries through
    the eigendecomposition computes; it differs from fixed_isometry_derivatives by terms of the
    order of the truncation. It exists only where no cut splits a degenerate eigenvalue pair."""

    def lnz(b, hh):
        return np.array(run(d, b, hh, Dcut, nsteps).lnz)

    def central(f, e):
        return (f(e) - f(-e)) / (2.0 * e)

    out = []
    for f in (lambda e: lnz(beta + e, h), lambda e: lnz(beta, h + e)):
        d1, d2 = central(f, eps), central(f, eps / 2)
        out.append((4.0 * d2 - d1) / 3.0)
    return out[0], out[1]


def dims_schedule(d: int, Dcut: int, nsteps: int, order: list[int] | None = None) -> list[list[int]]:
    """Bond dimensions after each step under chi = min(D^2, Dcut) (reading R3)."""
    order = default_order(d) if order is None else order
    dims = [2] * d
    out = [list(dims)]
    for n in range(nsteps):
        a = order[n % len(order)]
        dims = [dims[b] if b == a else min(dims[b] ** 2, Dcut) for b in range(d)]
        out.append(list(dims))
    return out


def squeeze_flops(dims_before: list[int], a: int, Dcut: int) -> float:
    """Algorithmic flops of the squeeze contraction of one step: 2 * prod(chi_b) * P^3
    (the O(Dcut^15) term of Sec. 2's cost statement)."""
    P = float(np.prod(dims_before))
    chi = 1.0
    for b, D in enumerate(dims_before):
        if b != a:
            chi *= min(D * D, Dcut)
    return 2.0 * chi * P ** 3
