"""Pins of the FP64 CPU oracle against what the paper and mathematics fix (no GPU).

Each test names the passage of arXiv:1906.06060 it checks. The references used here
(enumeration, Onsager, transfer matrix, closed forms) are in oracle/exact.py and share no code
with the tensor-network oracle in oracle/hotrg_ref.py.
"""
import math

import numpy as np
import pytest

from oracle import exact as E
from oracle import hotrg_ref as R
from tests.inputs import random_site_tensor


# ------------------------------------------------------------------ Sec. 2: T^(0) and W
@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.44, 0.3), (1.0, -0.2), (0.05, 1e-6)])
def test_initial_tensor_closed_form(d, beta, h):
    T = R.initial_tensor(d, beta, h)
    C = E.initial_tensor_closed_form(d, beta, h)
    # the oracle sums e^{bh} and -e^{-bh}: odd entries carry its cancellation, so the
    # tolerance is relative to the largest entry
    np.testing.assert_allclose(T, C, rtol=1e-14, atol=1e-15 * np.abs(C).max())


@pytest.mark.parametrize("beta", [0.01, 0.1497, 0.7])
def test_bond_weight_factorises_boltzmann_weight(beta):
    W = R.bond_weight(beta)
    s = np.array([1.0, -1.0])
    np.testing.assert_allclose(W @ W.T, np.exp(beta * np.outer(s, s)), rtol=1e-15)


# ------------------------------------------------------------------ Eqs. (TNrep), (tTr): exact
@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.3, 0.01), (0.3, -0.2), (0.8, 0.05)])
def test_4d_lossless_steps_match_enumeration(beta, h):
    """After k lossless steps, Eq. (tTr) is Z of a lattice with L_a = 2^{k_a}."""
    f = R.run(4, beta, h, 16, 2)
    assert f.dims == [(4, 4, 4, 2), (16, 16, 4, 4)]
    assert abs(2 * f.lnz[1] - E.lnz_bruteforce(beta, h, (1, 1, 1, 2))) < 1e-13 * 4
    assert abs(4 * f.lnz[2] - E.lnz_bruteforce(beta, h, (1, 1, 2, 2))) < 1e-13 * 6


@pytest.mark.parametrize("beta,h", [(0.2, 0.0), (0.5, 0.1)])
def test_3d_lossless_steps_match_enumeration(beta, h):
    f = R.run(3, beta, h, 16, 3)
    for n, L in [(1, (1, 1, 2)), (2, (1, 2, 2)), (3, (2, 2, 2))]:
        assert abs(2 ** n * f.lnz[n] - E.lnz_bruteforce(beta, h, L)) < 1e-12


@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.4407, 0.0), (0.44, 0.05), (0.9, -0.3)])
def test_2d_4x4_lattice_matches_enumeration(beta, h):
    """4 lossless steps (Dcut=16) give the periodic 4x4 lattice, 65,536 configurations."""
    f = R.run(2, beta, h, 16, 4)
    assert f.dims[-1] == (16, 16)
    assert abs(16 * f.lnz[4] - E.lnz_bruteforce(beta, h, (4, 4))) < 1e-12


@pytest.mark.slow
@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.3, 0.01), (0.3, -0.01)])
def test_4d_periodic_2to4_lattice_matches_enumeration(beta, h):
    """The 16-site periodic 2^4 lattice (65,536 configurations): two lossless steps (t, z),
    then the exact periodic 2x2 contraction in (x, y)."""
    f = R.run(4, beta, h, 16, 2, keep_tensor=True)
    L = sum(math.ldexp(c, -k) for k, c in enumerate(f.ln_c))
    lnz = 16 * L + E.lnz_periodic_2x2_xy(f.tensor)
    assert abs(lnz - E.lnz_bruteforce(beta, h, (2, 2, 2, 2))) < 1e-12 * 20


@pytest.mark.parametrize("n", [1, 2, 3, 6, 12, 30])
@pytest.mark.parametrize("beta,h", [(0.5, 0.1), (1.3, -0.02)])
def test_1d_chain_matches_transfer_matrix(n, beta, h):
    f = R.run(1, beta, h, 4, n)
    assert abs(f.lnz[-1] - E.lnz_1d(beta, h, 2 ** n) / 2 ** n) < 1e-14


@pytest.mark.parametrize("d,Dcut", [(2, 3), (3, 4), (4, 3)])
def test_infinite_temperature_gives_ln2(d, Dcut):
    f = R.run(d, 0.0, 0.0, Dcut, 4 * d)
    assert abs(f.lnz[-1] - math.log(2.0)) < 1e-14


# ------------------------------------------------------------------ truncated flows
def test_onsager_forms_agree():
    for beta in (0.2, 0.3, 0.6):
        assert abs(E.lnz_onsager(beta) - E.lnz_onsager_double(beta)) < 1e-11


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_2d_flow_converges_to_onsager(beta):
    """Off-critical 2D flow: the error against Onsager falls as Dcut grows (the paper's
    monotone delta f, Sec. 3) and is below 1e-8 at Dcut=16 after 40 steps (2^40 sites)."""
    errs = [abs(R.run(2, beta, 0.0, D, 40).lnz[-1] - E.lnz_onsager(beta)) for D in (4, 8, 16)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8


def test_4d_high_temperature_series():
    f = R.run(4, 0.1497, 0.0, 5, 16)
    assert abs(f.lnz[-1] - E.lnz_high_temperature_4d(0.1497)) < 1e-3


def test_field_reversal_symmetry():
    """Z(h) = Z(-h) (spin-flip symmetry of Eq. (pf))."""
    a = R.run(4, 0.1497, 0.01, 5, 8)
    b = R.run(4, 0.1497, -0.01, 5, 8)
    assert abs(a.lnz[-1] - b.lnz[-1]) < 1e-13 * abs(a.lnz[-1])


def test_axis_order_invariance():
    """T^(0) is isotropic, so any axis cycle gives the same flow (relabelled axes)."""
    a = R.run(4, 0.1497, 0.0, 5, 8, order=[3, 2, 1, 0])
    b = R.run(4, 0.1497, 0.0, 5, 8, order=[0, 1, 2, 3])
    assert abs(a.lnz[-1] - b.lnz[-1]) < 1e-13


def test_normalisation_invariance():
    """Isometries are scale-invariant, so the ln Z estimate does not depend on the norm used."""
    a = R.run(4, 0.1497, 0.0, 5, 8)
    b = R.run(4, 0.1497, 0.0, 5, 8, norm=lambda T: float(np.max(np.abs(T))))
    assert abs(a.lnz[-1] - b.lnz[-1]) < 1e-13


def test_isometries_orthonormal_and_left_right_spectra_equal():
    T = R.initial_tensor(4, 0.1497, 0.0)
    T /= R.frobenius(T)
    for a in (3, 2, 1):
        for b in range(4):
            if b == a:
                continue
            G = R.gram(T, a, b)
            Gp = R.gram(T, a, b, side="primed")
            l1, l2 = np.linalg.eigvalsh(G), np.linalg.eigvalsh(Gp)
            np.testing.assert_allclose(l1, l2, rtol=1e-12, atol=1e-14 * l1.max())
            iso = R.isometry_from_gram(G, T.shape[b], 5)
            U = iso.U.reshape(-1, iso.chi)
            np.testing.assert_allclose(U.T @ U, np.eye(iso.chi), atol=1e-13)
        T, _ = R.coarse_grain(T, a, 5)
        T /= R.frobenius(T)


# ------------------------------------------------------------------ contraction pins (random)
@pytest.mark.parametrize("d,dims,a", [(2, (3, 2), 1), (3, (2, 3, 2), 0), (4, (2, 2, 3, 2), 3),
                                      (4, (3, 2, 2, 2), 1)])
def test_gram_half_contractions_match_two_site_unfolding(d, dims, a):
    T = random_site_tensor(dims, seed=d * 10 + a)
    M = R.two_site_tensor(T, T, a)
    # position of (b1, b2) in M's unprimed block
    pos = 0
    for b in range(d):
        if b == a:
            pos += 1
            continue
        X = np.moveaxis(M, (pos, pos + 1), (0, 1)).reshape(dims[b] ** 2, -1)
        np.testing.assert_allclose(R.gram(T, a, b), X @ X.T, rtol=1e-12, atol=1e-12)
        pos += 2


@pytest.mark.parametrize("Dcut", [2, 3])
def test_isometry_keeps_the_dominant_subspace(Dcut):
    """U spans the top-chi eigenvectors: the weight it keeps equals the sum of kept
    eigenvalues, computed on the explicit two-site tensor."""
    dims, a, b = (2, 2, 2, 2), 3, 1
    T = random_site_tensor(dims, seed=7)
    M = R.two_site_tensor(T, T, a)
    X = np.moveaxis(M, (2, 3), (0, 1)).reshape(4, -1)
    iso = R.isometry_from_gram(R.gram(T, a, b), 2, Dcut)
    kept = np.linalg.norm(iso.U.reshape(4, -1).T @ X) ** 2
    assert abs(kept - iso.eigenvalues[:iso.chi].sum()) < 1e-11 * kept
    assert np.all(np.diff(iso.eigenvalues) <= 0)


@pytest.mark.parametrize("d,dims,a,Dcut", [(2, (3, 2), 1, 4), (2, (3, 3), 0, 5), (3, (2, 3, 2), 0, 3),
                                           (4, (2, 2, 2, 2), 3, 3), (4, (2, 3, 2, 2), 1, 4),
                                           (4, (3, 2, 2, 3), 0, 16)])
def test_sliced_squeeze_matches_whole_network(d, dims, a, Dcut):
    T = random_site_tensor(dims, seed=100 + d + a)
    U = {}
    for b in range(d):
        if b != a:
            U[b] = R.isometry_from_gram(R.gram(T, a, b), dims[b], Dcut).U
    np.testing.assert_allclose(R.squeeze(T, T, a, U), R.squeeze_direct(T, T, a, U),
                               rtol=1e-12, atol=1e-12)
    # distinct site tensors too (the contraction must not rely on T1 == T2)
    T2 = random_site_tensor(dims, seed=200 + d + a)
    np.testing.assert_allclose(R.squeeze(T, T2, a, U), R.squeeze_direct(T, T2, a, U),
                               rtol=1e-12, atol=1e-12)


def test_squeeze_slice_selection_picks_the_same_slices():
    """The slice selection used by the full-size parity tests only chooses which slices to
    compute: the selected slices equal those of the whole squeeze, the others stay zero."""
    d, dims, a, Dcut = 4, (3, 2, 3, 2), 1, 5
    T = random_site_tensor(dims, seed=77)
    U = {b: R.isometry_from_gram(R.gram(T, a, b), dims[b], Dcut).U for b in range(d) if b != a}
    full = R.squeeze(T, T, a, U)
    pick = {(0, 0, 1), (4, 2, 3)}
    part = R.squeeze(T, T, a, U, slices=pick)
    for k0 in range(full.shape[0]):
        for k2 in range(full.shape[2]):
            for k3 in range(full.shape[3]):
                sl = (k0, slice(None), k2, k3)
                if (k0, k2, k3) in pick:
                    assert np.array_equal(part[sl], full[sl])
                else:
                    assert not np.any(part[sl])


def test_x_indicator_phases():
    """X^(n) -> 1 in the disordered and -> 2 in the ordered phase (Sec. 3, Eq. (x))."""
    hot = R.run(4, 0.10, 0.0, 4, 24)
    cold = R.run(4, 0.25, 0.0, 4, 24)
    assert abs(hot.x[-1] - 1.0) < 1e-3
    assert abs(cold.x[-1] - 2.0) < 1e-3


@pytest.mark.parametrize("beta,h", [(0.5, 0.1), (1.3, -0.02), (0.2, 0.3), (0.9, 0.0)])
def test_x_indicator_1d_matches_transfer_matrix(beta, h):
    """Exact pin of X^(n) (Eqs. (matA), (x)): in d = 1 the flow's tensor is the site matrix to the
    power 2^n, so X is fixed by the transfer-matrix eigenvalues at every step (values well
    between 1 and 2 at the first steps)."""
    f = R.run(1, beta, h, 4, 8)
    for n in range(1, 9):
        assert abs(f.x[n - 1] - E.x_1d(beta, h, 2 ** n)) < 1e-13, n
    assert 1.01 < f.x[0] < 1.99


def test_dims_schedule_reaches_dcut_at_step_3():
    assert R.dims_schedule(4, 10, 4) == [[2, 2, 2, 2], [4, 4, 4, 2], [10, 10, 4, 4],
                                         [10, 10, 10, 10], [10, 10, 10, 10]]
    assert R.squeeze_flops([10] * 4, 0, 10) == pytest.approx(2e15)


# ------------------------------------------------------------------ zero-field spin-flip structure
def _odd_entries_max(T, par):
    """Largest |T| over entries whose legs' parities (par[b][index], both copies of leg b) add
    up to odd."""
    d = T.ndim // 2
    tot = np.zeros(T.shape, dtype=int)
    for slot in range(2 * d):
        shape = [1] * (2 * d)
        shape[slot] = T.shape[slot]
        tot = tot + par[slot % d].reshape(shape)
    odd = (tot % 2) == 1
    return np.abs(T[odd]).max() if odd.any() else 0.0


@pytest.mark.parametrize("d,Dcut,nsteps", [(2, 8, 8), (3, 6, 6), (4, 5, 6)])
def test_zero_field_flow_keeps_the_spin_flip_block_structure(d, Dcut, nsteps):
    """Sec. 2's T^(0) at h = 0: the site weight is even in s, so entries with an odd number of
    odd legs vanish; Gram matrices then commute with the fused parity and every kept
    eigenvector lies in one parity sector, so the structure survives each step with the new
    bond's parities read off the isometry. This is what the block-sparse squeeze relies on. At
    h != 0 the odd entries are present from the start."""
    beta = {2: 0.4, 3: 0.22, 4: 0.1497}[d]
    T = R.initial_tensor(d, beta, 0.0)
    assert _odd_entries_max(R.initial_tensor(d, beta, 0.05), [np.array([0, 1])] * d) > 1e-3
    par = [np.array([0, 1]) for _ in range(d)]
    order = R.default_order(d)
    for n in range(nsteps):
        assert _odd_entries_max(T, par) <= 1e-13 * np.abs(T).max(), n
        a = order[n % d]
        T, info = R.coarse_grain(T, a, Dcut)
        T = T / R.frobenius(T)
        for b, iso in info.isometries.items():
            U = iso.U
            fused = (par[b][:, None] ^ par[b][None, :]).astype(bool)
            w_odd = (U ** 2)[fused].sum(axis=0)
            w_even = (U ** 2)[~fused].sum(axis=0)
            assert np.all(np.minimum(w_odd, w_even) < 1e-20), (n, b)
            par[b] = (w_odd > w_even).astype(int)
    assert _odd_entries_max(T, par) <= 1e-13 * np.abs(T).max()
    # both sectors are kept on a truncated bond
    assert any(0 < p.sum() < p.size for p in par)


# ------------------------------------------------------------------ planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """A dropped weight, a transposed operand or a wrong leg must fail one of the pins above."""
    beta, h = 0.3, 0.01
    ref = E.lnz_bruteforce(beta, h, (1, 1, 2, 2))

    # (1) dropped 2^{-n} weight on ln c_n
    orig_ldexp = R.math.ldexp
    monkeypatch.setattr(R.math, "ldexp", lambda x, n: x)
    bad = R.run(4, beta, h, 16, 2)
    monkeypatch.setattr(R.math, "ldexp", orig_ldexp)
    assert abs(4 * bad.lnz[2] - ref) > 1e-3

    # (2) second site's tensor transposed (u <-> p) in the squeeze: caught by the random pin
    T = random_site_tensor((2, 3, 2, 2), seed=5)
    d = 4
    Tt = np.transpose(T, list(range(d, 2 * d)) + list(range(d)))
    U = {b: R.isometry_from_gram(R.gram(T, 1, b), T.shape[b], 4).U for b in (0, 2, 3)}
    assert not np.allclose(R.squeeze(T, Tt, 1, U), R.squeeze_direct(T, T, 1, U), atol=1e-6)

    # (3) Gram half-contraction on the wrong leg of site 1 (u_a instead of p_a)
    Tr = random_site_tensor((2, 2, 3, 2), seed=6)
    good = R.gram(Tr, 3, 1)
    Q1 = R.half_gram(Tr, 1, 3)
    Q2 = R.half_gram(Tr, 1, 3)
    wrong = np.einsum("ikab,jlab->ijkl", Q1, Q2).reshape(4, 4)
    assert not np.allclose(wrong, good, rtol=1e-6)


# ------------------------------------------------------------------ derivatives (reading R9)
@pytest.mark.parametrize("beta,h", [(0.7, 0.2), (0.3, 0.0), (1.1, -0.05)])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_dlnz_1d_matches_enumeration(beta, h, N):
    """The differentiated transfer-matrix result against thermal averages by enumeration:
    d(lnZ/N)/d beta = <sum s s'>/N + h <s>, d(lnZ/N)/d h = beta <s>."""
    e, m = E.moments_bruteforce(beta, h, (N,))
    db, dh = E.dlnz_1d(beta, h, N)
    assert abs(db - (e + h * m)) < 1e-13
    assert abs(dh - beta * m) < 1e-13


@pytest.mark.parametrize("beta,h", [(0.7, 0.2), (0.3, 0.0)])
def test_dlnz_1d_matches_difference_quotient_of_lnz_1d(beta, h):
    N, eps = 2 ** 20, 1e-4
    f = lambda b, hh: E.lnz_1d(b, hh, N) / N
    db, dh = E.dlnz_1d(beta, h, N)
    assert abs(db - (f(beta + eps, h) - f(beta - eps, h)) / (2 * eps)) < 1e-7
    assert abs(dh - (f(beta, h + eps) - f(beta, h - eps)) / (2 * eps)) < 1e-7


def test_moments_bruteforce_symmetry_and_difference_quotient():
    """<s> = 0 at h = 0 (Z2 symmetry); the moments are the derivatives of lnz_bruteforce."""
    L = (2, 2, 2)
    e0, m0 = E.moments_bruteforce(0.3, 0.0, L)
    assert abs(m0) < 1e-15 and e0 > 0
    beta, h, eps, N = 0.3, 0.07, 1e-4, 8
    e, m = E.moments_bruteforce(beta, h, L)
    f = lambda b, hh: E.lnz_bruteforce(b, hh, L) / N
    assert abs((f(beta + eps, h) - f(beta - eps, h)) / (2 * eps) - (e + h * m)) < 1e-7
    assert abs((f(beta, h + eps) - f(beta, h - eps)) / (2 * eps) - beta * m) < 1e-7


@pytest.mark.parametrize("beta,h", [(0.7, 0.2), (0.44, 0.0)])
def test_fixed_isometry_derivatives_1d_match_transfer_matrix(beta, h):
    """d = 1 has no transverse legs: every step is exact and after n steps the flow describes a
    ring of 2^n sites."""
    db, dh = R.fixed_isometry_derivatives(1, beta, h, 2, 12)
    for n in range(13):
        rb, rh = E.dlnz_1d(beta, h, 2 ** n)
        assert abs(db[n] - rb) < 1e-10 * max(1.0, abs(rb))
        assert abs(dh[n] - rh) < 1e-10 * max(1.0, abs(rh))


@pytest.mark.parametrize("beta,h", [(0.4407, 0.05), (0.3, 0.0)])
def test_fixed_isometry_derivatives_2d_lossless_match_enumeration(beta, h):
    """Lossless steps (Dcut = 16) give the 2x2 and 4x4 periodic lattices; with square
    orthogonal U the frozen-U derivative is the exact one."""
    db, dh = R.fixed_isometry_derivatives(2, beta, h, 16, 4)
    for n, L in ((2, (2, 2)), (4, (4, 4))):
        e, m = E.moments_bruteforce(beta, h, L)
        assert abs(db[n] - (e + h * m)) < 1e-10
        assert abs(dh[n] - beta * m) < 1e-10


def test_fixed_isometry_derivatives_4d_lossless_match_enumeration():
    beta, h = 0.3, 0.01
    db, dh = R.fixed_isometry_derivatives(4, beta, h, 16, 1)
    e, m = E.moments_bruteforce(beta, h, (1, 1, 1, 2))
    assert abs(db[1] - (e + h * m)) < 1e-10
    assert abs(dh[1] - beta * m) < 1e-10


def test_fixed_isometry_derivative_detects_a_dropped_field_term(monkeypatch):
    """Planted mistake: a site weight that forgets the field must fail the enumeration pin."""
    beta, h = 0.4407, 0.05
    orig = R.site_weight
    monkeypatch.setattr(R, "site_weight", lambda b, hh: orig(b, 0.0))
    db, _ = R.fixed_isometry_derivatives(2, beta, h, 16, 2)
    monkeypatch.setattr(R, "site_weight", orig)
    e, m = E.moments_bruteforce(beta, h, (2, 2))
    assert abs(db[2] - (e + h * m)) > 1e-4


def test_fixed_isometries_reproduce_the_free_flow():
    """Freezing U at the values the flow itself chose changes nothing at the same (beta, h)."""
    f = R.run(4, 0.1497, 0.0, 3, 6)
    g = R.run(4, 0.1497, 0.0, 3, 6, isometries=f.isometries)
    assert f.lnz == g.lnz


@pytest.mark.parametrize("d,beta,h,Dcut,nsteps,L", [(1, 0.7, 0.2, 2, 10, (1024,)),
                                                    (2, 0.4407, 0.05, 16, 4, (4, 4))])
def test_flow_derivatives_lossless_match_exact(d, beta, h, Dcut, nsteps, L):
    """Without truncation the flow's derivative is the lattice's: transfer matrix or enumeration."""
    db, dh = R.flow_derivatives(d, beta, h, Dcut, nsteps)
    if d == 1:
        rb, rh = E.dlnz_1d(beta, h, L[0])
    else:
        e, m = E.moments_bruteforce(beta, h, L)
        rb, rh = e + h * m, beta * m
    assert abs(db[-1] - rb) < 1e-9 and abs(dh[-1] - rh) < 1e-9


def test_flow_and_fixed_isometry_derivatives_differ_by_truncation_terms():
    """Under truncation the two derivatives are different quantities (reading R9): at Dcut = 3
    they part from step 2 on by far more than either's error."""
    fb, fh = R.flow_derivatives(4, 0.16, 0.01, 3, 4)
    xb, xh = R.fixed_isometry_derivatives(4, 0.16, 0.01, 3, 4)
    assert abs(fb[0] - xb[0]) < 1e-10           # T^(0): nothing truncated yet
    for n in (2, 3, 4):
        assert abs(fb[n] - xb[n]) > 1e-3 and abs(fh[n] - xh[n]) > 1e-6


# ------------------------------------------------------------------ impure tensors (Eqs. (impTN)-(spin))
@pytest.mark.parametrize("beta,h", [(0.4407, 0.05), (0.3, 0.0)])
def test_impurity_flow_2d_lossless_matches_enumeration(beta, h):
    """Without truncation Eqs. (energy), (spin) are exact on the 2^n-site lattice: the pair sits
    along the first coarse-graining axis (axis 1 in 2D)."""
    f = R.impurity_flow(2, beta, h, 16, 4)
    for n, L in ((1, (1, 2)), (2, (2, 2)), (3, (2, 4)), (4, (4, 4))):
        pe, ps = E.pair_and_spin_bruteforce(beta, h, L, 1)
        assert abs(f.nn[n - 1] - pe) < 1e-13
        assert abs(f.spin[n] - ps) < 1e-13


def test_impurity_flow_4d_lossless_matches_enumeration():
    beta, h = 0.3, 0.01
    f = R.impurity_flow(4, beta, h, 16, 2)
    for n, L in ((1, (1, 1, 1, 2)), (2, (1, 1, 2, 2))):
        pe, ps = E.pair_and_spin_bruteforce(beta, h, L, 3)
        assert abs(f.nn[n - 1] - pe) < 1e-13 and abs(f.spin[n] - ps) < 1e-13


def test_pair_and_spin_bruteforce_consistent_with_moments():
    """On an isotropic lattice d <s s'> along one axis + h <s> is d(lnZ/N)/d beta."""
    beta, h, L = 0.35, 0.02, (2, 2, 2, 2)
    pe, ps = E.pair_and_spin_bruteforce(beta, h, L, 0)
    e, m = E.moments_bruteforce(beta, h, L)
    # N d bonds (with L = 2 each neighbour pair is joined twice), each with mean <s s'>
    assert abs(e - 4 * pe) < 1e-13 and abs(m - ps) < 1e-14


def test_impurity_flow_symmetries_and_a_planted_mistake():
    """<s> = 0 at h = 0 (Z2) at every step; merging the energy impurity with a pure tensor at
    step 1 (instead of with the second impurity, Eq. (SS)) fails the enumeration pin."""
    f = R.impurity_flow(4, 0.1497, 0.0, 3, 6)
    assert max(abs(x) for x in f.spin) < 1e-15
    assert all(0 < x < 1 for x in f.nn)
    beta, h = 0.4407, 0.05
    good = R.impurity_flow(2, beta, h, 16, 1).nn[0]
    T0 = R.initial_tensor(2, beta, h)
    S0 = R.initial_tensor(2, beta, h, spin_insertion=True)
    _, info = R.coarse_grain(T0, 1, 16)
    U = {b: iso.U for b, iso in info.isometries.items()}
    bad = R.trace(R.squeeze(S0, T0, 1, U)) / R.trace(R.squeeze(T0, T0, 1, U))
    pe, _ = E.pair_and_spin_bruteforce(beta, h, (1, 2), 1)
    assert abs(good - pe) < 1e-13 and abs(bad - pe) > 1e-3
