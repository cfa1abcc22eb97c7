"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage it rests on.  None of them compares the oracle with
itself through a retyped formula: they use closed forms, library routines,
finite differences, invariances and identities that a wrong sign, a dropped
term or a transposed operand would break.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import ddlpb as O
from oracle import sph
from paper_2203_00552_gb300 import synth

from expansions import harmonic_expansions, plane_wave_expansions

A2B = synth.ANGSTROM_TO_BOHR
KAPPA = 0.104 / A2B
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- basis and quadrature
@pytest.mark.parametrize("n,lmax", [(50, 5), (110, 8), (302, 14), (590, 20)])
def test_lebedev_orthonormality(n, lmax):
    """Sec. 2.2: the Lebedev rule integrates Y_lm Y_l'm' exactly up to its degree."""
    s, w, deg = sph.lebedev(n)
    assert 2 * lmax <= deg
    Y = sph.ylm(lmax, s)
    G = (Y * w[:, None]).T @ Y
    assert abs(G - np.eye(G.shape[0])).max() < 1e-12
    assert abs(w.sum() - 4 * math.pi) < 1e-13


def test_ylm_against_scipy_complex():
    """Real Y_lm of the appendix normalisation vs scipy's complex harmonics."""
    sph_harm_y = getattr(special, "sph_harm_y", None)
    if sph_harm_y is None:
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    u = rng.normal(size=(40, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    th, ph = np.arccos(u[:, 2]), np.arctan2(u[:, 1], u[:, 0])
    Y = sph.ylm(9, u)
    for l in range(10):
        for m in range(-l, l + 1):
            c = sph_harm_y(l, abs(m), th, ph)
            ref = c.real if m == 0 else math.sqrt(2) * (-1) ** m * (c.real if m > 0 else c.imag)
            assert abs(Y[:, l * l + l + m] - ref).max() < 1e-12


def test_ylm_polynomial_vs_legendre():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(64, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    u[0] = [0, 0, 1.0]
    u[1] = [0, 0, -1.0]
    assert abs(sph.solid_harmonics(12, u) - sph.ylm_scipy(12, u)).max() < 1e-11


def test_solid_harmonic_gradient_fd():
    """Eq. derivative_ylm rests on grad Y(x/|x|) = (grad_S Y)/|x|; check the polynomial gradient."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(6, 3))
    R, dR = sph.solid_harmonics(7, x, grad=True)
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (sph.solid_harmonics(7, x + e) - sph.solid_harmonics(7, x - e)) / (2 * h)
        assert abs(fd - dR[..., a]).max() < 1e-7 * max(1.0, abs(R).max())
    u = x / np.linalg.norm(x, axis=1)[:, None]
    Y, gS = sph.ylm_and_grad(7, u)
    assert abs(np.einsum("pbc,pc->pb", gS, u)).max() < 1e-12  # tangential


def test_bessel_closed_forms_and_wronskian():
    """Sec. 2.2 / appendix: i_0 = sinh x / x, k_0 ~ e^-x / x, the small-argument law
    i_n(x) ~ x^n/(2n+1)!!, and the Wronskian i_n k_n' - i_n' k_n = -pi/(2 x^2)."""
    x = np.array([0.01, 0.1, 0.5, 1.0, 3.0, 10.0])
    assert np.allclose(sph.bessel_i(0, x), np.sinh(x) / x, rtol=1e-14)
    assert np.allclose(sph.bessel_i(1, x), (x * np.cosh(x) - np.sinh(x)) / x ** 2, rtol=1e-9)
    assert np.allclose(sph.bessel_k(0, x), math.pi / 2 * np.exp(-x) / x, rtol=1e-14)
    for n in range(0, 12):
        wr = sph.bessel_i(n, x) * sph.bessel_k_deriv(n, x) - sph.bessel_i_deriv(n, x) * sph.bessel_k(n, x)
        assert np.allclose(wr, -math.pi / (2 * x ** 2), rtol=1e-10)
        df = 1.0
        for k in range(1, 2 * n + 2, 2):
            df *= k
        assert abs(sph.bessel_i(n, 1e-4) / (1e-4 ** n / df) - 1) < 1e-7


# ---------------------------------------------------------------- smooth switch (Eq. regular_char_function)
@pytest.mark.parametrize("eta", [0.1, 0.3, 0.7])
def test_chi_eta_c2(eta):
    """chi_eta must be C^2: value 1 / 0 and zero first and second derivative at both ends."""
    a, b = 1 - eta, 1.0
    h = 1e-6
    for t0, v in ((a, 1.0), (b, 0.0)):
        for t in (t0 - h, t0 + h):
            assert abs(O.chi_eta(np.array([t]), eta)[0] - v) < 1e-5
        d = O.dchi_eta(np.array([t0 - h, t0 + h]), eta)
        assert abs(d).max() < 1e-4
    tt = np.linspace(a + 1e-4, b - 1e-4, 50)
    fd = (O.chi_eta(tt + 1e-7, eta) - O.chi_eta(tt - 1e-7, eta)) / 2e-7
    assert abs(fd - O.dchi_eta(tt, eta)).max() < 1e-5
    # second derivative vanishes at the ends: chi'(end +- h)/h = O(h), not O(1/eta^2)
    d2 = (O.dchi_eta(np.array([a + 1e-7, b - 1e-7]), eta)) / 1e-7
    assert abs(d2).max() < 1e-3 / eta ** 2


def test_printed_p_eta_constant_is_not_continuous():
    """The literal constant 1 - eta^2 - 15 eta + 6 gives p_eta(1 - eta) != 1; the reading 10 eta^2 - 15 eta + 6 gives 1."""
    eta = 0.1
    t = 1 - eta
    lit = eta ** -5 * (1 - t) ** 3 * (6 * t * t + (15 * eta - 12) * t + 1 - eta ** 2 - 15 * eta + 6)
    assert abs(lit - 1) > 1.0
    assert abs(O.chi_eta(np.array([t + 1e-12]), eta)[0] - 1) < 1e-9


# ---------------------------------------------------------------- physics pins
def _born(q, a, eps2, kappa, eps1=1.0):
    return q * q / (2 * a) * (1.0 / (eps2 * (1 + kappa * a)) - 1.0 / eps1)


@pytest.mark.parametrize("lmax,n", [(0, 6), (2, 26), (6, 110)])
def test_born_debye_hueckel_exact(lmax, n):
    """One ion in one sphere: the discrete system reproduces the Born/DH energy for every lmax."""
    with open(os.path.join(GOLDEN, "born_dh.json")) as f:
        gold = json.load(f)
    for c in gold["cases"]:
        a = c["a_angstrom"] * A2B
        kap = max(c["kappa_per_angstrom"] / A2B, 1e-12)
        E, F, _ = O.run([[0.3, -0.2, 0.1]], [a], [c["q"]], c["eps_solvent"], kap, lmax, n)
        assert abs(E - _born(c["q"], a, c["eps_solvent"], kap)) < 1e-12
        assert abs(E - c["energy"]) < 2e-10
        assert abs(F).max() < 1e-12


def test_born_scaling_in_q_and_a():
    for q, a, kap in ((-0.7, 3.1, 0.02), (2.0, 1.5, 0.3)):
        E, _, _ = O.run([[0, 0, 0]], [a], [q], 40.0, kap, 3, 50, forces=False)
        assert abs(E - _born(q, a, 40.0, kap)) < 1e-12 * abs(E) + 1e-15


def test_two_distant_ions_asymptotics():
    """Two non-overlapping ions: E - E_Born1 - E_Born2 tends to the screened pair term
    q1 q2 [exp(kappa (a1 + a2 - d)) / (eps2 d (1 + kappa a1)(1 + kappa a2)) - 1/(eps1 d)]."""
    q1, q2, a1, a2, eps2 = 0.8, -0.6, 3.0, 2.5, 78.54
    kap = 0.08
    resid = []
    for d in (12.0, 24.0, 48.0):
        E, _, _ = O.run([[0, 0, 0], [d, 0.0, 0.0]], [a1, a2], [q1, q2], eps2, kap, 6, 110, forces=False)
        pair = q1 * q2 * (math.exp(kap * (a1 + a2 - d)) / (eps2 * d * (1 + kap * a1) * (1 + kap * a2)) - 1.0 / d)
        r = E - _born(q1, a1, eps2, kap) - _born(q2, a2, eps2, kap) - pair
        resid.append(abs(r) / abs(pair))
    assert resid[0] < 0.05
    assert resid[2] < resid[1] < resid[0]


def test_isolated_spheres_have_identity_AB():
    """Eq. definition_of_A_matrix: with no overlaps A = B = I."""
    p = O.DDLPB([[0, 0, 0], [20, 0, 0]], [3, 3], [0.5, -0.5], 78.54, KAPPA, 3, 50)
    X = np.random.default_rng(0).normal(size=(2, p.nb))
    assert np.allclose(p.apply_A(X), X, atol=0)
    assert np.allclose(p.apply_B(X), X, atol=0)
    assert np.allclose(p.chi, 1.0)


@pytest.fixture(scope="module")
def chain8():
    c, r, q = synth.molecule(8, 3, "chain")
    return c, r, q


def test_dense_equals_matrix_free_and_transpose(chain8):
    """The assembled L (entry formulas of Sec. 2.2) equals the matrix-free product, and
    <L x, y> = <x, L* y> with L* of Eq. AstarXg."""
    c, r, q = chain8
    p = O.DDLPB(c, r, q, 78.54, KAPPA, 3, 50)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(2 * p.M, p.nb))
    Yv = rng.normal(size=(2 * p.M, p.nb))
    L = p.assemble_L()
    assert abs(L @ X.ravel() - p.apply_L(X).ravel()).max() < 1e-12
    lhs = (p.apply_L(X) * Yv).sum()
    rhs = (X * p.apply_LT(Yv)).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the two blocks of C are not symmetric, so a transposed operand is caught
    assert abs(L - L.T).max() > 1e-3


def test_sampled_rows_equal_the_full_products():
    """The sampled-row forms used at full size (rows of A X, B X, A^T Y, B^T Y and of the coupling
    and its transpose, summed over sources in blocks) equal the rows of the full products above,
    on a globule with buried, partly covered and exposed spheres."""
    c, r, q = synth.molecule(30, 3, "globule", None, "sas")
    p = O.DDLPB(c, r, q, 78.54, KAPPA, 4, 50, surface="sas")
    n_ext = (p.chi > 0).sum(axis=1)
    rows = [int(n_ext.argmin()), int(n_ext.argmax()), int(np.abs(n_ext - p.N // 2).argmin()), p.M - 1]
    assert n_ext[rows[0]] == 0 and n_ext[rows[1]] > 0
    rng = np.random.default_rng(4)
    Y = rng.normal(size=(p.M, p.nb))
    for kind in "ri":
        assert np.abs(p.apply_A_rows(Y, rows, kind) - p.apply_A(Y, kind)[rows]).max() < 1e-13
        assert np.abs(p.apply_AT_rows(Y, rows, kind) - p.apply_AT(Y, kind)[rows]).max() < 1e-13
    for got, want in ((p.apply_K_rows(Y, rows), p.apply_K(Y)[rows]), (p.apply_KT_rows(Y, rows), p.apply_KT(Y)[rows])):
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_gmres_matches_dense(chain8):
    c, r, q = chain8
    p1 = O.DDLPB(c, r, q, 78.54, KAPPA, 3, 50)
    p1.solve(dense=True)
    p2 = O.DDLPB(c, r, q, 78.54, KAPPA, 3, 50)
    p2.solve(dense=False)
    assert abs(p1.X - p2.X).max() < 1e-11 * abs(p1.X).max()


def test_forces_central_fd_and_net_force(chain8):
    """Sec. 4.1.1: analytical forces equal finite differences of the discrete energy
    (central differences here, so O(h^2)), and the net force vanishes (translation invariance)."""
    c, r, q = chain8
    E, F, p = O.run(c, r, q, 78.54, KAPPA, 3, 50)
    assert abs(F.sum(0)).max() < 1e-12 * abs(F).max()
    # E is only C^0 where some f^i crosses 1 (the min in Eq. di); this seed keeps every
    # switching point at least 1e-5 away from that kink
    assert np.min(np.abs(p.f[(p.f > 0) & (np.abs(p.f - 1) > 1e-12)] - 1)) > 1e-5
    h = 1e-4
    for k, a in ((0, 0), (2, 1), (5, 2), (7, 0), (3, 2)):
        cp = c.copy()
        cp[k, a] += h
        cm = c.copy()
        cm[k, a] -= h
        Ep, _, _ = O.run(cp, r, q, 78.54, KAPPA, 3, 50, forces=False)
        Em, _, _ = O.run(cm, r, q, 78.54, KAPPA, 3, 50, forces=False)
        assert abs(-(Ep - Em) / (2 * h) - F[k, a]) < 1e-9


def test_translation_invariance(chain8):
    c, r, q = chain8
    E0, _, _ = O.run(c, r, q, 78.54, KAPPA, 3, 50, forces=False)
    E1, _, _ = O.run(c + np.array([1.7, -3.2, 0.4]), r, q, 78.54, KAPPA, 3, 50, forces=False)
    assert abs(E1 - E0) < 1e-12 * abs(E0)


def test_rotation_fluctuation_shrinks_with_discretisation():
    """Sec. 4.1.3: the energy of a diatomic under rotation fluctuates (the grid is fixed),
    and the fluctuation shrinks as (lmax, N_leb) grows."""
    rH, rF = 1.2 * 1.1 * A2B, 1.47 * 1.1 * A2B
    d = 0.92 * A2B
    spreads = []
    for lmax, n in ((6, 110), (10, 302)):
        Es = []
        for th in np.linspace(0.1, 3.0, 7):
            xf = [d * math.sin(th) * math.cos(0.3 * th), d * math.sin(th) * math.sin(0.3 * th), d * math.cos(th)]
            E, _, _ = O.run([[0, 0, 0], xf], [rH, rF], [0.4, -0.4], 78.54, KAPPA, lmax, n, forces=False)
            Es.append(E)
        spreads.append(np.ptp(Es))
    assert spreads[1] < spreads[0]


def _kirkwood_tanford(q, a, b, eps2, kappa, lmax, eps1=1.0):
    """Energy and radial force of a charge q at distance b from the centre of a dielectric
    ball of radius a (eps1 inside) in a screened solvent (eps2, kappa), truncated at lmax:
    E = q^2/(2 eps1) sum_l R_l b^(2l) / a^(2l+1),
    R_l = [(eps1/eps2)(l+1)/a + beta_l] / [(eps1/eps2) l/a - beta_l], beta_l = kappa k_l'(kappa a)/k_l(kappa a)."""
    E = 0.0
    dE = 0.0
    for l in range(lmax + 1):
        beta = kappa * special.spherical_kn(l, kappa * a, derivative=True) / special.spherical_kn(l, kappa * a)
        R = ((eps1 / eps2) * (l + 1) / a + beta) / ((eps1 / eps2) * l / a - beta)
        E += R * b ** (2 * l) / a ** (2 * l + 1)
        if l > 0:
            dE += R * 2 * l * b ** (2 * l - 1) / a ** (2 * l + 1)
    return q * q / (2 * eps1) * E, q * q / (2 * eps1) * dE


@pytest.mark.parametrize("lmax,n", [(3, 110), (6, 302)])  # quadrature degree >= lmax + 14: aliasing < 1e-12
def test_kirkwood_tanford_off_centre_charge(lmax, n):
    """A charged atom with a tiny sphere buried inside a large neutral sphere: the large sphere
    behaves as an isolated dielectric ball and the small one samples its reaction field at the
    charge, so the discrete energy equals the Kirkwood-Tanford multipole sum up to lmax (this pins
    every l > 0 factor of C1, C2, F0 and the A coupling) and the analytical force equals -dE/db."""
    a, eps2, kap = 6.0, 78.54, 0.09
    b_dir = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    b = 0.25 * a
    c = np.array([[0.0, 0.0, 0.0], b * b_dir])
    r = np.array([a, 0.2 * a])
    q = np.array([0.0, 0.7])
    E, F, p = O.run(c, r, q, eps2, kap, lmax, n)
    E_ref, dE_ref = _kirkwood_tanford(0.7, a, b, eps2, kap, lmax)
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref)
    assert np.allclose(F[1], -dE_ref * b_dir, rtol=1e-8, atol=1e-12)
    assert np.allclose(F[0], -F[1], rtol=1e-10, atol=1e-14)
    # the l > 0 terms matter: dropping them changes the energy well beyond the tolerance
    E0, _ = _kirkwood_tanford(0.7, a, b, eps2, kap, 0)
    assert abs(E_ref - E0) > 1e-4 * abs(E_ref)


# ---------------------------------------------------------------- A and B entry by entry
# Eqs. definition_of_A_matrix, definition_of_B_matrix with the switch weights of Eqs.
# regular_omega_ij, di, regular_chi_e: sum_j omega_ij^eta = 1 - chi_i^eta at every grid point
# (d^i = min(f, 1)/f), and each neighbour's expansion of a harmonic polynomial (basis r_l Y) or
# of a plane wave exp(kappa u.x) (basis i-ratio Y, an exact solution of the screened equation)
# is exact, so (A X_h)_i = analysis_i(chi_i h) and (B X_pw)_i = analysis_i(chi_i pw) sphere by
# sphere.  A wrong omega (e.g. d = 1/f also where f < 1), a wrong radial scaling or a wrong
# Y_lm convention breaks these identities on any geometry with partly covered spheres.

def _dense_globule(lmax=4, n=50):
    c, r, q = synth.molecule(14, 2, "eden", None, "vdw")
    P = O.DDLPB(c, r, q, 78.54, KAPPA, lmax, n)
    f = P.f
    # the geometry must reach both branches of d^i and partial covering
    assert (f > 1.0).any() and ((f > 0.0) & (f < 1.0)).any()
    return P


@pytest.mark.parametrize("L,M", [(0, 0), (1, -1), (2, 1), (3, 0), (4, -3)])
def test_A_reproduces_harmonic_polynomials(L, M):
    P = _dense_globule()
    vals, X = harmonic_expansions(P, np.array([0.7, -1.3, 2.1]), L, M)
    lhs = P.apply_A(X)
    rhs = np.stack([P.analysis(P.chi[i] * vals[i]) for i in range(P.M)])
    assert np.abs(lhs - rhs).max() <= 1e-12 * max(np.abs(X).max(), 1.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_B_reproduces_plane_waves(seed):
    P = _dense_globule(8, 110)
    rng = np.random.default_rng(seed)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    vals, X = plane_wave_expansions(P, u)
    lhs = P.apply_B(X)
    rhs = np.stack([P.analysis(P.chi[i] * vals[i]) for i in range(P.M)])
    # truncation at lmax = 8 of the plane wave: about (kappa rho)^9 / 19!! with kappa rho < 0.35,
    # below 1e-12 (at lmax = 4 it is 1e-7)
    assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(X).max()
