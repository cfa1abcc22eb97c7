"""Pins of the oracle's tree (FMM-mode) approximation of the Yukawa far field: exactness of
the projection that forms a multipole, geometric decay of the truncation error with the
expansion order, exact transposition, and convergence of the FMM-mode coupling and energy to
the direct ones."""
import numpy as np
import pytest

from oracle import ddlpb as O
from oracle import fmm
from paper_2203_00552_gb300 import synth

KAPPA = synth.KAPPA_PER_ANGSTROM / synth.ANGSTROM_TO_BOHR


def test_multipole_of_one_source_about_its_centre_is_itself():
    """A node holding one source, centred on it: the projection onto k_l Y_lm must return the
    source's own coefficients (identity embedding into order p), which pins the quadrature,
    the Y_lm normalisation and the radial division at once."""
    from oracle import sph
    L, p = 4, 10
    t = fmm.YukawaTree(np.array([[0.3, -1.2, 2.0]]), KAPPA, L, p)
    nb = (L + 1) ** 2
    E = np.zeros(((p + 1) ** 2, nb))
    E[:nb, :nb] = np.eye(nb)
    # compare in the basis normalised at the check radius: k_l(kappa rho) grows steeply with l
    # at small kappa rho, so entry (a, b) carries the scale k_lb / k_la of the rounding
    ls = np.arange(p + 1)
    k = sph.bessel_k(ls, KAPPA * t.root.rho)[np.repeat(ls, 2 * ls + 1)]
    D = (t.root.P - E) * k[:, None] / k[None, :nb]
    assert np.abs(D).max() <= 1e-12


@pytest.fixture(scope="module")
def cluster():
    rng = np.random.default_rng(0)
    X = rng.uniform(-6, 6, size=(40, 3))
    mu = rng.normal(size=(40, 16))
    T = rng.normal(size=(400, 3))
    T = T / np.linalg.norm(T, axis=1)[:, None] * rng.uniform(8, 30, size=(400, 1))
    return X, mu, T


def test_truncation_error_decays_geometrically_in_p(cluster):
    """The error of a node's multipole at an admissible target is of order theta^(p+1)
    (theta = 1/2): against the direct sum it must fall at every step of p and by more than
    50x from p = 8 to p = 16."""
    X, mu, T = cluster
    err = {}
    for p in (4, 8, 12, 16):
        tr = fmm.YukawaTree(X, 0.055, 3, p)
        ref = tr.potential_direct(mu, T)
        err[p] = np.abs(tr.potential(mu, T) - ref).max() / np.abs(ref).max()
    assert err[4] > err[8] > err[12] > err[16]
    assert err[16] <= err[8] / 50 and err[16] <= 1e-5


def test_tree_products_are_exact_transposes(cluster):
    X, mu, T = cluster
    tr = fmm.YukawaTree(X, 0.055, 3, 8)
    z = np.random.default_rng(1).normal(size=len(T))
    lhs = tr.potential(mu, T) @ z
    rhs = np.sum(mu * tr.potential_T(z, T))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.fixture(scope="module")
def chain():
    c, r, q = synth.molecule(12, 6, "chain")
    return c, r, q


def test_fmm_coupling_converges_to_direct(chain):
    """K (the common map of C1, C2) in FMM mode approaches the direct one as p grows, and
    its transpose stays exact."""
    c, r, q = chain
    d = O.DDLPB(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 50)
    y = np.random.default_rng(2).normal(size=(d.M, d.nb))
    ref = d.apply_K(y)
    err = {}
    for p in (4, 8, 16):
        f = O.DDLPB(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 50, fmm_order=p)
        err[p] = np.abs(f.apply_K(y) - ref).max() / np.abs(ref).max()
    # geometric decay: about one half per order (theta = 1/2), so well over 50x from 8 to 16
    assert err[4] > err[8] > err[16] and err[16] <= err[8] / 50 and err[16] <= 1e-4
    lam = np.random.default_rng(3).normal(size=(d.M, d.nb))
    lhs = np.sum(f.apply_K(y) * lam)
    rhs = np.sum(y * f.apply_KT(lam))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_fmm_energy_converges_to_direct(chain):
    c, r, q = chain
    d = O.DDLPB(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 50)
    d.solve()
    E = d.energy()
    errs = []
    for p in (4, 8, 16):
        f = O.DDLPB(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 50, fmm_order=p)
        f.solve()
        errs.append(abs(f.energy() - E) / abs(E))
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 1e-7
    with pytest.raises(NotImplementedError):
        f.adjoint()
        f.forces()
