"""Pins of the oracle's FMM mode (the Yukawa far field of the coupling by multipole and local
expansions over a binary tree, Appendix): the tree specification (coverage of every pair,
admissibility), a translation against the textbook addition theorem, geometric decay of the
far-field error with the expansion order, exact transposition of the adjoint pass, the gradient
map against finite differences, and FMM-mode energy and forces against the direct ones and
against finite differences of the FMM-mode energy."""
import numpy as np
import pytest

from oracle import ddlpb as O
from oracle import fmm, sph
from paper_2203_00552_gb300 import synth

KAPPA = synth.KAPPA_PER_ANGSTROM / synth.ANGSTROM_TO_BOHR


@pytest.fixture(scope="module")
def globule24():
    c, r, q = synth.molecule(24, 7, "globule", None, "vdw")
    return c, r, q


def _leaves_below(F, k):
    if F.leaf_sphere[k] >= 0:
        return [int(F.leaf_sphere[k])]
    return [s for ch in F.child[k] for s in _leaves_below(F, ch)]


def test_tree_covers_every_pair_once_and_respects_admissibility(globule24):
    c, r, _ = globule24
    F = fmm.YukawaFMM(c, r, KAPPA, 3, 6)
    M = len(c)
    assert sorted(F.order.tolist()) == list(range(M))
    cover = np.zeros((M, M), dtype=int)
    for A, B in F.m2l:
        d = np.linalg.norm(F.c[A] - F.c[B])
        assert F.Rt[A] + F.Rs[B] < F.theta * d
        for i in _leaves_below(F, A):
            for j in _leaves_below(F, B):
                cover[i, j] += 1
    for i in range(M):
        for j in F.near[i]:
            cover[i, j] += 1
            d = np.linalg.norm(c[i] - c[j])
            assert not (r[i] < F.theta * d)      # a near pair of leaves is not admissible
    assert (cover == 1).all()
    # node geometry: every sphere of a node lies within Rs of its centre, its ball within Rt
    for k in range(len(F.a)):
        idx = F.order[F.a[k]:F.b[k]]
        d = np.linalg.norm(c[idx] - F.c[k], axis=1)
        assert (d <= F.Rs[k] + 1e-12).all() and (d + r[idx] <= F.Rt[k] + 1e-12).all()


def test_monopole_m2l_equals_the_gegenbauer_addition_theorem():
    """k_0(kappa |x - y|) = sum_n (2n+1) i_n(kappa |x|) k_n(kappa |y|) P_n(cos gamma) for |x| < |y|
    (the textbook addition theorem of the modified spherical Bessel functions): the projected
    M2L of the unit monopole Y_00 k_0(kappa|x - y|)/k_0(kappa R_S) at y = d e_z onto the origin's
    locals (scale R_T) must carry, at (n, 0), the coefficient
    Y_00 (2n+1) k_n(kappa d) sqrt(4 pi / (2n+1)) i_n(kappa R_T) / k_0(kappa R_S), and nothing at m != 0."""
    d = 9.0
    c = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]])
    r = np.array([2.5, 1.5])
    F = fmm.YukawaFMM(c, r, KAPPA, 0, 10)
    A = int(F.leaf_node[0])
    B = int(F.leaf_node[1])
    T = F.translation("M2L", B, A)
    for n in range(11):
        want = (np.sqrt(1 / (4 * np.pi)) * (2 * n + 1) * sph.bessel_k(n, KAPPA * d) * np.sqrt(4 * np.pi / (2 * n + 1))
                * sph.bessel_i(n, KAPPA * r[0]) / sph.bessel_k(0, KAPPA * r[1]))
        got = T[n * n + n, 0]
        assert abs(got - want) <= 1e-9 * abs(want) + 1e-13, (n, got, want)
        for m in range(-n, n + 1):
            if m != 0:
                assert abs(T[n * n + n + m, 0]) <= 1e-13


def _far_error(c, r, p, lmax=3, seed=1):
    rng = np.random.default_rng(seed)
    mu = rng.normal(size=(len(c), (lmax + 1) ** 2))
    F = fmm.YukawaFMM(c, r, KAPPA, lmax, p)
    L = F.locals(mu)
    s, w, _ = sph.lebedev(38)
    err = 0.0
    for i in range(len(c)):
        pts = c[i] + r[i] * s
        far = [j for j in range(len(c)) if j not in F.near[i]]
        err = max(err, np.abs(sph.ylm(p, s) @ L[i] - F.potential_direct(mu, pts, far)).max())
    return err


def test_far_field_error_decays_with_the_order(globule24):
    """The truncation error of the multipole/local expansions: measured 0.36 -> 5e-3 from
    p = 4 to 12 on a 16-atom globule; it must fall at each step and by more than 20x."""
    c, r, _ = synth.molecule(16, 7, "globule", None, "vdw")
    e = [_far_error(c, r, p) for p in (4, 8, 12)]
    assert e[0] > e[1] > e[2]
    assert e[2] < e[0] / 20.0


def test_adjoint_pass_is_the_exact_transpose(globule24):
    c, r, _ = globule24
    F = fmm.YukawaFMM(c, r, KAPPA, 3, 5)
    rng = np.random.default_rng(3)
    mu = rng.normal(size=(len(c), 16))
    lam = rng.normal(size=(len(c), 36))
    lhs = float((F.locals(mu) * lam).sum())
    rhs = float((mu * F.locals_T(lam)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the degree-p leaves of the full adjoint truncate to the adjoint of the degree-lmax leaves
    assert np.allclose(F.locals_T_full(lam)[:, :16], F.locals_T(lam), rtol=0, atol=1e-14 * np.abs(lam).max())


def test_gradient_map_against_finite_differences():
    c = np.array([[0.4, -0.3, 0.2], [8.0, 1.0, -2.0]])
    r = np.array([2.2, 1.7])
    F = fmm.YukawaFMM(c, r, KAPPA, 3, 6)
    D = F.gradient_map(0, 3)                                   # [3, 16, 25]
    x = c[0] + np.array([[3.1, -2.2, 1.4], [-1.0, 4.0, 2.5]])
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (fmm.basis("S", 3, KAPPA, x + e - c[0], r[0]) - fmm.basis("S", 3, KAPPA, x - e - c[0], r[0])) / (2 * h)
        via = fmm.basis("S", 4, KAPPA, x - c[0], r[0]) @ D[a].T
        assert np.abs(fd - via).max() <= 1e-7 * np.abs(via).max()
    # each gradient reaches only the degrees l - 1 and l + 1
    for l in range(4):
        for lp in range(5):
            if abs(lp - l) != 1:
                blk = D[:, l * l:(l + 1) ** 2, lp * lp:(lp + 1) ** 2]
                assert np.abs(blk).max() <= 1e-10 * np.abs(D).max()


@pytest.fixture(scope="module")
def direct16():
    c, r, q = synth.molecule(16, 7, "globule", None, "vdw")
    E, F, _ = O.run(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 38)
    return c, r, q, E, F


def test_fmm_mode_energy_and_forces_track_the_direct_ones(direct16):
    """Measured at p = 8: energy 1.9e-6 relative, forces 1.1e-6 against max |F| = 8.6e-3."""
    c, r, q, E, F = direct16
    P = O.DDLPB(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 38, fmm_order=8)
    P.solve()
    P.adjoint()
    Ef, Ff = P.energy(), P.forces()
    assert abs(Ef - E) <= 2e-5 * abs(E)
    assert np.abs(Ff - F).max() <= 1e-3 * np.abs(F).max()
    assert np.abs(Ff.sum(axis=0)).max() <= 1e-3 * np.abs(F).max()


def test_fmm_mode_forces_against_finite_differences_of_the_fmm_energy(direct16):
    """The FMM-mode forces evaluate the exact force expression with FMM fields, so they equal the
    derivative of the FMM-mode energy up to the FMM error (measured 2.6e-8 at p = 6)."""
    c, r, q, _, _ = direct16
    p = 6
    P = O.DDLPB(c, r, q, synth.EPS_SOLVENT, KAPPA, 3, 38, fmm_order=p)
    P.solve()
    P.adjoint()
    F = P.forces()
    h = 1e-4
    for k, a in ((0, 0), (5, 2)):
        ep = []
        for s in (1, -1):
            cc = c.copy()
            cc[k, a] += s * h
            Q = O.DDLPB(cc, r, q, synth.EPS_SOLVENT, KAPPA, 3, 38, fmm_order=p)
            Q.solve()
            ep.append(Q.energy())
        fd = -(ep[0] - ep[1]) / (2 * h)
        assert abs(fd - F[k, a]) <= 1e-6, (k, a, fd, F[k, a])
