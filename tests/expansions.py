"""Exact expansions about every sphere of functions the blocks A and B reproduce: solid
harmonics (harmonic polynomials, regular basis of A) and plane waves exp(kappa u.x) (solutions
of the screened equation, regular i-basis of B).  Used by the oracle pins and by the GPU tests
of the same identities."""
import numpy as np

from oracle import sph


def harmonic_expansions(P, centre, L, M):
    """Coefficients about every sphere of the solid harmonic R_LM(x - centre) (degree L <= lmax)
    in the basis (rho/r_j)^l Y_lm, from its values on each sphere (exact: a polynomial of degree
    <= lmax), and those values [M, N]."""
    vals = np.stack([sph.solid_harmonics(L, P.pts[j] - centre)[:, L * L + L + M] for j in range(P.M)])
    return vals, np.stack([P.analysis(vals[j]) for j in range(P.M)])


def plane_wave_expansions(P, u):
    """exp(kappa u.x) about every sphere in the basis i_l(kappa rho)/i_l(kappa r_j) Y_lm:
    X_j,lm = exp(kappa u.x_j) 4 pi i_l(kappa r_j) Y_lm(u) (the plane-wave expansion), and its
    values at every grid point."""
    Yu = sph.ylm(P.lmax, u[None, :])[0]
    X = np.stack([np.exp(P.kappa * u @ P.x[j]) * 4 * np.pi * P.lexpand(P.i_r[j]) * Yu for j in range(P.M)])
    vals = np.exp(P.kappa * P.pts @ u)
    return vals, X


def masked_analysis(P, vals):
    """analysis(chi_i vals_i) for every sphere: what A (or B) applied to the exact expansion of
    vals gives."""
    return P.analysis(P.chi * vals)
