"""GPU FMM (far field of the coupling by multipole/local expansions, Appendix) against the
oracle's FMM mode, which shares the tree specification but computes every translation by
numerical projection instead of the rotation + coaxial (Gaunt) scheme of the CUDA path.

Tolerances: FP64 operators element by element at 1e-10 of the vector's max-norm (the two sides
form each translation by different arithmetic, whose rounding is amplified up to ~1e5 in the
high-degree coefficients of the projections); FP64 energy 1e-10 relative; the mixed form
(FP32 FMM in the Krylov solves, FP64 FMM in the refinement residuals) 1e-6 relative energy
against the FP64 FMM path on the same input.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ddlpb as O
from paper_2203_00552_gb300 import synth
import paper_2203_00552_gb300 as G

pytestmark = pytest.mark.gpu

KAPPA = synth.KAPPA_PER_ANGSTROM / synth.ANGSTROM_TO_BOHR
EPS = synth.EPS_SOLVENT
DEV = "cuda:0"


def _rand(nvec, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(nvec, generator=g, dtype=torch.float64).to(DEV)


CASES = {
    # name: (M, seed, kind, surface, lmax, n_lebedev, p)
    "globule24_l3_38_p6": (24, 7, "globule", "vdw", 3, 38, 6),
    "globule40_sas_l4_50_p8": (40, 11, "globule", "sas", 4, 50, 8),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def fcase(request):
    M, seed, kind, surf, lmax, n, p = CASES[request.param]
    c, r, q = synth.molecule(M, seed, kind, None, surf)
    P = O.DDLPB(c, r, q, EPS, KAPPA, lmax, n, surface=surf, fmm_order=p)
    ctx = G.Context(c, r, q, EPS, KAPPA, lmax, n, surface=surf, tol=1e-13, fmm_order=p)
    return dict(c=c, r=r, q=q, P=P, ctx=ctx, lmax=lmax, n=n, surf=surf, p=p)


def _apply_both(fc, op, seed):
    P, ctx = fc["P"], fc["ctx"]
    M, nb = P.M, P.nb
    x = _rand(2 * M * nb, seed)
    y = torch.empty_like(x)
    ctx.apply(op, x, y)
    X = x.cpu().numpy().reshape(2 * M, nb)
    if op == G.OP_C:
        cx = P.apply_K(P.ycoef(X[:M], X[M:]))
        ref = np.concatenate([cx, cx])
    elif op == G.OP_CT:
        kt = P.apply_KT(X[:M] + X[M:])
        c1 = (P.eps1 / P.eps2) * P.lidx[None, :] / P.r[:, None]
        ref = np.concatenate([c1 * kt, -P.lexpand(P.di) * kt])
    elif op == G.OP_L:
        ref = P.apply_L(X)
    else:
        ref = P.apply_LT(X)
    return y.cpu().numpy().reshape(2 * M, nb), ref


@pytest.mark.parametrize("op", [G.OP_C, G.OP_CT, G.OP_L, G.OP_LT])
def test_fmm_operators_match_oracle_fmm(fcase, op):
    got, ref = _apply_both(fcase, op, 10 + op)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, err


def test_fmm_rhs_matches_oracle_fmm(fcase):
    P, ctx = fcase["P"], fcase["ctx"]
    g = P.rhs().reshape(-1)
    gd = torch.empty(g.size, dtype=torch.float64, device=DEV)
    ctx.vector(0, gd)
    err = np.abs(gd.cpu().numpy() - g).max() / np.abs(g).max()
    assert err <= 1e-10, err


def test_fmm_energy_matches_oracle_fmm(fcase):
    P, ctx = fcase["P"], fcase["ctx"]
    P.solve()
    E0 = P.energy()
    ctx.solve()
    E = ctx.energy()
    assert abs(E - E0) <= 1e-10 * abs(E0), (E, E0)


def test_fmm_forces_match_oracle_fmm(fcase):
    """Forces in FMM mode: the target-side gradients of the local expansions and the source-side
    gradients through the degree lmax + 1 adjoint (Appendix), near pairs directly; the oracle
    computes the same from its projection-based translations and a projected gradient map."""
    P, ctx = fcase["P"], fcase["ctx"]
    P.solve()
    P.adjoint()
    F0 = P.forces()
    ctx.solve()
    ctx.adjoint()
    F = ctx.forces()
    assert np.abs(F - F0).max() <= 1e-8, np.abs(F - F0).max()


def test_fmm_mixed_matches_fp64_fmm():
    """The mixed form (FP32 FMM inside the Krylov solves, FP64 residuals) on a 200-atom globule at
    lmax 6, p = 8, against the FP64 FMM path on the same input, both solved to the workloads'
    tolerance 1e-8."""
    c, r, q = synth.molecule(200, 21, "globule", None, "vdw")
    kw = dict(tol=1e-8, fmm_order=8, gmres_restart=200)
    a = G.Context(c, r, q, EPS, KAPPA, 6, 110, **kw)
    a.solve()
    E64 = a.energy()
    a.adjoint()
    F64 = a.forces()
    b = G.Context(c, r, q, EPS, KAPPA, 6, 110, precision=G.DDLPB_MIXED, **kw)
    b.solve()
    Em = b.energy()
    b.adjoint()
    Fm = b.forces()
    assert abs(Em - E64) <= 1e-6 * abs(E64), (Em, E64)
    assert np.linalg.norm(Fm - F64) <= 1e-5 * np.linalg.norm(F64)
