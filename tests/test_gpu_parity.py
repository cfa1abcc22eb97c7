"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path): relative energy error <= 1e-10 and max force error
<= 1e-8 Hartree/Bohr against the oracle on the same seeded inputs; every
operator and the right-hand side element by element at 1e-11 of the vector's
max-norm (a few hundred FP64 roundings of O(1) terms).
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


def _ctx(c, r, q, lmax, n, surface="vdw", **kw):
    kw.setdefault("tol", 1e-13)
    return G.Context(c, r, q, EPS, KAPPA, lmax, n, surface=surface, **kw)


def _flat(p, X):
    return np.asarray(X).reshape(-1)


def _rand(nvec, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(nvec, generator=g, dtype=torch.float64).to(DEV)


CASES = {
    # name: (M, seed, kind, surface, lmax, n_lebedev)
    "chain20_l6_110": (20, 0, "chain", "vdw", 6, 110),
    "chain37_l5_86": (37, 5, "chain", "vdw", 5, 86),
    "globule45_sas_l4_50": (45, 7, "globule", "sas", 4, 50),
    "globule60_l3_38": (60, 9, "globule", "vdw", 3, 38),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    M, seed, kind, surf, lmax, n = CASES[request.param]
    c, r, q = synth.molecule(M, seed, kind, None, surf)
    p = O.DDLPB(c, r, q, EPS, KAPPA, lmax, n, surface=surf)
    g = p.rhs()
    ctx = _ctx(c, r, q, lmax, n, surf)
    return dict(name=request.param, c=c, r=r, q=q, p=p, g=g, ctx=ctx, lmax=lmax, n=n, surf=surf)


def test_counts_match_oracle(case):
    p, ctx = case["p"], case["ctx"]
    info = ctx.info()
    assert info["n_neighbour_pairs"] == sum(len(x) for x in p.nbrs)
    assert info["n_external"] == int((p.chi > 0).sum())
    hits = sum(int((p.t(i, j) < 1).sum()) for i in range(p.M) for j in p.nbrs[i])
    assert info["n_hits"] == hits


def test_rhs_parity(case):
    ctx, g = case["ctx"], case["g"]
    out = torch.empty(ctx.nvec, dtype=torch.float64, device=DEV)
    ctx.vector(0, out)
    ref = g.reshape(-1)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("op", ["L", "LT", "AB", "ABT", "C", "CT"])
def test_operator_parity(case, op):
    p, ctx = case["p"], case["ctx"]
    M, nb = p.M, p.nb
    x = _rand(ctx.nvec, 11)
    xn = x.cpu().numpy().reshape(2 * M, nb)
    if op == "L":
        ref = p.apply_L(xn)
        code = G.OP_L
    elif op == "LT":
        ref = p.apply_LT(xn)
        code = G.OP_LT
    elif op == "AB":
        ref = np.concatenate([p.apply_A(xn[:M]), p.apply_B(xn[M:])])
        code = G.OP_AB
    elif op == "ABT":
        ref = np.concatenate([p.apply_AT(xn[:M]), p.apply_AT(xn[M:], kind="i")])
        code = G.OP_ABT
    elif op == "C":
        k = p.apply_K(p.ycoef(xn[:M], xn[M:]))
        ref = np.concatenate([k, k])
        code = G.OP_C
    else:
        kt = p.apply_KT(xn[:M] + xn[M:])
        c1 = (p.eps1 / p.eps2) * p.lidx[None, :] / p.r[:, None]
        ref = np.concatenate([c1 * kt, -p.lexpand(p.di) * kt])
        code = G.OP_CT
    y = torch.empty_like(x)
    ctx.apply(code, x, y)
    yn = y.cpu().numpy().reshape(2 * M, nb)
    assert np.abs(yn - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1.0)


def test_energy_and_forces_parity(case):
    p, ctx = case["p"], case["ctx"]
    p.solve()
    E_ref = p.energy()
    p.adjoint()
    F_ref = p.forces()
    case["F_ref"] = F_ref
    ctx.solve()
    E = ctx.energy()
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref)
    ctx.adjoint()
    F = ctx.forces()
    assert np.abs(F - F_ref).max() <= 1e-8
    assert np.abs(F.sum(0)).max() <= 1e-10 * max(np.abs(F).max(), 1e-12) * F.shape[0]
    X = torch.empty(ctx.nvec, dtype=torch.float64, device=DEV)
    ctx.vector(1, X)
    assert np.abs(X.cpu().numpy() - p.X.reshape(-1)).max() <= 1e-9 * np.abs(p.X).max()
    info = ctx.info()
    assert info["solve_residual"] <= 1e-12 and info["adjoint_residual"] <= 1e-12


def test_single_ion_born():
    a = 2.0 * synth.ANGSTROM_TO_BOHR
    ctx = _ctx(np.array([[0.5, -1.0, 2.0]]), np.array([a]), np.array([1.0]), 4, 50)
    ctx.solve()
    E = ctx.energy()
    ref = 1.0 / (2 * a) * (1.0 / (EPS * (1 + KAPPA * a)) - 1.0)
    assert abs(E - ref) <= 1e-12 * abs(ref)
    ctx.adjoint()
    assert np.abs(ctx.forces()).max() < 1e-12


def test_isolated_and_nested_spheres():
    # two isolated ions (no hits) and one sphere swallowed by another (no external points)
    c = np.array([[0.0, 0, 0], [30.0, 0, 0], [30.5, 0.2, 0.0]])
    r = np.array([3.0, 4.0, 1.5])
    q = np.array([0.4, -0.3, 0.2])
    p = O.DDLPB(c, r, q, EPS, KAPPA, 4, 50)
    p.solve()
    p.adjoint()
    ctx = _ctx(c, r, q, 4, 50)
    assert ctx.info()["n_external"] == int((p.chi > 0).sum())
    ctx.solve()
    assert abs(ctx.energy() - p.energy()) <= 1e-10 * abs(p.energy())
    ctx.adjoint()
    assert np.abs(ctx.forces() - p.forces()).max() <= 1e-8
    # mixed precision with no hits at all (two far ions): the stored FP32/FP16 paths are empty
    c2, r2, q2 = c[:2], r[:2], q[:2]
    p2 = O.DDLPB(c2, r2, q2, EPS, KAPPA, 4, 50)
    p2.solve()
    m = _ctx(c2, r2, q2, 4, 50, precision=G.DDLPB_MIXED, tol=1e-12)
    assert m.info()["n_hits"] == 0
    m.solve()
    assert abs(m.energy() - p2.energy()) <= 1e-10 * abs(p2.energy())


@pytest.mark.parametrize("precision", [0, 1])
def test_max_degree_parity(precision):
    """The largest degree the library takes (lmax 16, 434-point grid, exact to degree 35) on a
    3-atom chain: energy and forces match the oracle, FP64 and mixed."""
    c, r, q = synth.molecule(3, 11, "chain")
    p = O.DDLPB(c, r, q, EPS, KAPPA, 16, 434)
    p.solve()
    p.adjoint()
    ctx = _ctx(c, r, q, 16, 434, precision=precision, tol=1e-12)
    assert ctx.info()["n_hits"] > 0
    ctx.solve()
    assert abs(ctx.energy() - p.energy()) <= 1e-10 * abs(p.energy())
    ctx.adjoint()
    F, F_ref = ctx.forces(), p.forces()
    assert np.abs(F - F_ref).max() <= 1e-8 * max(1.0, np.abs(F_ref).max())


def test_high_degree_globule_parity():
    """lmax 10 on a 30-atom globule (590 points), the degree at which the energy of these dense
    globules starts to drift with lmax (a property of the discretisation, which the oracle
    shows too): the GPU energy equals the oracle's dense solve to 1e-10 relative."""
    c, r, q = synth.molecule(30, 3, "globule", None, "vdw")
    p = O.DDLPB(c, r, q, EPS, KAPPA, 10, 590)
    p.solve(dense=True)
    ctx = _ctx(c, r, q, 10, 590, tol=1e-12, gmres_restart=300, max_iter=4000)
    ctx.solve()
    assert abs(ctx.energy() - p.energy()) <= 1e-10 * abs(p.energy())


def test_device_setup_and_outputs_match_host():
    c, r, q = synth.molecule(12, 4, "chain")
    h = _ctx(c, r, q, 4, 50)
    h.solve()
    h.adjoint()
    d = G.Context(torch.tensor(c, device=DEV), torch.tensor(r, device=DEV), torch.tensor(q, device=DEV), EPS, KAPPA,
                  4, 50, tol=1e-13)
    d.solve()
    d.adjoint()
    e = torch.empty(1, dtype=torch.float64, device=DEV)
    d.energy_device(e)
    f = torch.empty((12, 3), dtype=torch.float64, device=DEV)
    d.forces_device(f)
    # same inputs, same result up to the order of the atomic accumulations
    assert abs(float(e) - h.energy()) <= 1e-13 * abs(h.energy())
    assert np.abs(f.cpu().numpy() - h.forces()).max() <= 1e-12 * np.abs(h.forces()).max()


def test_error_paths():
    c, r, q = synth.molecule(6, 1, "chain")
    ctx = _ctx(c, r, q, 3, 50)
    with pytest.raises(G.DDLPBError) as e:
        ctx.adjoint()
    assert e.value.status == 5
    with pytest.raises(G.DDLPBError) as e:
        ctx.forces()
    assert e.value.status == 5
    bad = _ctx(c, r, q, 3, 50, max_iter=1, tol=1e-14)
    with pytest.raises(G.DDLPBError) as e:
        bad.solve()
    assert e.value.status == 3
    rr = r.copy()
    rr[2] = np.nan
    with pytest.raises(G.DDLPBError) as e:
        _ctx(c, rr, q, 3, 50)
    assert e.value.status == 1


def test_mixed_precision_refinement_parity(case):
    """FP32 Krylov solves inside FP64 refinement reach the FP64 solution: at a tight
    tolerance the energy matches the oracle to 1e-10 relative; at the default 1e-8 the
    mixed form stays within 1e-6 relative energy and 1e-5 relative force norm."""
    p = case["p"]
    if "F_ref" not in case:
        p.solve()
        p.adjoint()
        case["F_ref"] = p.forces()
    E_ref = p.energy()
    F_ref = case["F_ref"]
    tight = _ctx(case["c"], case["r"], case["q"], case["lmax"], case["n"], case["surf"], precision=G.DDLPB_MIXED,
                 tol=1e-12)
    tight.solve()
    assert abs(tight.energy() - E_ref) <= 1e-10 * abs(E_ref)
    info = tight.info()
    assert info["refinement_steps"] >= 1 and info["solve_residual"] <= 1e-12
    loose = _ctx(case["c"], case["r"], case["q"], case["lmax"], case["n"], case["surf"], precision=G.DDLPB_MIXED,
                 tol=1e-8)
    loose.solve()
    assert abs(loose.energy() - E_ref) <= 1e-6 * abs(E_ref)
    loose.adjoint()
    F = loose.forces()
    assert np.linalg.norm(F - F_ref) <= 1e-5 * np.linalg.norm(F_ref)


@pytest.mark.parametrize("op", range(6))
def test_fp32_operators_track_fp64(case, op):
    """The FP32 operators of the mixed-precision form agree with the FP64 ones to
    single-precision accuracy (1e-5 of the output's max-norm)."""
    ctx = case["ctx"]
    x = _rand(ctx.nvec, 3 + op)
    y64 = torch.empty_like(x)
    y32 = torch.empty_like(x)
    ctx.apply(op, x, y64)
    ctx.apply(op + 8, x, y32)
    scale = float(y64.abs().max())
    assert float((y64 - y32).abs().max()) <= 1e-5 * scale


def test_fp16_preconditioner_operators(case):
    """A/B with the FP16 stored basis of the mixed-precision preconditioner: within 3e-3 of
    the FP64 operators (FP16 rounding of the basis, 2^-11 relative), and the forward and
    transposed kernels are exact transposes of each other (they stream the same FP16 values),
    <A16 x, y> = <x, A16^T y> to FP32 accumulation accuracy."""
    ctx = case["ctx"]
    x = _rand(ctx.nvec, 21)
    z = _rand(ctx.nvec, 22)
    for op64, op16 in ((G.OP_AB, G.OP_AB_F16), (G.OP_ABT, G.OP_ABT_F16)):
        y64 = torch.empty_like(x)
        y16 = torch.empty_like(x)
        ctx.apply(op64, x, y64)
        ctx.apply(op16, x, y16)
        assert float((y64 - y16).abs().max()) <= 3e-3 * float(y64.abs().max())
    # the identity part (x itself) cancels in the transpose check: compare (I - A16) forms
    ax = torch.empty_like(x)
    atz = torch.empty_like(x)
    ctx.apply(G.OP_AB_F16, x, ax)
    ctx.apply(G.OP_ABT_F16, z, atz)
    lhs = float(torch.dot(x - ax, z))
    rhs = float(torch.dot(x, z - atz))
    scale = float(torch.linalg.norm(x - ax) * torch.linalg.norm(z))
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_mixed_with_fp32_preconditioner(case):
    """The mixed form with the FP32 stored basis in the preconditioner (precond_fp16 = 0)
    reaches the same energy as with the FP16 one."""
    p = case["p"]
    p.solve()
    E_ref = p.energy()
    for fp16 in (0, 1):
        ctx = _ctx(case["c"], case["r"], case["q"], case["lmax"], case["n"], case["surf"], precision=G.DDLPB_MIXED,
                   tol=1e-11, precond_fp16=fp16)
        ctx.solve()
        assert abs(ctx.energy() - E_ref) <= 1e-9 * abs(E_ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_kirkwood_tanford(precision):
    """The GPU path reproduces the Kirkwood-Tanford multipole energy and force of an
    off-centre charge (tiny charged sphere buried in a neutral one), FP64 and mixed."""
    from scipy import special
    a, eps2, kap, lmax = 6.0, 78.54, 0.09, 6
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    b = 0.25 * a
    c = np.array([[0.0, 0.0, 0.0], b * d])
    ctx = G.Context(c, np.array([a, 0.2 * a]), np.array([0.0, 0.7]), eps2, kap, lmax, 302, tol=1e-12,
                    precision=precision)
    ctx.solve()
    ctx.adjoint()
    E, F = ctx.energy(), ctx.forces()
    Eref = dE = 0.0
    for l in range(lmax + 1):
        beta = kap * special.spherical_kn(l, kap * a, derivative=True) / special.spherical_kn(l, kap * a)
        R = ((l + 1) / (eps2 * a) + beta) / (l / (eps2 * a) - beta)
        Eref += 0.49 / 2 * R * b ** (2 * l) / a ** (2 * l + 1)
        dE += 0.49 / 2 * R * 2 * l * b ** (2 * l - 1) / a ** (2 * l + 1) if l else 0.0
    assert abs(E - Eref) <= 1e-10 * abs(Eref)
    assert np.allclose(F[1], -dE * d, rtol=1e-8, atol=1e-12)
