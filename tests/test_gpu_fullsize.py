"""Parity at the full sizes of the workloads, in the launch configuration bench.py times (mixed
precision, FMM coupling of the workload's order), on sampled outputs the oracle computes one by
one, and on properties that hold at any size.

Sampled outputs: rows of A X, B X, A^T Y, B^T Y and of the coupling C and its transpose for a
few spheres (first, last, fully exposed, partly covered, buried), the coupling rows summed by
the oracle directly over every source sphere.  Tolerances, relative to the largest reference
entry of the op:
  FP64, direct coupling      1e-11  (rounding of sums over N x neighbours terms)
  FP32 arithmetic (ops 8+)   TOL_F32 (inputs and basis rounded to FP32, u = 6e-8, sums of a few
                             hundred terms per entry)
  FP16 stored basis (16, 17) 3e-3   (half-precision rounding, u = 4.9e-4, of each basis entry)
  FMM coupling               FMM_TOL[(p, op)]: the far field truncated at degree p under the
                             admissibility ratio theta = 0.4; the bounds are five times the
                             errors these rows show on a GB300 (C^T rows sum every target point
                             and cancel, so their largest entry understates their terms); the
                             requirement itself is the energy and force check below
Properties: the A block reproduces solid harmonics of degree <= lmax and the B block plane waves
exp(kappa u.x) (the identities the oracle is pinned to) in every precision of the operators; the
central difference of the energy along a random displacement field equals -sum F.v (FP64,
direct coupling, where the forces are the exact gradient of the discrete energy); zero net
force (exact for the direct coupling, to the FMM error in FMM mode); the bench configuration's
energy and forces against the FP64 direct result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ddlpb as O
import paper_2203_00552_gb300 as G
from paper_2203_00552_gb300 import synth

from expansions import harmonic_expansions, masked_analysis, plane_wave_expansions

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
BENCH_OPTS = dict(gmres_restart=300, precond_tol=0.4, max_iter=4000)
TOL_F64 = 1e-11
TOL_F32 = 2e-5
TOL_F16 = 3e-3
FMM_TOL = {(16, G.OP_C): 2e-6, (16, G.OP_CT): 4e-5, (20, G.OP_C): 3e-7, (20, G.OP_CT): 3e-7}


def oracle(w):
    return O.DDLPB(w["centres"], w["radii"], w["charges"], w["eps_solvent"], w["kappa"], w["lmax"],
                   w["n_lebedev"], surface=w["surface"])


def context(w, **kw):
    opts = dict(BENCH_OPTS, tol=1e-8, precision=G.DDLPB_MIXED, fmm_order=w["fmm_order"])
    opts.update(kw)
    return G.Context(w["centres"], w["radii"], w["charges"], w["eps_solvent"], w["kappa"], w["lmax"],
                     w["n_lebedev"], surface=w["surface"], **opts)


def sample_rows(p):
    """First and last sphere, the most exposed, one about half covered and one buried (if any)."""
    n_ext = (p.chi > 0).sum(axis=1)
    rows = [0, p.M - 1, int(n_ext.argmax()), int(np.abs(n_ext - p.N // 2).argmin())]
    buried = np.nonzero(n_ext == 0)[0]
    if len(buried):
        rows.append(int(buried[0]))
    return sorted(set(rows))


def oracle_rows(p, op, X, rows):
    """Rows `rows` of both halves of op (2: A/B, 3: A^T/B^T, 4: C, 5: C^T) applied to X [2M, nb],
    the coupling summed directly."""
    M = p.M
    Xr, Xe = X[:M], X[M:]
    if op == G.OP_AB:
        return p.apply_A_rows(Xr, rows), p.apply_A_rows(Xe, rows, kind="i")
    if op == G.OP_ABT:
        return p.apply_AT_rows(Xr, rows), p.apply_AT_rows(Xe, rows, kind="i")
    if op == G.OP_C:
        k = p.apply_K_rows(p.ycoef(Xr, Xe), rows)
        return k, k
    kt = p.apply_KT_rows(Xr + Xe, rows)
    c1 = (p.eps1 / p.eps2) * p.lidx[None, :] / p.r[rows, None]
    return c1 * kt, -p.lexpand(p.di[rows]) * kt


def base_op(op):
    """The FP64 operator whose rows an op of another precision approximates."""
    return {G.OP_AB_F16: G.OP_AB, G.OP_ABT_F16: G.OP_ABT}.get(op, op % G.OP_FP32)


def rows_error(ctx, op, x, ref, rows, M):
    """Largest deviation of rows `rows` of ctx's op x from ref, relative to ref's largest entry."""
    y = torch.empty_like(x)
    ctx.apply(op, x, y)
    yn = y.cpu().numpy().reshape(2 * M, -1)
    got_r, got_e = yn[rows], yn[M + np.asarray(rows)]
    scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max(), 1e-300)
    return max(np.abs(got_r - ref[0]).max(), np.abs(got_e - ref[1]).max()) / scale


def identity_errors(p, ctx, ops):
    """Largest error, relative to the largest coefficient, of [A X_h ; B X_pw] against
    [analysis(chi X_h) ; analysis(chi pw)] for solid harmonics R_LM of degree <= lmax about the
    molecule's centroid and a plane wave, through each op in ops (2, 10, 16)."""
    centre = p.x.mean(axis=0) + np.array([0.7, -1.3, 2.1])
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    pw_vals, Xpw = plane_wave_expansions(p, u)
    pw_want = masked_analysis(p, pw_vals)
    errs = {op: 0.0 for op in ops}
    for L, Mq in ((0, 0), (1, 1), (3, -2), (p.lmax, p.lmax - 1)):
        h_vals, Xh = harmonic_expansions(p, centre, L, Mq)
        h_want = masked_analysis(p, h_vals)
        x = torch.from_numpy(np.concatenate([Xh, Xpw]).reshape(-1)).to(DEV)
        y = torch.empty_like(x)
        for op in ops:
            ctx.apply(op, x, y)
            yn = y.cpu().numpy().reshape(2 * p.M, -1)
            e = max(np.abs(yn[:p.M] - h_want).max() / np.abs(Xh).max(),
                    np.abs(yn[p.M:] - pw_want).max() / np.abs(Xpw).max())
            errs[op] = max(errs[op], e)
    return errs


@pytest.fixture(scope="module")
def w1000():
    w = synth.workload("globule1000_sas")
    p = oracle(w)
    rows = sample_rows(p)
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn(2 * p.M * p.nb, generator=g, dtype=torch.float64)
    X = x.numpy().reshape(2 * p.M, p.nb)
    refs = {op: oracle_rows(p, op, X, rows) for op in (G.OP_AB, G.OP_ABT, G.OP_C, G.OP_CT)}
    return dict(w=w, p=p, rows=rows, x=x.to(DEV), refs=refs)


def test_1000_sas_direct_fp64_rows(w1000):
    w, p = w1000["w"], w1000["p"]
    ctx = context(w, precision=G.DDLPB_FP64, fmm_order=0)
    for op in (G.OP_AB, G.OP_ABT, G.OP_C, G.OP_CT):
        err = rows_error(ctx, op, w1000["x"], w1000["refs"][op], w1000["rows"], p.M)
        assert err <= TOL_F64, (op, err)
    ctx.close()


def test_1000_sas_bench_configuration_rows(w1000):
    """The operators of the bench configuration (mixed, FMM of order 16): FP64 A/B and their
    transposes, the FP64 FMM coupling (refinement residuals), the FP32 operators of the Krylov
    solves and the FP16-basis preconditioner blocks, against the oracle's direct rows."""
    w, p = w1000["w"], w1000["p"]
    fc, fct = FMM_TOL[(w["fmm_order"], G.OP_C)], FMM_TOL[(w["fmm_order"], G.OP_CT)]
    tol = {G.OP_AB: TOL_F64, G.OP_ABT: TOL_F64, G.OP_C: fc, G.OP_CT: fct,
           G.OP_AB + G.OP_FP32: TOL_F32, G.OP_ABT + G.OP_FP32: TOL_F32,
           G.OP_C + G.OP_FP32: fc + TOL_F32, G.OP_CT + G.OP_FP32: fct + TOL_F32,
           G.OP_AB_F16: TOL_F16, G.OP_ABT_F16: TOL_F16}
    ctx = context(w)
    for op, t in tol.items():
        err = rows_error(ctx, op, w1000["x"], w1000["refs"][base_op(op)], w1000["rows"], p.M)
        assert err <= t, (op, err, t)
    errs = identity_errors(p, ctx, (G.OP_AB, G.OP_AB + G.OP_FP32, G.OP_AB_F16))
    assert errs[G.OP_AB] <= TOL_F64, errs
    assert errs[G.OP_AB + G.OP_FP32] <= TOL_F32, errs
    assert errs[G.OP_AB_F16] <= TOL_F16, errs
    ctx.close()


def test_1000_sas_energy_forces(w1000):
    """The bench configuration's energy and forces against the FP64 direct solution (FMM
    truncation plus the 1e-8 solver tolerance), zero net force (exact for the direct coupling,
    to the FMM error with the FMM), and the directional derivative of the FP64 direct energy
    along a random displacement field by central differences (h = 3e-4 bohr: the O(h^2)
    truncation is about 2e-6 of |F| |v| there, the solver noise 1e-11 |E| / h below 1e-7)."""
    w = w1000["w"]
    ctx = context(w)
    ctx.solve()
    ctx.adjoint()
    E, F = ctx.energy(), ctx.forces()
    ctx.close()
    ref = context(w, precision=G.DDLPB_FP64, fmm_order=0, tol=1e-11)
    ref.solve()
    ref.adjoint()
    E64, F64 = ref.energy(), ref.forces()
    ref.close()
    # zero net force: exact for the direct coupling (to rounding); in FMM mode the far field is
    # approximated and the net force is of the order of the FMM error (4e-7 relative measured)
    assert np.abs(F64.sum(0)).max() <= 1e-12 * np.abs(F64).max()
    assert np.abs(F.sum(0)).max() <= 2e-6 * np.abs(F).max()
    assert abs(E - E64) <= 1e-6 * abs(E64), (E, E64)
    assert np.linalg.norm(F - F64) <= 1e-5 * np.linalg.norm(F64)

    v = np.random.default_rng(3).normal(size=F64.shape)
    h = 3e-4
    Es = []
    for s in (1.0, -1.0):
        ws = dict(w, centres=w["centres"] + s * h * v)
        c = context(ws, precision=G.DDLPB_FP64, fmm_order=0, tol=1e-11)
        c.solve()
        Es.append(c.energy())
        c.close()
    dE = (Es[0] - Es[1]) / (2 * h)
    assert abs(dE + np.sum(F64 * v)) <= 1e-5 * np.linalg.norm(F64) * np.linalg.norm(v), (dE, -np.sum(F64 * v))


def test_10000_fmm_rows():
    """globule10000 (lmax 10, 590 points, FMM of order 20), mixed: FP64 A/B and transposes, the
    FP64 and FP32 FMM coupling and its transpose, on a partly covered and a buried sphere."""
    w = synth.workload("globule10000")
    p = oracle(w)
    n_ext = (p.chi > 0).sum(axis=1)
    rows = [int(np.abs(n_ext - p.N // 4).argmin()), int(np.nonzero(n_ext == 0)[0][0])]
    g = torch.Generator(device="cpu").manual_seed(6)
    x = torch.randn(2 * p.M * p.nb, generator=g, dtype=torch.float64)
    X = x.numpy().reshape(2 * p.M, p.nb)
    refs = {op: oracle_rows(p, op, X, rows) for op in (G.OP_AB, G.OP_ABT, G.OP_C, G.OP_CT)}
    x = x.to(DEV)
    fc, fct = FMM_TOL[(w["fmm_order"], G.OP_C)], FMM_TOL[(w["fmm_order"], G.OP_CT)]
    ctx = context(w)
    for op, t in ((G.OP_AB, TOL_F64), (G.OP_ABT, TOL_F64), (G.OP_C, fc), (G.OP_CT, fct),
                  (G.OP_C + G.OP_FP32, fc + TOL_F32), (G.OP_CT + G.OP_FP32, fct + TOL_F32)):
        err = rows_error(ctx, op, x, refs[base_op(op)], rows, p.M)
        assert err <= t, (op, err, t)
    ctx.close()
