"""Parity at the full sizes of the workloads, in the launch configuration bench.py uses,
on sampled outputs the oracle computes one by one (rows of A X, B X and of the dense
coupling for a few spheres), plus properties that hold at any size (zero net force,
agreement of the mixed-precision and FP64 results)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ddlpb as O
import paper_2203_00552_gb300 as G
from paper_2203_00552_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
BENCH_OPTS = dict(gmres_restart=300, precond_tol=0.4, max_iter=4000)


def _rows_check(w, rows, ops=(G.OP_AB, G.OP_C)):
    ctx = G.Context(w["centres"], w["radii"], w["charges"], w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"],
                    surface=w["surface"], tol=1e-8, precision=G.DDLPB_MIXED, **BENCH_OPTS)
    p = O.DDLPB(w["centres"], w["radii"], w["charges"], w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"],
                surface=w["surface"])
    M, nb = p.M, p.nb
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn(ctx.nvec, generator=g, dtype=torch.float64).to(DEV)
    xn = x.cpu().numpy().reshape(2 * M, nb)
    for op in ops:
        y = torch.empty_like(x)
        ctx.apply(op, x, y)
        yn = y.cpu().numpy().reshape(2 * M, nb)
        if op == G.OP_AB:
            ref_r = p.apply_A_rows(xn[:M], rows)
            ref_e = p.apply_A_rows(xn[M:], rows, kind="i")
            got_r, got_e = yn[rows], yn[M + np.array(rows)]
        else:
            k = p.apply_K_rows(p.ycoef(xn[:M], xn[M:]), rows)
            ref_r = ref_e = k
            got_r, got_e = yn[rows], yn[M + np.array(rows)]
        scale = max(np.abs(ref_r).max(), np.abs(ref_e).max(), 1.0)
        assert np.abs(got_r - ref_r).max() <= 1e-11 * scale, op
        assert np.abs(got_e - ref_e).max() <= 1e-11 * scale, op
    return ctx


def test_globule1000_sas_sampled_rows_and_properties():
    w = synth.workload("globule1000_sas")
    rows = [0, 17, 503, 999]
    ctx = _rows_check(w, rows)
    ctx.solve()
    ctx.adjoint()
    E = ctx.energy()
    F = ctx.forces()
    assert np.abs(F.sum(0)).max() <= 1e-8 * np.abs(F).max()
    ref = G.Context(w["centres"], w["radii"], w["charges"], w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"],
                    surface=w["surface"], tol=1e-10, precision=G.DDLPB_FP64, **BENCH_OPTS)
    ref.solve()
    ref.adjoint()
    E64, F64 = ref.energy(), ref.forces()
    assert abs(E - E64) <= 1e-6 * abs(E64)
    assert np.linalg.norm(F - F64) <= 1e-5 * np.linalg.norm(F64)


def test_globule10000_sampled_rows():
    w = synth.workload("globule10000")
    _rows_check(w, [4321, 9396])   # a buried sphere and the one with the most external points
