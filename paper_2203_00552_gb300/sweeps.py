"""Convergence and size sweeps of the GPU path on seeded synthetic globules.

  lmax: the energy of one solute for every (lmax, Lebedev grid) pair of the given lists whose
        grid is exact to degree 2 lmax (the convergence study of Sec. 4); FP64, tolerance 1e-11.
  size: atoms/s of a whole step (setup, both solves, energy, forces; mixed precision, tolerance
        1e-8) for globules of M atoms at one (lmax, grid): the growth of the cost with M.
  fmm:  for every (admissibility theta, order p): the FP64 FMM solution against the FP64 direct
        one (energy and forces, tolerance 1e-11; the p_max study of Sec. 4), and the wall time of
        one step of the mixed form (tolerance 1e-8) after one warm-up step.

    python -m paper_2203_00552_gb300.sweeps lmax --atoms 100 --lmax 2 4 6 8 10 12 --grid 302 590 770
    python -m paper_2203_00552_gb300.sweeps size --lmax 6 --grid 110 --atoms 100 300 1000 3000
    python -m paper_2203_00552_gb300.sweeps fmm --workload globule1000_sas --theta 0.5 0.4 0.3 0.25 --order 12 16 20

Each prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

from . import synth


def _kappa():
    return synth.KAPPA_PER_ANGSTROM / synth.ANGSTROM_TO_BOHR


DEGREE = {6: 3, 14: 5, 26: 7, 38: 9, 50: 11, 74: 13, 86: 15, 110: 17, 146: 19, 170: 21, 194: 23, 230: 25,
          266: 27, 302: 29, 350: 31, 434: 35, 590: 41, 770: 47}   # exactness of the Lebedev rules


def lmax_sweep(atoms: int, seed: int, lmaxes, grids):
    from . import _binding as B
    c, r, q = synth.molecule(atoms, seed, "globule", None, "vdw")
    rows = []
    for N in grids:
        for L in lmaxes:
            if DEGREE[N] < 2 * L:
                continue
            t0 = time.perf_counter()
            ctx = B.Context(c, r, q, synth.EPS_SOLVENT, _kappa(), L, N, tol=1e-11, precision=B.DDLPB_FP64,
                            gmres_restart=300, max_iter=4000)
            try:
                ctx.solve()
                e = ctx.energy()
                info = ctx.info()
            finally:
                ctx.close()
            rows.append({"lmax": L, "grid": N, "energy_hartree": e, "iterations": info["solve_iterations"],
                         "seconds": time.perf_counter() - t0})
    return {"sweep": "lmax", "atoms": atoms, "seed": seed, "rows": rows}


def size_sweep(sizes, seed: int, lmax: int, grid: int):
    import torch

    from . import _binding as B
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    rows = []
    for M in sizes:
        c, r, q = synth.molecule(M, seed, "globule", None, "vdw")
        e_out = torch.empty(1, dtype=torch.float64, device=dev)
        f_out = torch.empty((M, 3), dtype=torch.float64, device=dev)

        def step():
            ctx = B.Context(c, r, q, synth.EPS_SOLVENT, _kappa(), lmax, grid, tol=1e-8, precision=B.DDLPB_MIXED,
                            gmres_restart=300, precond_tol=0.4, max_iter=4000, stream=stream.cuda_stream)
            ctx.solve()
            ctx.adjoint()
            ctx.energy_device(e_out)
            ctx.forces_device(f_out)
            return ctx

        step().close()   # warm-up
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        info = ctx.info()
        ctx.close()
        rows.append({"atoms": M, "ms_per_step": ms, "atoms_per_s": M / (ms / 1e3),
                     "outer": info["solve_iterations"], "adjoint_outer": info["adjoint_iterations"],
                     "hits": info["n_hits"], "external_fraction": info["n_external"] / (M * grid)})
        print(json.dumps(rows[-1]), flush=True)   # one line per size as it completes
    return {"sweep": "size", "lmax": lmax, "grid": grid, "seed": seed, "precision": "mixed", "tol": 1e-8,
            "rows": rows}


def fmm_sweep(workload: str, thetas, orders):
    import numpy as np
    import torch

    from . import _binding as B
    w = synth.workload(workload)
    opts = dict(gmres_restart=300, precond_tol=0.4, max_iter=4000)

    def ctx(**kw):
        return B.Context(w["centres"], w["radii"], w["charges"], w["eps_solvent"], w["kappa"], w["lmax"],
                         w["n_lebedev"], surface=w["surface"], **dict(opts, **kw))

    def energy_forces(**kw):
        c = ctx(**kw)
        try:
            c.solve()
            c.adjoint()
            return c.energy(), c.forces(), c.info()
        finally:
            c.close()

    E0, F0, _ = energy_forces(precision=B.DDLPB_FP64, tol=1e-11, fmm_order=0)
    rows = []
    for theta in thetas:
        for p in orders:
            E, F, info = energy_forces(precision=B.DDLPB_FP64, tol=1e-11, fmm_order=p, fmm_theta=theta)
            energy_forces(precision=B.DDLPB_MIXED, tol=1e-8, fmm_order=p, fmm_theta=theta)   # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            energy_forces(precision=B.DDLPB_MIXED, tol=1e-8, fmm_order=p, fmm_theta=theta)
            torch.cuda.synchronize()
            rows.append({"theta": theta, "order": p, "energy_rel_err": abs(E - E0) / abs(E0),
                         "force_rel_err": float(np.linalg.norm(F - F0) / np.linalg.norm(F0)),
                         "force_max_abs_err": float(np.abs(F - F0).max()), "mixed_step_s": time.perf_counter() - t0,
                         "m2l": info["fmm_m2l"], "near_pairs": info["fmm_near_pairs"]})
            print(json.dumps(rows[-1]), flush=True)
    return {"sweep": "fmm", "workload": workload, "energy_direct_hartree": E0, "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="what", required=True)
    a = sub.add_parser("lmax")
    a.add_argument("--atoms", type=int, default=100)
    a.add_argument("--seed", type=int, default=3)
    a.add_argument("--lmax", type=int, nargs="+", default=[2, 4, 6, 8, 10, 12])
    a.add_argument("--grid", type=int, nargs="+", default=[302, 590, 770])
    b = sub.add_parser("size")
    b.add_argument("--atoms", type=int, nargs="+", default=[100, 300, 1000, 3000])
    b.add_argument("--seed", type=int, default=4)
    b.add_argument("--lmax", type=int, default=6)
    b.add_argument("--grid", type=int, default=110)
    f = sub.add_parser("fmm")
    f.add_argument("--workload", default="globule1000_sas")
    f.add_argument("--theta", type=float, nargs="+", default=[0.5, 0.4, 0.3, 0.25])
    f.add_argument("--order", type=int, nargs="+", default=[12, 16, 20])
    args = ap.parse_args()
    if args.what == "lmax":
        out = lmax_sweep(args.atoms, args.seed, sorted(args.lmax), args.grid)
    elif args.what == "size":
        out = size_sweep(args.atoms, args.seed, args.lmax, args.grid)
    else:
        out = fmm_sweep(args.workload, args.theta, args.order)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
