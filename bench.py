"""Benchmark: ddLPB energy + analytical forces, atoms/s.

Default workload (named in config.workload): `globule1000_sas`, the 1000-atom globule (chain
growth rule, then compacted onto the 18 A ball, seed 1), SAS radii (U[1.2, 2.0] A + 1.4 A
probe), charges U[-0.5, 0.5] e with zero net charge, eps = 78.54, kappa = 0.104 1/A, lmax = 8,
302-point Lebedev grid, the coupling's far field by the FMM of order 16 (admissibility ratio
0.4), outer tolerance 1e-8
(FP64 relative residual).  The 10,000-atom globule (lmax 10, 590 points, FMM order 20;
`--workload globule10000`) fits one GPU, but its preconditioned system needs thousands of
Krylov iterations (their count grows with the atom count and lmax), far beyond a bench run.
One step = setup (neighbour lists, switch functions, hit lists, right-hand side) + primal
solve + adjoint solve + energy + forces, from inputs already resident in HBM.  The mixed
form runs the Krylov solves in FP32 inside FP64 iterative refinement; --precision fp64
times the plain FP64 path.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own copy of the workload (replicas:
one molecule is not split across GPUs); value = all atoms / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_00552_gb300 import synth  # noqa: E402

METRIC = "ddLPB energy+forces atoms/s at 10k atoms (mixed vs FP64, 1e-6); served p99 ms"
UNIT = "atoms/s"
WORKLOAD = "globule1000_sas"
FP32_PEAK_TFLOPS_AT_MAX_CLOCK = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
# Algorithmic FP32 flops per unit of the hot kernels (see the kernel roofline table):
#   per (hit, basis function) for the A/B kernels (two bases, 8 flops each),
#   per (target, source, basis function) for the Yukawa kernels.
FLOPS_PER_UNIT = {"ab_apply": 16, "ab_transpose": 16, "yukawa_pot": 8, "yukawa_adj": 8,
                  "fmm_m2l": 1, "fmm_m2l_T": 1}   # the FMM translations count their flops themselves
HBM_PEAK_GBS = 6789.6   # measured copy bandwidth of this machine's GB300 (read + write bytes)
# dram bytes per launch from the committed ncu capture (profiles/), keyed by (kernel, workload),
# with the digest of the kernel's source text they were taken on; null once that text changes.
NCU_TRAFFIC = {("ab_transpose_f16", "globule1000_sas"): {"bytes_per_launch": 1082074368, "digest": "707bf782404a2be7"}}
# CUDA functions whose source text a timed kernel name stands for
KERNEL_SOURCES = {"ab_apply_f32": ["load8_f", "load8", "k_ab_hits_chunk"],
                  "ab_apply_f16": ["half8_to_float", "load8_h", "load8", "k_ab_hits_chunk"],
                  "ab_transpose_f32": ["load8_f", "load8", "k_ab_transpose_chunk"],
                  "ab_transpose_f16": ["half8_to_float", "load8_h", "load8", "k_ab_transpose_chunk"]}
# every group of launches the library times at kernel_timing = 2 (setup and forces as one group each)
BREAKDOWN_NAMES = ([b + sfx for b in ("ab_apply", "ab_transpose", "yukawa_pot", "yukawa_adj", "krylov_dot",
                                      "krylov_update", "ab_project", "synthesis", "masked_analysis",
                                      "coupling_projection", "store", "fmm_m2l", "fmm_m2l_T", "fmm_tree",
                                      "fmm_near") for sfx in ("_f16", "_f32", "_f64")]
                   + ["setup_f64", "forces_f64"])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--restart", type=int, default=300)
    ap.add_argument("--precond-tol", type=float, default=0.4)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fmm-order", type=int, default=None,
                    help="FMM expansion order (default: the workload's; 0 = direct summation)")
    ap.add_argument("--fmm-theta", type=float, default=0.4,
                    help="FMM admissibility ratio: M2L when Rt_A + Rs_B < theta |c_A - c_B|")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-breakdown", action="store_true", help="skip the instrumented breakdown step")
    ap.add_argument("--no-fp64", action="store_true", help="skip the one-step FP64 comparison")
    ap.add_argument("--ops-only", action="store_true",
                    help="setup plus one application of each FP32 operator, then exit (for ncu captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample(w, atoms=12):
    """The oracle (FP64, dense, CPU) on the first `atoms` atoms of the workload."""
    from oracle import ddlpb as O
    c, r, q = w["centres"][:atoms], w["radii"][:atoms], w["charges"][:atoms]
    t = time.perf_counter()
    O.run(c, r, q, w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"], surface=w["surface"])
    return time.perf_counter() - t


def reference_arm(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    atoms = 12
    for _ in range(args.warmup):
        oracle_sample(w, atoms)
    times = [oracle_sample(w, atoms) for _ in range(args.steps)]
    dt = sum(times) / len(times)
    value = atoms / dt
    cores = os.cpu_count()
    sample = ("oracle energy+forces (dense LU, FP64 numpy) on the first %d atoms of the %d-atom globule, "
              "lmax %d, %d Lebedev points; its cost grows like M^3 (dense solve) and M^2 (coupling), so this "
              "is the rate on the sample, not on the whole workload" % (atoms, w["n"], w["lmax"], w["n_lebedev"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s (oracle sample: first %d atoms)" % (args.workload, atoms), "lmax": w["lmax"],
                       "n_lebedev": w["n_lebedev"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def clocks_start():
    """Sample SM clocks and throttle reasons every 200 ms into a temporary CSV (nvidia-smi)."""
    import tempfile
    fd, path = tempfile.mkstemp(prefix="ddlpb_clocks_", suffix=".csv")
    f = os.fdopen(fd, "w")
    try:
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                              "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f, path
    except Exception:
        f.close()
        os.remove(path)
        return None, None, None


def clocks_stop(p, f, path, dev_index):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(dev_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for k, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(k)
    os.remove(path)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def whole_job(atoms_per_rank, ms_local, world, dist=None, device="cpu"):
    """Max step time over ranks and the whole-job throughput (all ranks' atoms / that time).
    Each rank solves its own copy of the workload (replicas), so the only collective is this
    reduction of one number; it works with any torch.distributed backend."""
    t_max = float(ms_local)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * atoms_per_rank / (t_max / 1e3)


def stored_bytes_names():
    """Timed kernels whose roofline is HBM bytes of a stored basis."""
    return {k + sfx for k in ("ab_apply", "ab_transpose") for sfx in ("_f32", "_f16")}


def kernel_digest(kernel):
    """Digest of the source text (definition through its closing brace) of the CUDA functions
    behind a timed kernel name; None if a function is not found."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2203_00552_gb300", "csrc", "operators.cu")) as f:
        text = f.read()
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES.get(kernel, []):
        i = text.find(" " + fn + "(")
        if i < 0:
            return None
        j = text.index("{", i)
        depth = 0
        for k in range(j, len(text)):
            depth += {"{": 1, "}": -1}.get(text[k], 0)
            if depth == 0:
                break
        h.update(text[i:k + 1].encode())
    return h.hexdigest()[:16] if kernel in KERNEL_SOURCES else None


def main():
    args = parse()
    w = synth.workload(args.workload)
    if args.impl == "reference":
        reference_arm(args, w)
        return
    import torch
    import paper_2203_00552_gb300 as G

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    if not os.path.exists(os.path.join(ROOT, "paper_2203_00552_gb300", "libddlpb.so")):
        if rank == 0:
            from paper_2203_00552_gb300 import build
            build.build()
        if pg:
            pg.barrier()
    G.library()
    prec = G.DDLPB_MIXED if args.precision == "mixed" else G.DDLPB_FP64
    fmm_order = w["fmm_order"] if args.fmm_order is None else args.fmm_order
    opts = dict(tol=1e-8, precision=prec, gmres_restart=args.restart, precond_tol=args.precond_tol, max_iter=4000,
                fmm_order=fmm_order, fmm_theta=args.fmm_theta)
    M = w["n"]
    cen = torch.tensor(w["centres"], device=dev)
    rad = torch.tensor(w["radii"], device=dev)
    chg = torch.tensor(w["charges"], device=dev)
    e_out = torch.empty(1, dtype=torch.float64, device=dev)
    f_out = torch.empty((M, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    if args.ops_only:
        ctx = G.Context(cen, rad, chg, w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"],
                        surface=w["surface"], stream=stream.cuda_stream, **opts)
        x = torch.randn(ctx.nvec, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)
        times = {}
        for op, name in ((10, "AB32"), (11, "ABT32"), (16, "AB16"), (17, "ABT16"), (12, "C32"), (13, "CT32"),
                         (2, "AB64"), (4, "C64")):
            ctx.apply(op, x, y)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 5
            for _ in range(reps):
                ctx.apply(op, x, y)
            torch.cuda.synchronize()
            times[name] = (time.perf_counter() - t0) / reps * 1e3
        print(json.dumps({"ops_only": args.workload, "ms_per_apply": times, "info": ctx.info()}), flush=True)
        ctx.close()
        return

    def step(timing=0, options=None):
        ctx = G.Context(cen, rad, chg, w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"],
                        surface=w["surface"], stream=stream.cuda_stream, kernel_timing=int(timing),
                        **(options or opts))
        ctx.solve()
        ctx.adjoint()
        ctx.energy_device(e_out)
        ctx.forces_device(f_out)
        return ctx

    for _ in range(args.warmup):
        step().close()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks_start() if rank == 0 else (None, None, None)
    times, kstats, launches, infos = [], {}, 0, []
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx = step(timing=1)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        info = ctx.info()
        infos.append(info)
        launches += info["kernel_launches"]
        for base in FLOPS_PER_UNIT:
            for suf in ("_f16", "_f32", "_f64"):
                n, ms = ctx.kernel_time(base + suf)
                if n:
                    a = kstats.setdefault(base + suf, [0, 0.0])
                    a[0] += n
                    a[1] += ms
        ctx.close()
    torch.cuda.synchronize()
    clocks = clocks_stop(*clk, local) if rank == 0 else None
    ms_step = sum(times) / len(times)
    t_max, value = whole_job(M, ms_step, world, pg, dev)

    # end to end through the C ABI with host buffers (copies inside the timed region): the
    # inputs sit in pinned host memory, the results come back to host arrays
    hc, hr, hq = (torch.from_numpy(np.ascontiguousarray(w[k], dtype=np.float64)).pin_memory().numpy()
                  for k in ("centres", "radii", "charges"))
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else args.steps
    e2e_times = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = G.Context(hc, hr, hq, w["eps_solvent"], w["kappa"], w["lmax"], w["n_lebedev"], surface=w["surface"],
                        stream=stream.cuda_stream, **opts)
        ctx.solve()
        ctx.adjoint()
        E = ctx.energy()
        F = ctx.forces()
        e2e_times.append(time.perf_counter() - t0)
        ctx.close()
    e2e = None
    if e2e_times:
        e2e = {"value": world * M / (sum(e2e_times) / len(e2e_times)), "unit": UNIT,
               "h2d_bytes_per_step": int(hc.nbytes + hr.nbytes + hq.nbytes),
               "d2h_bytes_per_step": int(F.nbytes + 8)}

    # the plain FP64 path on the same workload, one step, for comparison with the mixed form
    fp64 = None
    if prec == G.DDLPB_MIXED and not args.no_fp64 and rank == 0:
        e_mixed = float(e_out.item())
        f_mixed = f_out.clone()
        o64 = dict(opts, precision=G.DDLPB_FP64)
        step(options=o64).close()   # warm-up of the FP64 kernels
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step(options=o64).close()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        e64 = float(e_out.item())
        fp64 = {"ms_per_step": ms64, "value": M / (ms64 / 1e3), "unit": UNIT, "speedup_of_mixed": ms64 / t_max,
                "energy_rel_diff_mixed_vs_fp64": abs(e_mixed - e64) / abs(e64),
                "force_rel_diff_mixed_vs_fp64": float((f_mixed - f_out).norm() / f_out.norm())}

    # breakdown of one more (untimed) step: CUDA events around every group of launches
    breakdown = None
    if rank == 0 and not args.no_breakdown:
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx = step(timing=2)
        ev1.record(stream)
        torch.cuda.synchronize()
        parts = {}
        for name in BREAKDOWN_NAMES:
            n, ms = ctx.kernel_time(name)
            if n:
                parts[name] = {"launches": n, "ms": round(ms, 2)}
        ctx.close()
        wall = ev0.elapsed_time(ev1)
        busy = sum(v["ms"] for v in parts.values())
        breakdown = {"step_ms": round(wall, 1), "timed_ms": round(busy, 1),
                     "other_ms": round(wall - busy, 1), "parts": parts,
                     "other": "launch gaps, host synchronisation and host work of the solver (GMRES "
                              "least squares, convergence checks), small untimed kernels"}

    # roofline of the dominant instrumented kernel
    info = infos[-1]
    nb = (w["lmax"] + 1) ** 2
    units = {"ab_apply": info["n_hits"] * nb, "ab_transpose": info["n_hits"] * nb,
             "yukawa_pot": info["n_external"] * info["n_sources"] * nb,
             "yukawa_adj": info["n_external"] * info["n_sources"] * nb,
             "fmm_m2l": info["fmm_m2l_flops"], "fmm_m2l_T": info["fmm_m2l_flops"]}
    roofline = None
    L = w["lmax"]
    # The stored A/B products of the FP32 set stream the basis (HBM-bound): algorithmic bytes
    # per hit are the basis row (nb + lmax + 1 values, 4 B in the FP32 copy, 2 B in the FP16
    # copy) plus the hit's point index (4 B; its sphere is stored once per group of 8 hits).
    stored_bytes = {name: info["n_hits"] * ((nb + L + 1) * (4 if name.endswith("_f32") else 2) + 4)
                    for name in stored_bytes_names()}
    if kstats:
        top = max(kstats, key=lambda k: kstats[k][1])
        n, ms = kstats[top]
        base = top.rsplit("_", 1)[0]
        tr = NCU_TRAFFIC.get((top, args.workload))
        traffic = tr["bytes_per_launch"] if tr and tr.get("digest") == kernel_digest(top) else None
        common = {"kernel": top, "traffic": traffic, "launches_per_step": n / len(times), "ms_per_launch": ms / n,
                  "share_of_step": ms / sum(times)}
        if top in stored_bytes:
            achieved = stored_bytes[top] / (ms / n / 1e3) / 1e9
            roofline = dict(bound="hbm", achieved=achieved, peak=HBM_PEAK_GBS, unit="GB/s",
                            frac=achieved / HBM_PEAK_GBS, peak_source="measured copy bandwidth", **common)
        else:
            flops_per_launch = units[base] * FLOPS_PER_UNIT[base]
            achieved = flops_per_launch / (ms / n / 1e3) / 1e12
            peak = FP32_PEAK_TFLOPS_AT_MAX_CLOCK if top.endswith("f32") else 1.25
            roofline = dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                            peak_source=("FP32: 152 SMs x 128 lanes x 2 flop x 2070 MHz" if top.endswith("f32")
                                         else "FP64 nominal 1.25 TFLOP/s"), **common)
        roofline["all_kernels"] = {k: {"launches": v[0], "ms": round(v[1], 2)} for k, v in kstats.items()}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        atoms = 12
        dt = oracle_sample(w, atoms)
        cpu = {"value": atoms / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "oracle energy+forces (dense LU, FP64 numpy) on the first %d atoms of this workload, "
                         "%.1f s; its cost grows like M^3 (dense solve) and M^2 (coupling), so this is the rate on "
                         "the sample, not on the whole workload" % (atoms, dt)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f16+f32+f64" if prec == G.DDLPB_MIXED else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "atoms": M, "lmax": w["lmax"], "n_lebedev": w["n_lebedev"],
                           "surface": w["surface"], "precision": args.precision,
                           "coupling": ("fmm" if fmm_order > 0 else "direct summation"), "fmm_order": fmm_order,
                           "fmm_theta": opts["fmm_theta"] if fmm_order > 0 else None,
                           "tol": 1e-8, "gmres_restart": args.restart, "precond_tol": args.precond_tol,
                           "l2": "512 MB buffer written between timed steps; working set > L2",
                           "parallelism": "replicas" if world > 1 else "single"},
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "breakdown": breakdown, "fp64_path": fp64,
                "cpu_baseline": cpu, "clocks": clocks,
                "solver": {"outer": info["solve_iterations"], "adjoint_outer": info["adjoint_iterations"],
                           "refinement": info["refinement_steps"], "residual": info["solve_residual"],
                           "adjoint_residual": info["adjoint_residual"], "external_points": info["n_external"],
                           "external_fraction": info["n_external"] / float(M * w["n_lebedev"]),
                           "hits": info["n_hits"], "sources": info["n_sources"], "fmm_m2l": info["fmm_m2l"],
                           "fmm_near_pairs": info["fmm_near_pairs"], "fmm_nodes": info["fmm_nodes"]},
                "energy_hartree": float(e_out.item())}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
