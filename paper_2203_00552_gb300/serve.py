"""Serving form: a stream of solutes of different sizes, solved as they arrive.

Requests (geometry, lmax, Lebedev grid) arrive as a Poisson process.  A dispatcher admits
them in arrival order into at most `slots` concurrent slots, as long as the estimated device
footprint of the requests in flight stays within an HBM budget; each admitted request runs
on its own host thread, CUDA stream and library context (setup, solve, adjoint, energy,
forces), so that requests that arrive while others are on the GPU overlap with them.  A
request that perturbs an earlier geometry starts its solves from that one's solutions X and
X_adj (kept on the device), the reuse of the previous iterate that Sec. 4 of the paper makes
inside its solver, carried across geometries.  Reported: per-request latency (arrival to
result), its p50 / p99, and atoms/s over the run.

    python -m paper_2203_00552_gb300.serve --rate 4 --duration 20 --size-max 600
    python -m paper_2203_00552_gb300.serve --batch 256 --size-max 300     # batched form
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth

GRIDS = {4: 50, 6: 110, 8: 302, 10: 590}


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    centres: np.ndarray            # Bohr
    radii: np.ndarray
    charges: np.ndarray
    lmax: int
    n_lebedev: int
    parent: int | None = None      # request whose geometry this one perturbs

    @property
    def atoms(self) -> int:
        return int(self.centres.shape[0])


@dataclass
class Result:
    rid: int
    atoms: int
    energy: float
    forces: np.ndarray
    start: float
    end: float
    latency: float
    warm: bool
    iterations: int = 0
    extra: dict = field(default_factory=dict)


def make_requests(seed: int, rate: float, duration: float, size_min: int, size_max: int,
                  lmax_choices=(6, 8), perturb_frac: float = 0.3, sigma_angstrom: float = 0.02):
    """Seeded Poisson stream: sizes log-uniform in [size_min, size_max], globules of the
    workload density, lmax drawn from lmax_choices (with their Lebedev grids); a fraction
    perturb_frac re-sends an earlier geometry moved by Gaussian noise of sigma_angstrom."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        if reqs and rng.random() < perturb_frac:
            p = reqs[int(rng.integers(0, len(reqs)))]
            c = p.centres + rng.normal(scale=sigma_angstrom * synth.ANGSTROM_TO_BOHR, size=p.centres.shape)
            reqs.append(Request(rid, t, c, p.radii, p.charges, p.lmax, p.n_lebedev, parent=p.rid))
        else:
            n = int(round(math.exp(rng.uniform(math.log(size_min), math.log(size_max)))))
            lmax = int(rng.choice(lmax_choices))
            c, r, q = synth.molecule(n, int(rng.integers(0, 2 ** 31)), "globule", None, "vdw")
            reqs.append(Request(rid, t, c, r, q, lmax, GRIDS[lmax]))
        rid += 1
    return reqs


def make_batch(seed: int, n: int, size_min: int, size_max: int, lmax_choices=(6, 8)):
    """A batch of n independent solutes, all present at time 0 (the batched form): sizes
    log-uniform in [size_min, size_max], lmax drawn from lmax_choices with their grids."""
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(n):
        m = int(round(math.exp(rng.uniform(math.log(size_min), math.log(size_max)))))
        lmax = int(rng.choice(lmax_choices))
        c, r, q = synth.molecule(m, int(rng.integers(0, 2 ** 31)), "globule", None, "vdw")
        reqs.append(Request(rid, 0.0, c, r, q, lmax, GRIDS[lmax]))
    return reqs


def footprint_bytes(atoms: int, lmax: int, n_lebedev: int, restart: int, hits_per_point: float = 8.0) -> int:
    """Conservative device footprint of one request (bytes): grid arrays, hit lists with the
    stored FP32 and FP64 bases, vectors, and the FP32/FP64 Krylov bases."""
    nb = (lmax + 1) ** 2
    points = atoms * n_lebedev
    hits = points * hits_per_point
    nvec = 2 * atoms * nb
    grid = points * 8 * 8
    hit_lists = hits * (4 * 6 + 8 * 2)
    stored = hits * (nb + lmax + 1) * (4 + 8) + hits * 16
    vectors = nvec * 8 * 16
    krylov = nvec * (4 * (2 * restart + 1) + 4 * 42 + 8 * 42)
    return int(grid + hit_lists + stored + vectors + krylov) + (64 << 20)


class Server:
    """Admission, slots and timing; `engine(request, warm)` does the work of one request
    and returns (energy, forces, solution handle, iterations)."""

    def __init__(self, engine, slots: int, hbm_budget: int, restart: int = 300):
        self.engine = engine
        self.slots = slots
        self.budget = hbm_budget
        self.restart = restart
        self.solutions = {}
        self.lock = threading.Lock()
        self.peak_inflight = 0
        self.peak_bytes = 0

    def run(self, requests):
        results = {}
        pending = list(requests)
        pending.sort(key=lambda r: r.arrival)
        inflight = {}
        used = 0
        cv = threading.Condition(self.lock)
        t0 = time.perf_counter()

        def worker(req, fp):
            start = time.perf_counter() - t0
            with self.lock:
                warm = self.solutions.get(req.parent) if req.parent is not None else None
            try:
                energy, forces, handle, iters = self.engine(req, warm)
                err = None
            except Exception as e:  # reported per request
                energy, forces, handle, iters, err = float("nan"), None, None, 0, repr(e)
            end = time.perf_counter() - t0
            with cv:
                if handle is not None:
                    self.solutions[req.rid] = handle
                res = Result(req.rid, req.atoms, energy, forces, start, end, end - req.arrival, warm is not None,
                             iters)
                if err:
                    res.extra["error"] = err
                results[req.rid] = res
                del inflight[req.rid]
                nonlocal used
                used -= fp
                cv.notify_all()

        i = 0
        with cv:
            while i < len(pending) or inflight:
                now = time.perf_counter() - t0
                if i < len(pending):
                    req = pending[i]
                    fp = footprint_bytes(req.atoms, req.lmax, req.n_lebedev, self.restart)
                    fits = used + fp <= self.budget or not inflight
                    if req.arrival <= now and len(inflight) < self.slots and fits:
                        inflight[req.rid] = fp
                        used += fp
                        self.peak_inflight = max(self.peak_inflight, len(inflight))
                        self.peak_bytes = max(self.peak_bytes, used)
                        th = threading.Thread(target=worker, args=(req, fp), daemon=True)
                        th.start()
                        i += 1
                        continue
                    wait = max(0.0, req.arrival - now) if req.arrival > now else None
                else:
                    wait = None
                cv.wait(timeout=wait if wait is not None else 0.05)
        makespan = time.perf_counter() - t0
        return [results[r.rid] for r in requests], makespan


def summary(results, makespan):
    lat = np.array([r.latency for r in results]) * 1e3
    atoms = sum(r.atoms for r in results)
    return {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "atoms_per_s": atoms / makespan, "makespan_s": makespan,
            "warm_started": int(sum(r.warm for r in results)),
            "errors": int(sum("error" in r.extra for r in results))}


def gpu_engine(device: int = 0, **options):
    """Engine that solves a request with the CUDA library on its own stream."""
    import torch

    from . import _binding as B

    opts = dict(tol=1e-8, precision=B.DDLPB_MIXED, gmres_restart=300, precond_tol=0.4, max_iter=4000)
    opts.update(options)
    kappa = synth.KAPPA_PER_ANGSTROM / synth.ANGSTROM_TO_BOHR

    def run(req: Request, warm):
        torch.cuda.set_device(device)
        stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(stream):
            ctx = B.Context(req.centres, req.radii, req.charges, synth.EPS_SOLVENT, kappa, req.lmax, req.n_lebedev,
                            stream=stream.cuda_stream, **opts)
            try:
                if warm is not None and warm[0].numel() == ctx.nvec:
                    ctx.set_vector(1, warm[0])
                    ctx.set_vector(2, warm[1])
                ctx.solve()
                ctx.adjoint()
                e = ctx.energy()
                f = ctx.forces()
                X = torch.empty(ctx.nvec, dtype=torch.float64, device=f"cuda:{device}")
                Xa = torch.empty_like(X)
                ctx.vector(1, X)
                ctx.vector(2, Xa)
                info = ctx.info()
            finally:
                ctx.close()
        return e, f, (X, Xa), info["solve_iterations"] + info["adjoint_iterations"]

    return run


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=4.0, help="requests per second")
    ap.add_argument("--duration", type=float, default=20.0, help="seconds of arrivals")
    ap.add_argument("--size-min", type=int, default=20)
    ap.add_argument("--size-max", type=int, default=600)
    ap.add_argument("--lmax", type=int, nargs="+", default=[6, 8])
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--hbm-gb", type=float, default=200.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0, help="batched form: this many solutes present at time 0")
    args = ap.parse_args()
    if args.batch:
        reqs = make_batch(args.seed, args.batch, args.size_min, args.size_max, tuple(args.lmax))
    else:
        reqs = make_requests(args.seed, args.rate, args.duration, args.size_min, args.size_max, tuple(args.lmax))
    server = Server(gpu_engine(), args.slots, int(args.hbm_gb * 2 ** 30))
    results, makespan = server.run(reqs)
    line = summary(results, makespan)
    if args.batch:
        line.update({"metric": "batched atoms/s", "unit": "atoms/s", "value": line["atoms_per_s"],
                     "molecules": args.batch})
    else:
        line.update({"metric": "served p99 latency", "unit": "ms", "rate_per_s": args.rate,
                     "duration_s": args.duration})
    line.update({"sizes": [args.size_min, args.size_max], "lmax": args.lmax, "slots": args.slots,
                 "hbm_budget_gb": args.hbm_gb, "peak_inflight": server.peak_inflight,
                 "peak_footprint_gb": server.peak_bytes / 2 ** 30, "precision": "mixed", "tol": 1e-8})
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
