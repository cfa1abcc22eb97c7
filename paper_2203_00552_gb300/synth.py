"""Seeded synthetic solutes (chains and globules of atom-centred spheres).

This module holds no arithmetic of the ddLPB method: it only draws geometries,
radii and charges, and converts Angstrom to Bohr.  Both the oracle-based tests
and the GPU path take its arrays as plain inputs.

Growth rule (stand-in for the protein structures of Sec. 4, which are not
available): atom 0 sits at the origin; every further atom is placed 1.5 A from
a uniformly chosen earlier atom, in a uniformly random direction, and the
candidate is rejected if it lies closer than 1.2 A to any atom already placed.

A globule of radius R ("globule") is that cluster compacted onto the ball of
radius R: the grown cluster (an Eden-type cluster whose core holds about 0.3
atoms/A^3) is mapped radially about its centroid, each atom keeping its
direction and its rank in distance, the k-th nearest (k = 0 .. n-1) moving to
radius R ((k + 1/2) / n)^(1/3).  The radial density is then uniform,
n / (4/3 pi R^3) (0.041 atoms/A^3 for 1000 atoms in 18 A, 0.037 for 10 000 in
40 A).  The map stretches the cluster's sparse rim inwards, so a few percent of
the atoms come closer than 1.2 A to another one: in growth order, an atom
closer than 1.2 A to an atom already accepted is re-drawn uniformly in the ball
until it is not.

The other reading ("eden") keeps the growth rule inside the ball: a candidate
outside the ball of radius R around atom 0 is rejected as well.  The cluster
then never reaches R (28.8 A of 40 A at 10 000 atoms) and its core is about
6.6 times denser than R implies; it is kept as a stress workload (45 overlapping
neighbours per atom, 4 % of the grid points external).
"""
from __future__ import annotations

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903
SAS_PROBE_ANGSTROM = 1.4


def _grow(n: int, rng: np.random.Generator, radius_limit: float | None,
          bond: float = 1.5, min_dist: float = 1.2) -> np.ndarray:
    """Grow n atom positions (Angstrom) by the chain/globule growth rule."""
    pos = np.zeros((n, 3))
    if n == 0:
        return pos
    # Uniform cell hash for the min-distance rejection.
    cell = min_dist
    grid: dict[tuple[int, int, int], list[int]] = {}

    def key(p):
        return (int(np.floor(p[0] / cell)), int(np.floor(p[1] / cell)), int(np.floor(p[2] / cell)))

    def too_close(p):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for q in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        d = p - pos[q]
                        if d @ d < min_dist * min_dist:
                            return True
        return False

    grid.setdefault(key(pos[0]), []).append(0)
    placed = 1
    failures = 0
    while placed < n:
        parent = int(rng.integers(0, placed))
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cand = pos[parent] + bond * v
        ok = not too_close(cand)
        if ok and radius_limit is not None:
            ok = float(np.linalg.norm(cand - pos[0])) <= radius_limit
        if not ok:
            failures += 1
            if failures > 200000:
                raise RuntimeError("growth rule could not place atom %d" % placed)
            continue
        failures = 0
        pos[placed] = cand
        grid.setdefault(key(cand), []).append(placed)
        placed += 1
    return pos


def _compact(pos: np.ndarray, radius: float, rng: np.random.Generator, min_dist: float = 1.2) -> np.ndarray:
    """Map a grown cluster onto the ball of the given radius (Angstrom), see the module text."""
    n = len(pos)
    if n == 0:
        return pos
    d = pos - pos.mean(axis=0)
    r = np.sqrt((d * d).sum(axis=1))
    order = np.argsort(r, kind="stable")
    out = np.empty_like(pos)
    new_r = radius * ((np.arange(n) + 0.5) / n) ** (1.0 / 3.0)
    u = d[order] / np.where(r[order] > 0.0, r[order], 1.0)[:, None]
    u[r[order] == 0.0] = (0.0, 0.0, 1.0)
    out[order] = u * new_r[:, None]
    # min-distance repair in growth order, with a cell hash of the accepted atoms
    cell = min_dist
    grid: dict[tuple[int, int, int], list[int]] = {}

    def key(p):
        return (int(np.floor(p[0] / cell)), int(np.floor(p[1] / cell)), int(np.floor(p[2] / cell)))

    def too_close(p):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for q in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        e = p - out[q]
                        if e @ e < min_dist * min_dist:
                            return True
        return False

    for k in range(n):
        tries = 0
        while too_close(out[k]):
            tries += 1
            if tries > 100000:
                raise RuntimeError("no room for atom %d in the ball" % k)
            v = rng.uniform(-radius, radius, size=3)
            if v @ v <= radius * radius:
                out[k] = v
        grid.setdefault(key(out[k]), []).append(k)
    return out


def molecule(n: int, seed: int, kind: str = "chain", globule_radius: float | None = None,
             surface: str = "vdw", vdw_scale: float = 1.1):
    """Return (centres[n,3], radii[n], charges[n]) in atomic units (Bohr, e).

    kind: "chain" (no outer ball), "globule" (the grown cluster compacted onto the ball
    of radius `globule_radius` A, default 18 * (n/1000)^(1/3)) or "eden" (grown inside
    that ball).
    surface: "vdw" scales the drawn radii by `vdw_scale`; "sas" leaves them as
    drawn (the library adds the 1.4 A probe when asked for an SAS cavity).
    Radii are U[1.2, 2.0] A, charges U[-0.5, 0.5] e shifted to zero net charge.
    """
    rng = np.random.default_rng(seed)
    ball = None
    if kind in ("globule", "eden"):
        ball = globule_radius if globule_radius is not None else 18.0 * (n / 1000.0) ** (1.0 / 3.0)
    elif kind != "chain":
        raise ValueError(kind)
    if kind == "globule":
        pos = _compact(_grow(n, rng, None), ball, rng)
    else:
        pos = _grow(n, rng, ball)
    radii = rng.uniform(1.2, 2.0, size=n)
    if surface == "vdw":
        radii = radii * vdw_scale
    elif surface != "sas":
        raise ValueError(surface)
    q = rng.uniform(-0.5, 0.5, size=n)
    if n > 0:
        q = q - q.mean()
    return (np.ascontiguousarray(pos * ANGSTROM_TO_BOHR), np.ascontiguousarray(radii * ANGSTROM_TO_BOHR),
            np.ascontiguousarray(q))


# The three single-molecule workloads (physical constants of Sec. 4: eps=78.54,
# kappa=0.104 1/A, probe 1.4 A).
KAPPA_PER_ANGSTROM = 0.104
EPS_SOLVENT = 78.54

WORKLOADS = {
    "chain20": dict(n=20, seed=0, kind="chain", surface="vdw", lmax=6, n_lebedev=110, fmm_order=0),
    "globule1000_sas": dict(n=1000, seed=1, kind="globule", globule_radius=18.0, surface="sas",
                            lmax=8, n_lebedev=302, fmm_order=16),
    "globule10000": dict(n=10000, seed=2, kind="globule", globule_radius=40.0, surface="vdw",
                         lmax=10, n_lebedev=590, fmm_order=20),
    # the same sizes grown inside the ball (the denser "eden" reading), stress cases
    "eden1000_sas": dict(n=1000, seed=1, kind="eden", globule_radius=18.0, surface="sas",
                         lmax=8, n_lebedev=302, fmm_order=16),
    "eden10000": dict(n=10000, seed=2, kind="eden", globule_radius=40.0, surface="vdw",
                      lmax=10, n_lebedev=590, fmm_order=20),
}


def workload(name: str):
    """Return a dict with the arrays and parameters of a named workload."""
    w = dict(WORKLOADS[name])
    c, r, q = molecule(w["n"], w["seed"], w["kind"], w.get("globule_radius"), w["surface"])
    w.update(centres=c, radii=r, charges=q, kappa=KAPPA_PER_ANGSTROM / ANGSTROM_TO_BOHR,
             eps_solvent=EPS_SOLVENT)
    return w
