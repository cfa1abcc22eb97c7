"""Oracle: fast multipole method for the Yukawa far field of the coupling C (FMM mode).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The coupling of Sec. 3 evaluates, at the external points of every sphere i, the potential of
the degree-lmax multipoles mu_j of all spheres j,
    phi(x) = sum_j sum_lm mu_jlm k_l(kappa |x - x_j|)/k_l(kappa r_j) Y_lm((x - x_j)/|x - x_j|),
and the paper makes it linear-cost with a fast multipole method over a binary tree whose
expansions are these k_l Y_lm (multipoles) and i_l Y_lm (locals) functions, moved between
centres by M2M, M2L and L2L translations (Appendix).  The reference the paper cites for the
tree and its traversal is not available, so this module fixes its own specification, which the
GPU path shares:

  * order: the spheres sorted by the Morton key of their centres (each coordinate quantised
    to 21 bits, floor(2^21 (x - lo)/side), lo the lower corner and side the largest edge of the
    centres' bounding box, clamped to 2^21 - 1; bits interleaved x, y, z from the most
    significant; ties by sphere index);
  * tree: the root holds the whole sorted list; a node [a, b) with b - a >= 2 has the children
    [a, a + (b-a)//2) and [a + (b-a)//2, b); the leaves are single spheres;
  * node geometry: c = midpoint of the bounding box of its sphere centres; Rs = the largest
    |x_j - c| (sources are the sphere centres); Rt = the largest |x_j - c| + r_j (targets lie on
    the spheres); a leaf has c = x_j, Rs = 0, Rt = r_j;
  * expansions of a node, order p >= lmax: multipole M_lm of
        sum_{l <= p} M_lm k_l(kappa |x - c|)/k_l(kappa Rt) Y_lm(unit(x - c)),
    local L_lm of  sum_{l <= p} L_lm i_l(kappa |x - c|)/i_l(kappa Rt) Y_lm(unit(x - c));
    a leaf's multipole is the sphere's mu_j itself (degree lmax, scale r_j), and a leaf's local
    evaluated on its own sphere is sum L_lm Y_lm(s_n);
  * dual traversal from (root, root): (A target, B source) is admissible when
    Rt_A + Rs_B < theta |c_A - c_B| (default theta = 0.4): one M2L; else two leaves: near pair, summed
    directly; else split A if B is a leaf or (A is not a leaf and Rt_A >= Rs_B), otherwise B.
Translations here are computed by projection: the source expansion is evaluated on a sphere of
radius rho about the new centre and projected onto Y_lm with a Gauss-Legendre x trapezoid rule
exact to degree p + 50 (rho = 2 Rt for M2M, Rt for M2L and L2L), then divided by the radial
factor at rho.  Since each re-expansion of a k_l Y_lm or i_l Y_lm about another centre is exact
in the infinite addition series, this gives the translation coefficients up to the truncation
at p (no closed form is used).  Forward and transposed passes use the same explicit matrices.
"""
from __future__ import annotations

import numpy as np

from . import sph


def product_rule(degree: int):
    """Points s[Q,3] and weights w[Q] (summing to 4 pi) of a rule on the unit sphere exact for
    polynomials of the given degree: Gauss-Legendre in cos(theta) x trapezoid in phi."""
    nt = degree // 2 + 1
    nphi = degree + 1
    t, wt = np.polynomial.legendre.leggauss(nt)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - t ** 2)
    s = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)), np.outer(t, np.ones(nphi))], axis=-1)
    w = np.outer(wt, np.full(nphi, 2 * np.pi / nphi))
    return s.reshape(-1, 3), w.reshape(-1)


def _lrep(p: int):
    ls = np.arange(p + 1)
    return ls, np.repeat(ls, 2 * ls + 1)


def radial(kind: str, p: int, kappa: float, rho, R: float):
    """k_l(kappa rho)/k_l(kappa R) (kind 'S') or i_l(kappa rho)/i_l(kappa R) (kind 'R'), l <= p."""
    ls = np.arange(p + 1)
    f = sph.bessel_k if kind == "S" else sph.bessel_i
    return f(ls, kappa * np.asarray(rho)[..., None]) / f(ls, kappa * R)


def basis(kind: str, p: int, kappa: float, d: np.ndarray, R: float) -> np.ndarray:
    """Expansion functions of order p about the origin with scale R at the offsets d[..., 3]."""
    rho = np.linalg.norm(d, axis=-1)
    _, lidx = _lrep(p)
    return radial(kind, p, kappa, rho, R)[..., lidx] * sph.ylm(p, d / rho[..., None])


def basis_grad(kind: str, p: int, kappa: float, d: np.ndarray, R: float) -> np.ndarray:
    """Spatial gradient of basis(kind, p, ...) at d[..., 3] -> [..., (p+1)^2, 3] (p <= 12)."""
    rho = np.linalg.norm(d, axis=-1)
    e = d / rho[..., None]
    ls, lidx = _lrep(p)
    if kind == "S":
        f, df = sph.bessel_k, sph.bessel_k_deriv
    else:
        f, df = sph.bessel_i, sph.bessel_i_deriv
    x = kappa * rho[..., None]
    Rr = (f(ls, x) / f(ls, kappa * R))[..., lidx]
    dR = (kappa * df(ls, x) / f(ls, kappa * R))[..., lidx]
    Yv, gS = sph.ylm_and_grad(p, e)
    return (dR * Yv)[..., None] * e[..., None, :] + (Rr / rho[..., None])[..., None] * gS


def morton_order(x: np.ndarray) -> np.ndarray:
    """Sphere indices sorted by the Morton key of their centres (ties by index)."""
    lo = x.min(axis=0)
    side = float((x.max(axis=0) - lo).max())
    if not side > 0.0:
        side = 1.0
    q = np.floor((x - lo) / side * 2097152.0)
    q = np.minimum(q, 2097151.0).astype(np.int64)
    key = np.zeros(len(x), dtype=np.int64)
    for k in range(21):
        for d in range(3):
            key |= ((q[:, d] >> k) & 1) << (3 * k + (2 - d))
    return np.lexsort((np.arange(len(x)), key))


class YukawaFMM:
    """Multipole and local expansions over the binary tree of the module docstring.

    centres[M,3], radii[M] (cavity radii), kappa, lmax (degree of the sphere multipoles),
    p (expansion order, >= lmax), theta.
    """

    def __init__(self, centres, radii, kappa, lmax, p, theta=0.4):
        if p < lmax:
            raise ValueError("the expansion order must be at least lmax")
        self.x = np.asarray(centres, dtype=float).reshape(-1, 3)
        self.r = np.asarray(radii, dtype=float).reshape(-1)
        self.kappa, self.lmax, self.p, self.theta = float(kappa), int(lmax), int(p), float(theta)
        self.M = len(self.x)
        self.nb, self.nbp = (lmax + 1) ** 2, (p + 1) ** 2
        self.order = morton_order(self.x)
        # nodes: ranges [a, b) of the sorted list; children; geometry
        self.a, self.b, self.child, self.parent = [], [], [], []
        stack = [(0, self.M, -1)]
        while stack:
            a, b, par = stack.pop()
            k = len(self.a)
            self.a.append(a)
            self.b.append(b)
            self.parent.append(par)
            self.child.append(None)
            if par >= 0:
                ch = self.child[par]
                self.child[par] = (k,) if ch is None else (ch[0], k)
            if b - a >= 2:
                m = a + (b - a) // 2
                stack.append((m, b, k))   # popped second: the left child is created first
                stack.append((a, m, k))
        n = len(self.a)
        self.c = np.zeros((n, 3))
        self.Rs = np.zeros(n)
        self.Rt = np.zeros(n)
        self.leaf_sphere = np.full(n, -1)
        for k in range(n):
            idx = self.order[self.a[k]:self.b[k]]
            pts = self.x[idx]
            c = 0.5 * (pts.min(axis=0) + pts.max(axis=0))
            d = np.sqrt(((pts - c) ** 2).sum(axis=1))
            self.c[k] = c
            self.Rs[k] = d.max()
            self.Rt[k] = (d + self.r[idx]).max()
            if self.b[k] - self.a[k] == 1:
                self.leaf_sphere[k] = idx[0]
                self.c[k] = self.x[idx[0]]
                self.Rs[k] = 0.0
                self.Rt[k] = self.r[idx[0]]
        self.leaf_node = np.zeros(self.M, dtype=int)
        for k in range(n):
            if self.leaf_sphere[k] >= 0:
                self.leaf_node[self.leaf_sphere[k]] = k
        # dual traversal
        self.m2l, near = [], []
        stack = [(0, 0)]
        while stack:
            A, B = stack.pop()
            dv = self.c[A] - self.c[B]
            d = np.sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2])
            if self.Rt[A] + self.Rs[B] < self.theta * d:
                self.m2l.append((A, B))
                continue
            la, lb = self.child[A] is None, self.child[B] is None
            if la and lb:
                near.append((self.leaf_sphere[A], self.leaf_sphere[B]))
                continue
            if lb or (not la and self.Rt[A] >= self.Rs[B]):
                for ch in self.child[A]:
                    stack.append((ch, B))
            else:
                for ch in self.child[B]:
                    stack.append((A, ch))
        self.near = [[] for _ in range(self.M)]      # near[i]: sources j summed directly at i
        for i, j in near:
            self.near[i].append(j)
        self._rule = product_rule(self.p + 50)
        self._T = {}

    def translation(self, kind: str, S: int, T: int) -> np.ndarray:
        """Matrix [(p+1)^2, (p+1)^2] of the translation kind ('M2M', 'M2L', 'L2L') from node S to
        node T.  A leaf multipole has degree lmax: its coefficients are the first (lmax+1)^2
        inputs (the columns of the higher degrees give the transposed pass at degree p)."""
        key = (kind, S, T)
        if key in self._T:
            return self._T[key]
        s, w = self._rule
        if kind == "M2M":
            rho, kin, kout = 2.0 * self.Rt[T], "S", "S"
        elif kind == "M2L":
            rho, kin, kout = self.Rt[T], "S", "R"
        else:
            rho, kin, kout = self.Rt[T], "R", "R"
        pts = self.c[T] + rho * s
        Bin = basis(kin, self.p, self.kappa, pts - self.c[S], self.Rt[S])        # [Q, nin]
        Yo = sph.ylm(self.p, s)                                                   # [Q, nout]
        _, lidx = _lrep(self.p)
        norm = radial(kout, self.p, self.kappa, rho, self.Rt[T])[lidx]
        Tm = ((Yo * w[:, None]).T @ Bin) / norm[:, None]
        self._T[key] = Tm
        return Tm

    # ---- far field: local expansions at the sphere centres, and the transpose
    def locals(self, mu: np.ndarray) -> np.ndarray:
        """mu[M, nb] (sphere multipoles) -> L[M, (p+1)^2], the far-field local expansion of
        every sphere (scale r_i): the sum over its admissible sources."""
        n = len(self.a)
        Mexp = [None] * n
        for k in range(n - 1, -1, -1):            # children have larger indices than parents
            if self.leaf_sphere[k] >= 0:
                Mexp[k] = np.zeros(self.nbp)
                Mexp[k][:self.nb] = mu[self.leaf_sphere[k]]
            else:
                Mexp[k] = sum(self.translation("M2M", ch, k) @ Mexp[ch] for ch in self.child[k])
        Lexp = [np.zeros(self.nbp) for _ in range(n)]
        for A, B in self.m2l:
            Lexp[A] += self.translation("M2L", B, A) @ Mexp[B]
        for k in range(1, n):                      # parents first
            Lexp[k] += self.translation("L2L", self.parent[k], k) @ Lexp[self.parent[k]]
        out = np.zeros((self.M, self.nbp))
        for i in range(self.M):
            out[i] = Lexp[self.leaf_node[i]]
        return out

    def locals_T(self, lam: np.ndarray) -> np.ndarray:
        """Transpose of `locals`: lam[M, (p+1)^2] -> Psi[M, nb], the far-field adjoint
        coefficients of the sphere multipoles."""
        return self.locals_T_full(lam)[:, :self.nb]

    def locals_T_full(self, lam: np.ndarray) -> np.ndarray:
        """Transpose of `locals` before the truncation of the leaf multipoles to lmax:
        Psi[M, (p+1)^2] (the degrees above lmax are the far part of sum_t c_t k_l Y_lm at the
        sphere centre, used for the source-side gradients)."""
        n = len(self.a)
        Lad = [np.zeros(self.nbp) for _ in range(n)]
        for i in range(self.M):
            Lad[self.leaf_node[i]] = lam[i].copy()
        for k in range(n - 1, 0, -1):              # children first
            Lad[self.parent[k]] += self.translation("L2L", self.parent[k], k).T @ Lad[k]
        Mad = [np.zeros(self.nbp) for _ in range(n)]
        for A, B in self.m2l:
            Mad[B] += self.translation("M2L", B, A).T @ Lad[A]
        for k in range(1, n):                      # parents first
            P = self.parent[k]
            Mad[k] += self.translation("M2M", k, P).T @ Mad[P]
        out = np.zeros((self.M, self.nbp))
        for i in range(self.M):
            out[i] = Mad[self.leaf_node[i]]
        return out

    def gradient_map(self, j: int, degree: int) -> np.ndarray:
        """D[3, (degree+1)^2, (degree+2)^2]: the gradient of each function
        k_l(kappa|x - x_j|)/k_l(kappa r_j) Y_lm (l <= degree) as a combination of the same
        functions of degree <= degree + 1, by projection of the exact gradient on a sphere about
        x_j (each gradient is a finite combination of degrees l - 1 and l + 1)."""
        s, w = product_rule(2 * degree + 20)
        rho = 2.0 * self.r[j]
        g = basis_grad("S", degree, self.kappa, rho * s, self.r[j])              # [Q, nin, 3]
        Yo = sph.ylm(degree + 1, s)
        _, lidx = _lrep(degree + 1)
        norm = radial("S", degree + 1, self.kappa, rho, self.r[j])[lidx]
        D = np.einsum("qo,qia->aio", Yo * w[:, None], g) / norm[None, None, :]
        return D

    # ---- direct sums (near field and checks)
    def potential_direct(self, mu: np.ndarray, targets: np.ndarray, sources=None) -> np.ndarray:
        """sum_j mu_j . k-ratio basis of sphere j at targets[T,3] (all spheres, or `sources`)."""
        phi = np.zeros(len(targets))
        for j in (range(self.M) if sources is None else sources):
            phi += basis("S", self.lmax, self.kappa, targets - self.x[j], self.r[j]) @ mu[j]
        return phi
