"""Oracle: tree approximation of the Yukawa far field of the coupling C (FMM mode).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The coupling of Sec. 3 evaluates, at the external points x of every sphere, the potential of
point multipoles of degree lmax at the sphere centres x_j,
    phi(x) = sum_j sum_lm mu'_jlm k_l(kappa |x - x_j|) Y_lm((x - x_j)/|x - x_j|),
(mu' = mu / k_l(kappa r_j) for the k-ratio basis), and the paper sums it with a fast multipole
method whose expansions are the same k_l Y_lm functions about tree-node centres.  This module
is the oracle's version of that approximation, plain and slow; its tree specification:

  * binary tree over the source centres: a node is split at the median of its centres along
    the longest axis of their bounding box until it holds at most `leaf` sources;
  * node centre c = midpoint of the bounding box of its centres; node radius R = the largest
    distance from c to one of its centres;
  * multipole of a node, order p >= lmax: the coefficients M_lm of
        phi_node(x) = sum_{l <= p} M_lm k_l(kappa |x - c|) Y_lm((x - c)/|x - c|),  |x - c| > R,
    by projection of the node's exact field onto the sphere of radius rho = max(R, r0)/theta
    about c, with a product Gauss-Legendre x trapezoid rule exact to degree p + 60
    (M_lm = <phi_node(c + rho s), Y_lm(s)> / k_l(kappa rho)); the expansion of a point multipole
    about another centre in k_l Y_lm is the addition theorem of the modified spherical Bessel
    functions, so the projection gives its coefficients up to truncation at p;
  * a target x uses the multipole of a node when |x - c| > R / theta (theta = 0.5), otherwise the
    node's children, and at a leaf it sums the node's sources directly.
The truncation error of one node at an admissible target is of order theta^(p+1).  Forward and
transposed products are built from the same explicit matrices, so they are exact transposes.
"""
from __future__ import annotations

import numpy as np

from . import sph


def _product_rule(degree: int):
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


def _kY(lmax: int, kappa: float, d: np.ndarray):
    """k_l(kappa |d|) Y_lm(d/|d|) for d[..., 3] -> [..., (lmax+1)^2]."""
    rho = np.linalg.norm(d, axis=-1)
    ls = np.arange(lmax + 1)
    K = sph.bessel_k(ls, kappa * rho[..., None])
    lidx = np.repeat(ls, 2 * ls + 1)
    return K[..., lidx] * sph.ylm(lmax, d / rho[..., None])


class Node:
    def __init__(self, idx, centres):
        self.idx = idx
        lo, hi = centres[idx].min(0), centres[idx].max(0)
        self.c = 0.5 * (lo + hi)
        self.R = float(np.linalg.norm(centres[idx] - self.c, axis=1).max())
        self.extent = hi - lo
        self.children = []


class YukawaTree:
    """Tree approximation of phi(x) = sum_j sum_lm mu'_jlm k_l Y_lm(x - x_j) (see the module
    docstring for the specification)."""

    def __init__(self, centres, kappa, lmax, p, theta=0.5, leaf=8, r0=1.0):
        if p < lmax:
            raise ValueError("the expansion order must be at least lmax")
        self.x = np.asarray(centres, dtype=float)
        self.kappa, self.lmax, self.p, self.theta, self.leaf = float(kappa), lmax, p, theta, leaf
        self.nb, self.nbp = (lmax + 1) ** 2, (p + 1) ** 2
        self.nodes = []
        self.root = self._build(np.arange(len(self.x)))
        s, w = _product_rule(p + 60)
        self._s, self._w = s, w
        for nd in self.nodes:
            nd.rho = max(nd.R, r0) / theta
            nd.P = self._projection(nd)

    def _build(self, idx):
        nd = Node(idx, self.x)
        self.nodes.append(nd)
        if len(idx) > self.leaf:
            ax = int(np.argmax(nd.extent))
            order = idx[np.argsort(self.x[idx, ax], kind="stable")]
            h = len(order) // 2
            nd.children = [self._build(order[:h]), self._build(order[h:])]
        return nd

    def _projection(self, nd):
        """P[(p+1)^2, S*nb]: node multipole from the node's source coefficients."""
        q = nd.c + nd.rho * self._s                                   # check points
        src = np.concatenate([_kY(self.lmax, self.kappa, q - self.x[j]) for j in nd.idx], axis=1)
        Yq = sph.ylm(self.p, self._s)                                 # [Q, nbp]
        ls = np.arange(self.p + 1)
        kr = sph.bessel_k(ls, self.kappa * nd.rho)[np.repeat(ls, 2 * ls + 1)]
        return ((Yq * self._w[:, None]).T @ src) / kr[:, None]

    # ---- the approximated potential and its transpose
    def potential(self, mu, targets):
        """phi at targets[T,3] from source coefficients mu[S, nb]."""
        phi = np.zeros(len(targets))
        self._walk(self.root, np.arange(len(targets)), targets, mu, phi, None)
        return phi

    def potential_T(self, z, targets):
        """The transpose: source coefficients nu[S, nb] = sum_x z(x) d phi(x) / d mu."""
        nu = np.zeros((len(self.x), self.nb))
        self._walk(self.root, np.arange(len(targets)), targets, None, None, (z, nu))
        return nu

    def _walk(self, nd, tidx, targets, mu, phi, adj):
        if len(tidx) == 0:
            return
        d = np.linalg.norm(targets[tidx] - nd.c, axis=1)
        far = d > nd.R / self.theta
        if far.any():
            rows = _kY(self.p, self.kappa, targets[tidx[far]] - nd.c) @ nd.P    # [Tf, S*nb]
            if adj is None:
                phi[tidx[far]] += rows @ mu[nd.idx].reshape(-1)
            else:
                z, nu = adj
                nu[nd.idx] += (z[tidx[far]] @ rows).reshape(len(nd.idx), self.nb)
        near = tidx[~far]
        if not nd.children:
            for j in nd.idx:
                B = _kY(self.lmax, self.kappa, targets[near] - self.x[j])
                if adj is None:
                    phi[near] += B @ mu[j]
                else:
                    z, nu = adj
                    nu[j] += z[near] @ B
            return
        for ch in nd.children:
            self._walk(ch, near, targets, mu, phi, adj)

    def potential_direct(self, mu, targets):
        """The same sum without the tree (for checks)."""
        phi = np.zeros(len(targets))
        for j in range(len(self.x)):
            phi += _kY(self.lmax, self.kappa, targets - self.x[j]) @ mu[j]
        return phi
