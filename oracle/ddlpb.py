"""Oracle: plain FP64 ddLPB energy and analytical forces on the CPU.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Jha, Nottoli, Mikhalev, Quan, Stamm (arXiv:2203.00552):
  Sec. 2.2    neighbour sets, omega_ij, chi_i^e, bases r_l, i_l, k_l, Y_lm,
              Lebedev sums, the block system L X = g (Eq. AXg), the matrices
              A, B (Eqs. definition_of_A_matrix / _B_matrix), C1, C2 through Q
              and P chi (Eqs. definition_of_C1/C2/Q/P_matrix), the right-hand
              side G0, F0 (Eqs. definition_of_G_0, _F_0, defintion_of_S,
              definition_of_c_0_l_0_m_0).
  Sec. 3      energy (Eq. energy_computation), adjoint system (Eqs.
              adjoint_system, AstarXg), force contraction (Eq. force_lpb) with
              the regularised chi_eta, omega_ij^eta, chi_i^eta (Eqs.
              regular_char_function .. regular_chi_e) and every derivative of
              Sec. 3.1 (Eqs. derivative_omegaij, derivative_ylm,
              derivative_radial, derivative_bessel, derivative_chi_i,
              Derivative_of_k_l0, derivative_psi_0, derivative_normal_psi_0).
Readings where the text is garbled or silent (each one is pinned by a test):
  * p_eta constant: 10 eta^2 - 15 eta + 6 (the printed "1 - eta^2 - 15 eta + 6"
    makes chi_eta discontinuous at t = 1 - eta).
  * Q_{j00} = q_j * Y_00, so that E_s = 1/2 sum_j q_j psi_r(x_j) (Eq.
    energy_computation written with the expansion of psi_r); this reproduces
    the Born / Debye-Hueckel energy of one ion exactly.
  * Every Bessel function takes kappa * distance, and the primes are d/dr, so
    i_l'(r_j)/i_l(r_j) = kappa i_l'(kappa r_j) / i_l(kappa r_j).
  * d^i = 1 where f^i = 0; the normal is the outward s_n; eps_1 divides
    grad dn psi0 as it divides psi0.
Forces are returned as -dE/dx_k (Sec. 4.1.1), in Hartree/Bohr.
"""
from __future__ import annotations

import numpy as np

from . import sph

SAS_PROBE_BOHR = 1.4 / 0.529177210903


# ---------------------------------------------------------------------------
# Sec. 3.1, Eq. regular_char_function: the smooth switch chi_eta and p_eta.
def chi_eta(t, eta):
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t <= 1.0 - eta, 1.0, 0.0)
    mid = (t > 1.0 - eta) & (t < 1.0)
    tm = t[mid] if out.ndim else t
    p = eta ** -5 * (1.0 - tm) ** 3 * (6.0 * tm ** 2 + (15.0 * eta - 12.0) * tm
                                        + 10.0 * eta ** 2 - 15.0 * eta + 6.0)
    if out.ndim:
        out[mid] = p
        return out
    return float(p) if mid else float(out)


def dchi_eta(t, eta):
    """d chi_eta / dt (zero outside the window 1-eta < t < 1)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    mid = (t > 1.0 - eta) & (t < 1.0)
    tm = t[mid]
    a = (1.0 - tm)
    poly = 6.0 * tm ** 2 + (15.0 * eta - 12.0) * tm + 10.0 * eta ** 2 - 15.0 * eta + 6.0
    dpoly = 12.0 * tm + 15.0 * eta - 12.0
    out[mid] = eta ** -5 * (-3.0 * a ** 2 * poly + a ** 3 * dpoly)
    return out


def gmres(apply, b, tol=1e-13, restart=60, maxiter=4000, x0=None):
    """Restarted GMRES with modified Gram-Schmidt (plain textbook form)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    it = 0
    while it < maxiter:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            return x, it
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        k_used = 0
        for k in range(restart):
            w = apply(V[k])
            for jj in range(k + 1):
                H[jj, k] = V[jj] @ w
                w = w - H[jj, k] * V[jj]
            H[k + 1, k] = np.linalg.norm(w)
            it += 1
            k_used = k + 1
            e1 = np.zeros(k + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)
            res = np.linalg.norm(H[:k + 2, :k + 1] @ y - e1)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            if res <= tol * bnorm or H[k + 1, k] == 0.0:
                break
        x = x + V[:k_used].T @ y
    return x, it


class DDLPB:
    """The discrete ddLPB problem for one solute (Sec. 2.2).

    centres [M,3] (Bohr), radii [M] (Bohr, vdW; the SAS cavity adds the 1.4 A
    probe), charges [M] (e), eps_solvent, kappa (1/Bohr), lmax, n_lebedev.
    """

    def __init__(self, centres, radii, charges, eps_solvent, kappa, lmax, n_lebedev,
                 surface="vdw", eta=0.1, eps_solute=1.0, fmm_order=0, fmm_theta=0.4):
        self.x = np.array(centres, dtype=np.float64).reshape(-1, 3)
        r = np.array(radii, dtype=np.float64).reshape(-1)
        if surface == "sas":
            r = r + SAS_PROBE_BOHR
        elif surface != "vdw":
            raise ValueError(surface)
        self.r = r
        self.q = np.array(charges, dtype=np.float64).reshape(-1)
        self.M = self.x.shape[0]
        self.eps1 = float(eps_solute)
        self.eps2 = float(eps_solvent)
        self.kappa = float(kappa)
        self.lmax = int(lmax)
        self.nb = sph.nbasis(lmax)
        self.eta = float(eta)
        self.fmm_order = int(fmm_order)   # > 0: Yukawa far field by the tree of oracle/fmm.py
        self.fmm_theta = float(fmm_theta)  # admissibility ratio of that tree
        self._tree = None
        self.s, self.w, self.degree = sph.lebedev(n_lebedev)
        self.N = self.s.shape[0]
        self.Y = sph.ylm(self.lmax, self.s)                     # [N, nb], Y_lm(s_n)
        self.lidx = np.array([int(np.sqrt(k)) for k in range(self.nb)])
        self.Y00 = 1.0 / np.sqrt(4.0 * np.pi)
        # Lebedev points x_i^n = x_i + r_i s_n
        self.pts = self.x[:, None, :] + self.r[:, None, None] * self.s[None, :, :]
        self._neighbours()
        self._switch()
        self._bessel()

    # ---- Sec. 2.2: N_i = spheres intersecting Omega_i, i excluded
    def _neighbours(self):
        M = self.M
        nb = []
        for i in range(M):
            d = np.linalg.norm(self.x - self.x[i], axis=1)
            js = np.nonzero((d < self.r + self.r[i]) & (np.arange(M) != i))[0]
            nb.append(js)
        self.nbrs = nb

    def t(self, i, j):
        """r_1^j(x_i^n) = |x_i^n - x_j| / r_j over n (Eq. definition_radial_scaling)."""
        return np.linalg.norm(self.pts[i] - self.x[j], axis=1) / self.r[j]

    def e(self, i, j):
        """e^j(x_i^n) = (x_i^n - x_j)/|x_i^n - x_j| over n."""
        d = self.pts[i] - self.x[j]
        return d / np.linalg.norm(d, axis=1)[:, None]

    # ---- Sec. 3.1, Eqs. regular_omega_ij .. regular_chi_e
    def _switch(self):
        M, N = self.M, self.N
        self.f = np.zeros((M, N))
        self.Z = np.zeros((M, N, 3))
        for i in range(M):
            js = self.nbrs[i]
            if len(js) == 0:
                continue
            d = self.pts[i][:, None, :] - self.x[js][None, :, :]        # [N, k, 3]
            dist = np.linalg.norm(d, axis=2)
            t = dist / self.r[js][None, :]                              # r_1^j(x_i^n)
            self.f[i] = chi_eta(t, self.eta).sum(1)
            # Z_n^i = sum_{k0 in N_i} chi'(r_1^k0) e^k0 / r_k0
            self.Z[i] = ((dchi_eta(t, self.eta) / self.r[js][None, :])[:, :, None] * d / dist[:, :, None]).sum(1)
        f = self.f
        self.d = np.where(f > 1.0, 1.0 / np.where(f > 1.0, f, 1.0), 1.0)
        # chi_i^eta = 1 - sum_j omega_ij = 1 - d f, which Sec. 3.1 (below Eq.
        # derivative_chi_i) notes is exactly zero wherever f > 1; written so that no
        # rounding residue of 1 - (1/f) f survives there
        self.chi = np.where(f >= 1.0, 0.0, 1.0 - self.d * f)
        self.delta_gt1 = (f > 1.0).astype(np.float64)

    def omega(self, i, j):
        """omega_ij^eta(x_i^n) over n (Eq. regular_omega_ij)."""
        return self.d[i] * chi_eta(self.t(i, j), self.eta)

    # ---- Bessel data per sphere (Sec. 2.2, C_ik; the readings in the header)
    def _bessel(self):
        M, L, k = self.M, self.lmax, self.kappa
        ls = np.arange(L + 1)
        x = k * self.r[:, None]
        self.i_r = sph.bessel_i(ls[None, :], x)                       # i_l(kappa r_j)
        self.k_r = sph.bessel_k(ls[None, :], x)                       # k_l(kappa r_j)
        self.di = k * sph.bessel_i_deriv(ls[None, :], x) / self.i_r   # i_l'(r_j)/i_l(r_j)
        self.dk = k * sph.bessel_k_deriv(ls[None, :], x) / self.k_r   # k_l'(r_j)/k_l(r_j)
        self.cik = 1.0 / (self.di - self.dk)                          # C_ik^j(l)

    def lexpand(self, a):
        """Spread a per-l array [..., lmax+1] to per-(l,m) [..., nb]."""
        return a[..., self.lidx]

    # ---- bases centred at sphere j, evaluated at points P[...,3]
    def basis(self, kind, j, P, grad=False):
        """kind 'r': r_l^j Y^j; 'i': i-ratio Y^j; 'k': k-ratio Y^j (Sec. 2.2).

        With grad, also the spatial gradient with respect to P
        (Eqs. derivative_ylm, derivative_radial, derivative_bessel,
        Derivative_of_k_l0 for the k = i case).
        """
        xj, rj = self.x[j], self.r[j]
        i_r, k_r = self.i_r[j], self.k_r[j]
        if np.ndim(j) == 1:   # several spheres at once: results [len(j), ..., nb]
            xj, rj = xj[:, None, :], rj[:, None, None]
            i_r, k_r = i_r[:, None, :], k_r[:, None, :]
        d = P - xj
        rho = np.linalg.norm(d, axis=-1)
        e = d / rho[..., None]
        ls = np.arange(self.lmax + 1)
        if kind == "r":
            R = (rho[..., None] / rj) ** ls
            dR = ls * (rho[..., None] / rj) ** np.maximum(ls - 1, 0) / rj
        elif kind == "i":
            R = sph.bessel_i(ls, self.kappa * rho[..., None]) / i_r
            dR = self.kappa * sph.bessel_i_deriv(ls, self.kappa * rho[..., None]) / i_r
        elif kind == "k":
            R = sph.bessel_k(ls, self.kappa * rho[..., None]) / k_r
            dR = self.kappa * sph.bessel_k_deriv(ls, self.kappa * rho[..., None]) / k_r
        else:
            raise ValueError(kind)
        R = self.lexpand(R)
        if not grad:
            return R * sph.ylm(self.lmax, e)
        dR = self.lexpand(dR)
        Yv, gS = sph.ylm_and_grad(self.lmax, e)
        B = R * Yv
        dB = (dR * Yv)[..., None] * e[..., None, :] + (R / rho[..., None])[..., None] * gS
        return B, dB

    # ---- projections on the Lebedev grid of one sphere
    def analysis(self, vals):
        """sum_n w_n vals(n) Y_lm(s_n) for vals[..., N] -> [..., nb]."""
        return (vals * self.w) @ self.Y

    def synthesis(self, coef):
        """sum_lm coef_lm Y_lm(s_n) for coef[..., nb] -> [..., N]."""
        return coef @ self.Y.T

    # ---------------------------------------------------------------- operators
    def apply_A(self, Xr, kind="r"):
        """A X (Eq. definition_of_A_matrix); kind 'i' gives B X (Eq. definition_of_B_matrix)."""
        out = Xr.copy()
        for i in range(self.M):
            v = np.zeros(self.N)
            for j in self.nbrs[i]:
                v += self.omega(i, j) * (self.basis(kind, j, self.pts[i]) @ Xr[j])
            out[i] -= self.analysis(v)
        return out

    def apply_A_rows(self, Xc, rows, kind="r"):
        """Rows `rows` of A X (kind 'r') or B X (kind 'i'), for sampled checks at full size."""
        out = []
        for i in rows:
            v = np.zeros(self.N)
            for j in self.nbrs[i]:
                v += self.omega(i, j) * (self.basis(kind, j, self.pts[i]) @ Xc[j])
            out.append(Xc[i] - self.analysis(v))
        return np.array(out)

    def apply_K_rows(self, y, rows):
        """Rows `rows` of apply_K(y) (all sources, sampled targets).  P chi_j y_j is formed as
        analysis(chi_j synthesis(y_j)), the same product as [P chi_j] y_j."""
        src = np.array([j for j in range(self.M) if np.any(self.chi[j] > 0)])
        mu = self.lexpand(self.cik) * self.analysis(self.chi * self.synthesis(y))
        out = []
        for i in rows:
            ext = self.chi[i] > 0
            phi = np.zeros(self.N)
            if ext.any():
                P = self.pts[i][ext]
                for s in range(0, len(src), 128):   # sources in blocks
                    js = src[s:s + 128]
                    phi[ext] += np.einsum("jpn,jn->p", self.basis("k", js, P), mu[js])
            out.append(self.analysis(self.chi[i] * phi))
        return np.array(out)

    def apply_B(self, Xe):
        return self.apply_A(Xe, kind="i")

    def apply_AT(self, Yr, kind="r"):
        """A^T Y (and B^T Y with kind 'i'), written from the entries of A."""
        out = Yr.copy()
        for i in range(self.M):
            zi = self.w * self.synthesis(Yr[i])            # sum_lm w_n Y_lm(s_n) Y_{i lm}
            for j in self.nbrs[i]:
                out[j] -= (self.omega(i, j) * zi) @ self.basis(kind, j, self.pts[i])
        return out

    def apply_AT_rows(self, Yc, rows, kind="r"):
        """Rows `rows` of A^T Y (kind 'r') or B^T Y (kind 'i'): row j collects the entries A_ij
        over the spheres i that overlap j (the overlap relation is symmetric)."""
        out = []
        for j in rows:
            acc = Yc[j].copy()
            for i in self.nbrs[j]:
                zi = self.w * self.synthesis(Yc[i])
                acc -= (self.omega(i, j) * zi) @ self.basis(kind, j, self.pts[i])
            out.append(acc)
        return np.array(out)

    def apply_KT_rows(self, lam, rows):
        """Rows `rows` of apply_KT(lam), every target sphere summed directly."""
        z = self.w * self.chi * self.synthesis(lam)      # [M, N]
        ext = self.chi > 0
        P, zf = self.pts[ext], z[ext]                     # every point with chi > 0
        out = []
        for j in rows:
            nu = np.zeros(self.nb)
            if not ext[j].any():          # P chi_j = 0: the row vanishes
                out.append(nu)
                continue
            for s in range(0, len(P), 65536):
                nu += zf[s:s + 65536] @ self.basis("k", j, P[s:s + 65536])
            out.append(self._pchi(j) @ (self.lexpand(self.cik[j]) * nu))
        return np.array(out)

    def _pchi(self, j):
        """[P chi_j^e] (Eq. definition_of_P_matrix), nb x nb."""
        return (self.Y * (self.w * self.chi[j])[:, None]).T @ self.Y

    def ycoef(self, Xr, Xe):
        """y_j = eps1/eps2 (l/r_j) X_r,j - i_l'(r_j)/i_l(r_j) X_e,j (Eq. def_c1_c2)."""
        c1 = (self.eps1 / self.eps2) * self.lidx[None, :] / self.r[:, None]
        return c1 * Xr - self.lexpand(self.di) * Xe

    # ---- FMM mode: the potential of the k-ratio multipoles at the points with chi > 0
    def _fmm(self):
        if self._tree is None:
            from .fmm import YukawaFMM
            self._tree = YukawaFMM(self.x, self.r, self.kappa, self.lmax, self.fmm_order, self.fmm_theta)
            self._ext = [np.nonzero(self.chi[i] > 0)[0] for i in range(self.M)]
            self._Yp = sph.ylm(self.fmm_order, self.s)                 # [N, (p+1)^2]
            # near sources of each target sphere, and the near targets of each source sphere
            self._near_t = [[] for _ in range(self.M)]
            for i in range(self.M):
                for j in self._tree.near[i]:
                    self._near_t[j].append(i)
        return self._tree

    def _potential(self, mu):
        """phi[i, n] = sum_j k-ratio basis of j at x_i^n times mu_j, at the points with chi > 0
        (zero elsewhere in FMM mode); far field by the FMM when fmm_order > 0, else directly."""
        phi = np.zeros((self.M, self.N))
        if self.fmm_order > 0:
            F = self._fmm()
            Lc = F.locals(mu)
            for i in range(self.M):
                e = self._ext[i]
                if len(e) == 0:
                    continue
                phi[i, e] = self._Yp[e] @ Lc[i] + F.potential_direct(mu, self.pts[i][e], F.near[i])
            return phi
        for i in range(self.M):
            for j in range(self.M):
                phi[i] += self.basis("k", j, self.pts[i]) @ mu[j]
        return phi

    def _potential_T(self, z, full=False):
        """Transpose of _potential for z[M, N] (only the entries with chi > 0 count).  With full
        (FMM mode), the far part is returned to degree fmm_order as a second array."""
        if self.fmm_order > 0:
            F = self._fmm()
            lam = np.zeros((self.M, F.nbp))
            for i in range(self.M):
                e = self._ext[i]
                lam[i] = z[i, e] @ self._Yp[e]
            far = F.locals_T_full(lam)
            nu = far[:, :self.nb].copy()
            for j in range(self.M):
                for i in self._near_t[j]:
                    e = self._ext[i]
                    if len(e):
                        nu[j] += z[i, e] @ self.basis("k", j, self.pts[i][e])
            return (nu, far) if full else nu
        nu = np.zeros((self.M, self.nb))
        for i in range(self.M):
            for j in range(self.M):
                nu[j] += z[i] @ self.basis("k", j, self.pts[i])
        return nu

    def apply_K(self, y):
        """The common dense map of C1 X_r + C2 X_e given y (Eqs. def_c1_c2, definition_of_Q_matrix):
        out_i = sum_n w_n chi_i(x_i^n) Y(s_n) sum_j sum_l0m0 C_ik^j [P chi_j y_j]_l0m0 k^j_l0 Y^j_l0m0 (x_i^n).
        """
        mu = np.stack([self.lexpand(self.cik[j]) * (self._pchi(j) @ y[j]) for j in range(self.M)])
        out = np.zeros((self.M, self.nb))
        if self.fmm_order > 0:
            phi = self._potential(mu)
            return np.stack([self.analysis(self.chi[i] * phi[i]) for i in range(self.M)])
        for i in range(self.M):
            phi = np.zeros(self.N)
            for j in range(self.M):
                phi += self.basis("k", j, self.pts[i]) @ mu[j]
            out[i] = self.analysis(self.chi[i] * phi)
        return out

    def apply_KT(self, lam):
        """K^T lam (transpose of apply_K)."""
        nu = np.zeros((self.M, self.nb))
        if self.fmm_order > 0:
            nu = self._potential_T(np.stack([self.w * self.chi[i] * self.synthesis(lam[i]) for i in range(self.M)]))
        for i in range(self.M if self.fmm_order == 0 else 0):
            zi = self.w * self.chi[i] * self.synthesis(lam[i])
            for j in range(self.M):
                nu[j] += zi @ self.basis("k", j, self.pts[i])
        return np.stack([self._pchi(j) @ (self.lexpand(self.cik[j]) * nu[j]) for j in range(self.M)])

    def apply_L(self, X):
        """L X (Eq. AXg), X = [X_r; X_e] of shape [2M, nb]."""
        M = self.M
        Xr, Xe = X[:M], X[M:]
        cx = self.apply_K(self.ycoef(Xr, Xe))
        return np.concatenate([self.apply_A(Xr) + cx, self.apply_B(Xe) + cx])

    def apply_LT(self, Yv):
        """L* Y (Eq. AstarXg)."""
        M = self.M
        Yr, Ye = Yv[:M], Yv[M:]
        kt = self.apply_KT(Yr + Ye)
        c1 = (self.eps1 / self.eps2) * self.lidx[None, :] / self.r[:, None]
        return np.concatenate([self.apply_AT(Yr) + c1 * kt,
                               self.apply_AT(Ye, kind="i") - self.lexpand(self.di) * kt])

    def assemble_L(self):
        """Dense L from the entry formulas (Eqs. definition_of_A_matrix .. _Q_matrix)."""
        M, nb, N = self.M, self.nb, self.N
        A = np.eye(M * nb)
        B = np.eye(M * nb)
        for i in range(M):
            WY = (self.Y * self.w[:, None]).T                     # [nb, N]
            for j in self.nbrs[i]:
                om = self.omega(i, j)
                A[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] -= (WY * om) @ self.basis("r", j, self.pts[i])
                B[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] -= (WY * om) @ self.basis("i", j, self.pts[i])
        C1 = np.zeros((M * nb, M * nb))
        C2 = np.zeros((M * nb, M * nb))
        for j in range(M):
            # Q_j^{in} as a matrix [N, nb] for each i: k_l0 Y_l0m0 (x_i^n) C_ik P chi_j
            PC = self.lexpand(self.cik[j])[:, None] * self._pchi(j)   # [l0m0, l'm']
            d1 = (self.eps1 / self.eps2) * self.lidx / self.r[j]
            d2 = -self.lexpand(self.di[j])
            for i in range(M):
                Q = self.basis("k", j, self.pts[i]) @ PC               # [N, l'm']
                blk = (self.Y * (self.w * self.chi[i])[:, None]).T @ Q  # [lm, l'm']
                C1[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = blk * d1[None, :]
                C2[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = blk * d2[None, :]
        top = np.hstack([A + C1, C2])
        bot = np.hstack([C1, B + C2])
        return np.vstack([top, bot])

    # ------------------------------------------------------------ right-hand side
    def psi0(self, P):
        """psi_0 (Eq. defintion_of_psi_0) at points P[...,3]."""
        d = P[..., None, :] - self.x
        return (self.q / np.linalg.norm(d, axis=-1)).sum(-1) / self.eps1

    def grad_psi0(self, P):
        d = P[..., None, :] - self.x
        rho = np.linalg.norm(d, axis=-1)
        return -(self.q[:, None] * d / rho[..., None] ** 3).sum(-2) / self.eps1

    def dn_psi0(self, i):
        """d_n psi_0 at x_i^n with the outward normal s_n."""
        return (self.grad_psi0(self.pts[i]) * self.s).sum(-1)

    def rhs(self):
        """g = [G0 + F0; F0] (Eqs. AXg, definition_of_G_0, definition_of_F_0, defintion_of_S, c_0)."""
        M = self.M
        G0 = np.stack([-self.analysis(self.chi[i] * self.psi0(self.pts[i])) for i in range(M)])
        C0 = np.stack([self.analysis(self.chi[j] * self.dn_psi0(j)) for j in range(M)])
        mu0 = self.lexpand(self.cik) * C0
        F0 = np.zeros((M, self.nb))
        if self.fmm_order > 0:
            S_all = self._potential(mu0)
            F0 = np.stack([-(self.eps1 / self.eps2) * self.analysis(self.chi[i] * S_all[i]) for i in range(M)])
        for i in range(M if self.fmm_order == 0 else 0):
            S = np.zeros(self.N)
            for j in range(M):
                S += self.basis("k", j, self.pts[i]) @ mu0[j]
            F0[i] = -(self.eps1 / self.eps2) * self.analysis(self.chi[i] * S)
        self.G0, self.F0, self.C0 = G0, F0, C0
        return np.concatenate([G0 + F0, F0])

    def qvec(self):
        """Q with Q_{j00} = q_j Y_00 (reading of Eq. energy_computation), zero on the X_e rows."""
        Q = np.zeros((2 * self.M, self.nb))
        Q[:self.M, 0] = self.q * self.Y00
        return Q

    # ------------------------------------------------------------------ solves
    def solve(self, dense=None, tol=1e-13):
        g = self.rhs()
        n = 2 * self.M * self.nb
        if dense is None:
            dense = n <= 6000 and self.fmm_order == 0
        if dense and self.fmm_order > 0:
            raise ValueError("the dense assembly is direct; FMM mode solves matrix-free")
        if dense:
            self.L = self.assemble_L()
            X = np.linalg.solve(self.L, g.reshape(-1))
        else:
            X, _ = gmres(lambda v: self.apply_L(v.reshape(2 * self.M, self.nb)).reshape(-1),
                         g.reshape(-1), tol=tol)
        self.X = X.reshape(2 * self.M, self.nb)
        return self.X

    def adjoint(self, dense=None, tol=1e-13):
        Q = self.qvec()
        n = 2 * self.M * self.nb
        if dense is None:
            dense = n <= 6000 and self.fmm_order == 0
        if dense and self.fmm_order > 0:
            raise ValueError("the dense assembly is direct; FMM mode solves matrix-free")
        if dense:
            if not hasattr(self, "L"):
                self.L = self.assemble_L()
            Xa = np.linalg.solve(self.L.T, Q.reshape(-1))
        else:
            Xa, _ = gmres(lambda v: self.apply_LT(v.reshape(2 * self.M, self.nb)).reshape(-1),
                          Q.reshape(-1), tol=tol)
        self.Xadj = Xa.reshape(2 * self.M, self.nb)
        return self.Xadj

    def energy(self, X=None):
        """E_s = 1/2 <X, Q> (Eq. energy_computation), Hartree."""
        X = self.X if X is None else X
        return 0.5 * float((X * self.qvec()).sum())

    # ------------------------------------------------------------------ forces
    def _acc_dchi(self, G, i, a):
        """G[k] += sum_n a(n) grad_k chi_i^eta(x_i^n) (Eq. derivative_chi_i)."""
        le1 = 1.0 - self.delta_gt1[i]
        G[i] += -((a * le1)[:, None] * self.Z[i]).sum(0)
        for k in self.nbrs[i]:
            gk = (dchi_eta(self.t(i, k), self.eta) / self.r[k])[:, None] * self.e(i, k)
            G[k] += ((a * le1)[:, None] * gk).sum(0)

    def _grad_sparse(self, G, Xc, xi, kind):
        """+1/2 sum_i sum_{j in N_i} sum_n xi_i(n) grad_k [omega_ij u_j](x_i^n): the A (kind 'r')
        or B (kind 'i') term, with the three cases of Eq. derivative_omegaij and the
        basis derivatives of Eqs. derivative_ylm, derivative_radial, derivative_bessel."""
        for i in range(self.M):
            for j in self.nbrs[i]:
                tj = self.t(i, j)
                ej = self.e(i, j)
                om = self.d[i] * chi_eta(tj, self.eta)
                dc = dchi_eta(tj, self.eta)
                B, dB = self.basis(kind, j, self.pts[i], grad=True)
                u = B @ Xc[j]
                gu = np.einsum("nbc,b->nc", dB, Xc[j])
                dl = self.delta_gt1[i]
                # k = i
                dom_i = self.d[i][:, None] * ((dc / self.r[j])[:, None] * ej
                                              - (dl * om)[:, None] * self.Z[i])
                G[i] += 0.5 * (xi[i][:, None] * (dom_i * u[:, None] + om[:, None] * gu)).sum(0)
                # k = j
                dom_j = -(self.d[i] * dc / self.r[j] * (1.0 - dl * om))[:, None] * ej
                G[j] += 0.5 * (xi[i][:, None] * (dom_j * u[:, None] - om[:, None] * gu)).sum(0)
                # k in N_i, k != j
                for k in self.nbrs[i]:
                    if k == j:
                        continue
                    dom_k = (om * dl * self.d[i] * dchi_eta(self.t(i, k), self.eta)
                             / self.r[k])[:, None] * self.e(i, k)
                    G[k] += 0.5 * (xi[i][:, None] * dom_k * u[:, None]).sum(0)

    def _grad_K(self, G, vsrc, zeta, scale):
        """G += scale * grad_k T with T = sum_i sum_n zeta_i(n) chi_i(x_i^n) phi(x_i^n),
        phi = sum_j sum_l0m0 mu_j k^j Y^j, mu_j = C_ik^j sum_n0 w_n0 chi_j(x_j^n0) vsrc_j(n0) Y(s_n0),
        holding vsrc fixed: the derivative of chi_i (Eq. derivative_chi_i), of
        P chi_j / C0 (through chi_j), of k^j (Eq. Derivative_of_k_l0) and of Y^j
        (Eq. derivative_ylm).  Returns the adjoint coefficients nu_j.  In FMM mode the far
        part of phi and of its gradient at the targets comes from the local expansions, and
        the far part of the source-side gradient from the adjoint pass (Appendix)."""
        M = self.M
        mu = np.stack([self.lexpand(self.cik[j]) * self.analysis(self.chi[j] * vsrc[j]) for j in range(M)])
        if self.fmm_order > 0:
            return self._grad_K_fmm(G, mu, vsrc, zeta, scale)
        nu = np.zeros((M, self.nb))
        for i in range(M):
            phi = np.zeros(self.N)
            c = zeta[i] * self.chi[i]
            for j in range(M):
                if j == i:
                    B = self.basis("k", j, self.pts[i])
                    phi += B @ mu[j]
                    nu[j] += c @ B
                    continue
                B, dB = self.basis("k", j, self.pts[i], grad=True)
                phi += B @ mu[j]
                nu[j] += c @ B
                gphi = np.einsum("nbc,b->nc", dB, mu[j])
                gg = (c[:, None] * gphi).sum(0)
                G[i] += scale * gg
                G[j] -= scale * gg
            # target mask chi_i
            Gt = np.zeros_like(G)
            self._acc_dchi(Gt, i, zeta[i] * phi)
            G += scale * Gt
        self._acc_source_mask(G, vsrc, nu, scale)
        return nu

    def _acc_source_mask(self, G, vsrc, nu, scale):
        """Source mask chi_j inside P chi_j / C0 (Eq. derivative_chi_i through Eq. definition_of_P_matrix)."""
        for j in range(self.M):
            a = self.w * vsrc[j] * self.synthesis(self.lexpand(self.cik[j]) * nu[j])
            Gs = np.zeros_like(G)
            self._acc_dchi(Gs, j, a)
            G += scale * Gs

    def _grad_K_fmm(self, G, mu, vsrc, zeta, scale):
        from .fmm import basis_grad
        F = self._fmm()
        M, p = self.M, self.fmm_order
        if p < self.lmax + 1:
            raise ValueError("FMM-mode forces need fmm_order >= lmax + 1")
        phi = self._potential(mu)
        c = zeta * self.chi                                             # [M, N]
        nu, far = self._potential_T(c, full=True)
        Lc = F.locals(mu)
        for i in range(M):
            e = self._ext[i]
            if len(e):
                # target side: far field from the local expansion of sphere i, near sources directly
                P = self.pts[i][e]
                g = np.einsum("nbc,b->nc", basis_grad("R", p, self.kappa, P - self.x[i], self.r[i]), Lc[i])
                for j in F.near[i]:
                    if j != i:
                        g += np.einsum("nbc,b->nc", self.basis("k", j, P, grad=True)[1], mu[j])
                G[i] += scale * (c[i, e][:, None] * g).sum(0)
            Gt = np.zeros_like(G)
            self._acc_dchi(Gt, i, zeta[i] * phi[i])
            G += scale * Gt
        nd = (self.lmax + 2) ** 2
        for j in range(M):
            # source side: sum_t c_t grad (mu_j . k-basis_j)(x_t), far part through the gradient
            # map of the degree lmax + 1 adjoint coefficients, near targets directly
            D = F.gradient_map(j, self.lmax)                            # [3, nb, nd]
            sg = np.einsum("anb,b,n->a", D, far[j, :nd], mu[j])
            for i in self._near_t[j]:
                e = self._ext[i]
                if i == j or len(e) == 0:
                    continue
                dB = self.basis("k", j, self.pts[i][e], grad=True)[1]
                sg += (c[i, e][:, None] * np.einsum("nbc,b->nc", dB, mu[j])).sum(0)
            G[j] -= scale * sg
        self._acc_source_mask(G, vsrc, nu, scale)
        return nu

    def hess_inv_r(self, d):
        """Hessian of 1/|d|: 3 d d^T/|d|^5 - I/|d|^3 (Eq. derivative_normal_psi_0)."""
        rho = np.linalg.norm(d, axis=-1)
        return 3.0 * d[..., :, None] * d[..., None, :] / rho[..., None, None] ** 5 \
            - np.eye(3) / rho[..., None, None] ** 3

    def energy_gradient(self, X=None, Xa=None):
        """dE_s/dx_k = 1/2 <grad g - grad L X, X_adj> (Eq. force_lpb), all k at once."""
        X = self.X if X is None else X
        Xa = self.Xadj if Xa is None else Xa
        M = self.M
        Xr, Xe = X[:M], X[M:]
        Ar, Ae = Xa[:M], Xa[M:]
        G = np.zeros((M, 3))
        xi_r = self.w * self.synthesis(Ar)
        xi_e = self.w * self.synthesis(Ae)
        zeta = xi_r + xi_e
        # -<grad A X_r, X_adj_r> and -<grad B X_e, X_adj_e> (Sec. 3.1.1)
        self._grad_sparse(G, Xr, xi_r, "r")
        self._grad_sparse(G, Xe, xi_e, "i")
        # -<grad (C1 X_r + C2 X_e), X_adj_r + X_adj_e> (Sec. 3.1.2)
        y = self.ycoef(Xr, Xe)
        vC = self.synthesis(y)
        self._grad_K(G, vC, zeta, -0.5)
        # +<grad G0, X_adj_r> (Sec. 3.1.3, Eq. derivative_psi_0)
        for i in range(M):
            p0 = self.psi0(self.pts[i])
            Gt = np.zeros_like(G)
            self._acc_dchi(Gt, i, -xi_r[i] * p0)
            G += 0.5 * Gt
            c = -xi_r[i] * self.chi[i]
            for j in range(M):
                if j == i:
                    continue
                d = self.pts[i] - self.x[j]
                rho = np.linalg.norm(d, axis=1)
                gp = -self.q[j] * d / rho[:, None] ** 3 / self.eps1   # grad_x q_j/(eps1|x-x_j|)
                gg = (c[:, None] * gp).sum(0)
                G[i] += 0.5 * gg
                G[j] -= 0.5 * gg
        # +<grad F0, X_adj_r + X_adj_e> (Sec. 3.1.3, Eq. derivative_normal_psi_0)
        sc = -(self.eps1 / self.eps2)
        vF = np.stack([self.dn_psi0(j) for j in range(M)])
        nu = self._grad_K(G, vF, zeta, 0.5 * sc)
        for j in range(M):
            a = self.w * self.chi[j] * self.synthesis(self.lexpand(self.cik[j]) * nu[j])
            for k in range(M):
                if k == j:
                    continue
                H = self.hess_inv_r(self.pts[j] - self.x[k])          # [N,3,3]
                hn = np.einsum("nab,nb->na", H, self.s) * self.q[k] / self.eps1
                gg = (a[:, None] * hn).sum(0)
                G[j] += 0.5 * sc * gg
                G[k] -= 0.5 * sc * gg
        return G

    def forces(self, X=None, Xa=None):
        """F_k = -dE_s/dx_k (Hartree/Bohr)."""
        return -self.energy_gradient(X, Xa)


def run(centres, radii, charges, eps_solvent, kappa, lmax, n_lebedev, surface="vdw", eta=0.1,
        forces=True, dense=None):
    """Energy (and forces) of one solute; returns (E, F or None, problem)."""
    p = DDLPB(centres, radii, charges, eps_solvent, kappa, lmax, n_lebedev, surface, eta)
    p.solve(dense=dense)
    E = p.energy()
    F = None
    if forces:
        p.adjoint(dense=dense)
        F = p.forces()
    return E, F, p
