"""Oracle: Lebedev grids, real orthonormal spherical harmonics and their
tangential gradients, modified spherical Bessel functions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (Sec. 2.2, Eqs. definition_ylm and the normalisation N~_l^m of the
appendix): Y_lm is real and orthonormal on the unit sphere,
    Y_l0  = sqrt((2l+1)/(4 pi)) P_l(cos t),
    Y_lm  = sqrt(2 (2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos t) cos(m p),   m > 0,
    Y_l-m = same with sin(m p),
where P_l^m carries no Condon-Shortley phase (the (-1)^m of N~ cancels it).
The flat index of (l, m) is l*l + l + m.

Values and gradients come from the regular solid harmonic R_lm(x) = |x|^l Y_lm
(x/|x|), written out as an explicit homogeneous polynomial of degree l:
    R_lm = c_lm * A_l^m(z, |x|^2) * B_m(x, y),
    A_l^m = sum_k a_k z^(l-m-2k) (|x|^2)^k        (m-th derivative of P_l),
    B_m   = Re (x + i y)^m  (m > 0),  Im (x + i y)^|m|  (m < 0),  1 (m = 0),
and differentiated term by term.  On the unit sphere the tangential gradient
is grad R(s) - l Y(s) s.
"""
from __future__ import annotations

import math
import os

import numpy as np
from scipy import special

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def lebedev(n: int):
    """Lebedev-Laikov grid with n points: (s[n,3] unit vectors, w[n], degree).

    Sec. 2.2: <f,g>_{n,i} = sum_n w_n f(x_i^n) g(x_i^n), x_i^n = x_i + r_i s_n.
    The weights sum to 4 pi.
    """
    path = os.path.join(_DATA, "lebedev_%d.txt" % n)
    if not os.path.exists(path):
        raise ValueError("no Lebedev grid with %d points" % n)
    with open(path) as f:
        head = f.readline()
    degree = int(head.split("degree")[1].split(";")[0])
    a = np.loadtxt(path, comments="#")
    return np.ascontiguousarray(a[:, :3]), np.ascontiguousarray(a[:, 3]), degree


def nbasis(lmax: int) -> int:
    return (lmax + 1) ** 2


def _legendre_deriv_coeffs(l: int, m: int):
    """Coefficients a_k of d^m/dt^m P_l(t) = sum_k a_k t^(l-m-2k)."""
    out = []
    for k in range(0, (l - m) // 2 + 1):
        num = math.factorial(2 * l - 2 * k)
        den = (2 ** l) * math.factorial(k) * math.factorial(l - k) * math.factorial(l - 2 * k - m)
        out.append(((-1) ** k) * num / den)
    return out


def _norm(l: int, m: int) -> float:
    am = abs(m)
    c = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    return c * (math.sqrt(2.0) if m != 0 else 1.0)


def solid_harmonics(lmax: int, x: np.ndarray, grad: bool = False):
    """Regular solid harmonics R_lm(x) = |x|^l Y_lm(x/|x|) for x[...,3].

    Returns R[..., nb] and, if grad, dR[..., nb, 3] (exact polynomial calculus).
    """
    x = np.asarray(x, dtype=np.float64)
    X, Yc, Z = x[..., 0], x[..., 1], x[..., 2]
    r2 = X * X + Yc * Yc + Z * Z
    shape = x.shape[:-1]
    nb = nbasis(lmax)
    R = np.zeros(shape + (nb,))
    dR = np.zeros(shape + (nb, 3)) if grad else None
    # powers of w = x + i y and their derivatives
    w = X + 1j * Yc
    wpow = [np.ones(shape, dtype=complex)]
    for m in range(1, lmax + 1):
        wpow.append(wpow[-1] * w)
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            a = _legendre_deriv_coeffs(l, m)
            A = np.zeros(shape)
            dAdz = np.zeros(shape)
            dAdr2 = np.zeros(shape)
            for k, ak in enumerate(a):
                p = l - m - 2 * k
                zp = Z ** p
                r2k = r2 ** k
                A += ak * zp * r2k
                if grad:
                    if p > 0:
                        dAdz += ak * p * Z ** (p - 1) * r2k
                    if k > 0:
                        dAdr2 += ak * zp * k * r2 ** (k - 1)
            for sgn in ((1, -1) if m > 0 else (1,)):
                mm = sgn * m
                c = _norm(l, mm)
                if m == 0:
                    B = np.ones(shape)
                elif sgn > 0:
                    B = wpow[m].real
                else:
                    B = wpow[m].imag
                idx = l * l + l + mm
                R[..., idx] = c * A * B
                if grad:
                    # d/dx (x+iy)^m = m w^(m-1), d/dy = i m w^(m-1)
                    if m == 0:
                        dBx = np.zeros(shape)
                        dBy = np.zeros(shape)
                    else:
                        dw = m * wpow[m - 1]
                        if sgn > 0:
                            dBx, dBy = dw.real, (1j * dw).real
                        else:
                            dBx, dBy = dw.imag, (1j * dw).imag
                    dAx = dAdr2 * 2 * X
                    dAy = dAdr2 * 2 * Yc
                    dAz = dAdz + dAdr2 * 2 * Z
                    dR[..., idx, 0] = c * (dAx * B + A * dBx)
                    dR[..., idx, 1] = c * (dAy * B + A * dBy)
                    dR[..., idx, 2] = c * (dAz * B)
    return (R, dR) if grad else R


def ylm(lmax: int, u: np.ndarray):
    """Y_lm at unit vectors u[...,3] -> [..., nb].

    Above degree 12 the explicit polynomial loses digits to cancellation, so
    the values there come from scipy's associated Legendre functions.
    """
    if lmax > 12:
        return ylm_scipy(lmax, u)
    return solid_harmonics(lmax, u)


def ylm_and_grad(lmax: int, u: np.ndarray):
    """Y_lm(u) and the tangential gradient (grad_S Y)(u) for unit u[...,3].

    grad of Y_lm(x/|x|) at a point x equals (grad_S Y)(x/|x|) / |x|
    (the identity used to obtain Eq. derivative_ylm).
    """
    R, dR = solid_harmonics(lmax, u, grad=True)
    l = np.array([int(math.isqrt(k)) for k in range(nbasis(lmax))], dtype=np.float64)
    gS = dR - (l[:, None] * R[..., None]) * u[..., None, :]
    return R, gS


def ylm_scipy(lmax: int, u: np.ndarray):
    """Y_lm from scipy's associated Legendre functions (used only as a pin)."""
    u = np.asarray(u, dtype=np.float64)
    ct = np.clip(u[..., 2], -1.0, 1.0)
    ph = np.arctan2(u[..., 1], u[..., 0])
    out = np.zeros(u.shape[:-1] + (nbasis(lmax),))
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            p = special.lpmv(am, l, ct) * (-1.0) ** am  # remove Condon-Shortley phase
            c = _norm(l, m)
            if m > 0:
                t = np.cos(am * ph)
            elif m < 0:
                t = np.sin(am * ph)
            else:
                t = 1.0
            out[..., l * l + l + m] = c * p * t
    return out


# ---- modified spherical Bessel functions (Sec. 2.2, Eqs. definition_of_bessel_func_first/second)
# All arguments are kappa * distance; derivatives below are d/dx of i_l(x), k_l(x).

def bessel_i(l, x):
    return special.spherical_in(l, x)


def bessel_i_deriv(l, x):
    return special.spherical_in(l, x, derivative=True)


def bessel_k(l, x):
    return special.spherical_kn(l, x)


def bessel_k_deriv(l, x):
    return special.spherical_kn(l, x, derivative=True)
