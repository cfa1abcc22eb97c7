// fmm_host.h -- host-side constant tables of the Yukawa FMM (no CUDA): the coaxial
// translation coefficients expressed through Gaunt integrals.
//
// The FMM of the Appendix of arXiv:2203.00552 moves k_l Y_lm (multipole) and i_l Y_lm (local)
// expansions between centres; a translation along the z axis keeps m, and the coefficient of
// an output degree a from an input degree l is a finite sum over b = l + a - 2j, j = 0..min(l,a),
// of Gaunt integrals times i_b or k_b of kappa times the translation length (the addition
// theorem of the modified spherical Bessel functions, written with the plane-wave expansion
// exp(kappa u.x) = 4 pi sum_l i_l(kappa |x|) sum_m Y_lm(x/|x|) Y_lm(u)).  This header builds
//   g[m][l][a][j] = 4 pi Y_b0(e_z) int Y_lm Y_am Y_b0 dOmega,   b = l + a - 2j,
// for the real orthonormal Y_lm of the library (Y_lm = sqrt(2) Q_l^m(cos th) cos(m phi) for
// m > 0, sin(|m| phi) for m < 0, Q_l^0 for m = 0, Q the fully normalised associated Legendre
// function without the Condon-Shortley phase).  The integral over phi is exact; the one over
// cos(theta) uses a Gauss-Legendre rule with 2p + 2 nodes (exact to degree 4p + 3 >= l + a + b).
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace fmmhost {

// Gauss-Legendre nodes and weights on [-1, 1], n >= 2 (Newton iteration on P_n).
inline void gauss_legendre(int n, std::vector<double>& z, std::vector<double>& w) {
    z.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double p0 = 1.0, p1 = x, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0;
            p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);   // P_n'(x)
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        p0 = 1.0;
        p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        z[i] = -x;
        z[n - 1 - i] = x;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

// Q_l^m(z) for l <= L, all m <= l, at one z: out[l * (L + 1) + m].
inline void legendre_q(int L, double z, std::vector<double>& out) {
    out.assign((size_t)(L + 1) * (L + 1), 0.0);
    const double s2 = 1.0 - z * z;
    double qmm = 1.0 / std::sqrt(4.0 * M_PI);
    for (int m = 0; m <= L; ++m) {
        if (m > 0) qmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m) * s2);
        out[(size_t)m * (L + 1) + m] = qmm;
        if (m + 1 <= L) out[(size_t)(m + 1) * (L + 1) + m] = std::sqrt(2.0 * m + 3.0) * z * qmm;
        for (int l = m + 2; l <= L; ++l) {
            const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
            const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            out[(size_t)l * (L + 1) + m] = a * (z * out[(size_t)(l - 1) * (L + 1) + m] - b * out[(size_t)(l - 2) * (L + 1) + m]);
        }
    }
}

// Offsets of the table g: for m = 0..p, l = m..p, a = m..p, j = 0..min(l, a).
struct CoaxIndex {
    int p = 0;
    std::vector<long long> off;   // [(p+1)^3]: start of (m, l, a)
    long long size = 0;
    void build(int pp) {
        p = pp;
        off.assign((size_t)(p + 1) * (p + 1) * (p + 1), -1);
        long long o = 0;
        for (int m = 0; m <= p; ++m)
            for (int l = m; l <= p; ++l)
                for (int a = m; a <= p; ++a) {
                    off[((size_t)m * (p + 1) + l) * (p + 1) + a] = o;
                    o += std::min(l, a) + 1;
                }
        size = o;
    }
};

inline void gaunt_coax_table(int p, CoaxIndex& idx, std::vector<double>& g) {
    idx.build(p);
    g.assign((size_t)idx.size, 0.0);
    const int L = 2 * p;
    std::vector<double> z, w;
    gauss_legendre(2 * p + 2, z, w);
    std::vector<std::vector<double>> Q(z.size());
    for (size_t i = 0; i < z.size(); ++i) legendre_q(L, z[i], Q[i]);
    auto q = [&](size_t i, int l, int m) { return Q[i][(size_t)l * (L + 1) + m]; };
    for (int m = 0; m <= p; ++m)
        for (int l = m; l <= p; ++l)
            for (int a = m; a <= p; ++a) {
                const long long o = idx.off[((size_t)m * (p + 1) + l) * (p + 1) + a];
                for (int j = 0; j <= std::min(l, a); ++j) {
                    const int b = l + a - 2 * j;
                    double s = 0.0;
                    for (size_t i = 0; i < z.size(); ++i) s += w[i] * q(i, l, m) * q(i, a, m) * q(i, b, 0);
                    // int Y_lm Y_am Y_b0 dOmega = 2 pi int Q_l^m Q_a^m Q_b^0 dz (also for m > 0:
                    // 2 int cos^2 = 2 pi); Y_b0(e_z) = sqrt((2b+1)/(4 pi))
                    g[(size_t)(o + j)] = 4.0 * M_PI * std::sqrt((2.0 * b + 1.0) / (4.0 * M_PI)) * 2.0 * M_PI * s;
                }
            }
}

// Real Y_lm (l <= L) at the unit vector (x, y, z): out[l*l + l + m].
inline void real_ylm(int L, double x, double y, double z, std::vector<double>& out) {
    std::vector<double> Q;
    legendre_q(L, z, Q);
    out.assign((size_t)(L + 1) * (L + 1), 0.0);
    const double phi = std::atan2(y, x);
    for (int l = 0; l <= L; ++l) {
        out[(size_t)l * l + l] = Q[(size_t)l * (L + 1)];
        for (int m = 1; m <= l; ++m) {
            const double q = std::sqrt(2.0) * Q[(size_t)l * (L + 1) + m];
            out[(size_t)l * l + l + m] = q * std::cos(m * phi);
            out[(size_t)l * l + l - m] = q * std::sin(m * phi);
        }
    }
}

// Offset of the degree-l block in the table of rotation matrices: sum_{k<l} (2k+1)^2.
inline long long jblock(int l) { return (long long)l * (4LL * l * l - 1) / 3; }

// J_l[mi][mj] = int Y_{l, mj-l}(P^T s) Y_{l, mi-l}(s) dOmega for l <= p, with P the rotation
// about x by -90 degrees (P e_z = e_y): the coefficients of f(P^T x) in terms of those of f,
// degree by degree.  A rotation about y by b is then J Rz(b) J^T with Rz the (cheap) rotation
// about z.  Product rule (Gauss-Legendre x trapezoid) exact to degree 2p.
inline void rotation_J(int p, std::vector<double>& J) {
    J.assign((size_t)jblock(p + 1), 0.0);
    const int nt = p + 1, nphi = 2 * p + 1;
    std::vector<double> z, wz, ya, yb;
    gauss_legendre(std::max(nt, 2), z, wz);
    for (size_t i = 0; i < z.size(); ++i)
        for (int k = 0; k < nphi; ++k) {
            const double ph = 2.0 * M_PI * k / nphi, st = std::sqrt(1.0 - z[i] * z[i]);
            const double sx = st * std::cos(ph), sy = st * std::sin(ph), sz = z[i];
            const double w = wz[i] * 2.0 * M_PI / nphi;
            real_ylm(p, sx, sy, sz, ya);
            real_ylm(p, sx, -sz, sy, yb);     // at P^T s = (s_x, -s_z, s_y)
            for (int l = 0; l <= p; ++l) {
                double* Jl = J.data() + jblock(l);
                const int n = 2 * l + 1;
                for (int mi = 0; mi < n; ++mi)
                    for (int mj = 0; mj < n; ++mj)
                        Jl[mi * n + mj] += w * yb[(size_t)l * l + mj] * ya[(size_t)l * l + mi];
            }
        }
}

// Entries of one stored coaxial block with input degree pin and output degree pout.
inline long long coax_block_size(int pin, int pout) {
    long long s = 0;
    for (int m = 0; m <= std::min(pin, pout); ++m) s += (long long)(pin + 1 - m) * (pout + 1 - m);
    return s;
}

// Gradient of f_l(r) Y_lm in the real basis (used for the source-side force terms of the FMM):
//   d_alpha (f_l Y_lm) = sum_m' c[alpha][l -> l+1][m][m'] g+ Y_{l+1,m'} + c[alpha][l -> l-1][m][m'] g- Y_{l-1,m'},
// g+ = f' - l f / r, g- = f' + (l+1) f / r (for f = k_l(kappa r): g+ = -kappa k_{l+1}, g- = -kappa k_{l-1}).
// The coefficients follow from the textbook gradient formula of the complex harmonics with the
// Condon-Shortley phase (z component and the ladder combinations d_x +- i d_y), converted to the
// library's real basis: R_l0 = Y_l^0, R_lm = ((-1)^m Y_l^m + Y_l^-m)/sqrt(2),
// R_l,-m = ((-1)^m Y_l^m - Y_l^-m)/(i sqrt(2)), m > 0.
// Layout: for l = 0..L, for the two targets lp = l+1 and lp = l-1 (the latter absent at l = 0),
// for alpha = x, y, z, a (2l+1) x (2lp+1) block (row: the input m, column: the output m').
struct GradIndex {
    int L = 0;
    std::vector<long long> off;   // [(L+1) * 2]: block triple of (l, up) (up = 1: lp = l+1), -1 if absent
    long long size = 0;
};

inline void gradient_table(int L, GradIndex& gi, std::vector<double>& tab) {
    typedef std::complex<double> cd;
    gi.L = L;
    gi.off.assign((size_t)(L + 1) * 2, -1);
    long long o = 0;
    for (int l = 0; l <= L; ++l)
        for (int up = 1; up >= 0; --up) {
            const int lp = up ? l + 1 : l - 1;
            if (lp < 0) continue;
            gi.off[(size_t)l * 2 + up] = o;
            o += 3LL * (2 * l + 1) * (2 * lp + 1);
        }
    gi.size = o;
    tab.assign((size_t)o, 0.0);
    auto Umat = [](int l) {   // real <- complex, rows real m' + l, columns complex m + l
        const int n = 2 * l + 1;
        std::vector<cd> U((size_t)n * n, cd(0.0, 0.0));
        U[(size_t)l * n + l] = 1.0;
        const double s = 1.0 / std::sqrt(2.0);
        for (int m = 1; m <= l; ++m) {
            const double sg = (m & 1) ? -1.0 : 1.0;
            U[(size_t)(l + m) * n + (l + m)] = sg * s;
            U[(size_t)(l + m) * n + (l - m)] = s;
            U[(size_t)(l - m) * n + (l + m)] = sg * s / cd(0.0, 1.0);
            U[(size_t)(l - m) * n + (l - m)] = -s / cd(0.0, 1.0);
        }
        return U;
    };
    auto inv_U = [](int l) {   // complex <- real (U is unitary)
        const int n = 2 * l + 1;
        std::vector<cd> V((size_t)n * n, cd(0.0, 0.0));
        V[(size_t)l * n + l] = 1.0;
        const double s = 1.0 / std::sqrt(2.0);
        for (int m = 1; m <= l; ++m) {
            const double sg = (m & 1) ? -1.0 : 1.0;
            // Y^m = sg (R_m + i R_-m)/sqrt2, Y^-m = (R_m - i R_-m)/sqrt2
            V[(size_t)(l + m) * n + (l + m)] = sg * s;
            V[(size_t)(l + m) * n + (l - m)] = sg * s * cd(0.0, 1.0);
            V[(size_t)(l - m) * n + (l + m)] = s;
            V[(size_t)(l - m) * n + (l - m)] = -s * cd(0.0, 1.0);
        }
        return V;
    };
    for (int l = 0; l <= L; ++l)
        for (int up = 1; up >= 0; --up) {
            const int lp = up ? l + 1 : l - 1;
            if (lp < 0) continue;
            const int n = 2 * l + 1, np = 2 * lp + 1;
            std::vector<cd> Gc((size_t)3 * n * np, cd(0.0, 0.0));   // complex: rows m, columns m'
            for (int m = -l; m <= l; ++m) {
                double z, pl, mi;
                if (up) {
                    const double den = (2.0 * l + 1) * (2.0 * l + 3);
                    z = std::sqrt(((l + 1.0) * (l + 1.0) - (double)m * m) / den);
                    pl = -std::sqrt((l + m + 1.0) * (l + m + 2.0) / den);
                    mi = std::sqrt((l - m + 1.0) * (l - m + 2.0) / den);
                } else {
                    const double den = (2.0 * l - 1) * (2.0 * l + 1);
                    z = std::sqrt(((double)l * l - (double)m * m) / den);
                    pl = std::sqrt(std::max(0.0, (l - m) * (l - m - 1.0)) / den);
                    mi = -std::sqrt(std::max(0.0, (l + m) * (l + m - 1.0)) / den);
                }
                auto at = [&](int a, int mm) -> cd& { return Gc[((size_t)a * n + (m + l)) * np + (mm + lp)]; };
                if (std::abs(m) <= lp) at(2, m) += z;
                if (std::abs(m + 1) <= lp) {   // (d_x + i d_y) -> Y^{m+1}
                    at(0, m + 1) += pl / 2.0;
                    at(1, m + 1) += pl / cd(0.0, 2.0);
                }
                if (std::abs(m - 1) <= lp) {   // (d_x - i d_y) -> Y^{m-1}
                    at(0, m - 1) += mi / 2.0;
                    at(1, m - 1) -= mi / cd(0.0, 2.0);
                }
            }
            const std::vector<cd> U = Umat(l), Vp = inv_U(lp);
            double* out = tab.data() + gi.off[(size_t)l * 2 + up];
            for (int a = 0; a < 3; ++a)
                for (int r = 0; r < n; ++r)
                    for (int cc = 0; cc < np; ++cc) {
                        cd s(0.0, 0.0);
                        for (int k = 0; k < n; ++k)
                            for (int q = 0; q < np; ++q)
                                s += U[(size_t)r * n + k] * Gc[((size_t)a * n + k) * np + q] * Vp[(size_t)q * np + cc];
                        out[((size_t)a * n + r) * np + cc] = s.real();
                    }
        }
}

}  // namespace fmmhost
