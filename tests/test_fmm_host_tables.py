"""Host-side tables of the GPU FMM (paper_2203_00552_gb300/csrc/fmm_host.h), compiled with g++
and checked against independent definitions (the Appendix's OZ-axis translation scheme rests
on them):
  * J, the rotation about x by -90 degrees, degree by degree: orthogonal, the coefficients of
    f(P^T x) from those of f (checked with the oracle's real Y_lm at random points), and
    J^T = S J S with S = diag(-1 for m < 0), the identity the batched translation kernels use to
    form every product with J from J^T;
  * the Gaunt sums of the coaxial translations, g = 4 pi Y_b0(e_z) int Y_lm Y_am Y_b0, against a
    Lebedev quadrature of the oracle's Y_lm.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_00552_gb300", "csrc")

HARNESS = r"""
#include "fmm_host.h"
#include <cstdio>
int main() {
    const int PMAX = 21, P = 6;
    std::vector<double> J;
    fmmhost::rotation_J(PMAX, J);
    double orth = 0, sym = 0;
    for (int l = 0; l <= PMAX; ++l) {
        const int n = 2 * l + 1;
        const double* Jl = J.data() + fmmhost::jblock(l);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0;
                for (int k = 0; k < n; ++k) s += Jl[i * n + k] * Jl[j * n + k];
                orth = std::max(orth, std::fabs(s - (i == j)));
                const double si = i < l ? -1 : 1, sj = j < l ? -1 : 1;
                sym = std::max(sym, std::fabs(Jl[j * n + i] - si * sj * Jl[i * n + j]));
            }
    }
    printf("{\"orth\": %.3e, \"sym\": %.3e, \"J\": [", orth, sym);
    for (long long k = 0; k < fmmhost::jblock(P + 1); ++k) printf("%s%.17g", k ? "," : "", J[k]);
    fmmhost::CoaxIndex gi;
    std::vector<double> g;
    fmmhost::gaunt_coax_table(P, gi, g);
    printf("], \"g\": [");
    bool first = true;
    for (int m = 0; m <= P; ++m)
        for (int l = m; l <= P; ++l)
            for (int a = m; a <= P; ++a) {
                const long long o = gi.off[((size_t)m * (P + 1) + l) * (P + 1) + a];
                for (int j = 0; j <= std::min(l, a); ++j) {
                    printf("%s[%d,%d,%d,%d,%.17g]", first ? "" : ",", m, l, a, j, g[(size_t)(o + j)]);
                    first = false;
                }
            }
    printf("]}\n");
}
"""


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fmmhost")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_rotation_table_is_orthogonal_and_S_symmetric(tables):
    assert tables["orth"] < 1e-12
    assert tables["sym"] < 1e-12


def test_rotation_table_rotates_expansions(tables):
    """sum_i (J c)_i Y_li(s) = sum_j c_j Y_lj(P^T s), P^T s = (s_x, -s_z, s_y), for l <= 6."""
    P = 6
    J = np.array(tables["J"])
    rng = np.random.default_rng(0)
    s = rng.normal(size=(50, 3))
    s /= np.linalg.norm(s, axis=1)[:, None]
    ps = np.stack([s[:, 0], -s[:, 2], s[:, 1]], axis=1)
    Y, Yp = sph.ylm(P, s), sph.ylm(P, ps)
    o = 0
    for l in range(P + 1):
        n = 2 * l + 1
        Jl = J[o:o + n * n].reshape(n, n)
        o += n * n
        c = rng.normal(size=n)
        lhs = Y[:, l * l:l * l + n] @ (Jl @ c)
        rhs = Yp[:, l * l:l * l + n] @ c
        assert np.abs(lhs - rhs).max() < 1e-12, l


def test_gaunt_sums_match_quadrature(tables):
    """g[m, l, a, j] = 4 pi Y_b0(e_z) int Y_lm Y_am Y_b0 with b = l + a - 2j, m >= 0 (the same
    value for -m), against the 590-point Lebedev rule (exact to degree 41 >= l + a + b)."""
    s, w, deg = sph.lebedev(590)
    P = 6
    assert 4 * P <= deg
    Y = sph.ylm(2 * P, s)
    for m, l, a, j, g in tables["g"]:
        b = l + a - 2 * j
        yb0_ez = np.sqrt((2 * b + 1) / (4 * np.pi))
        for mm in ((m, -m) if m > 0 else (0,)):
            want = 4 * np.pi * yb0_ez * np.sum(w * Y[:, l * l + l + mm] * Y[:, a * a + a + mm] * Y[:, b * b + b])
            assert abs(g - want) < 1e-12 * max(1.0, abs(want)), (m, l, a, j, mm, g, want)


def test_translation_with_JT_only_equals_the_rotation_sequence(tables):
    """The batched kernels translate as Rz(a) J Rz(b) J^T Z J Rz(-b) J^T Rz(-a) but form every
    product with J as S J^T S and fold the two S into the neighbouring steps; the folded sequence
    gives the same operator (Z any m-preserving coaxial map, same block for +m and -m)."""
    P = 6
    nb = (P + 1) ** 2
    J = np.array(tables["J"])
    Jf = np.zeros((nb, nb))
    o = 0
    for l in range(P + 1):
        n = 2 * l + 1
        Jf[l * l:l * l + n, l * l:l * l + n] = J[o:o + n * n].reshape(n, n)
        o += n * n
    lidx = np.array([int(np.sqrt(i)) for i in range(nb)])
    midx = np.arange(nb) - lidx * lidx - lidx
    S = np.diag(np.where(midx < 0, -1.0, 1.0))

    def Rz(ang, s):
        R = np.eye(nb)
        for i in range(nb):
            l, m = lidx[i], midx[i]
            if m > 0:
                j = l * l + l - m
                c, sn = np.cos(m * ang), s * np.sin(m * ang)
                R[i, i], R[i, j], R[j, i], R[j, j] = c, -sn, sn, c
        return R

    rng = np.random.default_rng(2)
    Z = np.zeros((nb, nb))
    for m in range(P + 1):
        for l in range(m, P + 1):
            for a in range(m, P + 1):
                v = rng.normal()
                Z[a * a + a + m, l * l + l + m] = v
                if m > 0:
                    Z[a * a + a - m, l * l + l - m] = v
    al, be = 0.7, 1.9
    x = rng.normal(size=nb)
    plain = Rz(al, 1) @ Jf @ Rz(be, 1) @ Jf.T @ Z @ Jf @ Rz(be, -1) @ Jf.T @ Rz(al, -1) @ x
    v = Jf.T @ (Rz(al, -1) @ x)
    v = Jf.T @ (S @ (Rz(be, -1) @ v))        # rotation with its output flipped, then J^T
    v = Jf.T @ (Z @ (S @ v))                 # the coaxial step reads the flipped input
    v = Jf.T @ (S @ (Rz(be, 1) @ v))
    folded = Rz(al, 1) @ (S @ v)             # the last rotation reads the flipped input
    assert np.abs(plain - folded).max() < 1e-12 * np.abs(plain).max()
