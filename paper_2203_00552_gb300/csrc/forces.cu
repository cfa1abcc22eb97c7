// forces.cu -- analytical forces F_k = -dE_s/dx_k = -1/2 <grad g - grad L X, X_adj>
// (Eq. force_lpb), assembled from the derivatives of Sec. 3.1 of arXiv:2203.00552.
//
// With xi_r, xi_e the weighted syntheses w_n sum_lm Y_lm(s_n) X_adj of the two
// adjoint blocks, zeta = xi_r + xi_e, and G = dE/dx:
//  * A and B (Eqs. derivative_omegaij, derivative_ylm, derivative_radial,
//    derivative_bessel): for every hit (i, n, k) with omega_ik^eta(x_i^n) > 0,
//      c = 1/2 xi [d chi'(t_ik) e_ik / r_k (delta_{f>1} U - u_k) - omega_ik grad u_k]
//    summed over both blocks, where u_k is the expansion of sphere k at x_i^n and
//    U = sum_k omega_ik u_k; G[k] += c and G[i] -= c.
//  * chi_i^eta (Eq. derivative_chi_i): at an external point (f < 1) a scalar a
//    collects every term multiplying grad chi_i (the C and F0 target masks, the
//    G0 mask, and the source masks inside P chi_j and C0); per hit
//    G[k] += a chi'(t_ik) e_ik / r_k, G[i] -= the same.
//  * k_l and Y of the Yukawa expansions (Eqs. Derivative_of_k_l0, derivative_ylm):
//    with mu = -1/2 mu_C + 1/2 (-eps1/eps2) mu_F0 and c_t = zeta chi at external
//    points, G[i] += c_t grad phi_j(x_t), G[j] -= the same, for j != i.
//  * psi_0 and d_n psi_0 (Eqs. derivative_psi_0, derivative_normal_psi_0): Coulomb
//    pair terms with the field and the field gradient, target side and source side.
#include <algorithm>

#include "common.cuh"

#define FB 128

// a, c', b and c = zeta chi at every external point (see the file comment).
// Per sphere i: sigma = synthesis of C_ik * nu_i and v = synthesis of y_i at each
// external point of i.
__global__ void k_force_ext_scalars(int M, int N, int nb, int L, double e12, double sc, const int* __restrict__ ext_ptr,
                                    const int* __restrict__ ext_p, const double4* __restrict__ ext_x,
                                    const double4* __restrict__ leb, const double* __restrict__ Y,
                                    const double* __restrict__ cik, const double* __restrict__ di,
                                    const double4* __restrict__ sph, const double* __restrict__ X,
                                    const double* __restrict__ nu, const double* __restrict__ xir,
                                    const double* __restrict__ xie, const double* __restrict__ phiC,
                                    const double* __restrict__ S0, const double* __restrict__ psi0,
                                    const double* __restrict__ dn, double4* __restrict__ fs) {
    extern __shared__ double sm[];
    const int i = blockIdx.x;
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    if (cnt == 0) return;
    double* u = sm;
    double* yv = u + nb;
    const double ri = sph[i].w;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        int l = (int)sqrtf((float)idx + 0.5f);
        u[idx] = cik[(size_t)i * (L + 1) + l] * nu[(size_t)i * nb + idx];
        yv[idx] = e12 * (double)l / ri * X[(size_t)i * nb + idx] - di[(size_t)i * (L + 1) + l] * X[(size_t)(M + i) * nb + idx];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, p = ext_p[t], n = p % N;
        double sg = 0, vc = 0;
        for (int idx = 0; idx < nb; ++idx) {
            double yy = Y[(size_t)n * nb + idx];
            sg += yy * u[idx];
            vc += yy * yv[idx];
        }
        double w = leb[n].w, chi = ext_x[t].w;
        double xr = xir[p], z = xr + xie[p];
        double a = -0.5 * z * phiC[t] + 0.5 * sc * z * S0[t] - 0.5 * xr * psi0[t] - 0.5 * w * vc * sg +
                   0.5 * sc * w * dn[t] * sg;
        fs[t] = make_double4(a, -0.5 * xr * chi, 0.5 * sc * w * chi * sg, z * chi);
    }
}

// Per-hit force vectors c_h of the A/B terms and of the chi_i^eta derivative.
__global__ void k_force_hits(int M, int N, int nb, int L, double kappa, double eta, const double4* __restrict__ sph,
                             const double4* __restrict__ leb, YTab yt, const int* __restrict__ hptr,
                             const int* __restrict__ hj, const double* __restrict__ hw, const double* __restrict__ fval,
                             const double* __restrict__ Sinv, const double* __restrict__ X,
                             const double* __restrict__ xir, const double* __restrict__ xie,
                             const double* __restrict__ UA, const double* __restrict__ UB,
                             const int* __restrict__ isext_pos, const double4* __restrict__ fs,
                             double* __restrict__ ch) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    double* rr = sm;
    double* drr = rr + (L + 1) * bd;
    double* ri = drr + (L + 1) * bd;
    double* dri = ri + (L + 1) * bd;
    const long long MN = (long long)M * N;
    const long long p = (long long)blockIdx.x * bd + tid;
    if (p >= MN) return;
    const int i = (int)(p / N), n = (int)(p % N);
    const int h0 = hptr[p], h1 = hptr[p + 1];
    if (h0 == h1) return;
    const double4 a4 = sph[i], s = leb[n];
    const double px = a4.x + a4.w * s.x, py = a4.y + a4.w * s.y, pz = a4.z + a4.w * s.z;
    const double f = fval[p];
    const double d = f > 1.0 ? 1.0 / f : 1.0;
    const double delta = f > 1.0 ? 1.0 : 0.0;
    const double xr = xir[p], xe = xie[p];
    const double ua = UA[p], ub = UB[p];
    const int ep = isext_pos[p];
    const double amask = ep >= 0 ? fs[ep].x : 0.0;
    for (int h = h0; h < h1; ++h) {
        const int k = hj[h];
        const double om = hw[h];
        const double4 b = sph[k];
        double dx = px - b.x, dy = py - b.y, dz = pz - b.z;
        double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
        double ex = dx * inv, ey = dy * inv, ez = dz * inv;
        double t = rho / b.w;
        double dc = dchi_eta(t, eta);
        radial<double>(0, L, rho, b.w, kappa, nullptr, rr + tid, drr + tid, bd);
        radial<double>(1, L, rho, b.w, kappa, Sinv + (size_t)k * (L + 2), ri + tid, dri + tid, bd);
        const double* Xr = X + (size_t)k * nb;
        const double* Xe = X + (size_t)(M + k) * nb;
        double uA = 0, aA = 0, bAx = 0, bAy = 0, bAz = 0;
        double uB = 0, aB = 0, bBx = 0, bBy = 0, bBz = 0;
        ylm_grad_stream<double>(L, ex, ey, ez, yt, [&](int idx, int l, double yv, double gx, double gy, double gz) {
            double cr = __ldg(Xr + idx), ce = __ldg(Xe + idx);
            double R = rr[tid + l * bd], dR = drr[tid + l * bd];
            double Ri = ri[tid + l * bd], dRi = dri[tid + l * bd];
            uA += cr * R * yv;
            aA += cr * dR * yv;
            double fa = cr * R * inv;
            bAx += fa * gx; bAy += fa * gy; bAz += fa * gz;
            uB += ce * Ri * yv;
            aB += ce * dRi * yv;
            double fb = ce * Ri * inv;
            bBx += fb * gx; bBy += fb * gy; bBz += fb * gz;
        });
        // spatial gradients: R' Y e + (R/rho)(G - (e.G) e)
        double pA = bAx * ex + bAy * ey + bAz * ez, pB = bBx * ex + bBy * ey + bBz * ez;
        double gAx = aA * ex + bAx - pA * ex, gAy = aA * ey + bAy - pA * ey, gAz = aA * ez + bAz - pA * ez;
        double gBx = aB * ex + bBx - pB * ex, gBy = aB * ey + bBy - pB * ey, gBz = aB * ez + bBz - pB * ez;
        double sA = d * dc / b.w * (delta * ua - uA), sB = d * dc / b.w * (delta * ub - uB);
        double msk = (1.0 - delta) * amask * dc / b.w;
        double cx = 0.5 * xr * (sA * ex - om * gAx) + 0.5 * xe * (sB * ex - om * gBx) + msk * ex;
        double cy = 0.5 * xr * (sA * ey - om * gAy) + 0.5 * xe * (sB * ey - om * gBy) + msk * ey;
        double cz = 0.5 * xr * (sA * ez - om * gAz) + 0.5 * xe * (sB * ez - om * gBz) + msk * ez;
        ch[3 * (size_t)h] = cx;
        ch[3 * (size_t)h + 1] = cy;
        ch[3 * (size_t)h + 2] = cz;
    }
}

// G[i] -= sum of c_h over the hits of sphere i; G[k] += sum of c_h over the hits into k.
__global__ void k_force_hits_gather(int M, int N, const int* __restrict__ hptr, const int* __restrict__ tptr,
                                    const int* __restrict__ th, const double* __restrict__ ch, double* __restrict__ G) {
    __shared__ double red[3][FB / 32];
    const int i = blockIdx.x;
    double gx = 0, gy = 0, gz = 0;
    const int a0 = hptr[(long long)i * N], a1 = hptr[(long long)(i + 1) * N];
    for (int h = a0 + threadIdx.x; h < a1; h += blockDim.x) {
        gx -= ch[3 * (size_t)h];
        gy -= ch[3 * (size_t)h + 1];
        gz -= ch[3 * (size_t)h + 2];
    }
    for (int q = tptr[i] + threadIdx.x; q < tptr[i + 1]; q += blockDim.x) {
        int h = th[q];
        gx += ch[3 * (size_t)h];
        gy += ch[3 * (size_t)h + 1];
        gz += ch[3 * (size_t)h + 2];
    }
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    gz = warp_sum(gz);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = gx;
        red[1][threadIdx.x >> 5] = gy;
        red[2][threadIdx.x >> 5] = gz;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int w = 0; w < FB / 32; ++w) s += red[threadIdx.x][w];
        G[3 * (size_t)i + threadIdx.x] += s;
    }
}

// Target side of the Yukawa and Coulomb pair terms: per external point t (on sphere i)
//   Ft = c_t sum_{j in src, j != i} grad (mu_j . B^k_j)(x_t)
//      + sum_{k != i} q_k [c'_t grad(1/|x - x_k|) + b_t H(x_t - x_k) s_n] / eps1
#define FT_TS 8
__global__ void k_force_targets(int E, int N, int M, int nb, int L, double kappa, double eps1,
                                const double4* __restrict__ ext_x, const int* __restrict__ ext_p,
                                const double4* __restrict__ leb, int n_src, const int* __restrict__ src,
                                const double4* __restrict__ sph, const double* __restrict__ q,
                                const double* __restrict__ mu, const double* __restrict__ Khinv, YTab yt,
                                const double4* __restrict__ fs, double* __restrict__ Ft) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    double4* sp = (double4*)sm;
    int* sid = (int*)(sp + FT_TS);
    double* smu = (double*)(sid + 2 * FT_TS);
    double* skh = smu + FT_TS * nb;
    double* rad = skh + FT_TS * (L + 2);
    double* drad = rad + (L + 1) * bd;
    const int t = blockIdx.x * bd + tid;
    const bool valid = t < E;
    const double4 xt = valid ? ext_x[t] : make_double4(0, 0, 0, 0);
    const int p = valid ? ext_p[t] : 0;
    const int it = p / N;
    const double4 sn = leb[p % N];
    const double4 w4 = valid ? fs[t] : make_double4(0, 0, 0, 0);
    double fx = 0, fy = 0, fz = 0;
    // Yukawa
    for (int base = 0; base < n_src; base += FT_TS) {
        int ns = min(FT_TS, n_src - base);
        __syncthreads();
        for (int k = tid; k < ns * nb; k += bd) smu[k] = mu[(size_t)src[base + k / nb] * nb + k % nb];
        for (int k = tid; k < ns * (L + 2); k += bd) skh[k] = Khinv[(size_t)src[base + k / (L + 2)] * (L + 2) + k % (L + 2)];
        if (tid < ns) {
            sp[tid] = sph[src[base + tid]];
            sid[tid] = src[base + tid];
        }
        __syncthreads();
        for (int s = 0; s < ns; ++s) {
            double4 b = sp[s];
            bool self = !valid || sid[s] == it;
            double dx = self ? b.w : xt.x - b.x, dy = self ? 0 : xt.y - b.y, dz = self ? 0 : xt.z - b.z;
            double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
            double ex = dx * inv, ey = dy * inv, ez = dz * inv;
            radial<double>(2, L, rho, b.w, kappa, skh + s * (L + 2), rad + tid, drad + tid, bd);
            const double* m = smu + s * nb;
            double A = 0, Bx = 0, By = 0, Bz = 0;
            ylm_grad_stream<double>(L, ex, ey, ez, yt, [&](int idx, int l, double yv, double gx, double gy, double gz) {
                double c = m[idx];
                A += c * drad[tid + l * bd] * yv;
                double fr = c * rad[tid + l * bd] * inv;
                Bx += fr * gx; By += fr * gy; Bz += fr * gz;
            });
            if (!self) {
                double pr = Bx * ex + By * ey + Bz * ez;
                fx += w4.w * (A * ex + Bx - pr * ex);
                fy += w4.w * (A * ey + By - pr * ey);
                fz += w4.w * (A * ez + Bz - pr * ez);
            }
        }
    }
    // Coulomb
    for (int base = 0; base < M; base += bd) {
        __syncthreads();
        double4* sa = (double4*)sm;
        int k = base + tid;
        if (k < M) {
            double4 b = sph[k];
            sa[tid] = make_double4(b.x, b.y, b.z, q[k]);
        }
        __syncthreads();
        int cnt = min(bd, M - base);
        for (int kk = 0; kk < cnt; ++kk) {
            if (!valid || base + kk == it) continue;
            double4 b = sa[kk];
            double dx = xt.x - b.x, dy = xt.y - b.y, dz = xt.z - b.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            double ir = rsqrt(r2), ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
            // grad(1/r) = -d/r^3 ; H s = 3 d (d.s)/r^5 - s/r^3
            double ds = dx * sn.x + dy * sn.y + dz * sn.z;
            double cq = b.w / eps1;
            fx += cq * (-w4.y * dx * ir3 + w4.z * (3.0 * dx * ds * ir5 - sn.x * ir3));
            fy += cq * (-w4.y * dy * ir3 + w4.z * (3.0 * dy * ds * ir5 - sn.y * ir3));
            fz += cq * (-w4.y * dz * ir3 + w4.z * (3.0 * dz * ds * ir5 - sn.z * ir3));
        }
    }
    if (valid) {
        Ft[3 * (size_t)t] = fx;
        Ft[3 * (size_t)t + 1] = fy;
        Ft[3 * (size_t)t + 2] = fz;
    }
}

// G[i] += sum of Ft over the external points of sphere i.
__global__ void k_force_targets_gather(const int* __restrict__ ext_ptr, const double* __restrict__ Ft,
                                       double* __restrict__ G) {
    __shared__ double red[3][FB / 32];
    const int i = blockIdx.x;
    double gx = 0, gy = 0, gz = 0;
    for (int t = ext_ptr[i] + threadIdx.x; t < ext_ptr[i + 1]; t += blockDim.x) {
        gx += Ft[3 * (size_t)t];
        gy += Ft[3 * (size_t)t + 1];
        gz += Ft[3 * (size_t)t + 2];
    }
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    gz = warp_sum(gz);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = gx;
        red[1][threadIdx.x >> 5] = gy;
        red[2][threadIdx.x >> 5] = gz;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int w = 0; w < FB / 32; ++w) s += red[threadIdx.x][w];
        G[3 * (size_t)i + threadIdx.x] += s;
    }
}

// Source side of the Yukawa pair terms: G[j] -= sum_{t not on j} c_t grad (mu_j . B^k_j)(x_t).
__global__ void k_force_yukawa_sources(int E, int N, int nb, int L, double kappa, const double4* __restrict__ ext_x,
                                       const int* __restrict__ ext_p, const int* __restrict__ src,
                                       const double4* __restrict__ sph, const double* __restrict__ mu,
                                       const double* __restrict__ Khinv, YTab yt, const double4* __restrict__ fs,
                                       double* __restrict__ G) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    double* m = sm;
    double* kh = m + nb;
    double* rad = kh + (L + 2);
    double* drad = rad + (L + 1) * bd;
    double* red = drad + (L + 1) * bd;
    const int j = src[blockIdx.x];
    const double4 b = sph[j];
    for (int k = tid; k < nb; k += bd) m[k] = mu[(size_t)j * nb + k];
    for (int k = tid; k < L + 2; k += bd) kh[k] = Khinv[(size_t)j * (L + 2) + k];
    __syncthreads();
    double fx = 0, fy = 0, fz = 0;
    for (int t = tid; t < E; t += bd) {
        if (ext_p[t] / N == j) continue;
        double4 xt = ext_x[t];
        double c = fs[t].w;
        double dx = xt.x - b.x, dy = xt.y - b.y, dz = xt.z - b.z;
        double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
        double ex = dx * inv, ey = dy * inv, ez = dz * inv;
        radial<double>(2, L, rho, b.w, kappa, kh, rad + tid, drad + tid, bd);
        double A = 0, Bx = 0, By = 0, Bz = 0;
        ylm_grad_stream<double>(L, ex, ey, ez, yt, [&](int idx, int l, double yv, double gx, double gy, double gz) {
            double cc = m[idx];
            A += cc * drad[tid + l * bd] * yv;
            double fr = cc * rad[tid + l * bd] * inv;
            Bx += fr * gx; By += fr * gy; Bz += fr * gz;
        });
        double pr = Bx * ex + By * ey + Bz * ez;
        fx += c * (A * ex + Bx - pr * ex);
        fy += c * (A * ey + By - pr * ey);
        fz += c * (A * ez + Bz - pr * ez);
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if ((tid & 31) == 0) {
        red[3 * (tid >> 5)] = fx;
        red[3 * (tid >> 5) + 1] = fy;
        red[3 * (tid >> 5) + 2] = fz;
    }
    __syncthreads();
    if (tid < 3) {
        double s = 0;
        for (int w = 0; w < bd / 32; ++w) s += red[3 * w + tid];
        G[3 * (size_t)j + tid] -= s;
    }
}

// Source side of the Coulomb pair terms: G[k] -= sum_{t not on k} q_k [c'_t grad(1/r) + b_t H s_n] / eps1.
__global__ void k_force_coulomb_sources(int E, int N, double eps1, const double4* __restrict__ ext_x,
                                        const int* __restrict__ ext_p, const double4* __restrict__ leb,
                                        const double4* __restrict__ sph, const double* __restrict__ q,
                                        const double4* __restrict__ fs, double* __restrict__ G) {
    __shared__ double red[3][FB / 32];
    const int k = blockIdx.x;
    const double4 b = sph[k];
    double fx = 0, fy = 0, fz = 0;
    for (int t = threadIdx.x; t < E; t += blockDim.x) {
        int p = ext_p[t];
        if (p / N == k) continue;
        double4 xt = ext_x[t], sn = leb[p % N], w4 = fs[t];
        double dx = xt.x - b.x, dy = xt.y - b.y, dz = xt.z - b.z;
        double r2 = dx * dx + dy * dy + dz * dz;
        double ir = rsqrt(r2), ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
        double ds = dx * sn.x + dy * sn.y + dz * sn.z;
        fx += -w4.y * dx * ir3 + w4.z * (3.0 * dx * ds * ir5 - sn.x * ir3);
        fy += -w4.y * dy * ir3 + w4.z * (3.0 * dy * ds * ir5 - sn.y * ir3);
        fz += -w4.y * dz * ir3 + w4.z * (3.0 * dz * ds * ir5 - sn.z * ir3);
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = fx;
        red[1][threadIdx.x >> 5] = fy;
        red[2][threadIdx.x >> 5] = fz;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int w = 0; w < FB / 32; ++w) s += red[threadIdx.x][w];
        G[3 * (size_t)k + threadIdx.x] -= s * q[k] / eps1;
    }
}

__global__ void k_ext_index(int E, const int* __restrict__ ext_p, int* __restrict__ pos) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < E) pos[ext_p[t]] = t;
}

__global__ void k_mu_comb(long long n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                          double* __restrict__ out) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = a * x[k] + b * y[k];
}

__global__ void k_negate(long long n, const double* __restrict__ G, double* __restrict__ F) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) F[k] = -G[k];
}

static ddlpb_status fsmem(ddlpb_ctx* c, const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) DDLPB_CK(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return DDLPB_OK;
}

ddlpb_status compute_forces(ddlpb_ctx* c, double* f_dev) {
    const int M = c->M, N = c->N, nb = c->nb, L = c->lmax;
    const long long MN = (long long)M * N;
    const long long half = (long long)M * nb;
    cudaStream_t st = c->stream;
    static_assert(sizeof(double4) == 32, "double4");
    // scratch (allocated once per context)
    if (!c->force_acc) DDLPB_TRY(ctx_alloc(c, &c->force_acc, 3 * (size_t)M));
    ForceScratch& s = c->fscr;
    if (!s.ready) {
        DDLPB_TRY(ctx_alloc(c, &s.xir, MN));
        DDLPB_TRY(ctx_alloc(c, &s.xie, MN));
        DDLPB_TRY(ctx_alloc(c, &s.UA, MN));
        DDLPB_TRY(ctx_alloc(c, &s.UB, MN));
        DDLPB_TRY(ctx_alloc(c, &s.ch, 3 * (size_t)c->H));
        DDLPB_TRY(ctx_alloc(c, &s.Ft, 3 * (size_t)c->E));
        DDLPB_TRY(ctx_alloc(c, &s.G, 3 * (size_t)M));
        DDLPB_TRY(ctx_alloc(c, &s.muC, half));
        DDLPB_TRY(ctx_alloc(c, &s.nu, half));
        DDLPB_TRY(ctx_alloc(c, &s.muc, half));
        DDLPB_TRY(ctx_alloc(c, &s.fs, c->E));
        DDLPB_TRY(ctx_alloc(c, &s.extpos, MN));
        s.ready = true;
    }
    DDLPB_CK(c, cudaMemsetAsync(s.G, 0, sizeof(double) * 3 * M, st));
    DDLPB_CK(c, cudaMemsetAsync(s.muC, 0, sizeof(double) * half, st));
    DDLPB_CK(c, cudaMemsetAsync(s.nu, 0, sizeof(double) * half, st));
    DDLPB_CK(c, cudaMemsetAsync(s.extpos, 0xff, sizeof(int) * MN, st));
    if (c->E > 0) {
        k_ext_index<<<ceil_div(c->E, 256), 256, 0, st>>>(c->E, c->ext_p, s.extpos);
        DDLPB_LAUNCHED(c, "ext_index");
    }
    const double e12 = c->eps1 / c->eps2, sc = -e12;

    // adjoint syntheses xi_r, xi_e and the A/B grid values U of X
    DDLPB_TRY(op_synthesis(c, c->Xa, M, s.xir, true));
    DDLPB_TRY(op_synthesis(c, c->Xa + half, M, s.xie, true));
    DDLPB_TRY(op_apply_AB(c, c->X, nullptr, false, s.UA, s.UB));

    if (c->E > 0) {
        // mu_C, its potential phi_C, the adjoint coefficients nu = K^T(zeta chi)
        DDLPB_TRY(op_source_multipoles(c, c->X, s.muC));
        DDLPB_TRY(op_yukawa_potential(c, s.muC, c->extA));
        DDLPB_TRY(op_ext_weights(c, c->Xa, c->extB));
        DDLPB_TRY(op_yukawa_adjoint(c, c->extB, s.nu));
        size_t sm1 = sizeof(double) * 2 * nb;
        k_force_ext_scalars<<<M, FB, sm1, st>>>(M, N, nb, L, e12, sc, c->ext_ptr, c->ext_p, c->ext_x, c->leb, c->Y,
                                                c->cik, c->di, c->sph, c->X, s.nu, s.xir, s.xie, c->extA, c->S0,
                                                c->psi0, c->dnpsi0, s.fs);
        DDLPB_LAUNCHED(c, "force_ext_scalars");
    }
    // per-hit terms
    if (c->H > 0) {
        size_t sm2 = sizeof(double) * 4 * (size_t)(L + 1) * FB;
        DDLPB_TRY(fsmem(c, (const void*)k_force_hits, sm2));
        k_force_hits<<<ceil_div(MN, FB), FB, sm2, st>>>(M, N, nb, L, c->kappa, c->eta, c->sph, c->leb, c->yt,
                                                        c->hit_ptr, c->hit_j, c->hit_w, c->fval, c->Sinv, c->X, s.xir,
                                                        s.xie, s.UA, s.UB, s.extpos, s.fs, s.ch);
        DDLPB_LAUNCHED(c, "force_hits");
        k_force_hits_gather<<<M, FB, 0, st>>>(M, N, c->hit_ptr, c->thit_ptr, c->thit_h, s.ch, s.G);
        DDLPB_LAUNCHED(c, "force_hits_gather");
    }
    if (c->E > 0) {
        // mu = -1/2 mu_C + 1/2 sc mu0
        k_mu_comb<<<ceil_div(half, 256), 256, 0, st>>>(half, -0.5, s.muC, 0.5 * sc, c->mu0, s.muc);
        DDLPB_LAUNCHED(c, "mu_comb");
        size_t sm3 = sizeof(double4) * FT_TS + sizeof(int) * 2 * FT_TS +
                     sizeof(double) * (FT_TS * (size_t)nb + FT_TS * (size_t)(L + 2) + 2 * (size_t)(L + 1) * FB);
        sm3 = std::max(sm3, sizeof(double4) * FB);
        DDLPB_TRY(fsmem(c, (const void*)k_force_targets, sm3));
        // with the FMM the Yukawa part is added below (far field from the expansions), so
        // this kernel keeps only the Coulomb part (no sources)
        k_force_targets<<<ceil_div(c->E, FB), FB, sm3, st>>>(c->E, N, M, nb, L, c->kappa, c->eps1, c->ext_x,
                                                             c->ext_p, c->leb, c->fmm.on ? 0 : c->n_src, c->src,
                                                             c->sph, c->q, s.muc, c->Khinv, c->yt, s.fs, s.Ft);
        DDLPB_LAUNCHED(c, "force_targets");
        if (c->fmm.on) DDLPB_TRY(fmm_force_terms(c, s.muc, s.fs, s.Ft, s.G));
        k_force_targets_gather<<<M, FB, 0, st>>>(c->ext_ptr, s.Ft, s.G);
        DDLPB_LAUNCHED(c, "force_targets_gather");
        if (!c->fmm.on) {
            size_t sm4 = sizeof(double) * (nb + (L + 2) + 2 * (size_t)(L + 1) * FB + 3 * (FB / 32));
            DDLPB_TRY(fsmem(c, (const void*)k_force_yukawa_sources, sm4));
            k_force_yukawa_sources<<<c->n_src, FB, sm4, st>>>(c->E, N, nb, L, c->kappa, c->ext_x, c->ext_p, c->src,
                                                              c->sph, s.muc, c->Khinv, c->yt, s.fs, s.G);
            DDLPB_LAUNCHED(c, "force_yukawa_sources");
        }
        k_force_coulomb_sources<<<M, FB, 0, st>>>(c->E, N, c->eps1, c->ext_x, c->ext_p, c->leb, c->sph, c->q, s.fs,
                                                  s.G);
        DDLPB_LAUNCHED(c, "force_coulomb_sources");
    }
    k_negate<<<ceil_div(3LL * M, 256), 256, 0, st>>>(3LL * M, s.G, f_dev);
    DDLPB_LAUNCHED(c, "negate");
    return DDLPB_OK;
}
