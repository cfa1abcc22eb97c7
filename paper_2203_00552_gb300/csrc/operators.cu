// operators.cu -- the operators of the ddLPB system L X = g (Eq. AXg) and its adjoint
// L* (Eq. AstarXg), applied matrix-free on the device.
//
//   A, B  (Eqs. definition_of_A_matrix, definition_of_B_matrix): identity minus the
//         projection onto Y_lm(s_n) of the neighbour expansions, weighted by
//         omega_ij^eta at each grid point; evaluated from the hit lists.
//   C1 X_r + C2 X_e (Eq. def_c1_c2 with Eqs. definition_of_Q_matrix, definition_of_P_matrix):
//         y_j = eps1/eps2 (l/r_j) X_r - i_l'/i_l X_e;  mu_j = C_ik P chi_j y_j;
//         phi = sum_j mu_j k^j Y^j at the external points (direct summation);
//         out_i = sum_n w_n chi_i phi Y_lm(s_n), added to both block rows.
//   The transposes follow the same data in reverse (gathers, no atomics).
#include "common.cuh"

#define BLK 128

// ---------------------------------------------------------------- projections

// grid[row][n] = (w_n if weighted) * sum_lm YT[lm][n] coef[row][lm]
__global__ void k_synthesis(int N, int nb, const double* __restrict__ YT, const double4* __restrict__ leb,
                            const double* __restrict__ coef, double* __restrict__ grid, int weighted) {
    extern __shared__ double sc[];
    int row = blockIdx.x;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) sc[k] = coef[(size_t)row * nb + k];
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double v = 0;
        for (int k = 0; k < nb; ++k) v += YT[(size_t)k * N + n] * sc[k];
        if (weighted) v *= leb[n].w;
        grid[(size_t)row * N + n] = v;
    }
}

// out[i][lm] (+)= scale * (cik[i][l]) * sum_{external t of i} w_n chi_t val[t] Y_lm(s_n)
__global__ void k_masked_analysis(int N, int nb, int L, const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                                  const double4* __restrict__ ext_x, const double4* __restrict__ leb,
                                  const double* __restrict__ Y, const double* __restrict__ val, double scale,
                                  const double* __restrict__ cik, double* __restrict__ out, int out_stride,
                                  int accumulate) {
    extern __shared__ double sm[];
    int i = blockIdx.x;
    int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    double* gv = sm;
    int* gn = (int*)(gv + N);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k;
        int n = ext_p[t] % N;
        gn[k] = n;
        gv[k] = leb[n].w * ext_x[t].w * val[t];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        double a = 0;
        for (int k = 0; k < cnt; ++k) a += Y[(size_t)gn[k] * nb + idx] * gv[k];
        int l = (int)sqrtf((float)idx + 0.5f);
        if (cik) a *= cik[(size_t)i * (L + 1) + l];
        a *= scale;
        double* o = out + (size_t)i * out_stride + idx;
        *o = accumulate ? *o + a : a;
    }
}

// ---------------------------------------------------------------- A and B

// One CTA per sphere i.  For every grid point n the neighbour expansions of X_r
// (basis r_l^j Y^j) and X_e (basis i-ratio Y^j) are summed with omega_ij^eta; the
// grid values are projected back and subtracted from the identity.
__global__ void k_ab_apply(int M, int N, int nb, int L, double kappa, const double4* __restrict__ sph,
                           const double4* __restrict__ leb, YTab yt, const int* __restrict__ hptr,
                           const int* __restrict__ hj, const double* __restrict__ hw, const double* __restrict__ Sinv,
                           const double* __restrict__ Y, const double* __restrict__ x, double* __restrict__ y,
                           double* __restrict__ gridR, double* __restrict__ gridE) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    double* vr = sm;
    double* ve = vr + N;
    double* rr = ve + N;
    double* ri = rr + (L + 1) * bd;
    const int i = blockIdx.x;
    const double4 a = sph[i];
    const double* xr = x;
    const double* xe = x + (size_t)M * nb;
    for (int n = tid; n < N; n += bd) {
        double4 s = leb[n];
        double px = a.x + a.w * s.x, py = a.y + a.w * s.y, pz = a.z + a.w * s.z;
        long long p = (long long)i * N + n;
        double sr = 0, se = 0;
        for (int h = hptr[p]; h < hptr[p + 1]; ++h) {
            int j = hj[h];
            double w = hw[h];
            double4 b = sph[j];
            double dx = px - b.x, dy = py - b.y, dz = pz - b.z;
            double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
            radial<double>(0, L, rho, b.w, kappa, nullptr, rr + tid, nullptr, bd);
            radial<double>(1, L, rho, b.w, kappa, Sinv + (size_t)j * (L + 2), ri + tid, nullptr, bd);
            const double* Xr = xr + (size_t)j * nb;
            const double* Xe = xe + (size_t)j * nb;
            double ur = 0, ue = 0;
            ylm_stream<double>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, double yv) {
                ur += __ldg(Xr + idx) * rr[tid + l * bd] * yv;
                ue += __ldg(Xe + idx) * ri[tid + l * bd] * yv;
            });
            sr += w * ur;
            se += w * ue;
        }
        vr[n] = sr;
        ve[n] = se;
        if (gridR) {
            gridR[p] = sr;
            gridE[p] = se;
        }
    }
    __syncthreads();
    if (!y) return;
    for (int idx = tid; idx < nb; idx += bd) {
        double ar = 0, ae = 0;
        for (int n = 0; n < N; ++n) {
            double wy = leb[n].w * Y[(size_t)n * nb + idx];
            ar += wy * vr[n];
            ae += wy * ve[n];
        }
        size_t o = (size_t)i * nb + idx;
        y[o] = xr[o] - ar;
        y[(size_t)M * nb + o] = xe[o] - ae;
    }
}

// A^T and B^T: one CTA per sphere j gathers every hit (i, n) -> j.
// zr, ze are the weighted syntheses w_n sum_lm Y_lm(s_n) x_{i lm} of the two blocks.
__global__ void k_ab_transpose(int M, int N, int nb, int L, double kappa, const double4* __restrict__ sph,
                               const double4* __restrict__ leb, YTab yt, const int* __restrict__ tptr,
                               const int* __restrict__ tp, const double* __restrict__ tw,
                               const double* __restrict__ Sinv, const double* __restrict__ zr,
                               const double* __restrict__ ze, const double* __restrict__ x, double* __restrict__ y) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    double* accR = sm;
    double* accE = accR + nw * nb;
    double* rr = accE + nw * nb;
    double* ri = rr + (L + 1) * bd;
    const int j = blockIdx.x;
    const double4 b = sph[j];
    for (int k = tid; k < 2 * nw * nb; k += bd) sm[k] = 0;
    __syncthreads();
    const int t0 = tptr[j], cnt = tptr[j + 1] - t0;
    const double* sinv = Sinv + (size_t)j * (L + 2);
    for (int base = 0; base < cnt; base += bd) {
        int h = base + tid;
        double dx = b.w, dy = 0, dz = 0, wr = 0, we = 0;
        if (h < cnt) {
            int p = tp[t0 + h];
            int i = p / N, n = p % N;
            double4 a = sph[i], s = leb[n];
            dx = a.x + a.w * s.x - b.x;
            dy = a.y + a.w * s.y - b.y;
            dz = a.z + a.w * s.z - b.z;
            double w = tw[t0 + h];
            wr = w * zr[p];
            we = w * ze[p];
        }
        double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
        radial<double>(0, L, rho, b.w, kappa, nullptr, rr + tid, nullptr, bd);
        radial<double>(1, L, rho, b.w, kappa, sinv, ri + tid, nullptr, bd);
        ylm_stream<double>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, double yv) {
            double vR = warp_sum(wr * rr[tid + l * bd] * yv);
            double vE = warp_sum(we * ri[tid + l * bd] * yv);
            if (lane == 0) {
                accR[warp * nb + idx] += vR;
                accE[warp * nb + idx] += vE;
            }
        });
    }
    __syncthreads();
    for (int idx = tid; idx < nb; idx += bd) {
        double sr = 0, se = 0;
        for (int w = 0; w < nw; ++w) {
            sr += accR[w * nb + idx];
            se += accE[w * nb + idx];
        }
        size_t o = (size_t)j * nb + idx;
        y[o] = x[o] - sr;
        y[(size_t)M * nb + o] = x[(size_t)M * nb + o] - se;
    }
}

// ---------------------------------------------------------------- dense coupling (L_C)

// mu_j = C_ik^j * P chi_j y_j with y_j = eps1/eps2 (l/r_j) X_r,j - i_l'/i_l X_e,j, for j in src.
__global__ void k_source_mu(int M, int N, int nb, int L, double e12, const int* __restrict__ src,
                            const double4* __restrict__ sph, const double* __restrict__ di,
                            const double* __restrict__ cik, const int* __restrict__ ext_ptr,
                            const int* __restrict__ ext_p, const double4* __restrict__ ext_x,
                            const double4* __restrict__ leb, const double* __restrict__ Y,
                            const double* __restrict__ x, double* __restrict__ mu) {
    extern __shared__ double sm[];
    const int j = src[blockIdx.x];
    double* yv = sm;
    double* gv = yv + nb;
    int* gn = (int*)(gv + N);
    const double rj = sph[j].w;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        int l = (int)sqrtf((float)idx + 0.5f);
        yv[idx] = e12 * (double)l / rj * x[(size_t)j * nb + idx] -
                  di[(size_t)j * (L + 1) + l] * x[(size_t)(M + j) * nb + idx];
    }
    __syncthreads();
    const int t0 = ext_ptr[j], cnt = ext_ptr[j + 1] - t0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, n = ext_p[t] % N;
        double v = 0;
        for (int idx = 0; idx < nb; ++idx) v += Y[(size_t)n * nb + idx] * yv[idx];
        gn[k] = n;
        gv[k] = leb[n].w * ext_x[t].w * v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        double a = 0;
        for (int k = 0; k < cnt; ++k) a += Y[(size_t)gn[k] * nb + idx] * gv[k];
        int l = (int)sqrtf((float)idx + 0.5f);
        mu[(size_t)j * nb + idx] = cik[(size_t)j * (L + 1) + l] * a;
    }
}

// phi(x_t) = sum_{j in src} sum_lm mu_j,lm k_l^j(x_t) Y_lm^j(x_t) at every external point t
// (the potential in Eqs. definition_of_Q_matrix / defintion_of_S).  Direct summation: one
// thread per target, source tiles staged in shared memory.
#define YK_TS 8
__global__ void k_yukawa_pot(int E, const double4* __restrict__ ext_x, int n_src, const int* __restrict__ src,
                             const double4* __restrict__ sph, const double* __restrict__ mu,
                             const double* __restrict__ Khinv, int nb, int L, double kappa, YTab yt,
                             double* __restrict__ phi) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    double4* sp = (double4*)sm;
    double* smu = (double*)(sp + YK_TS);
    double* skh = smu + YK_TS * nb;
    double* rad = skh + YK_TS * (L + 2);
    const int t = blockIdx.x * bd + tid;
    const bool valid = t < E;
    const double4 xt = valid ? ext_x[t] : make_double4(0, 0, 0, 0);
    double acc = 0;
    for (int base = 0; base < n_src; base += YK_TS) {
        int ns = min(YK_TS, n_src - base);
        __syncthreads();
        for (int k = tid; k < ns * nb; k += bd) {
            int s = k / nb, idx = k % nb;
            smu[k] = mu[(size_t)src[base + s] * nb + idx];
        }
        for (int k = tid; k < ns * (L + 2); k += bd) {
            int s = k / (L + 2), l = k % (L + 2);
            skh[k] = Khinv[(size_t)src[base + s] * (L + 2) + l];
        }
        if (tid < ns) sp[tid] = sph[src[base + tid]];
        __syncthreads();
        for (int s = 0; s < ns; ++s) {
            double4 b = sp[s];
            double dx = valid ? xt.x - b.x : b.w, dy = valid ? xt.y - b.y : 0, dz = valid ? xt.z - b.z : 0;
            double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
            radial<double>(2, L, rho, b.w, kappa, skh + s * (L + 2), rad + tid, nullptr, bd);
            const double* m = smu + s * nb;
            double v = 0;
            ylm_stream<double>(L, dx * inv, dy * inv, dz * inv, yt,
                               [&](int idx, int l, double yv) { v += m[idx] * rad[tid + l * bd] * yv; });
            acc += v;
        }
    }
    if (valid) phi[t] = acc;
}

// nu_j = sum_t c_t k_l^j(x_t) Y_lm^j(x_t) (transpose of k_yukawa_pot), one CTA per source j.
__global__ void k_yukawa_adj(int E, const double4* __restrict__ ext_x, const double* __restrict__ cext,
                             const int* __restrict__ src, const double4* __restrict__ sph,
                             const double* __restrict__ Khinv, int nb, int L, double kappa, YTab yt,
                             double* __restrict__ nu) {
    extern __shared__ double sm[];
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    double* acc = sm;
    double* kh = acc + nw * nb;
    double* rad = kh + (L + 2);
    const int j = src[blockIdx.x];
    const double4 b = sph[j];
    for (int k = tid; k < nw * nb; k += bd) acc[k] = 0;
    for (int k = tid; k < L + 2; k += bd) kh[k] = Khinv[(size_t)j * (L + 2) + k];
    __syncthreads();
    for (int base = 0; base < E; base += bd) {
        int t = base + tid;
        double dx = b.w, dy = 0, dz = 0, c = 0;
        if (t < E) {
            double4 xt = ext_x[t];
            dx = xt.x - b.x;
            dy = xt.y - b.y;
            dz = xt.z - b.z;
            c = cext[t];
        }
        double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
        radial<double>(2, L, rho, b.w, kappa, kh, rad + tid, nullptr, bd);
        ylm_stream<double>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, double yv) {
            double v = warp_sum(c * rad[tid + l * bd] * yv);
            if (lane == 0) acc[warp * nb + idx] += v;
        });
    }
    __syncthreads();
    for (int idx = tid; idx < nb; idx += bd) {
        double s = 0;
        for (int w = 0; w < nw; ++w) s += acc[w * nb + idx];
        nu[(size_t)j * nb + idx] = s;
    }
}

// c_t = w_n chi_t sum_lm Y_lm(s_n) (x_r + x_e)_{i lm} at the external points of sphere i.
__global__ void k_ext_weights(int M, int N, int nb, const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                              const double4* __restrict__ ext_x, const double4* __restrict__ leb,
                              const double* __restrict__ Y, const double* __restrict__ x, double* __restrict__ cext) {
    extern __shared__ double sm[];
    const int i = blockIdx.x;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x)
        sm[idx] = x[(size_t)i * nb + idx] + x[(size_t)(M + i) * nb + idx];
    __syncthreads();
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, n = ext_p[t] % N;
        double v = 0;
        for (int idx = 0; idx < nb; ++idx) v += Y[(size_t)n * nb + idx] * sm[idx];
        cext[t] = leb[n].w * ext_x[t].w * v;
    }
}

// y_r,j += eps1/eps2 (l/r_j) z_j, y_e,j += -i_l'/i_l z_j with z_j = P chi_j (C_ik nu_j).
__global__ void k_ct_finish(int M, int N, int nb, int L, double e12, const int* __restrict__ src,
                            const double4* __restrict__ sph, const double* __restrict__ di,
                            const double* __restrict__ cik, const int* __restrict__ ext_ptr,
                            const int* __restrict__ ext_p, const double4* __restrict__ ext_x,
                            const double4* __restrict__ leb, const double* __restrict__ Y,
                            const double* __restrict__ nu, double* __restrict__ y) {
    extern __shared__ double sm[];
    const int j = src[blockIdx.x];
    double* u = sm;
    double* gv = u + nb;
    int* gn = (int*)(gv + N);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        int l = (int)sqrtf((float)idx + 0.5f);
        u[idx] = cik[(size_t)j * (L + 1) + l] * nu[(size_t)j * nb + idx];
    }
    __syncthreads();
    const int t0 = ext_ptr[j], cnt = ext_ptr[j + 1] - t0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, n = ext_p[t] % N;
        double v = 0;
        for (int idx = 0; idx < nb; ++idx) v += Y[(size_t)n * nb + idx] * u[idx];
        gn[k] = n;
        gv[k] = leb[n].w * ext_x[t].w * v;
    }
    __syncthreads();
    const double rj = sph[j].w;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        double a = 0;
        for (int k = 0; k < cnt; ++k) a += Y[(size_t)gn[k] * nb + idx] * gv[k];
        int l = (int)sqrtf((float)idx + 0.5f);
        y[(size_t)j * nb + idx] += e12 * (double)l / rj * a;
        y[(size_t)(M + j) * nb + idx] += -di[(size_t)j * (L + 1) + l] * a;
    }
}

// ---------------------------------------------------------------- host wrappers

static ddlpb_status set_smem(ddlpb_ctx* c, const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) DDLPB_CK(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return DDLPB_OK;
}

ddlpb_status op_synthesis(ddlpb_ctx* c, const double* coef, int rows, double* grid, bool weighted) {
    if (rows <= 0) return DDLPB_OK;
    k_synthesis<<<rows, BLK, sizeof(double) * c->nb, c->stream>>>(c->N, c->nb, c->YT, c->leb, coef, grid, weighted);
    DDLPB_LAUNCHED(c, "synthesis");
    return DDLPB_OK;
}

ddlpb_status op_masked_analysis(ddlpb_ctx* c, const double* val_ext, double scale, const double* cik_scale,
                                double* out, int out_stride, int accumulate) {
    size_t smem = (sizeof(double) + sizeof(int)) * c->N;
    k_masked_analysis<<<c->M, BLK, smem, c->stream>>>(c->N, c->nb, c->lmax, c->ext_ptr, c->ext_p, c->ext_x, c->leb,
                                                      c->Y, val_ext, scale, cik_scale, out, out_stride, accumulate);
    DDLPB_LAUNCHED(c, "masked_analysis");
    return DDLPB_OK;
}

ddlpb_status op_apply_AB(ddlpb_ctx* c, const double* x, double* y, bool transpose, double* gridR, double* gridE) {
    const int L = c->lmax;
    if (!transpose) {
        size_t smem = sizeof(double) * (2 * (size_t)c->N + 2 * (size_t)(L + 1) * BLK);
        DDLPB_TRY(set_smem(c, (const void*)k_ab_apply, smem));
        k_ab_apply<<<c->M, BLK, smem, c->stream>>>(c->M, c->N, c->nb, L, c->kappa, c->sph, c->leb, c->yt, c->hit_ptr,
                                                   c->hit_j, c->hit_w, c->Sinv, c->Y, x, y, gridR, gridE);
        DDLPB_LAUNCHED(c, "ab_apply");
        return DDLPB_OK;
    }
    // weighted syntheses of both blocks into gridA (X_r rows) and gridB (X_e rows)
    DDLPB_TRY(op_synthesis(c, x, c->M, c->gridA, true));
    DDLPB_TRY(op_synthesis(c, x + (size_t)c->M * c->nb, c->M, c->gridB, true));
    size_t smem = sizeof(double) * (2 * (size_t)(BLK / 32) * c->nb + 2 * (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_ab_transpose, smem));
    k_ab_transpose<<<c->M, BLK, smem, c->stream>>>(c->M, c->N, c->nb, L, c->kappa, c->sph, c->leb, c->yt, c->thit_ptr,
                                                   c->thit_p, c->thit_w, c->Sinv, c->gridA, c->gridB, x, y);
    DDLPB_LAUNCHED(c, "ab_transpose");
    return DDLPB_OK;
}

ddlpb_status op_source_multipoles(ddlpb_ctx* c, const double* x, double* mu) {
    if (c->n_src == 0) return DDLPB_OK;
    size_t smem = sizeof(double) * (c->nb + c->N) + sizeof(int) * c->N;
    k_source_mu<<<c->n_src, BLK, smem, c->stream>>>(c->M, c->N, c->nb, c->lmax, c->eps1 / c->eps2, c->src, c->sph,
                                                    c->di, c->cik, c->ext_ptr, c->ext_p, c->ext_x, c->leb, c->Y, x,
                                                    mu);
    DDLPB_LAUNCHED(c, "source_mu");
    return DDLPB_OK;
}

ddlpb_status op_yukawa_potential(ddlpb_ctx* c, const double* mu, double* phi_ext) {
    if (c->E == 0) return DDLPB_OK;
    const int L = c->lmax;
    size_t smem = sizeof(double4) * YK_TS + sizeof(double) * (YK_TS * (size_t)c->nb + YK_TS * (size_t)(L + 2) +
                                                              (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_yukawa_pot, smem));
    k_yukawa_pot<<<ceil_div(c->E, BLK), BLK, smem, c->stream>>>(c->E, c->ext_x, c->n_src, c->src, c->sph, mu,
                                                                c->Khinv, c->nb, L, c->kappa, c->yt, phi_ext);
    DDLPB_LAUNCHED(c, "yukawa_pot");
    return DDLPB_OK;
}

ddlpb_status op_yukawa_adjoint(ddlpb_ctx* c, const double* c_ext, double* nu) {
    if (c->n_src == 0) return DDLPB_OK;
    const int L = c->lmax;
    size_t smem = sizeof(double) * ((size_t)(BLK / 32) * c->nb + (L + 2) + (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_yukawa_adj, smem));
    k_yukawa_adj<<<c->n_src, BLK, smem, c->stream>>>(c->E, c->ext_x, c_ext, c->src, c->sph, c->Khinv, c->nb, L,
                                                     c->kappa, c->yt, nu);
    DDLPB_LAUNCHED(c, "yukawa_adj");
    return DDLPB_OK;
}

ddlpb_status op_ext_weights(ddlpb_ctx* c, const double* x, double* cext) {
    k_ext_weights<<<c->M, BLK, sizeof(double) * c->nb, c->stream>>>(c->M, c->N, c->nb, c->ext_ptr, c->ext_p, c->ext_x,
                                                                    c->leb, c->Y, x, cext);
    DDLPB_LAUNCHED(c, "ext_weights");
    return DDLPB_OK;
}

// y (+)= [K y ; K y] (forward) or y (+)= [D1 K^T (x_r + x_e) ; D2 K^T (x_r + x_e)] (transpose)
ddlpb_status op_apply_C(ddlpb_ctx* c, const double* x, double* y, bool transpose, bool accumulate) {
    const size_t half = (size_t)c->M * c->nb;
    if (!transpose) {
        DDLPB_TRY(op_source_multipoles(c, x, c->mu));
        DDLPB_TRY(op_yukawa_potential(c, c->mu, c->extA));
        DDLPB_TRY(op_masked_analysis(c, c->extA, 1.0, nullptr, y, c->nb, accumulate ? 1 : 0));
        DDLPB_TRY(op_masked_analysis(c, c->extA, 1.0, nullptr, y + half, c->nb, accumulate ? 1 : 0));
        return DDLPB_OK;
    }
    if (!accumulate) DDLPB_CK(c, cudaMemsetAsync(y, 0, sizeof(double) * 2 * half, c->stream));
    if (c->n_src == 0) return DDLPB_OK;
    DDLPB_TRY(op_ext_weights(c, x, c->extA));
    DDLPB_TRY(op_yukawa_adjoint(c, c->extA, c->mu));
    size_t smem = sizeof(double) * (c->nb + c->N) + sizeof(int) * c->N;
    k_ct_finish<<<c->n_src, BLK, smem, c->stream>>>(c->M, c->N, c->nb, c->lmax, c->eps1 / c->eps2, c->src, c->sph,
                                                    c->di, c->cik, c->ext_ptr, c->ext_p, c->ext_x, c->leb, c->Y, c->mu,
                                                    y);
    DDLPB_LAUNCHED(c, "ct_finish");
    return DDLPB_OK;
}

ddlpb_status op_apply_L(ddlpb_ctx* c, const double* x, double* y, bool transpose) {
    DDLPB_TRY(op_apply_AB(c, x, y, transpose, nullptr, nullptr));
    DDLPB_TRY(op_apply_C(c, x, y, transpose, true));
    return DDLPB_OK;
}
