// solve.cu -- restarted GMRES for L X = g and L* X_adj = Q, the energy, and the C ABI.
//
// The paper solves its system with DIIS preconditioned by L_AB (Sec. 4); any Krylov
// method that reaches the same discrete solution X gives the same energy and forces,
// and GMRES on the full operator needs no inner solves.  The stopping rule is the
// relative FP64 residual ||b - L x|| / ||b|| <= tol.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

#define RBLK 256
#define RGRID 592   // 4 x 148 resident CTAs

// partial[k * G + g] = sum over the g-th grid stride of V_k . w
__global__ void k_multidot(long long n, int kk, const double* __restrict__ V, const double* __restrict__ w,
                           double* __restrict__ partial) {
    __shared__ double red[RBLK / 32];
    const int k = blockIdx.y;
    const double* v = V + (size_t)k * n;
    double s = 0;
    for (long long i = (long long)blockIdx.x * RBLK + threadIdx.x; i < n; i += (long long)gridDim.x * RBLK)
        s += v[i] * w[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < RBLK / 32; ++q) t += red[q];
        partial[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
}

// out[k] = (add ? out[k] : 0) + sum_g partial[k * G + g]; optional sqrt
__global__ void k_reduce(int G, const double* __restrict__ partial, double* __restrict__ out, int add, int take_sqrt) {
    __shared__ double red[RBLK / 32];
    const int k = blockIdx.x;
    double s = 0;
    for (int g = threadIdx.x; g < G; g += RBLK) s += partial[(size_t)k * G + g];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < RBLK / 32; ++q) t += red[q];
        if (take_sqrt) t = sqrt(t);
        out[k] = add ? out[k] + t : t;
    }
}

// w -= sum_k V_k h[k]
__global__ void k_sub_combination(long long n, int kk, const double* __restrict__ V, const double* __restrict__ h,
                                  double* __restrict__ w) {
    __shared__ double sh[128];
    for (int k = threadIdx.x; k < kk; k += blockDim.x) sh[k] = h[k];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k < kk; ++k) s -= V[(size_t)k * n + i] * sh[k];
        w[i] = s;
    }
}

// x += sum_k V_k y[k]
__global__ void k_add_combination(long long n, int kk, const double* __restrict__ V, const double* __restrict__ y,
                                  double* __restrict__ x) {
    __shared__ double sh[128];
    for (int k = threadIdx.x; k < kk; k += blockDim.x) sh[k] = y[k];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int k = 0; k < kk; ++k) s += V[(size_t)k * n + i] * sh[k];
        x[i] = s;
    }
}

// out = a * x (+ b * y)
__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// out = x / s[0]
__global__ void k_scale_by(long long n, const double* __restrict__ x, const double* __restrict__ s,
                           double* __restrict__ out) {
    double inv = 1.0 / s[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = x[i] * inv;
}

__global__ void k_add_vec(int kk, const double* __restrict__ a, double* __restrict__ b) {
    int k = threadIdx.x;
    if (k < kk) b[k] += a[k];
}

// E = 1/2 sum_j q_j Y_00 X_r[j, 00] (Eq. energy_computation with Q_{j00} = q_j Y_00)
__global__ void k_energy(int M, int nb, const double* __restrict__ q, const double* __restrict__ X,
                         double* __restrict__ e) {
    __shared__ double red[RBLK / 32];
    double s = 0;
    for (int j = threadIdx.x; j < M; j += RBLK) s += q[j] * X[(size_t)j * nb];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < RBLK / 32; ++k) t += red[k];
        e[0] = 0.5 * 0.28209479177387814 * t;
    }
}

// ---------------------------------------------------------------- host side

static ddlpb_status dots(ddlpb_ctx* c, int kk, const double* V, const double* w, double* out, bool add, bool sq) {
    dim3 grid(RGRID, kk);
    k_multidot<<<grid, RBLK, 0, c->stream>>>(c->nvec, kk, V, w, c->gm_red);
    DDLPB_LAUNCHED(c, "multidot");
    k_reduce<<<kk, RBLK, 0, c->stream>>>(RGRID, c->gm_red, out, add ? 1 : 0, sq ? 1 : 0);
    DDLPB_LAUNCHED(c, "reduce");
    return DDLPB_OK;
}

static ddlpb_status ensure_krylov(ddlpb_ctx* c) {
    if (c->gm_V) return DDLPB_OK;
    const int m = c->opt.gmres_restart;
    DDLPB_TRY(ctx_alloc(c, &c->gm_V, (size_t)(m + 1) * c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->gm_w, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->gm_r, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->gm_red, (size_t)RGRID * (m + 2)));
    DDLPB_TRY(ctx_alloc(c, &c->gm_h, 4 * (size_t)(m + 2)));
    DDLPB_CK(c, cudaMallocHost((void**)&c->h_pinned, sizeof(double) * 4 * (m + 2)));
    return DDLPB_OK;
}

// GMRES(m) with classical Gram-Schmidt and one re-orthogonalisation pass.
ddlpb_status solve_system(ddlpb_ctx* c, bool transpose, const double* b, double* x, int* iters, double* resid) {
    DDLPB_TRY(ensure_krylov(c));
    const long long n = c->nvec;
    const int m = c->opt.gmres_restart;
    cudaStream_t st = c->stream;
    double* V = c->gm_V;
    double* w = c->gm_w;
    double* h1 = c->gm_h;            // [m+2]
    double* h2 = c->gm_h + (m + 2);  // [m+2]
    double* nrm = c->gm_h + 2 * (m + 2);
    double* hp = c->h_pinned;
    const int VG = 1184, VB = 256;

    // ||b||
    DDLPB_TRY(dots(c, 1, b, b, nrm, false, true));
    DDLPB_CK(c, cudaMemcpyAsync(hp, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    DDLPB_CK(c, cudaStreamSynchronize(st));
    const double bnorm = hp[0];
    *iters = 0;
    if (!(bnorm > 0.0)) {
        DDLPB_CK(c, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        *resid = 0.0;
        DDLPB_CK(c, cudaStreamSynchronize(st));
        return bnorm == 0.0 ? DDLPB_OK : DDLPB_EINVAL;
    }
    const double tol = c->opt.tol;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1), yv(m);
    int total = 0;
    double rel = 1.0;
    for (;;) {
        // r = b - L x ; beta = ||r||
        DDLPB_TRY(op_apply_L(c, x, c->gm_r, transpose));
        k_axpby<<<VG, VB, 0, st>>>(n, 1.0, b, -1.0, c->gm_r, c->gm_r);
        DDLPB_LAUNCHED(c, "axpby");
        DDLPB_TRY(dots(c, 1, c->gm_r, c->gm_r, nrm, false, true));
        DDLPB_CK(c, cudaMemcpyAsync(hp, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
        DDLPB_CK(c, cudaStreamSynchronize(st));
        const double beta = hp[0];
        rel = beta / bnorm;
        if (!std::isfinite(beta)) {
            c->err = "non-finite residual in GMRES";
            *resid = rel;
            return DDLPB_ENOTCONV;
        }
        if (rel <= tol) break;
        if (total >= c->opt.max_iter) {
            *iters = total;
            *resid = rel;
            c->err = "GMRES reached max_iter";
            return DDLPB_ENOTCONV;
        }
        k_scale_by<<<VG, VB, 0, st>>>(n, c->gm_r, nrm, V);
        DDLPB_LAUNCHED(c, "scale");
        std::fill(gvec.begin(), gvec.end(), 0.0);
        gvec[0] = beta;
        int k = 0;
        for (; k < m && total < c->opt.max_iter; ++k) {
            ++total;
            double* vk = V + (size_t)k * n;
            DDLPB_TRY(op_apply_L(c, vk, w, transpose));
            // CGS2
            DDLPB_TRY(dots(c, k + 1, V, w, h1, false, false));
            k_sub_combination<<<VG, VB, 0, st>>>(n, k + 1, V, h1, w);
            DDLPB_LAUNCHED(c, "sub_comb");
            DDLPB_TRY(dots(c, k + 1, V, w, h2, false, false));
            k_sub_combination<<<VG, VB, 0, st>>>(n, k + 1, V, h2, w);
            DDLPB_LAUNCHED(c, "sub_comb2");
            k_add_vec<<<1, 128, 0, st>>>(k + 1, h2, h1);
            DDLPB_LAUNCHED(c, "add_vec");
            DDLPB_TRY(dots(c, 1, w, w, nrm, false, true));
            k_scale_by<<<VG, VB, 0, st>>>(n, w, nrm, V + (size_t)(k + 1) * n);
            DDLPB_LAUNCHED(c, "scale2");
            DDLPB_CK(c, cudaMemcpyAsync(hp, h1, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
            DDLPB_CK(c, cudaMemcpyAsync(hp + (m + 2), nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
            DDLPB_CK(c, cudaStreamSynchronize(st));
            for (int q = 0; q <= k; ++q) H[(size_t)q * m + k] = hp[q];
            double hk1 = hp[m + 2];
            // apply previous rotations
            for (int q = 0; q < k; ++q) {
                double a = H[(size_t)q * m + k], bb = H[(size_t)(q + 1) * m + k];
                H[(size_t)q * m + k] = cs[q] * a + sn[q] * bb;
                H[(size_t)(q + 1) * m + k] = -sn[q] * a + cs[q] * bb;
            }
            double a = H[(size_t)k * m + k];
            double den = std::sqrt(a * a + hk1 * hk1);
            cs[k] = den > 0 ? a / den : 1.0;
            sn[k] = den > 0 ? hk1 / den : 0.0;
            H[(size_t)k * m + k] = den;
            gvec[k + 1] = -sn[k] * gvec[k];
            gvec[k] = cs[k] * gvec[k];
            double est = std::fabs(gvec[k + 1]) / bnorm;
            if (!std::isfinite(est)) {
                c->err = "non-finite Krylov residual";
                return DDLPB_ENOTCONV;
            }
            if (est <= 0.5 * tol || hk1 == 0.0) {
                ++k;
                break;
            }
        }
        // back substitution, x += V y
        for (int q = k - 1; q >= 0; --q) {
            double s = gvec[q];
            for (int r = q + 1; r < k; ++r) s -= H[(size_t)q * m + r] * yv[r];
            yv[q] = s / H[(size_t)q * m + q];
        }
        DDLPB_CK(c, cudaMemcpyAsync(h2, yv.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        k_add_combination<<<VG, VB, 0, st>>>(n, k, V, h2, x);
        DDLPB_LAUNCHED(c, "add_comb");
        DDLPB_CK(c, cudaStreamSynchronize(st));
    }
    *iters = total;
    *resid = rel;
    return DDLPB_OK;
}

// ---------------------------------------------------------------- C ABI

static thread_local std::string g_setup_err;

extern "C" void ddlpb_default_options(ddlpb_options* o) {
    if (!o) return;
    o->eta = 0.1;
    o->tol = 1e-8;
    o->max_iter = 500;
    o->gmres_restart = 40;
    o->precision = DDLPB_FP64;
    o->fmm_order = 0;
    o->cuda_stream = nullptr;
}

static ddlpb_status setup_common(int n, const double* centres, const double* radii, const double* charges,
                                 double eps_solvent, double kappa, int lmax, int n_lebedev, ddlpb_surface surface,
                                 const ddlpb_options* opt, ddlpb_ctx** out, bool device) {
    g_setup_err.clear();
    if (!out) {
        g_setup_err = "out is NULL";
        return DDLPB_EINVAL;
    }
    *out = nullptr;
    auto fail = [&](const std::string& m) {
        g_setup_err = m;
        return DDLPB_EINVAL;
    };
    if (n < 1) return fail("n must be >= 1");
    if (!centres || !radii || !charges) return fail("NULL input array");
    if (!(eps_solvent > 1.0) || !std::isfinite(eps_solvent)) return fail("eps_solvent must be > 1");
    if (!(kappa > 0.0) || !std::isfinite(kappa)) return fail("kappa must be > 0");
    if (lmax < 0 || lmax > DDLPB_LMAX_MAX) return fail("lmax out of range [0, 16]");
    if (surface != DDLPB_VDW && surface != DDLPB_SAS) return fail("unknown surface");
    ddlpb_options o;
    ddlpb_default_options(&o);
    if (opt) o = *opt;
    if (!(o.eta > 0.0 && o.eta <= 1.0)) return fail("eta must be in (0, 1]");
    if (!(o.tol > 0.0)) return fail("tol must be > 0");
    if (o.max_iter < 1) return fail("max_iter must be >= 1");
    if (o.gmres_restart < 1 || o.gmres_restart > 120) return fail("gmres_restart must be in [1, 120]");
    if (o.precision != DDLPB_FP64 && o.precision != DDLPB_MIXED) return fail("unknown precision");
    if (o.fmm_order != 0) return fail("fmm_order must be 0 (direct summation)");
    ddlpb_ctx* c = new ddlpb_ctx();
    c->M = n;
    c->lmax = lmax;
    c->nb = (lmax + 1) * (lmax + 1);
    c->N = n_lebedev;
    c->eps2 = eps_solvent;
    c->kappa = kappa;
    c->eta = o.eta;
    c->opt = o;
    c->stream = (cudaStream_t)o.cuda_stream;
    cudaGetDevice(&c->device);
    ddlpb_status s = ddlpb_internal_setup(c, centres, radii, charges, device, (int)surface);
    if (s != DDLPB_OK) {
        g_setup_err = c->err;
        ddlpb_free(c);
        return s;
    }
    *out = c;
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_setup(int n, const double* centres, const double* radii, const double* charges,
                                    double eps_solvent, double kappa, int lmax, int n_lebedev, ddlpb_surface surface,
                                    const ddlpb_options* opt, ddlpb_ctx** out) {
    return setup_common(n, centres, radii, charges, eps_solvent, kappa, lmax, n_lebedev, surface, opt, out, false);
}

extern "C" ddlpb_status ddlpb_setup_device(int n, const double* centres, const double* radii, const double* charges,
                                           double eps_solvent, double kappa, int lmax, int n_lebedev,
                                           ddlpb_surface surface, const ddlpb_options* opt, ddlpb_ctx** out) {
    return setup_common(n, centres, radii, charges, eps_solvent, kappa, lmax, n_lebedev, surface, opt, out, true);
}

extern "C" ddlpb_status ddlpb_solve(ddlpb_ctx* c) {
    if (!c) return DDLPB_EINVAL;
    c->err.clear();
    int it = 0;
    double res = 0;
    ddlpb_status s = solve_system(c, false, c->g, c->X, &it, &res);
    c->info.solve_iterations = it;
    c->info.solve_residual = res;
    c->solved = (s == DDLPB_OK);
    c->adjoint_done = false;
    return s;
}

extern "C" ddlpb_status ddlpb_adjoint(ddlpb_ctx* c) {
    if (!c) return DDLPB_EINVAL;
    c->err.clear();
    if (!c->solved) {
        c->err = "ddlpb_adjoint before a successful ddlpb_solve";
        return DDLPB_EORDER;
    }
    int it = 0;
    double res = 0;
    ddlpb_status s = solve_system(c, true, c->Qv, c->Xa, &it, &res);
    c->info.adjoint_iterations = it;
    c->info.adjoint_residual = res;
    c->adjoint_done = (s == DDLPB_OK);
    return s;
}

extern "C" ddlpb_status ddlpb_energy_device(ddlpb_ctx* c, double* e) {
    if (!c || !e) return DDLPB_EINVAL;
    c->err.clear();
    if (!c->solved) {
        c->err = "ddlpb_energy before a successful ddlpb_solve";
        return DDLPB_EORDER;
    }
    k_energy<<<1, RBLK, 0, c->stream>>>(c->M, c->nb, c->q, c->X, e);
    DDLPB_LAUNCHED(c, "energy");
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_energy(ddlpb_ctx* c, double* e) {
    if (!c || !e) return DDLPB_EINVAL;
    c->err.clear();
    if (!c->solved) {
        c->err = "ddlpb_energy before a successful ddlpb_solve";
        return DDLPB_EORDER;
    }
    k_energy<<<1, RBLK, 0, c->stream>>>(c->M, c->nb, c->q, c->X, c->gm_h ? c->gm_h + 3 * (c->opt.gmres_restart + 2) : c->tmpv);
    DDLPB_LAUNCHED(c, "energy");
    const double* src = c->gm_h ? c->gm_h + 3 * (c->opt.gmres_restart + 2) : c->tmpv;
    DDLPB_CK(c, cudaMemcpyAsync(e, src, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_forces_device(ddlpb_ctx* c, double* f) {
    if (!c || !f) return DDLPB_EINVAL;
    c->err.clear();
    if (!c->adjoint_done) {
        c->err = "ddlpb_forces before a successful ddlpb_adjoint";
        return DDLPB_EORDER;
    }
    DDLPB_TRY(compute_forces(c, f));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_forces(ddlpb_ctx* c, double* f) {
    if (!c || !f) return DDLPB_EINVAL;
    c->err.clear();
    if (!c->adjoint_done) {
        c->err = "ddlpb_forces before a successful ddlpb_adjoint";
        return DDLPB_EORDER;
    }
    if (!c->force_acc) DDLPB_TRY(ctx_alloc(c, &c->force_acc, 3 * (size_t)c->M));
    DDLPB_TRY(compute_forces(c, c->force_acc));
    DDLPB_CK(c, cudaMemcpyAsync(f, c->force_acc, sizeof(double) * 3 * c->M, cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_apply_device(ddlpb_ctx* c, int op, const double* x, double* y) {
    if (!c || !x || !y || op < 0 || op > 5) return DDLPB_EINVAL;
    c->err.clear();
    switch (op) {
        case 0: DDLPB_TRY(op_apply_L(c, x, y, false)); break;
        case 1: DDLPB_TRY(op_apply_L(c, x, y, true)); break;
        case 2: DDLPB_TRY(op_apply_AB(c, x, y, false, nullptr, nullptr)); break;
        case 3: DDLPB_TRY(op_apply_AB(c, x, y, true, nullptr, nullptr)); break;
        case 4: DDLPB_TRY(op_apply_C(c, x, y, false, false)); break;
        case 5: DDLPB_TRY(op_apply_C(c, x, y, true, false)); break;
    }
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_get_vector_device(ddlpb_ctx* c, int which, double* y) {
    if (!c || !y || which < 0 || which > 2) return DDLPB_EINVAL;
    const double* s = which == 0 ? c->g : (which == 1 ? c->X : c->Xa);
    DDLPB_CK(c, cudaMemcpyAsync(y, s, sizeof(double) * c->nvec, cudaMemcpyDeviceToDevice, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_get_info(const ddlpb_ctx* c, ddlpb_info* info) {
    if (!c || !info) return DDLPB_EINVAL;
    *info = c->info;
    return DDLPB_OK;
}

extern "C" const char* ddlpb_last_error(const ddlpb_ctx* c) { return c ? c->err.c_str() : ""; }

extern "C" const char* ddlpb_last_setup_error(void) { return g_setup_err.c_str(); }

extern "C" void ddlpb_free(ddlpb_ctx* c) {
    if (!c) return;
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
}
