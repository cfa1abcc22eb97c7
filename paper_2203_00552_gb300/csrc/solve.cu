// solve.cu -- Krylov solves of L X = g and L* X_adj = Q, the energy, and the C ABI.
//
// The paper solves its system with DIIS preconditioned by L_AB = diag(A, B), whose
// inverse is applied by inner (micro) iterations (Sec. 4).  Here the outer method is
// flexible GMRES, right-preconditioned by the same L_AB, whose inverse is applied by
// an inner GMRES on the sparse blocks; any method that reaches the same discrete
// solution X gives the same energy and forces.  The stopping rule is the relative
// FP64 residual ||b - L x|| / ||b|| <= tol.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cstdio>
#include <cstdlib>

#include "common.cuh"

// DDLPB_TRACE=1 in the environment prints the restart residuals of every Krylov solve.
static bool trace_on() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("DDLPB_TRACE");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

#define RBLK 256
#define RGRID 608   // 4 x 152 SMs
#define VG 1184
#define VB 256

// partial[k * G + g] = sum over the g-th grid stride of V_k . w (accumulated in FP64)
// Partial dot products <V_k, w>, k < kk: block b owns one contiguous slice of the rows for
// all k; its warps take (k, sub-slice) tasks (sub-slices when kk is below the warp count),
// lanes sum a few products in the vectors' precision, the lane sums are added in FP64.
template <typename T>
__global__ void __launch_bounds__(RBLK) k_multidot(long long n, int kk, const T* __restrict__ V,
                                                   const T* __restrict__ w, double* __restrict__ partial) {
    extern __shared__ double sacc[];   // [kk]
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * per, i1 = i0 + per < n ? i0 + per : n;
    for (int k = threadIdx.x; k < kk; k += RBLK) sacc[k] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = RBLK / 32;
    const int P = kk < nw ? nw / kk : 1;
    const long long len = i1 > i0 ? i1 - i0 : 0, plen = (len + P - 1) / P;
    for (int t = warp; t < kk * P; t += nw) {
        const int k = t / P, part = t % P;
        const long long a = i0 + part * plen, b = a + plen < i1 ? a + plen : i1;
        const T* v = V + (size_t)k * n;
        T s = 0;
#pragma unroll 4
        for (long long i = a + lane; i < b; i += 32) s += v[i] * w[i];
        const double d = warp_sum((double)s);
        if (lane == 0) atomicAdd(&sacc[k], d);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kk; k += RBLK) partial[(size_t)k * gridDim.x + blockIdx.x] = sacc[k];
}
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

// w -= sum_k V_k h[k]  (dynamic shared memory: kk coefficients)
template <typename T>
__global__ void k_sub_combination(long long n, int kk, const T* __restrict__ V, const double* __restrict__ h,
                                  T* __restrict__ w) {
    extern __shared__ unsigned char shraw[];
    T* sh = (T*)shraw;
    for (int k = threadIdx.x; k < kk; k += blockDim.x) sh[k] = (T)h[k];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T s = w[i];
        for (int k = 0; k < kk; ++k) s -= V[(size_t)k * n + i] * sh[k];
        w[i] = s;
    }
}

// x += sum_k V_k y[k]  (dynamic shared memory: kk coefficients)
template <typename T>
__global__ void k_add_combination(long long n, int kk, const T* __restrict__ V, const double* __restrict__ y,
                                  T* __restrict__ x) {
    extern __shared__ unsigned char shraw[];
    T* sh = (T*)shraw;
    for (int k = threadIdx.x; k < kk; k += blockDim.x) sh[k] = (T)y[k];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T s = x[i];
        for (int k = 0; k < kk; ++k) s += V[(size_t)k * n + i] * sh[k];
        x[i] = s;
    }
}

// out = a * x (+ b * y)
template <typename T>
__global__ void k_axpby(long long n, double a, const T* __restrict__ x, double b, const T* __restrict__ y,
                        T* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)(a * (double)x[i] + (y ? b * (double)y[i] : 0.0));
}

// out = x / s[0]
template <typename T>
__global__ void k_scale_by(long long n, const T* __restrict__ x, const double* __restrict__ s, T* __restrict__ out) {
    T inv = (T)(1.0 / s[0]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = x[i] * inv;
}

// FP64 <-> FP32 transfers of the refinement: r32 = r64 / s[0];  x64 += s[0] * d32
__global__ void k_to_f32_scaled(long long n, const double* __restrict__ a, const double* __restrict__ s,
                                float* __restrict__ b) {
    double inv = 1.0 / s[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)(a[i] * inv);
}

__global__ void k_add_f32_scaled(long long n, const float* __restrict__ d, const double* __restrict__ s,
                                 double* __restrict__ x) {
    double sc = s[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += sc * (double)d[i];
}

__global__ void k_add_vec(int kk, const double* __restrict__ a, double* __restrict__ b) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
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

// ---------------------------------------------------------------- Krylov engine

template <typename T>
struct Krylov {
    int m = 0;
    long long n = 0;
    T* V = nullptr;     // [(m+1)][n]
    T* Z = nullptr;     // [m][n] preconditioned directions (flexible variant), or nullptr
    T* w = nullptr;
    T* r = nullptr;
    double* red = nullptr;
    double* h = nullptr;   // h1 | h2 | nrm | scalar slots
    double* hp = nullptr;  // host mirror
};

template <typename T>
static ddlpb_status krylov_alloc(ddlpb_ctx* c, Krylov<T>& K, int m, long long n, bool flexible) {
    K.m = m;
    K.n = n;
    DDLPB_TRY(ctx_alloc(c, &K.V, (size_t)(m + 1) * n));
    if (flexible) DDLPB_TRY(ctx_alloc(c, &K.Z, (size_t)m * n));
    DDLPB_TRY(ctx_alloc(c, &K.w, n));
    DDLPB_TRY(ctx_alloc(c, &K.r, n));
    DDLPB_TRY(ctx_alloc(c, &K.red, (size_t)RGRID * (m + 2)));
    DDLPB_TRY(ctx_alloc(c, &K.h, 4 * (size_t)(m + 2)));
    // pageable host mirror: every copy into it is followed by a stream synchronisation anyway
    K.hp = new double[4 * (size_t)(m + 2)];
    c->host_bufs.push_back(K.hp);
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status dots(ddlpb_ctx* c, Krylov<T>& K, int kk, const T* V, const T* w, double* out, bool sq) {
    KernelTimer kt(c, "krylov_dot", sizeof(T) == 4, 2);
    k_multidot<T><<<RGRID, RBLK, sizeof(double) * kk, c->stream>>>(K.n, kk, V, w, K.red);
    DDLPB_LAUNCHED(c, "multidot");
    k_reduce<<<kk, RBLK, 0, c->stream>>>(RGRID, K.red, out, 0, sq ? 1 : 0);
    DDLPB_LAUNCHED(c, "reduce");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status norm_host(ddlpb_ctx* c, Krylov<T>& K, const T* v, double* dev_slot, double* host) {
    DDLPB_TRY(dots<T>(c, K, 1, v, v, dev_slot, true));
    DDLPB_CK(c, cudaMemcpyAsync(K.hp + 3 * (K.m + 2), dev_slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    *host = K.hp[3 * (K.m + 2)];
    return DDLPB_OK;
}

// Restarted (flexible) GMRES with classical Gram-Schmidt and one re-orthogonalisation
// pass (skipped when reorth is false: the few iterations of a loose inner solve).  apply(in, out) is the operator, precond(in, out) the right preconditioner
// (used only when K.Z is set).  x holds the initial guess (all zero if x_zero).
// Stops when the Krylov estimate of ||b - A x|| / ||b|| <= tol; the true residual
// is recomputed at every restart.
template <typename T, typename Apply, typename Prec>
static ddlpb_status gmres_T(ddlpb_ctx* c, Krylov<T>& K, Apply apply, Prec precond, const T* b, T* x, double tol,
                            int maxit, bool x_zero, int* iters, double* rel_out, bool stall_exit = false,
                            bool reorth = true) {
    const long long n = K.n;
    const int m = K.m;
    cudaStream_t st = c->stream;
    double* h1 = K.h;
    double* h2 = K.h + (m + 2);
    double* nrm = K.h + 2 * (m + 2);
    double* hp = K.hp;
    double bnorm = 0;
    DDLPB_TRY(norm_host<T>(c, K, b, nrm, &bnorm));
    *iters = 0;
    if (!(bnorm > 0.0)) {
        DDLPB_CK(c, cudaMemsetAsync(x, 0, sizeof(T) * n, st));
        *rel_out = 0.0;
        if (!(bnorm == 0.0)) {
            c->err = "non-finite right-hand side";
            return DDLPB_ENOTCONV;
        }
        return DDLPB_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1), yv(m);
    int total = 0;
    double rel = 1.0, prev_rel = -1.0;
    bool first = true;
    for (;;) {
        if (first && x_zero) {
            DDLPB_CK(c, cudaMemcpyAsync(K.r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            DDLPB_TRY(apply(x, K.r));
            KernelTimer kt(c, "krylov_update", sizeof(T) == 4, 2);
            k_axpby<T><<<VG, VB, 0, st>>>(n, 1.0, b, -1.0, K.r, K.r);
            DDLPB_LAUNCHED(c, "axpby");
        }
        first = false;
        double beta = 0;
        DDLPB_TRY(norm_host<T>(c, K, K.r, nrm, &beta));
        rel = beta / bnorm;
        if (trace_on())
            std::fprintf(stderr, "[ddlpb] gmres<%s>%s m=%d it=%d true_rel=%.3e tol=%.1e\n",
                         sizeof(T) == 8 ? "f64" : "f32", K.Z ? " flexible" : "", m, total, rel, tol);
        if (!std::isfinite(beta)) {
            c->err = "non-finite residual in GMRES";
            *rel_out = rel;
            return DDLPB_ENOTCONV;
        }
        if (rel <= tol) break;
        if (stall_exit && prev_rel > 0 && rel > 0.5 * prev_rel) {
            *iters = total;
            *rel_out = rel;
            c->err = "GMRES stagnated (relative residual " + std::to_string(rel) + ")";
            return DDLPB_ENOTCONV;
        }
        prev_rel = rel;
        if (total >= maxit) {
            *iters = total;
            *rel_out = rel;
            c->err = "GMRES reached max_iter (relative residual " + std::to_string(rel) + ")";
            return DDLPB_ENOTCONV;
        }
        {
            KernelTimer kt(c, "krylov_update", sizeof(T) == 4, 2);
            k_scale_by<T><<<VG, VB, 0, st>>>(n, K.r, nrm, K.V);
            DDLPB_LAUNCHED(c, "scale");
        }
        std::fill(gvec.begin(), gvec.end(), 0.0);
        gvec[0] = beta;
        int k = 0;
        for (; k < m && total < maxit; ++k) {
            ++total;
            T* vk = K.V + (size_t)k * n;
            if (K.Z) {
                T* zk = K.Z + (size_t)k * n;
                DDLPB_TRY(precond(vk, zk));
                DDLPB_TRY(apply(zk, K.w));
            } else {
                DDLPB_TRY(apply(vk, K.w));
            }
            DDLPB_TRY(dots<T>(c, K, k + 1, K.V, K.w, h1, false));
            {
                KernelTimer kt(c, "krylov_update", sizeof(T) == 4, 2);
                k_sub_combination<T><<<VG, VB, sizeof(T) * (k + 1), st>>>(n, k + 1, K.V, h1, K.w);
                DDLPB_LAUNCHED(c, "sub_comb");
            }
            if (reorth) {
                DDLPB_TRY(dots<T>(c, K, k + 1, K.V, K.w, h2, false));
                KernelTimer kt(c, "krylov_update", sizeof(T) == 4, 2);
                k_sub_combination<T><<<VG, VB, sizeof(T) * (k + 1), st>>>(n, k + 1, K.V, h2, K.w);
                DDLPB_LAUNCHED(c, "sub_comb2");
                k_add_vec<<<ceil_div(k + 1, 256), 256, 0, st>>>(k + 1, h2, h1);
                DDLPB_LAUNCHED(c, "add_vec");
            }
            DDLPB_TRY(dots<T>(c, K, 1, K.w, K.w, nrm, true));
            {
                KernelTimer kt(c, "krylov_update", sizeof(T) == 4, 2);
                k_scale_by<T><<<VG, VB, 0, st>>>(n, K.w, nrm, K.V + (size_t)(k + 1) * n);
                DDLPB_LAUNCHED(c, "scale2");
            }
            DDLPB_CK(c, cudaMemcpyAsync(hp, h1, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
            DDLPB_CK(c, cudaMemcpyAsync(hp + (m + 2), nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
            DDLPB_CK(c, cudaStreamSynchronize(st));
            for (int q = 0; q <= k; ++q) H[(size_t)q * m + k] = hp[q];
            double hk1 = hp[m + 2];
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
        for (int q = k - 1; q >= 0; --q) {
            double s = gvec[q];
            for (int r = q + 1; r < k; ++r) s -= H[(size_t)q * m + r] * yv[r];
            yv[q] = s / H[(size_t)q * m + q];
        }
        DDLPB_CK(c, cudaMemcpyAsync(h2, yv.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        {
            KernelTimer kt(c, "krylov_update", sizeof(T) == 4, 2);
            k_add_combination<T><<<VG, VB, sizeof(T) * std::max(k, 1), st>>>(n, k, K.Z ? K.Z : K.V, h2, x);
            DDLPB_LAUNCHED(c, "add_comb");
        }
        DDLPB_CK(c, cudaStreamSynchronize(st));
    }
    *iters = total;
    *rel_out = rel;
    return DDLPB_OK;
}

struct SolverState {
    Krylov<double> outer64, inner64;
    Krylov<float> outer32, inner32;
    bool ready64 = false, ready32 = false;
    float* r32 = nullptr;
    float* d32 = nullptr;
    double* r64 = nullptr;
    int inner_iters = 0;
};

static SolverState* state(ddlpb_ctx* c) {
    if (!c->solver) c->solver = new SolverState();
    return (SolverState*)c->solver;
}

void solver_state_free(ddlpb_ctx* c) {
    delete (SolverState*)c->solver;
    c->solver = nullptr;
}

static const int kInnerRestart = 40;
static const int kInnerMaxit = 200;

// Right preconditioner: z = P^{-1} v with P = L_AB = diag(A, B) of Sec. 4, plus (when
// precond_coupling is set) the near part of the coupling C1/C2 between each sphere and
// its neighbours; applied by an inner GMRES on that sparse operator.
template <typename T>
static ddlpb_status precond_apply(ddlpb_ctx* c, OpSet<T>& S, Krylov<T>& inner, bool transpose, const T* v, T* z,
                                  int* inner_count) {
    int it = 0;
    double rel = 0;
    auto ab = [&](const T* in, T* out) {
        if (c->opt.precond_coupling) return op_apply_P_T<T>(c, S, in, out, transpose);
        return op_apply_AB_precond<T>(c, S, in, out, transpose);
    };
    auto none = [&](const T*, T*) { return DDLPB_OK; };
    DDLPB_CK(c, cudaMemsetAsync(z, 0, sizeof(T) * inner.n, c->stream));
    ddlpb_status s = gmres_T<T>(c, inner, ab, none, v, z, c->opt.precond_tol, kInnerMaxit, true, &it, &rel, false,
                                c->opt.precond_tol < 1e-2);
    *inner_count += it;
    if (s == DDLPB_ENOTCONV) {
        c->err.clear();  // an inexact preconditioner is allowed in flexible GMRES
        return DDLPB_OK;
    }
    return s;
}

// FP64 flexible GMRES on L (or L*) with the L_AB preconditioner.
static ddlpb_status solve_fp64(ddlpb_ctx* c, bool transpose, const double* b, double* x, bool x_zero, int* iters,
                               double* resid) {
    SolverState* S = state(c);
    if (!S->ready64) {
        DDLPB_TRY(krylov_alloc<double>(c, S->outer64, c->opt.gmres_restart, c->nvec, true));
        DDLPB_TRY(krylov_alloc<double>(c, S->inner64, kInnerRestart, c->nvec, false));
        S->ready64 = true;
    }
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    auto L = [&](const double* in, double* out) { return op_apply_L_T<double>(c, c->d64, in, out, transpose); };
    auto P = [&](const double* in, double* out) {
        return precond_apply<double>(c, c->d64, S->inner64, transpose, in, out, &S->inner_iters);
    };
    if (c->opt.precond_tol >= 1.0) {
        Krylov<double> plain = S->outer64;
        plain.Z = nullptr;
        return gmres_T<double>(c, plain, L, P, b, x, c->opt.tol, c->opt.max_iter, x_zero, iters, resid);
    }
    return gmres_T<double>(c, S->outer64, L, P, b, x, c->opt.tol, c->opt.max_iter, x_zero, iters, resid);
}

// Mixed precision: FP64 iterative refinement around an FP32 flexible GMRES (FP32
// operators, FP32 L_AB preconditioner).  Only the residual r = b - L x, the update
// of x and the norms are FP64.
static ddlpb_status solve_mixed(ddlpb_ctx* c, bool transpose, const double* b, double* x, bool x_zero, int* iters,
                                double* resid, int* steps) {
    SolverState* S = state(c);
    const long long n = c->nvec;
    if (!S->ready32) {
        DDLPB_TRY(krylov_alloc<float>(c, S->outer32, c->opt.gmres_restart, n, true));
        DDLPB_TRY(krylov_alloc<float>(c, S->inner32, kInnerRestart, n, false));
        DDLPB_TRY(ctx_alloc(c, &S->r32, n));
        DDLPB_TRY(ctx_alloc(c, &S->d32, n));
        DDLPB_TRY(ctx_alloc(c, &S->r64, n));
        if (!S->ready64) {
            DDLPB_TRY(krylov_alloc<double>(c, S->outer64, 1, n, false));
        }
        S->ready32 = true;
    }
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    DDLPB_TRY(opset_prepare<float>(c, c->f32));
    Krylov<double>& K64 = S->outer64;
    double* slot = K64.h + 2 * (K64.m + 2);
    double bnorm = 0;
    DDLPB_TRY(norm_host<double>(c, K64, b, slot, &bnorm));
    *iters = 0;
    *steps = 0;
    if (!(bnorm > 0.0)) {
        DDLPB_CK(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
        *resid = 0;
        return bnorm == 0.0 ? DDLPB_OK : DDLPB_ENOTCONV;
    }
    auto L32 = [&](const float* in, float* out) { return op_apply_L_T<float>(c, c->f32, in, out, transpose); };
    auto P32 = [&](const float* in, float* out) {
        return precond_apply<float>(c, c->f32, S->inner32, transpose, in, out, &S->inner_iters);
    };
    // The attainable accuracy of an FP32 Krylov solve is about cond(L) * 6e-8; on dense
    // globules at lmax = 10 that is ~1e-4, so each refinement step asks for 1e-3 (three
    // digits per FP64 residual evaluation) and stops early if a restart shows no progress.
    const double inner_tol = 1e-3;
    const int step_cap = c->opt.max_iter;
    for (int step = 0;; ++step) {
        // r = b - L x in FP64
        if (step == 0 && x_zero) {
            DDLPB_CK(c, cudaMemcpyAsync(S->r64, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        } else {
            DDLPB_TRY(op_apply_L_T<double>(c, c->d64, x, S->r64, transpose));
            k_axpby<double><<<VG, VB, 0, c->stream>>>(n, 1.0, b, -1.0, S->r64, S->r64);
            DDLPB_LAUNCHED(c, "axpby64");
        }
        double rn = 0;
        DDLPB_TRY(norm_host<double>(c, K64, S->r64, slot, &rn));
        double rel = rn / bnorm;
        *resid = rel;
        if (trace_on()) std::fprintf(stderr, "[ddlpb] refinement step %d fp64_rel=%.3e\n", step, rel);
        if (!std::isfinite(rel)) {
            c->err = "non-finite residual in refinement";
            return DDLPB_ENOTCONV;
        }
        if (rel <= c->opt.tol) break;
        if (step >= 20) {
            c->err = "mixed-precision refinement stalled at relative residual " + std::to_string(rel);
            return DDLPB_ENOTCONV;
        }
        k_to_f32_scaled<<<VG, VB, 0, c->stream>>>(n, S->r64, slot, S->r32);
        DDLPB_LAUNCHED(c, "to_f32");
        DDLPB_CK(c, cudaMemsetAsync(S->d32, 0, sizeof(float) * n, c->stream));
        int it = 0;
        double r32rel = 0;
        Krylov<float> K32 = S->outer32;
        if (c->opt.precond_tol >= 1.0) K32.Z = nullptr;   // plain GMRES, no L_AB preconditioner
        ddlpb_status st = gmres_T<float>(c, K32, L32, P32, S->r32, S->d32, inner_tol, step_cap, true, &it, &r32rel,
                                         true);
        *iters += it;
        if (st != DDLPB_OK && st != DDLPB_ENOTCONV) return st;
        c->err.clear();
        k_add_f32_scaled<<<VG, VB, 0, c->stream>>>(n, S->d32, slot, x);
        DDLPB_LAUNCHED(c, "add_f32");
        *steps = step + 1;
    }
    return DDLPB_OK;
}

ddlpb_status solve_system(ddlpb_ctx* c, bool transpose, const double* b, double* x, int* iters, double* resid) {
    SolverState* S = state(c);
    S->inner_iters = 0;
    int steps = 0;
    ddlpb_status s;
    bool& zero = transpose ? c->Xa_zero : c->X_zero;
    if (c->opt.precision == DDLPB_MIXED) {
        s = solve_mixed(c, transpose, b, x, zero, iters, resid, &steps);
    } else {
        s = solve_fp64(c, transpose, b, x, zero, iters, resid);
    }
    zero = false;
    c->info.refinement_steps = steps;
    c->info.inner_iterations = S->inner_iters;
    return s;
}

// ---------------------------------------------------------------- C ABI

static thread_local std::string g_setup_err;

extern "C" void ddlpb_default_options(ddlpb_options* o) {
    if (!o) return;
    o->eta = 0.1;
    o->tol = 1e-8;
    o->max_iter = 500;
    o->gmres_restart = 150;
    o->precision = DDLPB_FP64;
    o->fmm_order = 0;
    o->cuda_stream = nullptr;
    o->precond_tol = 1e-3;
    o->kernel_timing = 0;
    o->precond_coupling = 0;
    o->precond_fp16 = 1;
    o->fmm_theta = 0.4;
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
    if (o.gmres_restart < 1 || o.gmres_restart > 2000) return fail("gmres_restart must be in [1, 2000]");
    if (o.precision != DDLPB_FP64 && o.precision != DDLPB_MIXED) return fail("unknown precision");
    if (o.fmm_order != 0 && (o.fmm_order < lmax + 1 || o.fmm_order > DDLPB_FMM_PMAX))
        return fail("fmm_order must be 0 (direct summation) or in [lmax + 1, 21]");
    if (o.fmm_order != 0 && !(o.fmm_theta > 0.0 && o.fmm_theta < 1.0)) return fail("fmm_theta must be in (0, 1)");
    if (!(o.precond_tol > 0.0 && o.precond_tol <= 1.0)) return fail("precond_tol must be in (0, 1]");
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
    ddlpb_status s;
    {
        KernelTimer kt(c, "setup", false, 2, true);
        s = ddlpb_internal_setup(c, centres, radii, charges, device, (int)surface);
    }
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
    k_energy<<<1, RBLK, 0, c->stream>>>(c->M, c->nb, c->q, c->X, c->tmpv);
    DDLPB_LAUNCHED(c, "energy");
    DDLPB_CK(c, cudaMemcpyAsync(e, c->tmpv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
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
    {
        KernelTimer kt(c, "forces", false, 2, true);
        DDLPB_TRY(compute_forces(c, f));
    }
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
    {
        KernelTimer kt(c, "forces", false, 2, true);
        DDLPB_TRY(compute_forces(c, c->force_acc));
    }
    DDLPB_CK(c, cudaMemcpyAsync(f, c->force_acc, sizeof(double) * 3 * c->M, cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_apply_device(ddlpb_ctx* c, int op, const double* x, double* y) {
    if (!c || !x || !y || op < 0 || op > 17 || (op > 5 && op < 8) || (op > 13 && op < 16)) return DDLPB_EINVAL;
    c->err.clear();
    if (op >= 8) {
        DDLPB_TRY(op_apply_fp32(c, op - 8, x, y));
        DDLPB_CK(c, cudaStreamSynchronize(c->stream));
        return DDLPB_OK;
    }
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

extern "C" ddlpb_status ddlpb_kernel_time(ddlpb_ctx* c, const char* name, long long* launches, double* ms) {
    if (!c || !name || !launches || !ms) return DDLPB_EINVAL;
    *launches = 0;
    *ms = 0.0;
    auto it = c->ktimes.find(name);
    if (it == c->ktimes.end()) return DDLPB_OK;
    KernelTimes& k = it->second;
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i + 1 < k.ev.size(); i += 2) {
        float t = 0.f;
        DDLPB_CK(c, cudaEventElapsedTime(&t, k.ev[i], k.ev[i + 1]));
        k.ms += t;
        k.launches += 1;
        cudaEventDestroy(k.ev[i]);
        cudaEventDestroy(k.ev[i + 1]);
    }
    k.ev.clear();
    *launches = k.launches;
    *ms = k.ms;
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_kernel_time_reset(ddlpb_ctx* c) {
    if (!c) return DDLPB_EINVAL;
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    for (auto& kv : c->ktimes) {
        for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
        kv.second = KernelTimes();
    }
    return DDLPB_OK;
}

extern "C" ddlpb_status ddlpb_set_vector_device(ddlpb_ctx* c, int which, const double* x) {
    if (!c || !x || (which != 1 && which != 2)) return DDLPB_EINVAL;
    c->err.clear();
    double* d = which == 1 ? c->X : c->Xa;
    DDLPB_CK(c, cudaMemcpyAsync(d, x, sizeof(double) * c->nvec, cudaMemcpyDeviceToDevice, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    if (which == 1) {
        c->X_zero = false;
        c->solved = false;
    } else {
        c->Xa_zero = false;
    }
    c->adjoint_done = false;
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
    for (auto& kv : c->ktimes)
        for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFreeAsync(p, c->stream);
    cudaStreamSynchronize(c->stream);
    for (double* p : c->host_bufs) delete[] p;
    solver_state_free(c);
    delete c;
}
