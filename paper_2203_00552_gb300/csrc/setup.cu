// setup.cu -- ddlpb_setup: validation, tables, neighbour lists, switch functions on
// the Lebedev grid, hit lists, external points and the right-hand side.
//
// Sec. 2.2 (cavity, N_i, omega_ij, chi_i^e, bases, Lebedev rule, G0, F0) and
// Sec. 3.1 (regularised chi_eta, omega_ij^eta, d^i, f^i, chi_i^eta) of
// arXiv:2203.00552.
#include <cub/cub.cuh>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "lebedev_tables.h"

static const double kSasProbeBohr = 1.4 / 0.529177210903;

// ---------------------------------------------------------------- kernels

__global__ void k_ylm_table(int N, int lmax, int nb, const double4* __restrict__ leb, YTab yt,
                            double* __restrict__ Y, double* __restrict__ YT) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double4 s = leb[n];
    ylm_stream<double>(lmax, s.x, s.y, s.z, yt, [&](int idx, int, double v) {
        Y[(size_t)n * nb + idx] = v;
        YT[(size_t)idx * N + n] = v;
    });
}

// Scaled Bessel data of every sphere (Sec. 2.2; C_ik of Eq. definition_of_Q_matrix).
__global__ void k_sphere_bessel(int M, int lmax, double kappa, const double4* __restrict__ sph,
                                double* __restrict__ Sinv, double* __restrict__ Khinv, double* __restrict__ di,
                                double* __restrict__ dk, double* __restrict__ cik) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    double r = sph[j].w, x = kappa * r, x2 = x * x;
    int L2 = lmax + 2;
    double S[DDLPB_LMAX_MAX + 3], K[DDLPB_LMAX_MAX + 3];
    for (int l = 0; l < L2; ++l) S[l] = scaled_i_series<double>(l, x);
    K[0] = 1.0;
    K[1] = 1.0 + x;
    for (int l = 1; l + 1 < L2; ++l) K[l + 1] = K[l] + x2 * K[l - 1] / (double)((2 * l + 1) * (2 * l - 1));
    for (int l = 0; l < L2; ++l) {
        Sinv[(size_t)j * L2 + l] = 1.0 / S[l];
        Khinv[(size_t)j * L2 + l] = 1.0 / K[l];
    }
    for (int l = 0; l <= lmax; ++l) {
        // i_l'/i_l and k_l'/k_l as d/dr at r (Bessel argument kappa r)
        double a = (double)l / r + kappa * kappa * r / (double)(2 * l + 3) * S[l + 1] / S[l];
        double b = ((double)l - (double)(2 * l + 1) * K[l + 1] / K[l]) / r;
        di[(size_t)j * (lmax + 1) + l] = a;
        dk[(size_t)j * (lmax + 1) + l] = b;
        cik[(size_t)j * (lmax + 1) + l] = 1.0 / (a - b);
    }
}

// N_i: spheres whose balls intersect ball i (Sec. 2.2), counted then listed in index order.
__global__ void k_nbr_count(int M, const double4* __restrict__ sph, int* __restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double4 a = sph[i];
    int c = 0;
    for (int j = 0; j < M; ++j) {
        if (j == i) continue;
        double4 b = sph[j];
        double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        double rr = a.w + b.w;
        if (dx * dx + dy * dy + dz * dz < rr * rr) ++c;
    }
    cnt[i] = c;
}

__global__ void k_nbr_fill(int M, const double4* __restrict__ sph, const int* __restrict__ ptr,
                           int* __restrict__ idx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double4 a = sph[i];
    int c = ptr[i];
    for (int j = 0; j < M; ++j) {
        if (j == i) continue;
        double4 b = sph[j];
        double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        double rr = a.w + b.w;
        if (dx * dx + dy * dy + dz * dz < rr * rr) idx[c++] = j;
    }
}

// Per grid point x_i^n = x_i + r_i s_n: f^i, chi_i^eta = 1 - d^i f^i, and the number
// of neighbours j with r_1^j(x_i^n) < 1 (nonzero omega_ij^eta).  Eqs. regular_omega_ij .. regular_chi_e.
__global__ void k_grid_switch(int M, int N, double eta, const double4* __restrict__ sph,
                              const double4* __restrict__ leb, const int* __restrict__ nptr,
                              const int* __restrict__ nidx, double* __restrict__ fval, double* __restrict__ chi,
                              int* __restrict__ nhit, int* __restrict__ isext) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)M * N) return;
    int i = (int)(p / N), n = (int)(p % N);
    double4 a = sph[i], s = leb[n];
    double px = a.x + a.w * s.x, py = a.y + a.w * s.y, pz = a.z + a.w * s.z;
    double f = 0.0;
    int h = 0;
    for (int k = nptr[i]; k < nptr[i + 1]; ++k) {
        double4 b = sph[nidx[k]];
        double dx = px - b.x, dy = py - b.y, dz = pz - b.z;
        double t = sqrt(dx * dx + dy * dy + dz * dz) / b.w;
        if (t < 1.0) {
            f += chi_eta(t, eta);
            ++h;
        }
    }
    double d = f > 1.0 ? 1.0 / f : 1.0;
    double c = 1.0 - d * f;
    if (f >= 1.0) c = 0.0;
    fval[p] = f;
    chi[p] = c;
    nhit[p] = h;
    isext[p] = c > 0.0 ? 1 : 0;
}

__global__ void k_hits_fill(int M, int N, double eta, const double4* __restrict__ sph, const double4* __restrict__ leb,
                            const int* __restrict__ nptr, const int* __restrict__ nidx, const double* __restrict__ fval,
                            const int* __restrict__ hptr, int* __restrict__ hj, double* __restrict__ hw,
                            int* __restrict__ hp, unsigned short* __restrict__ hs) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)M * N) return;
    int i = (int)(p / N), n = (int)(p % N);
    double4 a = sph[i], s = leb[n];
    double px = a.x + a.w * s.x, py = a.y + a.w * s.y, pz = a.z + a.w * s.z;
    double f = fval[p];
    double d = f > 1.0 ? 1.0 / f : 1.0;
    int o = hptr[p];
    for (int k = nptr[i]; k < nptr[i + 1]; ++k) {
        int j = nidx[k];
        double4 b = sph[j];
        double dx = px - b.x, dy = py - b.y, dz = pz - b.z;
        double t = sqrt(dx * dx + dy * dy + dz * dz) / b.w;
        if (t < 1.0) {
            hj[o] = j;
            hw[o] = d * chi_eta(t, eta);
            hp[o] = (int)p;
            hs[o] = (unsigned short)(k - nptr[i]);
            ++o;
        }
    }
}

// Transposed hit list: the hits sorted (stably) by their target sphere j, so that within
// each j the points stay in point-major order.  Filled from the sorted hit indices.
__global__ void k_iota(int n, int* __restrict__ v) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) v[k] = k;
}

__global__ void k_thits_gather(int H, const int* __restrict__ order, const int* __restrict__ hp,
                               const double* __restrict__ hw, int* __restrict__ tp, double* __restrict__ tw) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < H) {
        int h = order[k];
        tp[k] = hp[h];
        tw[k] = hw[h];
    }
}

// thit_ptr[j] = first position of key j in the sorted keys (keys are sphere indices).
__global__ void k_segment_starts(int H, int M, const int* __restrict__ keys, int* __restrict__ ptr) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > H) return;
    int cur = k < H ? keys[k] : M;
    int prev = k > 0 ? keys[k - 1] : -1;
    for (int j = prev + 1; j <= cur; ++j) ptr[j] = k;
}

__global__ void k_ext_fill(int M, int N, const double4* __restrict__ sph, const double4* __restrict__ leb,
                           const double* __restrict__ chi, const int* __restrict__ isext,
                           const int* __restrict__ epos, int* __restrict__ ext_p, double4* __restrict__ ext_x,
                           int* __restrict__ ext_ptr) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)M * N) return;
    int i = (int)(p / N), n = (int)(p % N);
    if (n == 0) ext_ptr[i] = epos[p];
    if (p == (long long)M * N - 1) ext_ptr[M] = epos[p] + isext[p];
    if (!isext[p]) return;
    double4 a = sph[i], s = leb[n];
    int e = epos[p];
    ext_p[e] = (int)p;
    ext_x[e] = make_double4(a.x + a.w * s.x, a.y + a.w * s.y, a.z + a.w * s.z, chi[p]);
}

__global__ void k_src_flag(int M, const int* __restrict__ ext_ptr, int* __restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) flag[i] = ext_ptr[i + 1] > ext_ptr[i] ? 1 : 0;
}

__global__ void k_src_fill(int M, const int* __restrict__ flag, const int* __restrict__ pos, int* __restrict__ src) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && flag[i]) src[pos[i]] = i;
}

// psi_0 (Eq. defintion_of_psi_0) and d_n psi_0 = grad psi_0 . s_n at the external points.
// One thread per point, atoms streamed through shared memory.
__global__ void k_coulomb_ext(int E, int N, int M, double eps1, const double4* __restrict__ ext_x,
                              const int* __restrict__ ext_p, const double4* __restrict__ leb,
                              const double4* __restrict__ sph, const double* __restrict__ q,
                              double* __restrict__ psi0, double* __restrict__ dn) {
    __shared__ double4 sa[256];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double4 x = t < E ? ext_x[t] : make_double4(0, 0, 0, 0);
    double4 s = t < E ? leb[ext_p[t] % N] : make_double4(0, 0, 1, 0);
    double pot = 0, gx = 0, gy = 0, gz = 0;
    for (int base = 0; base < M; base += 256) {
        int k = base + threadIdx.x;
        if (k < M) {
            double4 b = sph[k];
            sa[threadIdx.x] = make_double4(b.x, b.y, b.z, q[k]);
        }
        __syncthreads();
        int cnt = min(256, M - base);
        for (int kk = 0; kk < cnt; ++kk) {
            double4 b = sa[kk];
            double dx = x.x - b.x, dy = x.y - b.y, dz = x.z - b.z;
            double ir = rsqrt(dx * dx + dy * dy + dz * dz);
            double qi = b.w * ir;
            pot += qi;
            double qi3 = qi * ir * ir;
            gx -= qi3 * dx;
            gy -= qi3 * dy;
            gz -= qi3 * dz;
        }
        __syncthreads();
    }
    if (t < E) {
        psi0[t] = pot / eps1;
        dn[t] = (gx * s.x + gy * s.y + gz * s.z) / eps1;
    }
}

__global__ void k_fill_q(int M, int nb, const double* __restrict__ q, double* __restrict__ Qv) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) Qv[(size_t)j * nb] = q[j] * 0.28209479177387814;  // q_j Y_00
}

// g = [G0 + F0 ; F0]
__global__ void k_rhs_combine(long long half, const double* __restrict__ G0, const double* __restrict__ F0,
                              double* __restrict__ g) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < half) {
        g[k] = G0[k] + F0[k];
        g[half + k] = F0[k];
    }
}

__global__ void k_chunk_count(int M, const int* __restrict__ tptr, int* __restrict__ cnt) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) cnt[j] = (tptr[j + 1] - tptr[j] + DDLPB_TCHUNK - 1) / DDLPB_TCHUNK;
}

__global__ void k_chunk_fill(int M, const int* __restrict__ tptr, const int* __restrict__ cpos,
                             int* __restrict__ cj, int* __restrict__ ct0, int* __restrict__ ccnt) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int o = cpos[j];
    for (int t = tptr[j]; t < tptr[j + 1]; t += DDLPB_TCHUNK, ++o) {
        cj[o] = j;
        ct0[o] = t;
        ccnt[o] = min(DDLPB_TCHUNK, tptr[j + 1] - t);
    }
}

// ---------------------------------------------------------------- host helpers

static ddlpb_status scan_exclusive(ddlpb_ctx* c, const int* in, int* out, long long n) {
    size_t bytes = 0;
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, c->stream));
    void* tmp = nullptr;
    DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)n, c->stream));
    return DDLPB_OK;
}

static ddlpb_status read_int(ddlpb_ctx* c, const int* d, int* h) {
    DDLPB_CK(c, cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    return DDLPB_OK;
}

static void build_ytab(std::vector<double>& h) {
    const int LT = DDLPB_LT;
    h.assign(2 * LT * LT + 2 * LT, 0.0);
    double* a = h.data();
    double* b = a + LT * LT;
    double* qmm = b + LT * LT;
    double* q1 = qmm + LT;
    for (int l = 0; l < LT; ++l)
        for (int m = 0; m + 2 <= l; ++m) {
            double L = l, Mm = m;
            a[l * LT + m] = std::sqrt((4 * L * L - 1) / (L * L - Mm * Mm));
            b[l * LT + m] = std::sqrt(((L - 1) * (L - 1) - Mm * Mm) / (4 * (L - 1) * (L - 1) - 1));
        }
    qmm[0] = 1.0 / std::sqrt(4.0 * M_PI);
    for (int m = 1; m < LT; ++m) qmm[m] = qmm[m - 1] * std::sqrt((2.0 * m + 1.0) / (2.0 * m));
    for (int m = 0; m < LT; ++m) q1[m] = std::sqrt(2.0 * m + 3.0);
}

// ---------------------------------------------------------------- setup driver

ddlpb_status ddlpb_internal_setup(ddlpb_ctx* c, const double* centres, const double* radii, const double* charges,
                                  bool device_ptrs, int surface) {
    const int M = c->M;
    // -- inputs to host for validation
    std::vector<double> hc(3 * (size_t)M), hr(M), hq(M);
    if (device_ptrs) {
        DDLPB_CK(c, cudaMemcpyAsync(hc.data(), centres, 3 * sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream));
        DDLPB_CK(c, cudaMemcpyAsync(hr.data(), radii, sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream));
        DDLPB_CK(c, cudaMemcpyAsync(hq.data(), charges, sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream));
        DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(hc.data(), centres, 3 * sizeof(double) * M);
        std::memcpy(hr.data(), radii, sizeof(double) * M);
        std::memcpy(hq.data(), charges, sizeof(double) * M);
    }
    for (int k = 0; k < M; ++k) {
        if (!std::isfinite(hc[3 * k]) || !std::isfinite(hc[3 * k + 1]) || !std::isfinite(hc[3 * k + 2]) ||
            !std::isfinite(hr[k]) || !std::isfinite(hq[k])) {
            c->err = "non-finite centre, radius or charge at atom " + std::to_string(k);
            return DDLPB_EINVAL;
        }
        if (hr[k] <= 0.0) {
            c->err = "radius <= 0 at atom " + std::to_string(k);
            return DDLPB_EINVAL;
        }
    }
    for (int a = 0; a < 3; ++a) {
        double sum = 0;
        for (int k = 0; k < M; ++k) sum += hc[3 * k + a];
        c->centroid[a] = sum / M;
    }
    std::vector<double4> hs(M);
    for (int k = 0; k < M; ++k)
        hs[k] = make_double4(hc[3 * k], hc[3 * k + 1], hc[3 * k + 2], hr[k] + (surface == DDLPB_SAS ? kSasProbeBohr : 0.0));

    // -- Lebedev rule (Sec. 2.2)
    const LebedevRule* rule = nullptr;
    for (int k = 0; k < kNumLebedevRules; ++k)
        if (kLebedevRules[k].n == c->N) rule = &kLebedevRules[k];
    if (!rule) {
        c->err = "unsupported n_lebedev " + std::to_string(c->N);
        return DDLPB_EINVAL;
    }
    if (rule->degree < 2 * c->lmax) {
        c->err = "Lebedev rule with " + std::to_string(c->N) + " points is exact to degree " +
                 std::to_string(rule->degree) + " < 2*lmax";
        return DDLPB_EINVAL;
    }
    c->degree = rule->degree;
    const int N = c->N, nb = c->nb, L = c->lmax;
    const long long MN = (long long)M * N;

    cudaStream_t st = c->stream;
    DDLPB_TRY(ctx_alloc(c, &c->sph, M));
    DDLPB_TRY(ctx_alloc(c, &c->q, M));
    DDLPB_TRY(ctx_alloc(c, &c->leb, N));
    DDLPB_CK(c, cudaMemcpyAsync(c->sph, hs.data(), sizeof(double4) * M, cudaMemcpyHostToDevice, st));
    DDLPB_CK(c, cudaMemcpyAsync(c->q, hq.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
    DDLPB_CK(c, cudaMemcpyAsync(c->leb, rule->xyzw, sizeof(double4) * N, cudaMemcpyHostToDevice, st));

    std::vector<double> ht;
    build_ytab(ht);
    DDLPB_TRY(ctx_alloc(c, &c->ytab, ht.size()));
    DDLPB_CK(c, cudaMemcpyAsync(c->ytab, ht.data(), sizeof(double) * ht.size(), cudaMemcpyHostToDevice, st));
    c->yt.a = c->ytab;
    c->yt.b = c->ytab + DDLPB_LT * DDLPB_LT;
    c->yt.qmm = c->yt.b + DDLPB_LT * DDLPB_LT;
    c->yt.q1 = c->yt.qmm + DDLPB_LT;

    DDLPB_TRY(ctx_alloc(c, &c->Y, (size_t)N * nb));
    DDLPB_TRY(ctx_alloc(c, &c->YT, (size_t)N * nb));
    k_ylm_table<<<ceil_div(N, 128), 128, 0, st>>>(N, L, nb, c->leb, c->yt, c->Y, c->YT);
    DDLPB_LAUNCHED(c, "ylm_table");

    // -- Bessel tables
    DDLPB_TRY(ctx_alloc(c, &c->Sinv, (size_t)M * (L + 2)));
    DDLPB_TRY(ctx_alloc(c, &c->Khinv, (size_t)M * (L + 2)));
    DDLPB_TRY(ctx_alloc(c, &c->di, (size_t)M * (L + 1)));
    DDLPB_TRY(ctx_alloc(c, &c->dk, (size_t)M * (L + 1)));
    DDLPB_TRY(ctx_alloc(c, &c->cik, (size_t)M * (L + 1)));
    k_sphere_bessel<<<ceil_div(M, 128), 128, 0, st>>>(M, L, c->kappa, c->sph, c->Sinv, c->Khinv, c->di, c->dk, c->cik);
    DDLPB_LAUNCHED(c, "sphere_bessel");

    // -- neighbour lists
    int* cnt = nullptr;
    DDLPB_TRY(ctx_alloc(c, &cnt, M + 1));
    DDLPB_CK(c, cudaMemsetAsync(cnt, 0, sizeof(int) * (M + 1), st));
    k_nbr_count<<<ceil_div(M, 128), 128, 0, st>>>(M, c->sph, cnt);
    DDLPB_LAUNCHED(c, "nbr_count");
    DDLPB_TRY(ctx_alloc(c, &c->nbr_ptr, M + 1));
    DDLPB_TRY(scan_exclusive(c, cnt, c->nbr_ptr, M + 1));
    int npairs = 0;
    DDLPB_TRY(read_int(c, c->nbr_ptr + M, &npairs));
    c->n_pairs = npairs;
    DDLPB_TRY(ctx_alloc(c, &c->nbr_idx, npairs));
    k_nbr_fill<<<ceil_div(M, 128), 128, 0, st>>>(M, c->sph, c->nbr_ptr, c->nbr_idx);
    DDLPB_LAUNCHED(c, "nbr_fill");

    // -- switch functions and hit lists
    DDLPB_TRY(ctx_alloc(c, &c->fval, MN));
    DDLPB_TRY(ctx_alloc(c, &c->chi, MN));
    int *nhit = nullptr, *isext = nullptr, *epos = nullptr;
    DDLPB_TRY(ctx_alloc(c, &nhit, MN + 1));
    DDLPB_TRY(ctx_alloc(c, &isext, MN + 1));
    DDLPB_TRY(ctx_alloc(c, &epos, MN + 1));
    DDLPB_CK(c, cudaMemsetAsync(nhit + MN, 0, sizeof(int), st));
    DDLPB_CK(c, cudaMemsetAsync(isext + MN, 0, sizeof(int), st));
    k_grid_switch<<<ceil_div(MN, 256), 256, 0, st>>>(M, N, c->eta, c->sph, c->leb, c->nbr_ptr, c->nbr_idx, c->fval,
                                                     c->chi, nhit, isext);
    DDLPB_LAUNCHED(c, "grid_switch");
    DDLPB_TRY(ctx_alloc(c, &c->hit_ptr, MN + 1));
    DDLPB_TRY(scan_exclusive(c, nhit, c->hit_ptr, MN + 1));
    int H = 0;
    DDLPB_TRY(read_int(c, c->hit_ptr + MN, &H));
    c->H = H;
    DDLPB_TRY(ctx_alloc(c, &c->hit_j, H));
    DDLPB_TRY(ctx_alloc(c, &c->hit_w, H));
    DDLPB_TRY(ctx_alloc(c, &c->hit_p, H));
    DDLPB_TRY(ctx_alloc(c, &c->hit_s, H));
    k_hits_fill<<<ceil_div(MN, 256), 256, 0, st>>>(M, N, c->eta, c->sph, c->leb, c->nbr_ptr, c->nbr_idx, c->fval,
                                                   c->hit_ptr, c->hit_j, c->hit_w, c->hit_p, c->hit_s);
    DDLPB_LAUNCHED(c, "hits_fill");

    // -- transposed hits (stable radix sort of the hit indices by target sphere)
    DDLPB_TRY(ctx_alloc(c, &c->thit_ptr, M + 1));
    DDLPB_TRY(ctx_alloc(c, &c->thit_p, H));
    DDLPB_TRY(ctx_alloc(c, &c->thit_w, H));
    DDLPB_TRY(ctx_alloc(c, &c->thit_h, H));
    {
        int *keys_out = nullptr, *vals_in = nullptr;
        DDLPB_TRY(ctx_alloc(c, &keys_out, H));
        DDLPB_TRY(ctx_alloc(c, &vals_in, H));
        if (H > 0) {
            k_iota<<<ceil_div(H, 256), 256, 0, st>>>(H, vals_in);
            DDLPB_LAUNCHED(c, "iota");
            size_t bytes = 0;
            int bits = 1;
            while ((1 << bits) < M + 1) ++bits;
            DDLPB_CK(c, cub::DeviceRadixSort::SortPairs(nullptr, bytes, c->hit_j, keys_out, vals_in, c->thit_h, H, 0,
                                                        bits, st));
            void* tmp = nullptr;
            DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
            DDLPB_CK(c, cub::DeviceRadixSort::SortPairs(tmp, bytes, c->hit_j, keys_out, vals_in, c->thit_h, H, 0, bits,
                                                        st));
            k_thits_gather<<<ceil_div(H, 256), 256, 0, st>>>(H, c->thit_h, c->hit_p, c->hit_w, c->thit_p, c->thit_w);
            DDLPB_LAUNCHED(c, "thits_gather");
        }
        k_segment_starts<<<ceil_div(H + 1, 256), 256, 0, st>>>(H, M, keys_out, c->thit_ptr);
        DDLPB_LAUNCHED(c, "segment_starts");
    }

    // -- chunks of the transposed hit list (work units of the transposed A/B product)
    {
        int *ccnt = nullptr, *cpos = nullptr;
        DDLPB_TRY(ctx_alloc(c, &ccnt, M + 1));
        DDLPB_TRY(ctx_alloc(c, &cpos, M + 1));
        DDLPB_CK(c, cudaMemsetAsync(ccnt, 0, sizeof(int) * (M + 1), st));
        k_chunk_count<<<ceil_div(M, 256), 256, 0, st>>>(M, c->thit_ptr, ccnt);
        DDLPB_LAUNCHED(c, "chunk_count");
        DDLPB_TRY(scan_exclusive(c, ccnt, cpos, M + 1));
        int nch = 0;
        DDLPB_TRY(read_int(c, cpos + M, &nch));
        c->n_chunks = nch;
        DDLPB_TRY(ctx_alloc(c, &c->chunk_j, nch));
        DDLPB_TRY(ctx_alloc(c, &c->chunk_t0, nch));
        DDLPB_TRY(ctx_alloc(c, &c->chunk_cnt, nch));
        k_chunk_fill<<<ceil_div(M, 256), 256, 0, st>>>(M, c->thit_ptr, cpos, c->chunk_j, c->chunk_t0, c->chunk_cnt);
        DDLPB_LAUNCHED(c, "chunk_fill");
    }

    // -- external points (chi_i^eta > 0) and the spheres that own them
    DDLPB_TRY(scan_exclusive(c, isext, epos, MN + 1));
    int E = 0;
    DDLPB_TRY(read_int(c, epos + MN, &E));
    c->E = E;
    DDLPB_TRY(ctx_alloc(c, &c->ext_p, E));
    DDLPB_TRY(ctx_alloc(c, &c->ext_x, E));
    DDLPB_TRY(ctx_alloc(c, &c->ext_ptr, M + 1));
    k_ext_fill<<<ceil_div(MN, 256), 256, 0, st>>>(M, N, c->sph, c->leb, c->chi, isext, epos, c->ext_p, c->ext_x,
                                                  c->ext_ptr);
    DDLPB_LAUNCHED(c, "ext_fill");
    int *sflag = nullptr, *spos = nullptr;
    DDLPB_TRY(ctx_alloc(c, &sflag, M + 1));
    DDLPB_TRY(ctx_alloc(c, &spos, M + 1));
    DDLPB_CK(c, cudaMemsetAsync(sflag, 0, sizeof(int) * (M + 1), st));
    k_src_flag<<<ceil_div(M, 128), 128, 0, st>>>(M, c->ext_ptr, sflag);
    DDLPB_LAUNCHED(c, "src_flag");
    DDLPB_TRY(scan_exclusive(c, sflag, spos, M + 1));
    int ns = 0;
    DDLPB_TRY(read_int(c, spos + M, &ns));
    c->n_src = ns;
    DDLPB_TRY(ctx_alloc(c, &c->src, ns));
    k_src_fill<<<ceil_div(M, 128), 128, 0, st>>>(M, sflag, spos, c->src);
    DDLPB_LAUNCHED(c, "src_fill");

    // -- FMM tree and interaction lists (far field of the coupling, Appendix)
    if (c->opt.fmm_order > 0) DDLPB_TRY(fmm_build(c, hc.data()));

    // -- vectors and scratch
    c->nvec = 2LL * M * nb;
    const long long half = (long long)M * nb;
    DDLPB_TRY(ctx_alloc(c, &c->g, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->X, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->Xa, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->Qv, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->tmpv, c->nvec));
    DDLPB_TRY(ctx_alloc(c, &c->mu, half));
    DDLPB_TRY(ctx_alloc(c, &c->mu0, half));
    DDLPB_TRY(ctx_alloc(c, &c->gridA, MN));
    DDLPB_TRY(ctx_alloc(c, &c->gridB, MN));
    DDLPB_TRY(ctx_alloc(c, &c->psi0, E));
    DDLPB_TRY(ctx_alloc(c, &c->dnpsi0, E));
    DDLPB_TRY(ctx_alloc(c, &c->S0, E));
    DDLPB_TRY(ctx_alloc(c, &c->extA, E));
    DDLPB_TRY(ctx_alloc(c, &c->extB, E));
    DDLPB_CK(c, cudaMemsetAsync(c->mu, 0, sizeof(double) * half, st));
    DDLPB_CK(c, cudaMemsetAsync(c->X, 0, sizeof(double) * c->nvec, st));
    DDLPB_CK(c, cudaMemsetAsync(c->Xa, 0, sizeof(double) * c->nvec, st));
    DDLPB_CK(c, cudaMemsetAsync(c->Qv, 0, sizeof(double) * c->nvec, st));
    k_fill_q<<<ceil_div(M, 128), 128, 0, st>>>(M, nb, c->q, c->Qv);
    DDLPB_LAUNCHED(c, "fill_q");

    // -- right-hand side (Eqs. definition_of_G_0 .. definition_of_c_0_l_0_m_0)
    if (E > 0) {
        k_coulomb_ext<<<ceil_div(E, 256), 256, 0, st>>>(E, N, M, c->eps1, c->ext_x, c->ext_p, c->leb, c->sph, c->q,
                                                        c->psi0, c->dnpsi0);
        DDLPB_LAUNCHED(c, "coulomb_ext");
    }
    double* G0 = c->tmpv;
    double* F0 = c->tmpv + half;
    // G0 = -analysis(chi psi0)
    DDLPB_TRY(op_masked_analysis(c, c->psi0, -1.0, nullptr, G0, nb, 0));
    // mu0 = C_ik * analysis(chi dn psi0)
    DDLPB_TRY(op_masked_analysis(c, c->dnpsi0, 1.0, c->cik, c->mu0, nb, 0));
    // S = sum_j mu0_j k^j Y^j at external points; F0 = -(eps1/eps2) analysis(chi S)
    DDLPB_TRY(op_yukawa_potential(c, c->mu0, c->S0));
    DDLPB_TRY(op_masked_analysis(c, c->S0, -c->eps1 / c->eps2, nullptr, F0, nb, 0));
    k_rhs_combine<<<ceil_div(half, 256), 256, 0, st>>>(half, G0, F0, c->g);
    DDLPB_LAUNCHED(c, "rhs_combine");
    DDLPB_CK(c, cudaStreamSynchronize(st));

    c->info.n_atoms = M;
    c->info.lmax = L;
    c->info.n_lebedev = N;
    c->info.n_neighbour_pairs = c->n_pairs;
    c->info.n_hits = c->H;
    c->info.n_external = c->E;
    c->info.n_sources = c->n_src;
    return DDLPB_OK;
}
