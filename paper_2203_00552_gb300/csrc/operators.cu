// operators.cu -- the operators of the ddLPB system L X = g (Eq. AXg) and its adjoint
// L* (Eq. AstarXg), applied matrix-free on the device, in FP64 or FP32.
//
//   A, B  (Eqs. definition_of_A_matrix, definition_of_B_matrix): identity minus the
//         projection onto Y_lm(s_n) of the neighbour expansions, weighted by
//         omega_ij^eta at each grid point; evaluated from the hit lists.
//   C1 X_r + C2 X_e (Eq. def_c1_c2 with Eqs. definition_of_Q_matrix, definition_of_P_matrix):
//         y_j = eps1/eps2 (l/r_j) X_r - i_l'/i_l X_e;  mu_j = C_ik P chi_j y_j;
//         phi = sum_j mu_j k^j Y^j at the external points (direct summation);
//         out_i = sum_n w_n chi_i phi Y_lm(s_n), added to both block rows.
//   The transposes follow the same data in reverse (gathers, no atomics).
#include <cub/cub.cuh>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

#define BLK 128
#define YK_TS 8

// ---------------------------------------------------------------- projections

// grid[row][n] = (w_n if weighted) * sum_lm YT[lm][n] coef[row][lm]
template <typename T, typename V4>
__global__ void k_synthesis(int N, int nb, const T* __restrict__ YT, const V4* __restrict__ leb,
                            const T* __restrict__ coef, T* __restrict__ grid, int weighted) {
    extern __shared__ unsigned char smraw[];
    T* sc = (T*)smraw;
    int row = blockIdx.x;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) sc[k] = coef[(size_t)row * nb + k];
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        T v = 0;
        for (int k = 0; k < nb; ++k) v += YT[(size_t)k * N + n] * sc[k];
        if (weighted) v *= leb[n].w;
        grid[(size_t)row * N + n] = v;
    }
}

// out[i][lm] (+)= scale * (cik[i][l]) * sum_{external t of i} w_n chi_t val[t] Y_lm(s_n)
template <typename T, typename V4>
__global__ void k_masked_analysis(int N, int nb, int L, const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                                  const V4* __restrict__ ext_x, const V4* __restrict__ leb,
                                  const T* __restrict__ Y, const T* __restrict__ val, T scale,
                                  const T* __restrict__ cik, T* __restrict__ out, int out_stride, int accumulate) {
    extern __shared__ unsigned char smraw[];
    int i = blockIdx.x;
    int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    T* gv = (T*)smraw;
    int* gn = (int*)(gv + N);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k;
        int n = ext_p[t] % N;
        gn[k] = n;
        gv[k] = leb[n].w * ext_x[t].w * val[t];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        T a = 0;
        for (int k = 0; k < cnt; ++k) a += Y[(size_t)gn[k] * nb + idx] * gv[k];
        int l = (int)sqrtf((float)idx + 0.5f);
        if (cik) a *= cik[(size_t)i * (L + 1) + l];
        a *= scale;
        T* o = out + (size_t)i * out_stride + idx;
        *o = accumulate ? *o + a : a;
    }
}

// ---------------------------------------------------------------- A and B

// One CTA per sphere i.  For every grid point n the neighbour expansions of X_r
// (basis r_l^j Y^j) and X_e (basis i-ratio Y^j) are summed with omega_ij^eta; the
// grid values are projected back and subtracted from the identity.
template <typename T, typename V4>
__global__ void k_ab_apply(int M, int N, int nb, int L, T kappa, const V4* __restrict__ sph,
                           const V4* __restrict__ leb, YTabT<T> yt, const int* __restrict__ hptr,
                           const int* __restrict__ hj, const T* __restrict__ hw, const T* __restrict__ Sinv,
                           const T* __restrict__ Y, const T* __restrict__ x, T* __restrict__ y,
                           T* __restrict__ gridR, T* __restrict__ gridE) {
    extern __shared__ unsigned char smraw[];
    T* sm = (T*)smraw;
    const int bd = blockDim.x, tid = threadIdx.x;
    T* vr = sm;
    T* ve = vr + N;
    T* rr = ve + N;
    T* ri = rr + (L + 1) * bd;
    const int i = blockIdx.x;
    const V4 a = sph[i];
    const T* xr = x;
    const T* xe = x + (size_t)M * nb;
    for (int n = tid; n < N; n += bd) {
        V4 s = leb[n];
        T px = a.x + a.w * s.x, py = a.y + a.w * s.y, pz = a.z + a.w * s.z;
        long long p = (long long)i * N + n;
        T sr = 0, se = 0;
        for (int h = hptr[p]; h < hptr[p + 1]; ++h) {
            int j = hj[h];
            T w = hw[h];
            V4 b = sph[j];
            T dx = px - b.x, dy = py - b.y, dz = pz - b.z;
            T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
            radial<T>(0, L, rho, b.w, kappa, nullptr, rr + tid, nullptr, bd);
            radial<T>(1, L, rho, b.w, kappa, Sinv + (size_t)j * (L + 2), ri + tid, nullptr, bd);
            const T* Xr = xr + (size_t)j * nb;
            const T* Xe = xe + (size_t)j * nb;
            T ur = 0, ue = 0;
            ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, T yv) {
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
        T ar = 0, ae = 0;
        for (int n = 0; n < N; ++n) {
            T wy = leb[n].w * Y[(size_t)n * nb + idx];
            ar += wy * vr[n];
            ae += wy * ve[n];
        }
        size_t o = (size_t)i * nb + idx;
        y[o] = xr[o] - ar;
        y[(size_t)M * nb + o] = xe[o] - ae;
    }
}

// A^T and B^T: the hits (i, n) -> j of every target sphere j, in chunks of at most
// DDLPB_TCHUNK hits (one CTA each, so that the work is balanced across SMs); each chunk adds
// its partial sums into acc (zeroed before), and k_ab_transpose_finish forms y = x - acc.
// zr, ze are the weighted syntheses w_n sum_lm Y_lm(s_n) x_{i lm} of the two blocks.
template <typename T, typename V4>
__global__ void k_ab_transpose(int M, int N, int nb, int L, T kappa, const V4* __restrict__ sph,
                               const V4* __restrict__ leb, YTabT<T> yt, const int* __restrict__ chunk_j,
                               const int* __restrict__ chunk_t0, const int* __restrict__ chunk_cnt,
                               const int* __restrict__ tp, const T* __restrict__ tw, const T* __restrict__ Sinv,
                               const T* __restrict__ zr, const T* __restrict__ ze, T* __restrict__ acc) {
    extern __shared__ unsigned char smraw[];
    T* sm = (T*)smraw;
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    T* accR = sm;
    T* accE = accR + nw * nb;
    T* rr = accE + nw * nb;          // rr | ri | rr (second hit) | ri (second hit), (L+1)*bd each
    T* ri = rr + (L + 1) * bd;
    const int j = chunk_j[blockIdx.x];
    const V4 b = sph[j];
    for (int k = tid; k < 2 * nw * nb; k += bd) sm[k] = 0;
    __syncthreads();
    const int t0 = chunk_t0[blockIdx.x], cnt = chunk_cnt[blockIdx.x];
    const T* sinv = Sinv + (size_t)j * (L + 2);
    // two hits per thread (base + tid and base + bd + tid), summed before each warp reduction
    for (int base = 0; base < cnt; base += 2 * bd) {
        T dx[2], dy[2], dz[2], wr[2], we[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            int h = base + u * bd + tid;
            dx[u] = b.w; dy[u] = 0; dz[u] = 0; wr[u] = 0; we[u] = 0;
            if (h < cnt) {
                int p = tp[t0 + h];
                int i = p / N, n = p % N;
                V4 a = sph[i], s = leb[n];
                dx[u] = a.x + a.w * s.x - b.x;
                dy[u] = a.y + a.w * s.y - b.y;
                dz[u] = a.z + a.w * s.z - b.z;
                T w = tw[t0 + h];
                wr[u] = w * zr[p];
                we[u] = w * ze[p];
            }
        }
        T e[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            T rho = sqrt(dx[u] * dx[u] + dy[u] * dy[u] + dz[u] * dz[u]), inv = (T)1 / rho;
            radial<T>(0, L, rho, b.w, kappa, nullptr, rr + tid + u * (L + 1) * bd * 2, nullptr, bd);
            radial<T>(1, L, rho, b.w, kappa, sinv, ri + tid + u * (L + 1) * bd * 2, nullptr, bd);
            e[u][0] = dx[u] * inv;
            e[u][1] = dy[u] * inv;
            e[u][2] = dz[u] * inv;
        }
        const T* rr1 = rr + (L + 1) * bd * 2;
        const T* ri1 = ri + (L + 1) * bd * 2;
        ylm_stream2<T>(L, e[0][0], e[0][1], e[0][2], e[1][0], e[1][1], e[1][2], yt,
                       [&](int idx, int l, T y0, T y1) {
                           T vR = warp_sum(wr[0] * rr[tid + l * bd] * y0 + wr[1] * rr1[tid + l * bd] * y1);
                           T vE = warp_sum(we[0] * ri[tid + l * bd] * y0 + we[1] * ri1[tid + l * bd] * y1);
                           if (lane == 0) {
                               accR[warp * nb + idx] += vR;
                               accE[warp * nb + idx] += vE;
                           }
                       });
    }
    __syncthreads();
    for (int idx = tid; idx < nb; idx += bd) {
        T sr = 0, se = 0;
        for (int w = 0; w < nw; ++w) {
            sr += accR[w * nb + idx];
            se += accE[w * nb + idx];
        }
        size_t o = (size_t)j * nb + idx;
        atomicAdd(acc + o, sr);
        atomicAdd(acc + (size_t)M * nb + o, se);
    }
}

template <typename T>
__global__ void k_ab_transpose_finish(long long n, const T* __restrict__ x, const T* __restrict__ acc,
                                      T* __restrict__ y) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] = x[k] - acc[k];
}

// ---------------------------------------------------------------- A and B, stored basis

// Stored ("incore", Sec. 4) form of the sparse blocks A and B: for every hit h = (i, n, j)
// the weighted basis omega_ij^eta r_l^j Y_lm^j at x_i^n and the i-ratio correction
// rat_l = i_l(kappa rho)/i_l(kappa r_j) / (rho/r_j)^l are computed once at setup, in
// coefficient-major layout [lm][H] (threads over hits read consecutive addresses).  Used by
// the FP64 set (the residuals of the mixed form and the FP64 form); its transposes evaluate
// the basis on the fly.
// Within each sphere the stored hits are ordered by neighbour j, then point n (order[k] is
// the hit index h stored at position k), so that the threads of a warp mostly read the same
// neighbour's coefficients.
__global__ void k_store_keys(int H, int N, const int* __restrict__ hp, const unsigned short* __restrict__ hs,
                             unsigned long long* __restrict__ key, int* __restrict__ val) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    const int p = hp[h];
    key[h] = ((unsigned long long)(p / N) << 32) | ((unsigned long long)hs[h] << 16) | (unsigned long long)(p % N);
    val[h] = h;
}

template <typename O> __device__ __forceinline__ O to_store(float v);
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <typename O> __device__ __forceinline__ O to_store(double v) { return (O)v; }
template <> __device__ __forceinline__ __half to_store<__half>(double v) { return __double2half(v); }

// Source position s in [0, H) takes hit order[s] and writes its row at dst[s] (s itself when
// dst is null) of arrays with row stride `stride`; hps / hjs (when not null) get the hit's
// point and neighbour sphere at that position.
template <typename T, typename V4, typename O>
__global__ void k_ab_store(int H, long long stride, int N, int nb, int L, T kappa, const V4* __restrict__ sph,
                           const V4* __restrict__ leb, YTabT<T> yt, const int* __restrict__ order,
                           const long long* __restrict__ dst, const int* __restrict__ hp, const int* __restrict__ hj,
                           const T* __restrict__ hw, const T* __restrict__ Sinv, O* __restrict__ Bp,
                           O* __restrict__ Rp, int* __restrict__ hps, int* __restrict__ hjs) {
    extern __shared__ unsigned char smraw[];
    T* sm = (T*)smraw;
    const int bd = blockDim.x, tid = threadIdx.x;
    T* rr = sm;
    T* ri = rr + (L + 1) * bd;
    const long long s = (long long)blockIdx.x * bd + tid;   // source position
    if (s >= H) return;
    const long long h = dst ? dst[s] : s;                   // storage position
    const int hh = order[s];
    const int p = hp[hh], i = p / N, n = p % N, j = hj[hh];
    if (hps) hps[h] = p;
    if (hjs) hjs[h] = j;
    const V4 a = sph[i], q = leb[n], b = sph[j];
    const T dx = a.x + a.w * q.x - b.x, dy = a.y + a.w * q.y - b.y, dz = a.z + a.w * q.z - b.z;
    const T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
    const T w = hw[hh];
    radial<T>(0, L, rho, b.w, kappa, nullptr, rr + tid, nullptr, bd);
    radial<T>(1, L, rho, b.w, kappa, Sinv + (size_t)j * (L + 2), ri + tid, nullptr, bd);
    for (int l = 0; l <= L; ++l) Rp[(size_t)l * stride + h] = to_store<O>(ri[tid + l * bd] / rr[tid + l * bd]);
    ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt,
                  [&](int idx, int l, T yv) { Bp[(size_t)idx * stride + h] = to_store<O>(w * rr[tid + l * bd] * yv); });
}

// Hit-parallel form of the stored A/B product, step 1: every thread takes hits in a grid
// stride over all spheres (balanced whatever the per-sphere hit counts) and adds
// omega u_j(x_i^n) into the global grid arrays gr, ge (zeroed before).
template <typename T>
__global__ void __launch_bounds__(256) k_ab_hits_stored(int nb, long long H, const int* __restrict__ hp,
                                                        const int* __restrict__ hj, const T* __restrict__ Bp,
                                                        const T* __restrict__ Rp, const T* __restrict__ xr,
                                                        const T* __restrict__ xe, T* __restrict__ gr,
                                                        T* __restrict__ ge) {
    for (long long h = (long long)blockIdx.x * blockDim.x + threadIdx.x; h < H; h += (long long)gridDim.x * blockDim.x) {
        const int p = hp[h], j = hj[h];
        const T* Xr = xr + (size_t)j * nb;
        const T* Xe = xe + (size_t)j * nb;
        T ur = 0, ue = 0;
        int l = 0, lend = 1;
        T rat = Rp[h];
#pragma unroll 8
        for (int idx = 0; idx < nb; ++idx) {
            if (idx == lend) {
                ++l;
                lend = (l + 1) * (l + 1);
                rat = Rp[(size_t)l * H + h];
            }
            const T bv = Bp[(size_t)idx * H + h];
            ur += __ldg(Xr + idx) * bv;
            ue += __ldg(Xe + idx) * bv * rat;
        }
        atomicAdd(gr + p, ur);
        atomicAdd(ge + p, ue);
    }
}

// Step 2: y_i = x_i - sum_n w_n Y_lm(s_n) g_i(n) for both blocks, one CTA per sphere.
template <typename T, typename V4>
__global__ void k_ab_project(int M, int N, int nb, const V4* __restrict__ leb, const T* __restrict__ Y,
                             const T* __restrict__ gr, const T* __restrict__ ge, const T* __restrict__ x,
                             T* __restrict__ y) {
    extern __shared__ unsigned char smraw[];
    T* vr = (T*)smraw;
    T* ve = vr + N;
    const int i = blockIdx.x;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        T w = leb[n].w;
        vr[n] = w * gr[(size_t)i * N + n];
        ve[n] = w * ge[(size_t)i * N + n];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        T ar = 0, ae = 0;
        for (int n = 0; n < N; ++n) {
            T yv = Y[(size_t)n * nb + idx];
            ar += yv * vr[n];
            ae += yv * ve[n];
        }
        size_t o = (size_t)i * nb + idx;
        y[o] = x[o] - ar;
        y[(size_t)M * nb + o] = x[(size_t)M * nb + o] - ae;
    }
}


// ---------------------------------------------------------------- A and B, chunk layout (FP32 set)

// Chunk layout of the stored basis (FP32 set), in the order of the transposed hit list: the
// hits of every target-sphere chunk (at most DDLPB_TCHUNK hits, one neighbour j) padded to
// an even number of groups of 8, so that one load gives one basis function at 8 hits of one
// neighbour
// (16 bytes in the FP16 copy of the preconditioner, 32 in the FP32 copy of the outer
// products).  Both directions stream the same copy.
__global__ void k_chunk_groups(int n_chunks, const int* __restrict__ chunk_cnt, int* __restrict__ cng) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_chunks) cng[k] = 2 * ((chunk_cnt[k] + 15) / 16);   // an even number of groups
}

// Storage position of every entry of the transposed hit list; the neighbour of every group.
__global__ void k_chunk_positions(const int* __restrict__ chunk_j, const int* __restrict__ chunk_t0,
                                  const int* __restrict__ chunk_cnt, const int* __restrict__ cg0,
                                  const int* __restrict__ cng, long long* __restrict__ tpos, int* __restrict__ gj) {
    const int k = blockIdx.x;
    const int t0 = chunk_t0[k], cnt = chunk_cnt[k], g0 = cg0[k];
    for (int u = threadIdx.x; u < cnt; u += blockDim.x) tpos[t0 + u] = 8LL * g0 + u;
    for (int g = threadIdx.x; g < cng[k]; g += blockDim.x) gj[g0 + g] = chunk_j[k];
}

// Point index of every stored position (the padding keeps -1).
__global__ void k_chunk_points(long long H, const long long* __restrict__ tpos, const int* __restrict__ tp,
                               int* __restrict__ hp8) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < H) hp8[tpos[t]] = tp[t];
}

__device__ __forceinline__ void half8_to_float(const uint4 v, float* f) {
    const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __half22float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

// 8 consecutive stored values (one basis function at the 8 hits of group q), as floats.
__device__ __forceinline__ void load8_h(const __half* base, size_t q, float* f) {
    half8_to_float(__ldcs(reinterpret_cast<const uint4*>(base) + q), f);
}

__device__ __forceinline__ void load8_f(const float* base, size_t q, float* f) {
    const float4* p = reinterpret_cast<const float4*>(base) + 2 * q;
    const float4 a = __ldcs(p), b = __ldcs(p + 1);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
}

template <typename S>
__device__ __forceinline__ void load8(const S* base, size_t q, float* f) {
    if constexpr (std::is_same<S, __half>::value) {
        load8_h(base, q, f);
    } else {
        load8_f(base, q, f);
    }
}

// Forward product: one thread per group of 8 hits (one neighbour j), FP32 accumulation;
// adds omega u_j(x_i^n) of both blocks into the grid arrays gr, ge (zeroed before).
// S: storage type of the basis copy (__half for the preconditioner, float for the outer
// products); GP: groups of 8 hits per thread (consecutive groups of one neighbour: the chunks
// hold an even number of groups), so that a thread loads 32 bytes per basis function.
template <typename S, int GP>
__global__ void __launch_bounds__(256) k_ab_hits_chunk(int nb, int L, long long G8, const int* __restrict__ hp8,
                                                       const int* __restrict__ gj, const S* __restrict__ Bh,
                                                       const S* __restrict__ Rh, const float* __restrict__ xr,
                                                       const float* __restrict__ xe, float* __restrict__ gr,
                                                       float* __restrict__ ge) {
    constexpr int NH = 8 * GP;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G8 / GP) return;
    const long long g = t * GP;
    const int j = gj[g];
    const float* Xr = xr + (size_t)j * nb;
    const float* Xe = xe + (size_t)j * nb;
    float ur[NH], ue[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) ur[k] = ue[k] = 0.f;
    int idx = 0;
    for (int l = 0; l <= L; ++l) {
        float rat[NH], pe[NH];
#pragma unroll
        for (int u = 0; u < GP; ++u) load8(Rh, (size_t)l * G8 + g + u, rat + 8 * u);
#pragma unroll
        for (int k = 0; k < NH; ++k) pe[k] = 0.f;
#pragma unroll 3
        for (int m = 0; m <= 2 * l; ++m, ++idx) {
            float b[NH];
#pragma unroll
            for (int u = 0; u < GP; ++u) load8(Bh, (size_t)idx * G8 + g + u, b + 8 * u);
            const float a = __ldg(Xr + idx), e = __ldg(Xe + idx);
#pragma unroll
            for (int k = 0; k < NH; ++k) {
                ur[k] = fmaf(b[k], a, ur[k]);
                pe[k] = fmaf(b[k], e, pe[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < NH; ++k) ue[k] = fmaf(rat[k], pe[k], ue[k]);
    }
    const int4* P = reinterpret_cast<const int4*>(hp8) + 2 * g;
#pragma unroll
    for (int v = 0; v < 2 * GP; ++v) {
        const int4 pv = P[v];
        const int p[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (p[k] >= 0) {
                atomicAdd(gr + p[k], ur[4 * v + k]);
                atomicAdd(ge + p[k], ue[4 * v + k]);
            }
    }
}

// Transposed product, the forward's mapping: one thread per group of 8 hits (consecutive lanes
// read consecutive 16-byte pieces of a basis function), all basis functions in turn.  The
// lanes of a warp holding the same neighbour j are contiguous; a segmented suffix sum over the
// warp (5 shuffle steps, same-segment masks computed once) leaves every segment's sum in its
// first lane, which adds it into acc (zeroed before) at sphere j.
template <typename S, int GP>
__global__ void __launch_bounds__(256) k_ab_transpose_chunk(int M, int nb, int L, long long G8,
                                                            const int* __restrict__ gj, const int* __restrict__ hp8,
                                                            const S* __restrict__ Bh, const S* __restrict__ Rh,
                                                            const float* __restrict__ zr,
                                                            const float* __restrict__ ze, float* __restrict__ acc) {
    constexpr int NH = 8 * GP;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long g = t * GP;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool act = t < G8 / GP;
    const int j = act ? gj[g] : -1;
    unsigned same = 0;   // bit s: lane + 2^s holds the same neighbour
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int tj = __shfl_down_sync(FULL, j, 1 << s);
        if (lane + (1 << s) < 32 && tj == j) same |= 1u << s;
    }
    const int jup = __shfl_up_sync(FULL, j, 1);   // every lane takes part in every shuffle
    const bool head = act && (lane == 0 || jup != j);
    float uR[NH], uE[NH];
#pragma unroll
    for (int q = 0; q < NH; ++q) uR[q] = uE[q] = 0.f;
    if (act) {
        const int4* P = reinterpret_cast<const int4*>(hp8) + 2 * g;
#pragma unroll
        for (int v = 0; v < 2 * GP; ++v) {
            const int4 pv = P[v];
            const int p[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (p[k] >= 0) {
                    uR[4 * v + k] = zr[p[k]];
                    uE[4 * v + k] = ze[p[k]];
                }
        }
    }
    float* accR = act ? acc + (size_t)j * nb : acc;
    float* accE = act ? acc + (size_t)M * nb + (size_t)j * nb : acc;
    int idx = 0;
    for (int l = 0; l <= L; ++l) {
        float w[NH];
        {
            float rat[NH];
            if (act) {
#pragma unroll
                for (int u = 0; u < GP; ++u) load8(Rh, (size_t)l * G8 + g + u, rat + 8 * u);
            } else {
#pragma unroll
                for (int q = 0; q < NH; ++q) rat[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < NH; ++q) w[q] = uE[q] * rat[q];
        }
#pragma unroll 3
        for (int m = 0; m <= 2 * l; ++m, ++idx) {
            float b[NH];
            if (act) {
#pragma unroll
                for (int u = 0; u < GP; ++u) load8(Bh, (size_t)idx * G8 + g + u, b + 8 * u);
            } else {
#pragma unroll
                for (int q = 0; q < NH; ++q) b[q] = 0.f;
            }
            float vR = 0.f, vE = 0.f;
#pragma unroll
            for (int q = 0; q < NH; ++q) {
                vR = fmaf(b[q], uR[q], vR);
                vE = fmaf(b[q], w[q], vE);
            }
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const float tR = __shfl_down_sync(FULL, vR, 1 << s);
                const float tE = __shfl_down_sync(FULL, vE, 1 << s);
                if (same & (1u << s)) {
                    vR += tR;
                    vE += tE;
                }
            }
            if (head) {
                atomicAdd(accR + idx, vR);
                atomicAdd(accE + idx, vE);
            }
        }
    }
}

// ---------------------------------------------------------------- dense coupling (L_C)

// mu_j = C_ik^j * P chi_j y_j with y_j = eps1/eps2 (l/r_j) X_r,j - i_l'/i_l X_e,j, for j in src.
template <typename T, typename V4>
__global__ void k_source_mu(int M, int N, int nb, int L, T e12, const int* __restrict__ src,
                            const V4* __restrict__ sph, const T* __restrict__ di, const T* __restrict__ cik,
                            const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                            const V4* __restrict__ ext_x, const V4* __restrict__ leb, const T* __restrict__ Y,
                            const T* __restrict__ x, T* __restrict__ mu) {
    extern __shared__ unsigned char smraw[];
    const int j = src[blockIdx.x];
    T* yv = (T*)smraw;
    T* gv = yv + nb;
    int* gn = (int*)(gv + N);
    const T rj = sph[j].w;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        int l = (int)sqrtf((float)idx + 0.5f);
        yv[idx] = e12 * (T)l / rj * x[(size_t)j * nb + idx] - di[(size_t)j * (L + 1) + l] * x[(size_t)(M + j) * nb + idx];
    }
    __syncthreads();
    const int t0 = ext_ptr[j], cnt = ext_ptr[j + 1] - t0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, n = ext_p[t] % N;
        T v = 0;
        for (int idx = 0; idx < nb; ++idx) v += Y[(size_t)n * nb + idx] * yv[idx];
        gn[k] = n;
        gv[k] = leb[n].w * ext_x[t].w * v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        T a = 0;
        for (int k = 0; k < cnt; ++k) a += Y[(size_t)gn[k] * nb + idx] * gv[k];
        int l = (int)sqrtf((float)idx + 0.5f);
        mu[(size_t)j * nb + idx] = cik[(size_t)j * (L + 1) + l] * a;
    }
}

// phi(x_t) = sum_{j in src} sum_lm mu_j,lm k_l^j(x_t) Y_lm^j(x_t) at every external point t
// (the potential in Eqs. definition_of_Q_matrix / defintion_of_S).  Direct summation: one
// thread per target, source tiles staged in shared memory.
template <typename T, typename V4>
__global__ void k_yukawa_pot(int E, const V4* __restrict__ ext_x, int n_src, const int* __restrict__ src,
                             const V4* __restrict__ sph, const T* __restrict__ mu, const T* __restrict__ Khinv,
                             int nb, int L, T kappa, YTabT<T> yt, T* __restrict__ phi) {
    extern __shared__ unsigned char smraw[];
    const int bd = blockDim.x, tid = threadIdx.x;
    V4* sp = (V4*)smraw;
    T* smu = (T*)(sp + YK_TS);
    T* skh = smu + YK_TS * nb;
    T* rad = skh + YK_TS * (L + 2);
    const int t = blockIdx.x * bd + tid;
    const bool valid = t < E;
    V4 xt;
    if (valid) xt = ext_x[t];
    else xt.x = xt.y = xt.z = xt.w = 0;
    T acc = 0;
    // sources of this CTA: group blockIdx.y of gridDim.y (partials added atomically when split)
    const int per = ((n_src + gridDim.y - 1) / gridDim.y + YK_TS - 1) / YK_TS * YK_TS;
    const int s_begin = blockIdx.y * per, s_end = min(n_src, s_begin + per);
    for (int base = s_begin; base < s_end; base += YK_TS) {
        int ns = min(YK_TS, s_end - base);
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
            V4 b = sp[s];
            T dx = valid ? xt.x - b.x : b.w, dy = valid ? xt.y - b.y : (T)0, dz = valid ? xt.z - b.z : (T)0;
            T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
            radial<T>(2, L, rho, b.w, kappa, skh + s * (L + 2), rad + tid, nullptr, bd);
            const T* m = smu + s * nb;
            T v = 0;
            ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt,
                          [&](int idx, int l, T yv) { v += m[idx] * rad[tid + l * bd] * yv; });
            acc += v;
        }
    }
    if (valid) {
        if (gridDim.y > 1) atomicAdd(phi + t, acc);
        else phi[t] = acc;
    }
}

// nu_j = sum_t c_t k_l^j(x_t) Y_lm^j(x_t) (transpose of k_yukawa_pot), one CTA per source j.
template <typename T, typename V4>
__global__ void k_yukawa_adj(int E, const V4* __restrict__ ext_x, const T* __restrict__ cext,
                             const int* __restrict__ src, const V4* __restrict__ sph, const T* __restrict__ Khinv,
                             int nb, int L, T kappa, YTabT<T> yt, T* __restrict__ nu) {
    extern __shared__ unsigned char smraw[];
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    T* acc = (T*)smraw;
    T* kh = acc + nw * nb;
    T* rad = kh + (L + 2);
    const int j = src[blockIdx.x];
    const V4 b = sph[j];
    for (int k = tid; k < nw * nb; k += bd) acc[k] = 0;
    for (int k = tid; k < L + 2; k += bd) kh[k] = Khinv[(size_t)j * (L + 2) + k];
    __syncthreads();
    // targets of this CTA: chunk blockIdx.y of gridDim.y (partials added atomically when split)
    const int per = ((E + gridDim.y - 1) / gridDim.y + bd - 1) / bd * bd;
    const int t_begin = blockIdx.y * per, t_end = min(E, t_begin + per);
    for (int base = t_begin; base < t_end; base += bd) {
        int t = base + tid;
        T dx = b.w, dy = 0, dz = 0, c = 0;
        if (t < t_end) {
            V4 xt = ext_x[t];
            dx = xt.x - b.x;
            dy = xt.y - b.y;
            dz = xt.z - b.z;
            c = cext[t];
        }
        T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
        radial<T>(2, L, rho, b.w, kappa, kh, rad + tid, nullptr, bd);
        ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, T yv) {
            T v = warp_sum(c * rad[tid + l * bd] * yv);
            if (lane == 0) acc[warp * nb + idx] += v;
        });
    }
    __syncthreads();
    for (int idx = tid; idx < nb; idx += bd) {
        T s = 0;
        for (int w = 0; w < nw; ++w) s += acc[w * nb + idx];
        if (gridDim.y > 1) atomicAdd(nu + (size_t)j * nb + idx, s);
        else nu[(size_t)j * nb + idx] = s;
    }
}

// The near part of the coupling, used inside the preconditioner: for an external point t
// of sphere i, phi_loc(t) = sum over j in {i} and N_i of mu_j . B^k_j(x_t).  mu_j is zero
// for spheres without external points.  One CTA per sphere i.
template <typename T, typename V4>
__global__ void k_yukawa_local(int N, int nb, int L, T kappa, const int* __restrict__ ext_ptr,
                               const V4* __restrict__ ext_x, const int* __restrict__ nptr,
                               const int* __restrict__ nidx, const V4* __restrict__ sph, const T* __restrict__ mu,
                               const T* __restrict__ Khinv, YTabT<T> yt, T* __restrict__ phi) {
    extern __shared__ unsigned char smraw[];
    const int bd = blockDim.x, tid = threadIdx.x;
    T* rad = (T*)smraw;
    const int i = blockIdx.x;
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    const int k0 = nptr[i], nn = nptr[i + 1] - k0;
    for (int t = t0 + tid; t < t0 + cnt; t += bd) {
        V4 xt = ext_x[t];
        T acc = 0;
        for (int k = -1; k < nn; ++k) {
            int j = k < 0 ? i : nidx[k0 + k];
            V4 b = sph[j];
            T dx = xt.x - b.x, dy = xt.y - b.y, dz = xt.z - b.z;
            T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
            radial<T>(2, L, rho, b.w, kappa, Khinv + (size_t)j * (L + 2), rad + tid, nullptr, bd);
            const T* m = mu + (size_t)j * nb;
            T v = 0;
            ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt,
                          [&](int idx, int l, T yv) { v += __ldg(m + idx) * rad[tid + l * bd] * yv; });
            acc += v;
        }
        phi[t] = acc;
    }
}

// Transpose of k_yukawa_local: nu_j = sum over i in {j} and N_j, t external on i, of
// c_t B^k_j(x_t).  One CTA per source sphere j (the neighbour relation is symmetric).
template <typename T, typename V4>
__global__ void k_yukawa_local_adj(int nb, int L, T kappa, const int* __restrict__ src,
                                   const int* __restrict__ ext_ptr, const V4* __restrict__ ext_x,
                                   const T* __restrict__ cext, const int* __restrict__ nptr,
                                   const int* __restrict__ nidx, const V4* __restrict__ sph,
                                   const T* __restrict__ Khinv, YTabT<T> yt, T* __restrict__ nu) {
    extern __shared__ unsigned char smraw[];
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    T* acc = (T*)smraw;
    T* kh = acc + nw * nb;
    T* rad = kh + (L + 2);
    const int j = src[blockIdx.x];
    const V4 b = sph[j];
    for (int k = tid; k < nw * nb; k += bd) acc[k] = 0;
    for (int k = tid; k < L + 2; k += bd) kh[k] = Khinv[(size_t)j * (L + 2) + k];
    __syncthreads();
    const int k0 = nptr[j], nn = nptr[j + 1] - k0;
    for (int k = -1; k < nn; ++k) {
        const int i = k < 0 ? j : nidx[k0 + k];
        const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
        for (int base = 0; base < cnt; base += bd) {
            int t = t0 + base + tid;
            T dx = b.w, dy = 0, dz = 0, c = 0;
            if (base + tid < cnt) {
                V4 xt = ext_x[t];
                dx = xt.x - b.x;
                dy = xt.y - b.y;
                dz = xt.z - b.z;
                c = cext[t];
            }
            T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
            radial<T>(2, L, rho, b.w, kappa, kh, rad + tid, nullptr, bd);
            ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, T yv) {
                T v = warp_sum(c * rad[tid + l * bd] * yv);
                if (lane == 0) acc[warp * nb + idx] += v;
            });
        }
    }
    __syncthreads();
    for (int idx = tid; idx < nb; idx += bd) {
        T s = 0;
        for (int w = 0; w < nw; ++w) s += acc[w * nb + idx];
        nu[(size_t)j * nb + idx] = s;
    }
}

// c_t = w_n chi_t sum_lm Y_lm(s_n) (x_r + x_e)_{i lm} at the external points of sphere i.
template <typename T, typename V4>
__global__ void k_ext_weights(int M, int N, int nb, const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                              const V4* __restrict__ ext_x, const V4* __restrict__ leb, const T* __restrict__ Y,
                              const T* __restrict__ x, T* __restrict__ cext) {
    extern __shared__ unsigned char smraw[];
    T* sm = (T*)smraw;
    const int i = blockIdx.x;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x)
        sm[idx] = x[(size_t)i * nb + idx] + x[(size_t)(M + i) * nb + idx];
    __syncthreads();
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, n = ext_p[t] % N;
        T v = 0;
        for (int idx = 0; idx < nb; ++idx) v += Y[(size_t)n * nb + idx] * sm[idx];
        cext[t] = leb[n].w * ext_x[t].w * v;
    }
}

// y_r,j += eps1/eps2 (l/r_j) z_j, y_e,j += -i_l'/i_l z_j with z_j = P chi_j (C_ik nu_j).
template <typename T, typename V4>
__global__ void k_ct_finish(int M, int N, int nb, int L, T e12, const int* __restrict__ src,
                            const V4* __restrict__ sph, const T* __restrict__ di, const T* __restrict__ cik,
                            const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                            const V4* __restrict__ ext_x, const V4* __restrict__ leb, const T* __restrict__ Y,
                            const T* __restrict__ nu, T* __restrict__ y) {
    extern __shared__ unsigned char smraw[];
    const int j = src[blockIdx.x];
    T* u = (T*)smraw;
    T* gv = u + nb;
    int* gn = (int*)(gv + N);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        int l = (int)sqrtf((float)idx + 0.5f);
        u[idx] = cik[(size_t)j * (L + 1) + l] * nu[(size_t)j * nb + idx];
    }
    __syncthreads();
    const int t0 = ext_ptr[j], cnt = ext_ptr[j + 1] - t0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        int t = t0 + k, n = ext_p[t] % N;
        T v = 0;
        for (int idx = 0; idx < nb; ++idx) v += Y[(size_t)n * nb + idx] * u[idx];
        gn[k] = n;
        gv[k] = leb[n].w * ext_x[t].w * v;
    }
    __syncthreads();
    const T rj = sph[j].w;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        T a = 0;
        for (int k = 0; k < cnt; ++k) a += Y[(size_t)gn[k] * nb + idx] * gv[k];
        int l = (int)sqrtf((float)idx + 0.5f);
        y[(size_t)j * nb + idx] += e12 * (T)l / rj * a;
        y[(size_t)(M + j) * nb + idx] += -di[(size_t)j * (L + 1) + l] * a;
    }
}

// ---------------------------------------------------------------- FP32 tables

template <typename S, typename D>
__global__ void k_convert(long long n, const S* __restrict__ a, D* __restrict__ b) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) b[k] = (D)a[k];
}

__global__ void k_convert_pos(int n, const double4* __restrict__ a, float4* __restrict__ b, double cx, double cy,
                              double cz) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        double4 v = a[k];
        b[k] = make_float4((float)(v.x - cx), (float)(v.y - cy), (float)(v.z - cz), (float)v.w);
    }
}

__global__ void k_convert_leb(int n, const double4* __restrict__ a, float4* __restrict__ b) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        double4 v = a[k];
        b[k] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
    }
}

// ---------------------------------------------------------------- host wrappers

static ddlpb_status set_smem(ddlpb_ctx* c, const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) DDLPB_CK(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return DDLPB_OK;
}

template <typename S, typename D>
static ddlpb_status convert(ddlpb_ctx* c, const S* a, D** b, long long n) {
    DDLPB_TRY(ctx_alloc(c, b, n));
    if (n > 0) {
        k_convert<S, D><<<ceil_div(n, 256), 256, 0, c->stream>>>(n, a, *b);
        DDLPB_LAUNCHED(c, "convert");
    }
    return DDLPB_OK;
}

template <>
ddlpb_status opset_prepare<double>(ddlpb_ctx* c, OpSet<double>& S) {
    if (S.ready) return DDLPB_OK;
    S.sph = c->sph;
    S.leb = c->leb;
    S.Y = c->Y;
    S.YT = c->YT;
    S.ytab = c->ytab;
    S.yt = c->yt;
    S.Sinv = c->Sinv;
    S.Khinv = c->Khinv;
    S.di = c->di;
    S.cik = c->cik;
    S.hit_w = c->hit_w;
    S.thit_w = c->thit_w;
    S.ext_x = c->ext_x;
    S.mu = c->mu;
    S.extA = c->extA;
    S.gridA = c->gridA;
    S.gridB = c->gridB;
    DDLPB_TRY(ctx_alloc(c, &S.acc, 2 * (size_t)c->M * c->nb));
    S.ready = true;
    return DDLPB_OK;
}

template <>
ddlpb_status opset_prepare<float>(ddlpb_ctx* c, OpSet<float>& S) {
    if (S.ready) return DDLPB_OK;
    const int M = c->M, N = c->N, nb = c->nb, L = c->lmax;
    const long long MN = (long long)M * N;
    DDLPB_TRY(ctx_alloc(c, &S.sph, M));
    k_convert_pos<<<ceil_div(M, 256), 256, 0, c->stream>>>(M, c->sph, S.sph, c->centroid[0], c->centroid[1],
                                                           c->centroid[2]);
    DDLPB_LAUNCHED(c, "convert_pos");
    DDLPB_TRY(ctx_alloc(c, &S.leb, N));
    k_convert_leb<<<ceil_div(N, 256), 256, 0, c->stream>>>(N, c->leb, S.leb);
    DDLPB_LAUNCHED(c, "convert_leb");
    DDLPB_TRY(ctx_alloc(c, &S.ext_x, c->E));
    if (c->E > 0) {
        k_convert_pos<<<ceil_div(c->E, 256), 256, 0, c->stream>>>(c->E, c->ext_x, S.ext_x, c->centroid[0],
                                                                  c->centroid[1], c->centroid[2]);
        DDLPB_LAUNCHED(c, "convert_ext");
    }
    const long long ntab = 2LL * DDLPB_LT * DDLPB_LT + 2 * DDLPB_LT;
    DDLPB_TRY(convert(c, c->ytab, &S.ytab, ntab));
    S.yt.a = S.ytab;
    S.yt.b = S.ytab + DDLPB_LT * DDLPB_LT;
    S.yt.qmm = S.yt.b + DDLPB_LT * DDLPB_LT;
    S.yt.q1 = S.yt.qmm + DDLPB_LT;
    DDLPB_TRY(convert(c, c->Y, &S.Y, (long long)N * nb));
    DDLPB_TRY(convert(c, c->YT, &S.YT, (long long)N * nb));
    DDLPB_TRY(convert(c, c->Sinv, &S.Sinv, (long long)M * (L + 2)));
    DDLPB_TRY(convert(c, c->Khinv, &S.Khinv, (long long)M * (L + 2)));
    DDLPB_TRY(convert(c, c->di, &S.di, (long long)M * (L + 1)));
    DDLPB_TRY(convert(c, c->cik, &S.cik, (long long)M * (L + 1)));
    DDLPB_TRY(convert(c, c->hit_w, &S.hit_w, c->H));
    DDLPB_TRY(convert(c, c->thit_w, &S.thit_w, c->H));
    DDLPB_TRY(ctx_alloc(c, &S.mu, (size_t)M * nb));
    DDLPB_TRY(ctx_alloc(c, &S.extA, c->E));
    DDLPB_TRY(ctx_alloc(c, &S.gridA, MN));
    DDLPB_TRY(ctx_alloc(c, &S.gridB, MN));
    DDLPB_TRY(ctx_alloc(c, &S.acc, 2 * (size_t)M * nb));
    DDLPB_CK(c, cudaMemsetAsync(S.mu, 0, sizeof(float) * M * nb, c->stream));
    S.ready = true;
    return DDLPB_OK;
}

// Stored basis of the forward A/B product (built on the first forward application).
template <typename T>
static ddlpb_status build_stored(ddlpb_ctx* c, OpSet<T>& S) {
    S.store_tried = true;
    KernelTimer kt(c, "store", sizeof(T) == 4, 2);
    const int N = c->N, nb = c->nb, L = c->lmax;
    const long long H = c->H;
    if (H <= 0) return DDLPB_OK;
    unsigned long long *kin = nullptr, *kout = nullptr;
    int *vin = nullptr, *order = nullptr;
    DDLPB_TRY(ctx_alloc(c, &kin, H));
    DDLPB_TRY(ctx_alloc(c, &kout, H));
    DDLPB_TRY(ctx_alloc(c, &vin, H));
    DDLPB_TRY(ctx_alloc(c, &order, H));
    k_store_keys<<<ceil_div(H, 256), 256, 0, c->stream>>>((int)H, N, c->hit_p, c->hit_s, kin, vin);
    DDLPB_LAUNCHED(c, "store_keys");
    size_t bytes = 0;
    DDLPB_CK(c, cub::DeviceRadixSort::SortPairs(nullptr, bytes, kin, kout, vin, order, (int)H, 0, 64, c->stream));
    void* tmp = nullptr;
    DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
    DDLPB_CK(c, cub::DeviceRadixSort::SortPairs(tmp, bytes, kin, kout, vin, order, (int)H, 0, 64, c->stream));
    DDLPB_TRY(ctx_alloc(c, &S.Bp, (size_t)nb * H));
    DDLPB_TRY(ctx_alloc(c, &S.Rp, (size_t)(L + 1) * H));
    DDLPB_TRY(ctx_alloc(c, &S.hps, H));
    DDLPB_TRY(ctx_alloc(c, &S.hjs, H));
    size_t smem = sizeof(T) * 2 * (size_t)(L + 1) * BLK;
    DDLPB_TRY(set_smem(c, (const void*)k_ab_store<T, typename OpSet<T>::V4, T>, smem));
    k_ab_store<T, typename OpSet<T>::V4, T><<<ceil_div(H, BLK), BLK, smem, c->stream>>>(
        (int)H, H, N, nb, L, (T)c->kappa, S.sph, S.leb, S.yt, order, nullptr, c->hit_p, c->hit_j, S.hit_w, S.Sinv,
        S.Bp, S.Rp, S.hps, S.hjs);
    DDLPB_LAUNCHED(c, "ab_store");
    S.stored = true;
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status synthesis_T(ddlpb_ctx* c, OpSet<T>& S, const T* coef, int rows, T* grid, bool weighted) {
    if (rows <= 0) return DDLPB_OK;
    KernelTimer kt(c, "synthesis", sizeof(T) == 4, 2);
    k_synthesis<T><<<rows, BLK, sizeof(T) * c->nb, c->stream>>>(c->N, c->nb, S.YT, S.leb, coef, grid, weighted);
    DDLPB_LAUNCHED(c, "synthesis");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status masked_analysis_T(ddlpb_ctx* c, OpSet<T>& S, const T* val_ext, T scale, const T* cik_scale,
                                      T* out, int out_stride, int accumulate) {
    size_t smem = (sizeof(T) + sizeof(int)) * c->N;
    KernelTimer kt(c, "masked_analysis", sizeof(T) == 4, 2);
    k_masked_analysis<T><<<c->M, BLK, smem, c->stream>>>(c->N, c->nb, c->lmax, c->ext_ptr, c->ext_p, S.ext_x, S.leb,
                                                         S.Y, val_ext, scale, cik_scale, out, out_stride, accumulate);
    DDLPB_LAUNCHED(c, "masked_analysis");
    return DDLPB_OK;
}

static ddlpb_status apply_AB_chunks(ddlpb_ctx* c, OpSet<float>& S, const float* x, float* y, bool transpose,
                                    bool fp16, bool* done);

template <typename T>
ddlpb_status op_apply_AB_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose, T* gridR, T* gridE) {
    DDLPB_TRY(opset_prepare<T>(c, S));
    const int L = c->lmax;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 set: both directions stream the FP32 copy in the chunk layout
        if (y && !gridR) {
            bool done = false;
            DDLPB_TRY(apply_AB_chunks(c, S, x, y, transpose, false, &done));
            if (done) return DDLPB_OK;
        }
    }
    if (!transpose && y && !gridR && !S.store_tried) DDLPB_TRY(build_stored<T>(c, S));
    if (S.stored && !gridR && y && !transpose) {
        using V4 = typename OpSet<T>::V4;
        {
            const long long MN = (long long)c->M * c->N;
            DDLPB_CK(c, cudaMemsetAsync(S.gridA, 0, sizeof(T) * MN, c->stream));
            DDLPB_CK(c, cudaMemsetAsync(S.gridB, 0, sizeof(T) * MN, c->stream));
            {
                KernelTimer kt(c, "ab_apply", sizeof(T) == 4);
                const int grid = (int)std::min<long long>(ceil_div(c->H, 256), 152LL * 8);
                k_ab_hits_stored<T><<<grid, 256, 0, c->stream>>>(c->nb, c->H, S.hps, S.hjs, S.Bp, S.Rp, x,
                                                                 x + (size_t)c->M * c->nb, S.gridA, S.gridB);
                DDLPB_LAUNCHED(c, "ab_hits_stored");
            }
            {
                KernelTimer kt(c, "ab_project", sizeof(T) == 4, 2);
                k_ab_project<T, V4><<<c->M, BLK, sizeof(T) * 2 * (size_t)c->N, c->stream>>>(c->M, c->N, c->nb, S.leb, S.Y,
                                                                                           S.gridA, S.gridB, x, y);
                DDLPB_LAUNCHED(c, "ab_project");
            }
            return DDLPB_OK;
        }
    }
    if (!transpose) {
        size_t smem = sizeof(T) * (2 * (size_t)c->N + 2 * (size_t)(L + 1) * BLK);
        DDLPB_TRY(set_smem(c, (const void*)k_ab_apply<T, typename OpSet<T>::V4>, smem));
        KernelTimer kt(c, "ab_apply", sizeof(T) == 4);
        k_ab_apply<T><<<c->M, BLK, smem, c->stream>>>(c->M, c->N, c->nb, L, (T)c->kappa, S.sph, S.leb, S.yt,
                                                      c->hit_ptr, c->hit_j, S.hit_w, S.Sinv, S.Y, x, y, gridR, gridE);
        DDLPB_LAUNCHED(c, "ab_apply");
        return DDLPB_OK;
    }
    DDLPB_TRY(synthesis_T<T>(c, S, x, c->M, S.gridA, true));
    DDLPB_TRY(synthesis_T<T>(c, S, x + (size_t)c->M * c->nb, c->M, S.gridB, true));
    size_t smem = sizeof(T) * (2 * (size_t)(BLK / 32) * c->nb + 4 * (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_ab_transpose<T, typename OpSet<T>::V4>, smem));
    const long long nv = 2LL * c->M * c->nb;
    DDLPB_CK(c, cudaMemsetAsync(S.acc, 0, sizeof(T) * nv, c->stream));
    if (c->n_chunks > 0) {
        KernelTimer kt(c, "ab_transpose", sizeof(T) == 4);
        k_ab_transpose<T><<<c->n_chunks, BLK, smem, c->stream>>>(c->M, c->N, c->nb, L, (T)c->kappa, S.sph, S.leb,
                                                                 S.yt, c->chunk_j, c->chunk_t0, c->chunk_cnt,
                                                                 c->thit_p, S.thit_w, S.Sinv, S.gridA, S.gridB,
                                                                 S.acc);
        DDLPB_LAUNCHED(c, "ab_transpose");
    }
    k_ab_transpose_finish<T><<<ceil_div(nv, 256), 256, 0, c->stream>>>(nv, x, S.acc, y);
    DDLPB_LAUNCHED(c, "ab_transpose_finish");
    return DDLPB_OK;
}

// Chunk layout of the stored basis (FP32 set): the target-major hit list cut into chunks of
// one neighbour, each padded to whole groups of 8 hits; built on the first stored product.
static ddlpb_status build_chunk_layout(ddlpb_ctx* c, OpSet<float>& S) {
    S.chunk_tried = true;
    const long long H = c->H;
    const int nch = c->n_chunks;
    if (H <= 0 || nch <= 0) return DDLPB_OK;
    DDLPB_TRY(ctx_alloc(c, &S.cng, nch));
    DDLPB_TRY(ctx_alloc(c, &S.cg0, nch));
    k_chunk_groups<<<ceil_div(nch, 256), 256, 0, c->stream>>>(nch, c->chunk_cnt, S.cng);
    DDLPB_LAUNCHED(c, "chunk_groups");
    size_t bytes = 0;
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(nullptr, bytes, S.cng, S.cg0, nch, c->stream));
    void* tmp = nullptr;
    DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(tmp, bytes, S.cng, S.cg0, nch, c->stream));
    int last[2] = {0, 0};
    DDLPB_CK(c, cudaMemcpyAsync(&last[0], S.cg0 + nch - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaMemcpyAsync(&last[1], S.cng + nch - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    S.G8 = (long long)last[0] + last[1];
    const size_t H8 = 8 * (size_t)S.G8;
    DDLPB_TRY(ctx_alloc(c, &S.tpos, H));
    DDLPB_TRY(ctx_alloc(c, &S.hp8, H8));
    DDLPB_TRY(ctx_alloc(c, &S.gj, (size_t)S.G8));
    DDLPB_CK(c, cudaMemsetAsync(S.hp8, 0xFF, sizeof(int) * H8, c->stream));
    k_chunk_positions<<<nch, 128, 0, c->stream>>>(c->chunk_j, c->chunk_t0, c->chunk_cnt, S.cg0, S.cng, S.tpos, S.gj);
    DDLPB_LAUNCHED(c, "chunk_positions");
    k_chunk_points<<<ceil_div(H, 256), 256, 0, c->stream>>>(H, S.tpos, c->thit_p, S.hp8);
    DDLPB_LAUNCHED(c, "chunk_points");
    S.chunk_ready = true;
    return DDLPB_OK;
}

// One copy of the basis in the chunk layout: O = float (outer products) or __half
// (preconditioner).
template <typename O>
static ddlpb_status build_chunk_copy(ddlpb_ctx* c, OpSet<float>& S, O** Bc, O** Rc) {
    const bool half = std::is_same<O, __half>::value;
    KernelTimer kt(c, std::string(half ? "store_f16" : "store_f32"), 2);
    const long long H = c->H;
    const int nb = c->nb, L = c->lmax;
    const size_t H8 = 8 * (size_t)S.G8;
    DDLPB_TRY(ctx_alloc(c, Bc, (size_t)nb * H8));
    DDLPB_TRY(ctx_alloc(c, Rc, (size_t)(L + 1) * H8));
    DDLPB_CK(c, cudaMemsetAsync(*Bc, 0, sizeof(O) * nb * H8, c->stream));
    DDLPB_CK(c, cudaMemsetAsync(*Rc, 0, sizeof(O) * (L + 1) * H8, c->stream));
    // evaluated in FP64 from the exact geometry and rounded once to the storage type
    size_t smem = sizeof(double) * 2 * (size_t)(L + 1) * BLK;
    DDLPB_TRY(set_smem(c, (const void*)k_ab_store<double, double4, O>, smem));
    k_ab_store<double, double4, O><<<ceil_div(H, BLK), BLK, smem, c->stream>>>(
        (int)H, (long long)H8, c->N, nb, L, c->kappa, c->sph, c->leb, c->yt, c->thit_h, S.tpos, c->hit_p, c->hit_j,
        c->hit_w, c->Sinv, *Bc, *Rc, nullptr, nullptr);
    DDLPB_LAUNCHED(c, half ? "ab_store_half" : "ab_store_chunk");
    return DDLPB_OK;
}

// A/B (or their transposes) with the basis copy in the chunk layout, FP32 vectors: the FP16
// copy (fp16) or the FP32 one.  *done = false when there is no layout (no hits at all).
// Groups of 8 hits per thread: one, except in the FP16 transpose, which takes two (half the
// warp reductions per byte streamed).
template <typename O>
static ddlpb_status apply_chunks(ddlpb_ctx* c, OpSet<float>& S, const O* Bc, const O* Rc, const char* tag,
                                 const float* x, float* y, bool transpose) {
    constexpr int GP = 1;
    constexpr int GPT = std::is_same<O, __half>::value ? 2 : 1;
    const int M = c->M, nb = c->nb, L = c->lmax;
    const float* xe = x + (size_t)M * nb;
    if (!transpose) {
        const long long MN = (long long)M * c->N;
        DDLPB_CK(c, cudaMemsetAsync(S.gridA, 0, sizeof(float) * MN, c->stream));
        DDLPB_CK(c, cudaMemsetAsync(S.gridB, 0, sizeof(float) * MN, c->stream));
        {
            KernelTimer kt(c, std::string("ab_apply_") + tag);
            k_ab_hits_chunk<O, GP><<<ceil_div(S.G8 / GP, 256), 256, 0, c->stream>>>(nb, L, S.G8, S.hp8, S.gj, Bc, Rc,
                                                                                     x, xe, S.gridA, S.gridB);
            DDLPB_LAUNCHED(c, "ab_hits_chunk");
        }
        {
            KernelTimer kt(c, "ab_project", true, 2);
            k_ab_project<float, float4><<<M, BLK, sizeof(float) * 2 * (size_t)c->N, c->stream>>>(M, c->N, nb, S.leb, S.Y,
                                                                                                S.gridA, S.gridB, x, y);
            DDLPB_LAUNCHED(c, "ab_project");
        }
        return DDLPB_OK;
    }
    DDLPB_TRY(synthesis_T<float>(c, S, x, M, S.gridA, true));
    DDLPB_TRY(synthesis_T<float>(c, S, xe, M, S.gridB, true));
    const long long nv = 2LL * M * nb;
    DDLPB_CK(c, cudaMemsetAsync(S.acc, 0, sizeof(float) * nv, c->stream));
    {
        KernelTimer kt(c, std::string("ab_transpose_") + tag);
        k_ab_transpose_chunk<O, GPT><<<ceil_div(S.G8 / GPT, 256), 256, 0, c->stream>>>(M, nb, L, S.G8, S.gj, S.hp8,
                                                                                        Bc, Rc, S.gridA, S.gridB,
                                                                                        S.acc);
        DDLPB_LAUNCHED(c, "ab_transpose_chunk");
    }
    k_ab_transpose_finish<float><<<ceil_div(nv, 256), 256, 0, c->stream>>>(nv, x, S.acc, y);
    DDLPB_LAUNCHED(c, "ab_transpose_finish");
    return DDLPB_OK;
}

static ddlpb_status apply_AB_chunks(ddlpb_ctx* c, OpSet<float>& S, const float* x, float* y, bool transpose,
                                    bool fp16, bool* done) {
    *done = false;
    DDLPB_TRY(opset_prepare<float>(c, S));
    if (!S.chunk_tried) DDLPB_TRY(build_chunk_layout(c, S));
    if (!S.chunk_ready) return DDLPB_OK;
    if (fp16) {
        if (!S.Bh) DDLPB_TRY(build_chunk_copy<__half>(c, S, &S.Bh, &S.Rh));
        DDLPB_TRY(apply_chunks<__half>(c, S, S.Bh, S.Rh, "f16", x, y, transpose));
    } else {
        if (!S.Bc) DDLPB_TRY(build_chunk_copy<float>(c, S, &S.Bc, &S.Rc));
        DDLPB_TRY(apply_chunks<float>(c, S, S.Bc, S.Rc, "f32", x, y, transpose));
    }
    *done = true;
    return DDLPB_OK;
}

// A/B (or their transposes) with the FP16 copy, FP32 vectors (FP32 products when there are no hits).
static ddlpb_status apply_AB_half(ddlpb_ctx* c, OpSet<float>& S, const float* x, float* y, bool transpose) {
    bool done = false;
    DDLPB_TRY(apply_AB_chunks(c, S, x, y, transpose, true, &done));
    if (done) return DDLPB_OK;
    return op_apply_AB_T<float>(c, S, x, y, transpose, nullptr, nullptr);
}

template <>
ddlpb_status op_apply_AB_precond<double>(ddlpb_ctx* c, OpSet<double>& S, const double* x, double* y,
                                         bool transpose) {
    return op_apply_AB_T<double>(c, S, x, y, transpose, nullptr, nullptr);
}

template <>
ddlpb_status op_apply_AB_precond<float>(ddlpb_ctx* c, OpSet<float>& S, const float* x, float* y, bool transpose) {
    if (c->opt.precond_fp16) return apply_AB_half(c, S, x, y, transpose);
    return op_apply_AB_T<float>(c, S, x, y, transpose, nullptr, nullptr);
}

template <typename T>
static ddlpb_status source_mu_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* mu) {
    if (c->n_src == 0) return DDLPB_OK;
    size_t smem = sizeof(T) * (c->nb + c->N) + sizeof(int) * c->N;
    KernelTimer kt(c, "coupling_projection", sizeof(T) == 4, 2);
    k_source_mu<T><<<c->n_src, BLK, smem, c->stream>>>(c->M, c->N, c->nb, c->lmax, (T)(c->eps1 / c->eps2), c->src,
                                                       S.sph, S.di, S.cik, c->ext_ptr, c->ext_p, S.ext_x, S.leb, S.Y,
                                                       x, mu);
    DDLPB_LAUNCHED(c, "source_mu");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status yukawa_pot_T(ddlpb_ctx* c, OpSet<T>& S, const T* mu, T* phi_ext) {
    if (c->E == 0) return DDLPB_OK;
    const int L = c->lmax;
    using V4 = typename OpSet<T>::V4;
    size_t smem = sizeof(V4) * YK_TS + sizeof(T) * (YK_TS * (size_t)c->nb + YK_TS * (size_t)(L + 2) +
                                                     (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_yukawa_pot<T, V4>, smem));
    // at least ~4 CTAs per SM: split the sources when the targets alone give too few CTAs
    const int cx = ceil_div(c->E, BLK);
    const int sy = std::max(1, std::min(ceil_div(608, cx), ceil_div(c->n_src, 4 * YK_TS)));
    if (sy > 1) DDLPB_CK(c, cudaMemsetAsync(phi_ext, 0, sizeof(T) * c->E, c->stream));
    KernelTimer kt(c, "yukawa_pot", sizeof(T) == 4);
    k_yukawa_pot<T><<<dim3(cx, sy), BLK, smem, c->stream>>>(c->E, S.ext_x, c->n_src, c->src, S.sph, mu, S.Khinv,
                                                            c->nb, L, (T)c->kappa, S.yt, phi_ext);
    DDLPB_LAUNCHED(c, "yukawa_pot");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status yukawa_adj_T(ddlpb_ctx* c, OpSet<T>& S, const T* c_ext, T* nu) {
    if (c->n_src == 0) return DDLPB_OK;
    const int L = c->lmax;
    using V4 = typename OpSet<T>::V4;
    size_t smem = sizeof(T) * ((size_t)(BLK / 32) * c->nb + (L + 2) + (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_yukawa_adj<T, V4>, smem));
    // at least ~4 CTAs per SM: split the targets when the sources alone give too few CTAs
    const int ty = std::max(1, std::min(ceil_div(608, c->n_src), ceil_div(c->E, 4 * BLK)));
    if (ty > 1) DDLPB_CK(c, cudaMemsetAsync(nu, 0, sizeof(T) * (size_t)c->M * c->nb, c->stream));
    KernelTimer kt(c, "yukawa_adj", sizeof(T) == 4);
    k_yukawa_adj<T><<<dim3(c->n_src, ty), BLK, smem, c->stream>>>(c->E, S.ext_x, c_ext, c->src, S.sph, S.Khinv,
                                                                  c->nb, L, (T)c->kappa, S.yt, nu);
    DDLPB_LAUNCHED(c, "yukawa_adj");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status ext_weights_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* cext) {
    KernelTimer kt(c, "coupling_projection", sizeof(T) == 4, 2);
    k_ext_weights<T><<<c->M, BLK, sizeof(T) * c->nb, c->stream>>>(c->M, c->N, c->nb, c->ext_ptr, c->ext_p, S.ext_x,
                                                                  S.leb, S.Y, x, cext);
    DDLPB_LAUNCHED(c, "ext_weights");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status yukawa_local_T(ddlpb_ctx* c, OpSet<T>& S, const T* mu, T* phi_ext) {
    if (c->E == 0) return DDLPB_OK;
    size_t smem = sizeof(T) * (size_t)(c->lmax + 1) * BLK;
    KernelTimer kt(c, "yukawa_local", sizeof(T) == 4);
    k_yukawa_local<T><<<c->M, BLK, smem, c->stream>>>(c->N, c->nb, c->lmax, (T)c->kappa, c->ext_ptr, S.ext_x,
                                                      c->nbr_ptr, c->nbr_idx, S.sph, mu, S.Khinv, S.yt, phi_ext);
    DDLPB_LAUNCHED(c, "yukawa_local");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status yukawa_local_adj_T(ddlpb_ctx* c, OpSet<T>& S, const T* c_ext, T* nu) {
    if (c->n_src == 0) return DDLPB_OK;
    const int L = c->lmax;
    using V4 = typename OpSet<T>::V4;
    size_t smem = sizeof(T) * ((size_t)(BLK / 32) * c->nb + (L + 2) + (size_t)(L + 1) * BLK);
    DDLPB_TRY(set_smem(c, (const void*)k_yukawa_local_adj<T, V4>, smem));
    k_yukawa_local_adj<T><<<c->n_src, BLK, smem, c->stream>>>(c->nb, L, (T)c->kappa, c->src, c->ext_ptr, S.ext_x,
                                                              c_ext, c->nbr_ptr, c->nbr_idx, S.sph, S.Khinv, S.yt,
                                                              nu);
    DDLPB_LAUNCHED(c, "yukawa_local_adj");
    return DDLPB_OK;
}

template <typename T>
static ddlpb_status apply_C_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose, bool accumulate,
                              bool local = false);

// y (+)= [K y ; K y] (forward) or y (+)= [D1 K^T (x_r + x_e) ; D2 K^T (x_r + x_e)] (transpose).
// With local, K keeps only the sources j in {i} and N_i of each target sphere i.  With the FMM
// (fmm_order > 0) the potential and its transpose come from fmm.cu.
template <typename T>
static ddlpb_status apply_C_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose, bool accumulate,
                              bool local) {
    DDLPB_TRY(opset_prepare<T>(c, S));
    const size_t half = (size_t)c->M * c->nb;
    if (!transpose) {
        DDLPB_TRY(source_mu_T<T>(c, S, x, S.mu));
        if (local) DDLPB_TRY(yukawa_local_T<T>(c, S, S.mu, S.extA));
        else if (c->fmm.on) DDLPB_TRY(fmm_potential<T>(c, S, S.mu, S.extA));
        else DDLPB_TRY(yukawa_pot_T<T>(c, S, S.mu, S.extA));
        DDLPB_TRY(masked_analysis_T<T>(c, S, S.extA, (T)1, nullptr, y, c->nb, accumulate ? 1 : 0));
        DDLPB_TRY(masked_analysis_T<T>(c, S, S.extA, (T)1, nullptr, y + half, c->nb, accumulate ? 1 : 0));
        return DDLPB_OK;
    }
    if (!accumulate) DDLPB_CK(c, cudaMemsetAsync(y, 0, sizeof(T) * 2 * half, c->stream));
    if (c->n_src == 0) return DDLPB_OK;
    DDLPB_TRY(ext_weights_T<T>(c, S, x, S.extA));
    if (local) DDLPB_TRY(yukawa_local_adj_T<T>(c, S, S.extA, S.mu));
    else if (c->fmm.on) DDLPB_TRY(fmm_adjoint<T>(c, S, S.extA, S.mu));
    else DDLPB_TRY(yukawa_adj_T<T>(c, S, S.extA, S.mu));
    size_t smem = sizeof(T) * (c->nb + c->N) + sizeof(int) * c->N;
    k_ct_finish<T><<<c->n_src, BLK, smem, c->stream>>>(c->M, c->N, c->nb, c->lmax, (T)(c->eps1 / c->eps2), c->src,
                                                       S.sph, S.di, S.cik, c->ext_ptr, c->ext_p, S.ext_x, S.leb, S.Y,
                                                       S.mu, y);
    DDLPB_LAUNCHED(c, "ct_finish");
    return DDLPB_OK;
}

template <typename T>
ddlpb_status op_apply_L_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose) {
    DDLPB_TRY(op_apply_AB_T<T>(c, S, x, y, transpose, nullptr, nullptr));
    DDLPB_TRY(apply_C_T<T>(c, S, x, y, transpose, true));
    return DDLPB_OK;
}

// The operator of the preconditioner: [A x_r ; B x_e] plus the near part of the coupling
// (or the transposes).
template <typename T>
ddlpb_status op_apply_P_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose) {
    DDLPB_TRY(op_apply_AB_T<T>(c, S, x, y, transpose, nullptr, nullptr));
    DDLPB_TRY(apply_C_T<T>(c, S, x, y, transpose, true, true));
    return DDLPB_OK;
}

template ddlpb_status op_apply_P_T<double>(ddlpb_ctx*, OpSet<double>&, const double*, double*, bool);
template ddlpb_status op_apply_P_T<float>(ddlpb_ctx*, OpSet<float>&, const float*, float*, bool);
template ddlpb_status op_apply_L_T<double>(ddlpb_ctx*, OpSet<double>&, const double*, double*, bool);
template ddlpb_status op_apply_L_T<float>(ddlpb_ctx*, OpSet<float>&, const float*, float*, bool);
template ddlpb_status op_apply_AB_T<double>(ddlpb_ctx*, OpSet<double>&, const double*, double*, bool, double*,
                                            double*);
template ddlpb_status op_apply_AB_T<float>(ddlpb_ctx*, OpSet<float>&, const float*, float*, bool, float*, float*);

// ---------------------------------------------------------------- FP64 entry points used by setup and forces

ddlpb_status op_synthesis(ddlpb_ctx* c, const double* coef, int rows, double* grid, bool weighted) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    return synthesis_T<double>(c, c->d64, coef, rows, grid, weighted);
}

ddlpb_status op_masked_analysis(ddlpb_ctx* c, const double* val_ext, double scale, const double* cik_scale,
                                double* out, int out_stride, int accumulate) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    return masked_analysis_T<double>(c, c->d64, val_ext, scale, cik_scale, out, out_stride, accumulate);
}

ddlpb_status op_apply_AB(ddlpb_ctx* c, const double* x, double* y, bool transpose, double* gridR, double* gridE) {
    return op_apply_AB_T<double>(c, c->d64, x, y, transpose, gridR, gridE);
}

ddlpb_status op_source_multipoles(ddlpb_ctx* c, const double* x, double* mu) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    return source_mu_T<double>(c, c->d64, x, mu);
}

// The potential of the sphere multipoles mu at the external points and its transpose, in FP64:
// direct sums, or the FP64 FMM.
ddlpb_status op_yukawa_potential(ddlpb_ctx* c, const double* mu, double* phi_ext) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    if (c->fmm.on) return fmm_potential<double>(c, c->d64, mu, phi_ext);
    return yukawa_pot_T<double>(c, c->d64, mu, phi_ext);
}

ddlpb_status op_yukawa_adjoint(ddlpb_ctx* c, const double* c_ext, double* nu) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    if (c->fmm.on) return fmm_adjoint<double>(c, c->d64, c_ext, nu);
    return yukawa_adj_T<double>(c, c->d64, c_ext, nu);
}

ddlpb_status op_ext_weights(ddlpb_ctx* c, const double* x, double* cext) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    return ext_weights_T<double>(c, c->d64, x, cext);
}

ddlpb_status op_apply_C(ddlpb_ctx* c, const double* x, double* y, bool transpose, bool accumulate) {
    return apply_C_T<double>(c, c->d64, x, y, transpose, accumulate);
}

ddlpb_status op_apply_L(ddlpb_ctx* c, const double* x, double* y, bool transpose) {
    DDLPB_TRY(opset_prepare<double>(c, c->d64));
    return op_apply_L_T<double>(c, c->d64, x, y, transpose);
}

// The FP32 operators on FP64 vectors (converted on the way in and out); used to
// check the FP32 inner operators of the mixed-precision form against the FP64 ones.
ddlpb_status op_apply_fp32(ddlpb_ctx* c, int op, const double* x, double* y) {
    DDLPB_TRY(opset_prepare<float>(c, c->f32));
    const long long n = c->nvec;
    if (!c->f32_vec) DDLPB_TRY(ctx_alloc(c, &c->f32_vec, 2 * (size_t)n));
    float* xf = c->f32_vec;
    float* yf = c->f32_vec + n;
    k_convert<double, float><<<ceil_div(n, 256), 256, 0, c->stream>>>(n, x, xf);
    DDLPB_LAUNCHED(c, "convert_in");
    switch (op) {
        case 0: DDLPB_TRY(op_apply_L_T<float>(c, c->f32, xf, yf, false)); break;
        case 1: DDLPB_TRY(op_apply_L_T<float>(c, c->f32, xf, yf, true)); break;
        case 2: DDLPB_TRY(op_apply_AB_T<float>(c, c->f32, xf, yf, false, nullptr, nullptr)); break;
        case 3: DDLPB_TRY(op_apply_AB_T<float>(c, c->f32, xf, yf, true, nullptr, nullptr)); break;
        case 4: DDLPB_TRY(apply_C_T<float>(c, c->f32, xf, yf, false, false)); break;
        case 5: DDLPB_TRY(apply_C_T<float>(c, c->f32, xf, yf, true, false)); break;
        case 8: DDLPB_TRY(apply_AB_half(c, c->f32, xf, yf, false)); break;
        case 9: DDLPB_TRY(apply_AB_half(c, c->f32, xf, yf, true)); break;
        default: c->err = "bad operator"; return DDLPB_EINVAL;
    }
    k_convert<float, double><<<ceil_div(n, 256), 256, 0, c->stream>>>(n, yf, y);
    DDLPB_LAUNCHED(c, "convert_out");
    return DDLPB_OK;
}
